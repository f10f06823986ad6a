"""The bounded completion wait of the tensor-core and TMA kernels gives up
without a fault: nothing arrives on the barrier, the wait ends after its 1 s
bound, FPTC_FLAG_TIMEOUT is reported, and the same context decodes a batch
exactly afterwards (no GPU fault, no hang: the barrier that nothing completes
is the only thing waited on)."""
import time

import numpy as np
import pytest

import siggen

from gpu_util import compare_with_oracle, encode_workload, gpu_decode, make_plan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_01086_gb300 import build
    build()


def test_wait_gives_up_and_the_context_stays_usable():
    from paper_2605_01086_gb300 import _lib, check_bounded_wait
    assert check_bounded_wait(0, arrive=True) == 0
    t0 = time.monotonic()
    flags = check_bounded_wait(0, arrive=False)
    dt = time.monotonic() - t0
    assert flags == _lib.FLAG_TIMEOUT
    assert 0.9 <= dt < 30.0   # the 1 s bound on GPU global time, plus launch and copy
    # the context still decodes, exactly
    b = encode_workload(siggen.mixed_10000_logu(n=6, lo=100, hi=20000))
    plan = make_plan(b)
    _, _, out, lv = gpu_decode(plan, b)
    assert plan.device_status()[0] == 0
    compare_with_oracle(plan, b, out, lv)
