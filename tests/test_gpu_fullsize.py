"""Full-size parity: the two large workloads decoded in one persistent launch
(the launch configuration of the benchmark: default options, then autotuned),
every stream's levels compared bit-exactly and every stream's samples within
1e-5 relative L2 against the FP64 oracle, chunk by chunk."""
import numpy as np
import pytest

import oracle
import siggen

from gpu_util import FP32_REL_L2, encode_workload, make_plan

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_01086_gb300 import build
    build()


def _full_check(b, autotune: bool):
    plan = make_plan(b)
    w, s = plan.to_device(b.words, b.symlen)
    out = plan.empty_out()
    lv = torch.empty(plan.info["n_levels_total"], dtype=torch.uint8, device=plan.device)
    if autotune:
        plan.autotune(w, s, out, trials=1)
    plan.decode(w, s, out=out, levels=lv)
    torch.cuda.synchronize()
    assert plan.device_status()[0] == 0
    n = b.n_streams
    worst = 0.0
    chunk = 64
    for c0 in range(0, n, chunk):
        idx = np.arange(c0, min(n, c0 + chunk))
        xs, out_off, olv, lv_off = oracle.decode_many(b, idx, want_levels=True)
        for j, i in enumerate(idx):
            S = int(b.lengths[i])
            seg = plan.segments[i]
            o = int(seg["out_offset"])
            g = out[o:o + S].double().cpu().numpy()
            r = xs[int(out_off[j]):int(out_off[j]) + S]
            rel = np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-30)
            worst = max(worst, rel)
            assert rel <= FP32_REL_L2, (i, rel)
            d = b.domains[b.domain_idx[i]]
            L = d.windows(S) * d.E
            a = int(plan.level_offsets[i])
            got = lv[a:a + L].cpu().numpy()
            assert np.array_equal(got, olv[int(lv_off[j]):int(lv_off[j]) + L]), i
    return worst


def test_eeg_2048_channels_of_1m_samples():
    b = encode_workload(siggen.eeg_2048x1m(), chunk=128)
    assert b.n_streams == 2048 and int(b.lengths.sum()) == 2048 * 2 ** 20
    _full_check(b, autotune=True)


def test_mixed_10000_signals():
    b = encode_workload(siggen.mixed_10000_logu(), chunk=500)
    assert b.n_streams == 10000
    _full_check(b, autotune=False)
