"""Precision forms of the inverse transform on 16,384 seismic traces x 4,096
samples, against the FP64 oracle: relative L2 and max-abs error of each form
over the whole batch (levels bit-exact in every form), and the decode time of
each.  Run with -s to see the table."""
import time

import numpy as np
import pytest

import oracle
import siggen

from gpu_util import encode_workload, make_plan

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

# bounds derived from each form's operand rounding (see test_gpu_tc.py)
BOUND = {"fp32": 1e-5, "tf32x3": 1e-5, "bf16x3": 2e-5, "tf32": 1e-3}


@pytest.fixture(scope="module")
def seismic():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_01086_gb300 import build
    build()
    b = encode_workload(siggen.seismic_16384x4096(), chunk=2048)
    xs, out_off, olv, lv_off = oracle.decode_many(b, want_levels=True)
    return b, xs, olv


def test_precision_table(seismic):
    b, xs, olv = seismic
    rows = []
    for mode in ("fp32", "tf32x3", "bf16x3", "tf32"):
        plan = make_plan(b, idct=mode, out_align=4)
        w, s = plan.to_device(b.words, b.symlen)
        out = plan.empty_out()
        lv = torch.empty(plan.info["n_levels_total"], dtype=torch.uint8, device=plan.device)
        plan.decode(w, s, out=out, levels=lv)
        for _ in range(3):
            plan.decode(w, s, out=out)
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(10):
            plan.decode(w, s, out=out)
        e.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(e) / 10
        # all streams are 4096 samples, packed back to back: the output is one array
        g = out[:xs.size].double().cpu().numpy()
        rel = float(np.linalg.norm(g - xs) / np.linalg.norm(xs))
        mx = float(np.max(np.abs(g - xs)))
        assert np.array_equal(lv.cpu().numpy()[:olv.size], olv)
        rows.append((mode, rel, mx, ms, 4.0 * xs.size / ms / 1e6))
        assert rel <= BOUND[mode], (mode, rel)
        plan.close()
    print("\nform     rel L2      max abs     ms      GB/s")
    for r in rows:
        print(f"{r[0]:8s} {r[1]:.3e}  {r[2]:.3e}  {r[3]:.3f}  {r[4]:.0f}")
