"""GPU parity of the tensor-core (tcgen05) inverse-transform forms against the
FP64 oracle: decoded levels bit-exact in every form; samples within a relative
L2 bound derived from each form's operand rounding:
  TF32    each operand rounded to 11 significant bits: ~2^-12 per product -> 1e-3
  BF16X3  hi/lo split, the lo*lo product (2^-16 relative) dropped   -> 2e-5
  TF32X3  big/small split (big by truncation, small read as TF32: 2^-20), the small*small
          product (2^-22) dropped                                     -> 1e-5 (the FP32 bound)
"""
import numpy as np
import pytest

import oracle
import siggen

from gpu_util import compare_with_oracle, encode_workload, gpu_decode, make_plan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"tf32": 1e-3, "bf16x3": 2e-5, "tf32x3": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_01086_gb300 import build
    build()


@pytest.mark.parametrize("threads", [128, 256, 512, 640, 768, 896])
@pytest.mark.parametrize("mode", ["tf32", "bf16x3", "tf32x3"])
def test_mixed_batch(mode, threads):
    wl = siggen.mixed_10000_logu(n=40, lo=1, hi=150000)
    b = encode_workload(wl)
    if mode == "tf32x3" and threads >= 768:
        # six or seven warpgroups of 3xTF32 operands need more than the 512 tensor-memory columns
        from paper_2605_01086_gb300 import _lib
        with pytest.raises(_lib.FptcError) as ei:
            make_plan(b, idct=mode, threads=threads)
        assert ei.value.status == _lib.UNSUPPORTED and "tensor-memory" in str(ei.value)
        return
    plan = make_plan(b, idct=mode, threads=threads)
    assert plan.info["kernel"] == 4 and plan.info["idct"] == {"tf32": 1, "bf16x3": 2, "tf32x3": 3}[mode]
    _, _, out, lv = gpu_decode(plan, b, out_fill=float("nan"))
    worst = compare_with_oracle(plan, b, out, lv, tol=TOL[mode])
    assert plan.device_status()[0] == 0
    print(mode, threads, "worst rel L2", worst)


@pytest.mark.parametrize("threads", [256, 512])
@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3"])
def test_edges_misaligned_and_levels(mode, threads):
    lengths = [0, 1, 5, 31, 32, 33, 1023, 1024, 1025, 4097, 131073, 7]
    n = len(lengths)
    wl = siggen.Workload("edges", 9, np.array([i % 4 for i in range(n)], np.int32),
                         np.array([siggen.stream_seed(9, 100 + i) for i in range(n)], np.uint64),
                         np.array(lengths, np.uint64))
    b = encode_workload(wl)
    for align, base in ((4, 0), (1, 3)):
        plan = make_plan(b, idct=mode, out_align=align, out_base=base, threads=threads)
        _, _, out, lv = gpu_decode(plan, b, out_fill=float("nan"))
        compare_with_oracle(plan, b, out, lv, tol=TOL[mode])
        h = out.cpu().numpy()
        mask = np.ones(h.size, bool)
        for s in plan.segments:
            mask[int(s["out_offset"]):int(s["out_offset"]) + int(s["n_samples"])] = False
        assert np.all(np.isnan(h[mask]))


@pytest.mark.parametrize("threads", [256, 512])
def test_corrupt_segment_flagged(threads):
    from paper_2605_01086_gb300 import _lib
    wl = siggen.mixed_10000_logu(n=6, lo=5000, hi=20000)
    b = encode_workload(wl)
    bad_word = int(b.word_off[2]) + 5
    b.symlen[bad_word] -= 1
    plan = make_plan(b, idct="tf32x3", threads=threads)
    w, s = plan.to_device(b.words, b.symlen)
    out = plan.empty_out().fill_(float("nan"))
    plan.decode(w, s, out=out)
    st, flags, first = plan.device_status()
    assert st == _lib.CORRUPT_STREAM and flags & _lib.FLAG_SYMBOL_COUNT and first == 2
    compare_with_oracle(plan, b, out, None, idx=[0, 1, 3, 4, 5], tol=TOL["tf32x3"])


def test_rejects_other_shapes():
    from paper_2605_01086_gb300 import _lib
    cl = np.full(256, 8, np.uint8)
    d = oracle.Domain(64, 8, 1, 6, 50.0, 0.01, (1.0, 1.0, 0.0), 8, cl)
    b = oracle.EncodedBatch(np.zeros(1, np.uint64), np.full(1, 8, np.uint8), np.zeros(1, np.uint64),
                            np.ones(1, np.uint64), np.array([64], np.uint64), np.zeros(1, np.int32), [d])
    with pytest.raises(_lib.FptcError):
        make_plan(b, idct="bf16x3")
