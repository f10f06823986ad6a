"""GPU parity of the warp-tile kernel for window shapes other than N = 32,
E = 16 (any N in [4, 128] for every domain of a plan, power-of-two or not,
several N in one batch, any E <= N per domain; Table 1 ranges), and of the
tensor-core transform for the shapes with E >= 32: levels bit-exact and samples within the
FP32 bound against the FP64 oracle, for random levels over every bin, ragged
lengths (partial windows, partial tiles, partial output steps), outputs at
128-byte boundaries (TMA stores) and at odd offsets (per-lane stores), several
kept-bin counts and window sizes in one batch, trained tables on synthetic signals, and tiles
chained across a segment the index rejects."""
import numpy as np
import pytest

import oracle
import siggen

from gpu_util import FP32_REL_L2, compare_with_oracle, crafted_batch, encode_workload, gpu_decode, make_plan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WARP_TILE = 3


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_01086_gb300 import build
    build()


def _random_batch(N, Es, seed, lens_of=None):
    """Uniform 8-bit codes (every level a codeword), random levels; per domain
    (same N, kept bins Es[d]) streams of ragged lengths."""
    cl = np.full(256, 8, np.uint8)
    doms = [oracle.Domain(N, E, min(2, E), max(1, E - (d % 2)), 30.0 + d, 0.02, (3.0 + d, 1.0 + 0.5 * d, 0.0), 8, cl)
            for d, E in enumerate(Es)]
    rng = np.random.default_rng(seed)
    lens, dom_idx, levels = [], [], []
    for d, dom in enumerate(doms):
        T = min(2048 // dom.E, 8192 // N)
        base = lens_of(N, T) if lens_of else [1, N - 1, N, N + 1, 1024 + 5, T * N, T * N + 3, 3 * T * N - N // 2,
                                               40000 + 17 * d]
        for S in base:
            lens.append(S)
            dom_idx.append(d)
            levels.append(rng.integers(0, 256, size=dom.windows(S) * dom.E).astype(np.uint8))
    return crafted_batch(doms, levels, lens, dom_idx)


@pytest.mark.parametrize("N,Es", [(4, [1]), (4, [3, 4]), (8, [8]), (8, [3, 6]), (16, [8, 16]), (16, [5]),
                                  (32, [8]), (32, [32, 12]), (64, [16, 32]), (64, [7]), (128, [32, 64]),
                                  (128, [128, 1]),
                                  # window sizes that are not a power of two (run-time-N transform)
                                  (5, [5]), (6, [3, 6]), (12, [5]), (24, [12, 24]), (48, [24, 7]), (100, [50, 33]),
                                  (127, [64, 127])])
@pytest.mark.parametrize("align", [32, 1])
def test_shape_random_levels(N, Es, align):
    b = _random_batch(N, Es, seed=N * 100 + sum(Es) + align)
    plan = make_plan(b, out_align=align, out_base=0 if align == 32 else 3, kernel="warp_tile")
    assert plan.info["kernel"] == WARP_TILE
    _, _, out, lv = gpu_decode(plan, b, out_fill=float("nan"))
    compare_with_oracle(plan, b, out, lv)
    # nothing outside the segments is written
    h = out.cpu().numpy()
    mask = np.ones(h.size, bool)
    for sg in plan.segments:
        mask[int(sg["out_offset"]):int(sg["out_offset"]) + int(sg["n_samples"])] = False
    assert np.all(np.isnan(h[mask]))
    assert plan.device_status()[0] == 0


@pytest.mark.parametrize("threads", [256, 512, 768])
def test_shape_thread_counts(threads):
    b = _random_batch(64, [32, 16], seed=7)
    plan = make_plan(b, out_align=32, kernel="warp_tile", threads=threads)
    assert plan.info["threads"] == threads
    _, _, out, lv = gpu_decode(plan, b)
    compare_with_oracle(plan, b, out, lv)


def test_shape_default_choice():
    """Plans whose domains all have a power-of-two N get the warp-tile kernel by
    default, several N in one plan included, window sizes that are not a power
    of two too."""
    b = _random_batch(16, [8], seed=3)
    assert make_plan(b).info["kernel"] == WARP_TILE
    cl = np.full(256, 8, np.uint8)
    for n2, want in ((64, WARP_TILE), (24, WARP_TILE), (100, WARP_TILE)):
        doms = [oracle.Domain(16, 8, 2, 8, 30.0, 0.02, (3.0, 1.0, 0.0), 8, cl),
                oracle.Domain(n2, 8, 2, 8, 30.0, 0.02, (3.0, 1.0, 0.0), 8, cl)]
        lv = [np.full(d.windows(1000) * d.E, 128, np.uint8) for d in doms]
        assert make_plan(crafted_batch(doms, lv, [1000, 1000], [0, 1])).info["kernel"] == want


@pytest.mark.parametrize("align", [32, 1])
def test_shape_mixed_window_sizes(align):
    """Domains of N = 4, 16, 32 (E = 16 and E = 8), 64, 128, 24 and 100 in one batch,
    streams interleaved in the output: each tile takes its domain's transform."""
    cl = np.full(256, 8, np.uint8)
    shapes = [(4, 4, 1, 3), (16, 8, 2, 8), (32, 16, 2, 16), (32, 8, 2, 6), (64, 24, 3, 20), (128, 64, 2, 64),
              (24, 12, 2, 12), (100, 50, 2, 40)]
    doms = [oracle.Domain(N, E, B1, B2, 25.0 + i, 0.03, (2.0 + i, 1.0 + 0.25 * i, 0.0), 8, cl)
            for i, (N, E, B1, B2) in enumerate(shapes)]
    rng = np.random.default_rng(99 + align)
    lens, idx, levels = [], [], []
    for r in range(5):
        for d, dom in enumerate(doms):
            S = int(rng.integers(1, 60000)) if r else dom.N * 300 + d
            lens.append(S)
            idx.append(d)
            levels.append(rng.integers(0, 256, size=dom.windows(S) * dom.E).astype(np.uint8))
    b = crafted_batch(doms, levels, lens, idx)
    plan = make_plan(b, out_align=align, out_base=0 if align == 32 else 1)
    assert plan.info["kernel"] == WARP_TILE
    _, _, out, lv = gpu_decode(plan, b)
    compare_with_oracle(plan, b, out, lv)
    assert plan.device_status()[0] == 0


@pytest.mark.parametrize("N,E", [(64, 32), (16, 8), (128, 64)])
def test_shape_trained_signals(N, E):
    """Tables trained on the synthetic domains at another shape, signals of all four domains."""
    doms = [oracle.trained_domain(i, N=N, E=E, B1=2, B2=E) for i in range(4)]
    wl = siggen.mixed_10000_logu(n=24, lo=100, hi=200000)
    b = encode_workload(wl, domains=doms)
    plan = make_plan(b, out_align=32)
    assert plan.info["kernel"] == WARP_TILE
    _, _, out, lv = gpu_decode(plan, b)
    compare_with_oracle(plan, b, out, lv)


def test_shape_chain_across_rejected_segment():
    """Several tiles per warp, a segment with a wrong symbol count in between:
    it is flagged and skipped, the others decode exactly."""
    from paper_2605_01086_gb300 import _lib
    b = _random_batch(64, [32], seed=11, lens_of=lambda N, T: [T * N * 62 + 5] * 40)
    bad = 17
    b.symlen[int(b.word_off[bad]) + 9] -= 1
    plan = make_plan(b, out_align=32, kernel="warp_tile", threads=256, ctas_per_sm=1)
    assert plan.info["n_tiles"] >= 2 * plan.info["grid"] * 8
    w, s = plan.to_device(b.words, b.symlen)
    out = plan.empty_out().fill_(float("nan"))
    lv = torch.empty(plan.info["n_levels_total"], dtype=torch.uint8, device=plan.device)
    plan.decode(w, s, out=out, levels=lv)
    st, flags, first = plan.device_status()
    assert st == _lib.CORRUPT_STREAM and flags & _lib.FLAG_SYMBOL_COUNT and first == bad
    compare_with_oracle(plan, b, out, lv, idx=[i for i in range(b.n_streams) if i != bad])


TC_TOL = {"tf32": 1e-3, "bf16x3": 2e-5, "tf32x3": 1e-5}  # as for N = 32, E = 16 (tests/test_gpu_tc.py)


@pytest.mark.parametrize("mode", ["tf32", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("N,E", [(32, 32), (64, 32), (128, 32), (128, 64)])
@pytest.mark.parametrize("align", ["window", "odd"])
def test_tensor_core_shapes(N, E, mode, align):
    """The tensor-core transform for shapes with E >= 32 (decode_tcs.cu): two
    domains of the same (N, E) with different scales and zone bounds (one with a
    zone-2 bin), ragged lengths; outputs on window boundaries (3-D TMA stores of
    whole steps) and at odd offsets (lane stores); levels bit-exact, samples
    within the form's bound, nothing written outside the segments."""
    b = _random_batch(N, [E, E], seed=N * 7 + E + len(mode))
    plan = make_plan(b, out_align=N if align == "window" else 1, out_base=0 if align == "window" else 3, idct=mode)
    assert plan.info["kernel"] == 4
    _, _, out, lv = gpu_decode(plan, b, out_fill=float("nan"))
    # TF32 bounds each sample's error by ~2^-10 sum_k |C_k B_kn|, not by the sample: a
    # stream of a few samples whose sums cancel can exceed the stream-level bound
    short = np.flatnonzero(b.lengths < 1024)
    longer = np.flatnonzero(b.lengths >= 1024)
    worst = compare_with_oracle(plan, b, out, lv, idx=longer, tol=TC_TOL[mode])
    compare_with_oracle(plan, b, out, lv, idx=short, tol=TC_TOL[mode] * (50 if mode == "tf32" else 1))
    h = out.cpu().numpy()
    mask = np.ones(h.size, bool)
    for sg in plan.segments:
        mask[int(sg["out_offset"]):int(sg["out_offset"]) + int(sg["n_samples"])] = False
    assert np.all(np.isnan(h[mask]))
    assert plan.device_status()[0] == 0
    print(N, E, mode, align, "worst rel L2", worst)


def test_tensor_core_shape_trained_signals():
    """(64, 32) on trained tables and EEG-like signals, against the FP32 kernel's output too."""
    wl = siggen.Workload("tcs", 11, np.zeros(6, np.int32),
                         np.array([siggen.stream_seed(11, i) for i in range(6)], np.uint64),
                         np.array([64 * 1000 + 3, 65536, 1, 200000, 64 * 64, 12345], np.uint64))
    ts = siggen.training_set(0)
    flat, offs = siggen.signals(ts.domains, ts.seeds, ts.lengths)
    dom = oracle.train_domain(flat, offs, ts.lengths, oracle.Domain(64, 32, 2, 32, 50.0, 0.004, (0.0, 0.0, 0.0), 12),
                              99.9)
    b = encode_workload(wl, domains=[dom])
    plan = make_plan(b, out_align=64, idct="tf32x3")
    assert plan.info["kernel"] == 4
    _, _, out, lv = gpu_decode(plan, b, out_fill=0.0)   # the gaps between segments compare equal
    compare_with_oracle(plan, b, out, lv, tol=TC_TOL["tf32x3"])
    ref = make_plan(b, out_align=64, kernel="warp_tile")
    _, _, out32, _ = gpu_decode(ref, b, out_fill=0.0)
    rel = float(torch.linalg.vector_norm((out - out32).double()) / torch.linalg.vector_norm(out32.double()))
    assert rel < 1e-6
