"""GPU parity of the batch decoder against the FP64 oracle (through the C ABI):
decoded levels bit-exact, samples within 1e-5 relative L2 per stream
(FP32 path).  Covers the EEG stream of 65,536 samples, mixed-domain batches
with ragged lengths, the three decode kernels (warp-tile and block-tile for
N = 32 / E = 16, generic for any shape), both schedules,
tile and CTA sizes, crafted codebooks (L_max-long codes, 64 one-bit codes per
word, incomplete codes, one-symbol windows), other (N, E) shapes, misaligned
outputs, run-time scales and corrupted streams."""
import numpy as np
import pytest

import oracle
import siggen

from gpu_util import (FP32_REL_L2, compare_with_oracle, crafted_batch, encode_workload, gpu_decode, make_plan,
                      oracle_domains, product_domain, segments_of)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_01086_gb300 import build
    build()


def test_eeg_single_stream():
    b = encode_workload(siggen.eeg_1x65536())
    for kernel in KERNELS:
        plan = make_plan(b, kernel=kernel)
        assert plan.info["kernel"] == KERNEL_IDS[kernel]
        _, _, out, lv = gpu_decode(plan, b)
        compare_with_oracle(plan, b, out, lv)
        assert plan.device_status()[0] == 0
    assert make_plan(b).info["kernel"] == KERNEL_IDS["warp_tile"]


KERNELS = ["warp_tile", "block_tile", "generic"]
KERNEL_IDS = {"generic": 1, "block_tile": 2, "warp_tile": 3}


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("schedule", ["persistent", "per_segment"])
def test_mixed_batch_ragged(kernel, schedule):
    wl = siggen.mixed_10000_logu(n=48, lo=1, hi=200000)
    b = encode_workload(wl)
    plan = make_plan(b, kernel=kernel, schedule=schedule)
    assert plan.info["kernel"] == KERNEL_IDS[kernel]
    _, _, out, lv = gpu_decode(plan, b, out_fill=float("nan"))
    compare_with_oracle(plan, b, out, lv)
    assert plan.device_status()[0] == 0


def test_warp_tile_28_warps_and_shared_memory_limit():
    """896 threads (28 warps per CTA) fit the tables of four Table 1 domains and decode them; 1024
    threads do not fit and are refused at plan creation with the sizes named (no launch)."""
    from paper_2605_01086_gb300 import _lib
    wl = siggen.mixed_10000_logu(n=24, lo=100, hi=100000)
    b = encode_workload(wl)
    assert len(b.domains) == 4
    assert make_plan(b).info["threads"] == 896  # the default: the most warps that fit without spills
    plan = make_plan(b, kernel="warp_tile", threads=896)
    assert plan.info["threads"] == 896 and plan.info["kernel"] == KERNEL_IDS["warp_tile"]
    _, _, out, lv = gpu_decode(plan, b, out_fill=float("nan"))
    compare_with_oracle(plan, b, out, lv)
    assert plan.device_status()[0] == 0
    with pytest.raises(_lib.FptcError) as ei:
        make_plan(b, kernel="warp_tile", threads=1024)
    assert ei.value.status == _lib.UNSUPPORTED
    assert "shared memory" in str(ei.value) and "1024 threads" in str(ei.value)


@pytest.mark.parametrize("tile_samples,threads", [(32, 128), (512, 256), (2048, 512), (4096, 256), (16384, 256),
                                                  (8192, 128)])
def test_tile_and_cta_sizes(tile_samples, threads):
    wl = siggen.mixed_10000_logu(n=24, lo=100, hi=100000)
    b = encode_workload(wl)
    for kernel in KERNELS:
        plan = make_plan(b, tile_samples=tile_samples, threads=threads, kernel=kernel)
        _, _, out, lv = gpu_decode(plan, b)
        compare_with_oracle(plan, b, out, lv)


def test_edge_lengths_and_misaligned_outputs():
    lengths = [0, 1, 5, 31, 32, 33, 4095, 4096, 4097, 131073, 0, 7]
    n = len(lengths)
    wl = siggen.Workload("edges", 9, np.array([i % 4 for i in range(n)], np.int32),
                         np.array([siggen.stream_seed(9, i) for i in range(n)], np.uint64),
                         np.array(lengths, np.uint64))
    b = encode_workload(wl)
    for align, base, kernel in ((4, 0, "warp_tile"), (1, 0, "warp_tile"), (1, 3, "warp_tile"), (1, 3, "block_tile"),
                                (1, 3, "generic")):
        plan = make_plan(b, out_align=align, out_base=base, kernel=kernel)
        _, _, out, lv = gpu_decode(plan, b, out_fill=float("nan"))
        compare_with_oracle(plan, b, out, lv)
        # nothing outside the segments' outputs was written
        h = out.cpu().numpy()
        mask = np.ones(h.size, bool)
        for s in plan.segments:
            mask[int(s["out_offset"]):int(s["out_offset"]) + int(s["n_samples"])] = False
        assert np.all(np.isnan(h[mask]))


def test_all_zero_signal():
    d = oracle_domains()
    x = np.zeros(10000, np.float32)
    words, symlen, lv = oracle.encode_stream(x, d[0])
    assert np.all(lv == 128)
    b = oracle.EncodedBatch(words, symlen, np.zeros(1, np.uint64), np.array([words.size], np.uint64),
                            np.array([10000], np.uint64), np.zeros(1, np.int32), d)
    plan = make_plan(b)
    _, _, out, lvg = gpu_decode(plan, b)
    assert torch.all(out[:10000] == 0)
    compare_with_oracle(plan, b, out, lvg)


def test_long_codes_lmax16():
    freq = np.ones(256, np.uint64)
    fib = [1, 1]
    while len(fib) < 40:
        fib.append(fib[-1] + fib[-2])
    freq[:24] = np.array(fib[16:40], np.uint64)
    o = oracle.Domain(32, 16, 2, 16, 50.0, 0.004, (3.0, 2.0, 0.0), 16, oracle.package_merge(freq, 16))
    assert o.code_len.max() == 16
    rng = np.random.default_rng(1)
    lens = [32 * 100, 32 * 77 + 5, 1]
    levels = [rng.integers(0, 256, size=((S + 31) // 32) * 16).astype(np.uint8) for S in lens]
    b = crafted_batch([o], levels, lens, [0, 0, 0])
    assert b.symlen.max() <= 13
    for kernel in KERNELS:
        plan = make_plan(b, kernel=kernel)
        _, _, out, lv = gpu_decode(plan, b)
        compare_with_oracle(plan, b, out, lv)


def test_sixty_four_one_bit_codes_per_word():
    cl = np.full(256, 9, np.uint8)
    cl[128] = 1
    o = oracle.Domain(32, 16, 2, 12, 50.0, 0.004, (3.0, 2.0, 0.0), 9, cl)
    rng = np.random.default_rng(2)
    S = 32 * 3000
    X = np.full((S // 32) * 16, 128, np.uint8)
    hot = rng.integers(0, X.size, size=200)
    X[hot] = rng.integers(0, 256, size=200)
    b = crafted_batch([o], [X, np.full(16 * 40, 128, np.uint8)], [S, 32 * 40], [0, 0])
    assert (b.symlen == 64).sum() > 100
    plan = make_plan(b)
    _, _, out, lv = gpu_decode(plan, b)
    compare_with_oracle(plan, b, out, lv)


@pytest.mark.parametrize("kernel", ["generic", "warp_tile"])
def test_incomplete_code_and_one_symbol_windows(kernel):
    cl = np.zeros(256, np.uint8)
    cl[128], cl[120], cl[140] = 1, 3, 3   # Kraft 3/4: incomplete
    o1 = oracle.Domain(4, 1, 1, 1, 20.0, 0.01, (5.0, 0.0, 0.0), 3, cl)  # E = 1: one symbol per window
    rng = np.random.default_rng(3)
    X = rng.choice(np.array([128, 120, 140], np.uint8), size=1000)
    b = crafted_batch([o1], [X, X[:1], X[:7]], [4000, 3, 27], [0, 0, 0])
    plan = make_plan(b, kernel=kernel)
    assert plan.info["kernel"] == KERNEL_IDS[kernel]
    _, _, out, lv = gpu_decode(plan, b)
    compare_with_oracle(plan, b, out, lv)


@pytest.mark.parametrize("N,E,B1,B2", [(4, 4, 1, 3), (8, 3, 1, 2), (13, 7, 2, 5), (64, 8, 2, 6), (128, 128, 4, 100),
                                       (128, 1, 0, 1), (32, 16, 2, 12), (16, 16, 16, 16)])
def test_other_shapes_random_levels(N, E, B1, B2):
    cl = np.full(256, 8, np.uint8)
    doms = [oracle.Domain(N, E, B1, B2, 37.0, 0.05, (4.0, 1.5, 0.0), 8, cl),
            oracle.Domain(32, 16, 2, 16, 50.0, 0.004, (2.0, 1.0, 0.0), 8, cl)]
    rng = np.random.default_rng(N * 1000 + E)
    lens = [N * 50 + 3, 5000, N - 1, 777]
    dom_idx = [0, 1, 0, 0]
    levels = [rng.integers(0, 256, size=doms[di].windows(S) * doms[di].E).astype(np.uint8)
              for S, di in zip(lens, dom_idx)]
    b = crafted_batch(doms, levels, lens, dom_idx)
    plan = make_plan(b)
    _, _, out, lv = gpu_decode(plan, b)
    compare_with_oracle(plan, b, out, lv)


def test_trained_non_default_shape():
    doms = [oracle.trained_domain(0, N=64, E=24, B1=3, B2=20), oracle.trained_domain(2, N=16, E=4, B1=1, B2=4)]
    wl = siggen.mixed_10000_logu(n=16, lo=10, hi=50000)
    idx = (wl.domains == 0) | (wl.domains == 2)
    sub = wl.subset(np.flatnonzero(idx))
    sub.domains = np.where(sub.domains == 0, 0, 1).astype(np.int32)
    flat, offs = siggen.signals(np.where(sub.domains == 0, 0, 2), sub.seeds, sub.lengths)
    b = oracle.encode_many(flat, offs, sub.lengths, sub.domains, doms)
    plan = make_plan(b)
    _, _, out, lv = gpu_decode(plan, b)
    compare_with_oracle(plan, b, out, lv)


def test_runtime_scale_override():
    wl = siggen.mixed_10000_logu(n=8, lo=1000, hi=50000)
    b = encode_workload(wl)
    plan = make_plan(b)
    factors = np.array([[2.0, 0.5, 1.0], [1.0, 3.0, 1.0], [0.25, 1.0, 1.0], [1.5, 1.5, 1.0]])
    base = np.array([d.A for d in b.domains])
    sc = torch.tensor((base * factors).astype(np.float32).ravel(), device=plan.device)
    _, _, out, lv = gpu_decode(plan, b, scale=sc)
    doms2 = [oracle.Domain(d.N, d.E, d.B1, d.B2, d.mu, d.alpha1, tuple(base[i] * factors[i]), d.lmax, d.code_len)
             for i, d in enumerate(b.domains)]
    compare_with_oracle(plan, b, out, lv, domains=doms2)


# ---- malformed payloads: sticky device status, no trap, writes confined

def _eight_bit_batch():
    cl = np.full(256, 8, np.uint8)   # every word holds exactly 8 codewords (64 bits)
    o = oracle.Domain(32, 16, 2, 16, 50.0, 0.004, (3.0, 2.0, 0.0), 8, cl)
    rng = np.random.default_rng(4)
    lens = [32 * 64, 32 * 64, 32 * 64]
    levels = [rng.integers(0, 256, size=64 * 16).astype(np.uint8) for _ in lens]
    return crafted_batch([o], levels, lens, [0, 0, 0])


def _run_corrupt(b, kernel="auto"):
    plan = make_plan(b, kernel=kernel)
    w, s = plan.to_device(b.words, b.symlen)
    out = plan.empty_out().fill_(float("nan"))
    plan.decode(w, s, out=out)
    return plan, out, plan.device_status()


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("case", ["symlen_range", "count", "overrun"])
def test_corrupt_segment_is_flagged_and_confined(case, kernel):
    from paper_2605_01086_gb300 import _lib
    b = _eight_bit_batch()
    bad_word = int(b.word_off[1]) + 10
    if case == "symlen_range":
        b.symlen[bad_word] = 65
        want = _lib.FLAG_SYMLEN_RANGE
    elif case == "count":
        b.symlen[bad_word] -= 1
        want = _lib.FLAG_SYMBOL_COUNT
    else:
        b.symlen[bad_word] += 1
        b.symlen[bad_word + 1] -= 1
        want = _lib.FLAG_BIT_OVERRUN
    plan, out, (st, flags, first) = _run_corrupt(b, kernel)
    assert st == _lib.CORRUPT_STREAM and flags & want and first == 1
    # the good segments decode exactly
    compare_with_oracle(plan, b, out, None, idx=[0, 2])
    h = out.cpu().numpy()
    s1 = plan.segments[1]
    lo, hi = int(s1["out_offset"]), int(s1["out_offset"]) + int(s1["n_samples"])
    if case != "overrun":   # a segment rejected by the index is not written at all
        assert np.all(np.isnan(h[lo:hi]))
    # status is cleared by reading it
    assert plan.device_status()[0] == 0


@pytest.mark.parametrize("form", ["warp_tile", "tensor"])
def test_tile_chain_across_rejected_segment(form):
    """Every warp decodes a run of consecutive tiles, each starting where the one
    before it ended; a segment the index rejects inside such a run is skipped and
    the tiles after it still start at the right words."""
    from paper_2605_01086_gb300 import _lib
    b = encode_workload(siggen.mixed_10000_logu(n=48, lo=100000, hi=200000))
    bad = 20
    b.symlen[int(b.word_off[bad]) + 7] -= 1
    opts = dict(kernel="warp_tile") if form == "warp_tile" else dict(idct="bf16x3")
    plan = make_plan(b, threads=128, ctas_per_sm=1, **opts)
    warps = plan.info["grid"] * 4
    assert plan.info["n_tiles"] >= 2 * warps
    w, s = plan.to_device(b.words, b.symlen)
    out = plan.empty_out().fill_(float("nan"))
    lv = torch.empty(plan.info["n_levels_total"], dtype=torch.uint8, device=plan.device)
    plan.decode(w, s, out=out, levels=lv)
    st, flags, first = plan.device_status()
    assert st == _lib.CORRUPT_STREAM and flags & _lib.FLAG_SYMBOL_COUNT and first == bad
    good = [i for i in range(b.n_streams) if i != bad]
    compare_with_oracle(plan, b, out, lv, idx=good, tol=FP32_REL_L2 if form == "warp_tile" else 2e-5)


def test_adjoint_redecode_chains_tiles():
    """The adjoint decoding the levels again, several tiles per warp: the same
    coefficient gradients as from the saved levels."""
    b = encode_workload(siggen.power_1024x65536(n=320, S=65536))
    plan = make_plan(b)
    w, s, out, lv = gpu_decode(plan, b)
    gx = torch.randn(out.numel(), generator=torch.Generator().manual_seed(5)).to(plan.device) * 1e-3
    gco = torch.empty(plan.info["n_levels_total"], dtype=torch.float32, device=plan.device)
    gco2 = torch.empty_like(gco)
    gsc, _ = plan.backward(gx, levels=lv, grad_coeffs=gco)
    gsc2, _ = plan.backward(gx, words=w, symlen=s, grad_coeffs=gco2)
    torch.cuda.synchronize()
    assert plan.info["n_tiles"] >= 2 * plan.info["sm_count"] * 16
    assert torch.equal(gco, gco2)
    assert torch.allclose(gsc, gsc2, rtol=1e-12, atol=0)
    assert plan.device_status()[0] == 0


def test_invalid_code_is_flagged():
    from paper_2605_01086_gb300 import _lib
    cl = np.zeros(256, np.uint8)
    cl[128], cl[0] = 1, 2   # prefixes 11.. are no codeword
    o = oracle.Domain(4, 1, 1, 1, 20.0, 0.01, (5.0, 0.0, 0.0), 2, cl)
    b = crafted_batch([o], [np.full(8, 128, np.uint8)], [32], [0])
    b.words[0] = np.uint64(0xC000000000000000)  # '11' first
    plan, out, (st, flags, first) = _run_corrupt(b)
    assert st == _lib.CORRUPT_STREAM and flags & _lib.FLAG_INVALID_CODE and first == 0


def test_misaligned_pointer_rejected():
    from paper_2605_01086_gb300 import _lib
    b = encode_workload(siggen.eeg_1x65536())
    plan = make_plan(b)
    w, s = plan.to_device(b.words, b.symlen)
    out = torch.empty(plan.info["out_extent"] + 8, dtype=torch.float32, device=plan.device)
    with pytest.raises(_lib.FptcError):
        plan.decode(w, s, out=out[1:])


def test_graph_capture_replay():
    wl = siggen.mixed_10000_logu(n=16, lo=100, hi=100000)
    b = encode_workload(wl)
    plan = make_plan(b)
    w, s = plan.to_device(b.words, b.symlen)
    out = plan.empty_out()
    lv = torch.empty(plan.info["n_levels_total"], dtype=torch.uint8, device=plan.device)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        plan.decode(w, s, out=out, levels=lv)  # warm-up outside capture
    torch.cuda.synchronize()
    out.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        plan.decode(w, s, out=out, levels=lv)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    compare_with_oracle(plan, b, out, lv)


def _words_reversed(b):
    """The same batch with the streams' words stored in reverse stream order."""
    order = np.arange(b.n_streams)[::-1]
    words, symlen, off = [], [], np.zeros(b.n_streams, np.uint64)
    pos = 0
    for i in order:
        a, n = int(b.word_off[i]), int(b.n_words[i])
        words.append(b.words[a:a + n])
        symlen.append(b.symlen[a:a + n])
        off[i] = pos
        pos += n
    return oracle.EncodedBatch(np.concatenate(words), np.concatenate(symlen), off, b.n_words.copy(),
                               b.lengths.copy(), b.domain_idx.copy(), b.domains)


@pytest.mark.parametrize("idct,layout", [("fp32", "ordered"), ("bf16x3", "ordered"), ("fp32", "words_reversed")])
def test_decode_host_buffers(idct, layout):
    """fptc_decode_host: compressed streams from pinned host memory, samples back
    to host memory (a piece's words go up and its samples come back while other
    pieces decode; with the words out of output order everything goes up first);
    equal to the device-buffer decode and within the oracle bound."""
    wl = siggen.mixed_10000_logu(n=60, lo=1, hi=300000)
    b = encode_workload(wl)
    if layout == "words_reversed":
        b = _words_reversed(b)
    plan = make_plan(b, idct=idct, out_align=32)
    w, s, out, lv = gpu_decode(plan, b)
    h_w = torch.from_numpy(b.words.view(np.int64)).pin_memory()
    h_s = torch.from_numpy(b.symlen).pin_memory()
    h_o = torch.full((plan.info["out_extent"],), float("nan"), dtype=torch.float32).pin_memory()
    d_w, d_s = torch.zeros_like(w), torch.zeros_like(s)
    d_o = torch.zeros_like(out)
    plan.decode_host(h_w, h_s, h_o, d_w, d_s, d_o)
    assert plan.device_status()[0] == 0
    ref = out.cpu()
    for seg in plan.segments:
        o, n = int(seg["out_offset"]), int(seg["n_samples"])
        assert torch.equal(h_o[o:o + n], ref[o:o + n])
    compare_with_oracle(plan, b, h_o, None, tol=FP32_REL_L2 if idct == "fp32" else 2e-5)


@pytest.mark.parametrize("levels", [True, False])
def test_three_kernel_schedule(levels):
    """The paper's three-kernel GPU design (per-word offsets, one thread per word,
    one thread per sample) kept for comparison: same levels and samples as the oracle,
    ragged lengths, misaligned outputs, an incomplete code."""
    lengths = [0, 1, 5, 31, 32, 33, 1023, 1024, 1025, 4097, 131073, 7, 250000]
    n = len(lengths)
    wl = siggen.Workload("edges3k", 11, np.array([i % 4 for i in range(n)], np.int32),
                         np.array([siggen.stream_seed(11, i) for i in range(n)], np.uint64),
                         np.array(lengths, np.uint64))
    b = encode_workload(wl)
    for align, base in ((32, 0), (1, 3)):
        plan = make_plan(b, schedule="three_kernel", out_align=align, out_base=base)
        assert plan.info["schedule"] == 2
        _, _, out, lv = gpu_decode(plan, b, want_levels=levels, out_fill=float("nan"))
        compare_with_oracle(plan, b, out, lv)
        assert plan.device_status()[0] == 0
        h = out.cpu().numpy()
        mask = np.ones(h.size, bool)
        for s in plan.segments:
            mask[int(s["out_offset"]):int(s["out_offset"]) + int(s["n_samples"])] = False
        assert np.all(np.isnan(h[mask]))


def test_three_kernel_matches_fused():
    wl = siggen.mixed_10000_logu(n=40, lo=4096, hi=400000)
    b = encode_workload(wl)
    fused = make_plan(b)
    paper = make_plan(b, schedule="three_kernel")
    _, _, out_f, _ = gpu_decode(fused, b, want_levels=False, out_fill=0.0)
    _, _, out_p, _ = gpu_decode(paper, b, want_levels=False, out_fill=0.0)
    rel = float(torch.linalg.vector_norm((out_f - out_p).double()) / torch.linalg.vector_norm(out_f.double()))
    assert rel < 1e-6, rel  # both within FP32 rounding of the same sums


def test_three_kernel_stages_apart():
    """The paper's lossless and lossy kernels run on their own (the stage split that
    the runtime breakdown of Sec. 6 times): index, then lossless, then lossy gives
    the samples of one whole decode; the fused schedules refuse these stages."""
    from paper_2605_01086_gb300 import STAGE_DECODE, STAGE_INDEX, STAGE_LOSSLESS, STAGE_LOSSY, FptcError
    wl = siggen.mixed_10000_logu(n=24, lo=4096, hi=200000)
    b = encode_workload(wl)
    paper = make_plan(b, schedule="three_kernel")
    w, s = paper.to_device(b.words, b.symlen)
    whole = paper.empty_out().fill_(float("nan"))
    paper.decode_stages(w, s, whole, STAGE_INDEX | STAGE_DECODE)
    apart = paper.empty_out().fill_(float("nan"))
    paper.decode_stages(w, s, apart, STAGE_INDEX)
    paper.decode_stages(w, s, apart, STAGE_LOSSLESS)
    paper.decode_stages(w, s, apart, STAGE_LOSSY)
    torch.cuda.synchronize()
    assert torch.equal(torch.nan_to_num(whole, 7.0), torch.nan_to_num(apart, 7.0))  # NaN: outside every segment
    compare_with_oracle(paper, b, apart, None)
    fused = make_plan(b)
    with pytest.raises(FptcError):
        fused.decode_stages(w, s, fused.empty_out(), STAGE_LOSSLESS)
