"""GPU encoder (Eq. 1, the zone quantizer of Sec. 3.2, Alg. 1) against the
oracle: packing given levels is bit-exact (ragged and empty streams, one-bit
and maximum-length codes); levels from signals equal the library's FP64 host
encoder's in every bin, and the oracle's except where the oracle's coefficient
lies within FP64 rounding of a level boundary; words and symbol counts are
exact wherever the levels are; the GPU decoder reads what the
GPU encoder wrote; rooms that are too small and levels without a codeword are
flagged on the device."""
import numpy as np
import pytest

import oracle
import siggen

from gpu_util import compare_with_oracle, make_plan, near_level_boundary, oracle_domains, product_domain

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_01086_gb300 import build
    build()


def _oracle_stream(x, d):
    return oracle.encode_stream(x, d)  # words, symlen, levels


def _room_words(enc, words, symlen, n_words, i):
    a, n = int(enc.room_offsets[i]), int(n_words[i])
    return words[a:a + n], symlen[a:a + n]


@pytest.mark.parametrize("case", ["trained", "one_bit", "max_length", "runs"])
def test_pack_matches_oracle(case):
    from paper_2605_01086_gb300 import Encoder
    rng = np.random.default_rng(5)
    if case == "trained":
        doms = oracle_domains()
        lens = [0, 1, 31, 32, 33, 4097, 70000, 1000, 12345, 2]
        idx = [i % 4 for i in range(len(lens))]
        levels = []
        for S, di in zip(lens, idx):
            x = siggen.signal(di, int(siggen.stream_seed(7, len(levels))), S)
            levels.append(_oracle_stream(x, doms[di])[2] if S else np.zeros(0, np.uint8))
    elif case == "runs":
        # runs of one level (3- or 5-bit codes: a packing block of 4096 such
        # codewords does not end on a word boundary, so a block entered in
        # another state than its reference never meets it) between runs of
        # mixed lengths (where they do meet): blocks packed again from the
        # true state, then entered as assumed once more
        cl = np.full(256, 12, np.uint8)
        cl[128], cl[127], cl[129], cl[126], cl[130], cl[:8] = 1, 3, 3, 5, 5, 11
        d = oracle.Domain(32, 16, 2, 16, 50.0, 0.004, (1.0, 1.0, 0.0), 12, cl)
        doms = [d]
        lens = [32 * 4096 * 5 + 96, 32 * 777, 32 * 4096 * 2]
        idx = [0] * len(lens)
        levels = []
        for si, S in enumerate(lens):
            W = d.windows(S) * d.E
            L = np.empty(W, np.uint8)
            i = 0
            while i < W:
                k = min(int(rng.integers(1, 3 * 4096)), W - i)
                if si == 2 or rng.random() < 0.5:
                    L[i:i + k] = 126 if si == 2 else rng.choice([127, 126, 129])
                else:
                    L[i:i + k] = rng.choice([126, 127, 128, 129, 130, 5, 200], size=k,
                                            p=[.1, .2, .4, .15, .1, .03, .02])
                i += k
            levels.append(L)
    else:
        cl = np.zeros(256, np.uint8)
        if case == "one_bit":   # levels 0 and 128 with one-bit codes: 64 codewords per word
            cl[128], cl[0] = 1, 1
            lmax, pool = 8, np.array([128, 0])
        else:                   # levels 128..255 with 16-bit codes (lmax): 4 codewords per word
            cl[:128], cl[128:] = 8, 16
            lmax, pool = 16, np.arange(128, 256)
        d = oracle.Domain(32, 16, 2, 16, 50.0, 0.004, (1.0, 1.0, 0.0), lmax, cl)
        doms = [d]
        # 32 * 257 samples: a last packing block of 16 symbols, which (one-bit codes)
        # may fit the word left open by the block before it
        lens = [0, 5, 3200, 32 * 999 + 7, 32 * 257, 32 * 256 + 1, 32 * 4096 * 3]
        idx = [0] * len(lens)
        levels = []
        for S in lens:
            W = d.windows(S) * d.E
            levels.append(rng.choice(pool, size=W).astype(np.uint8) if W else np.zeros(0, np.uint8))
    enc = Encoder([product_domain(d) for d in doms], lens, idx)
    lv = np.zeros(max(1, enc.n_levels), np.uint8)
    for i, L in enumerate(levels):
        lv[int(enc.level_offsets[i]):int(enc.level_offsets[i]) + L.size] = L
    words, symlen, n_words = enc.pack(torch.from_numpy(lv).to(enc.device))
    assert enc.status()[0] == 0
    wh, sh, nh = words.cpu().numpy().view(np.uint64), symlen.cpu().numpy(), n_words.cpu().numpy()
    for i, L in enumerate(levels):
        codes = oracle.canonical_codes(doms[idx[i]].code_len, doms[idx[i]].lmax)
        w_o, s_o = oracle.pack_symlen(L, codes, doms[idx[i]].code_len) if L.size else (np.zeros(0, np.uint64),
                                                                                       np.zeros(0, np.uint8))
        w_g, s_g = _room_words(enc, wh, sh, nh, i)
        np.testing.assert_array_equal(w_g, w_o, err_msg=f"words of stream {i}")
        np.testing.assert_array_equal(s_g, s_o, err_msg=f"symlen of stream {i}")


def test_encode_matches_oracle_and_round_trips():
    """Levels of every bin equal the library's FP64 host encoder's bit for bit (the
    reading the kernel implements: cosine argument pi (2n + 1) k / 2N), and so do
    the packed words; where the oracle (cosine argument pi/N (n + 1/2) k) gives
    another level, its FP64 coefficient lies within the FP64 rounding bound of a
    level boundary (Eq. 1-3)."""
    from paper_2605_01086_gb300 import Encoder, Plan, codec
    doms = oracle_domains()
    pd = [product_domain(d) for d in doms]
    wl = siggen.mixed_10000_logu(n=40, lo=1, hi=150000)
    flat, offs = siggen.signals(wl.domains, wl.seeds, wl.lengths)
    enc = Encoder(pd, wl.lengths, wl.domains)
    x = torch.from_numpy(flat).to(enc.device)
    lv = torch.empty(max(1, enc.n_levels), dtype=torch.uint8, device=enc.device)
    words, symlen, n_words = enc.encode(x, levels=lv)
    assert enc.status()[0] == 0
    wh, sh, nh, lh = (words.cpu().numpy().view(np.uint64), symlen.cpu().numpy(), n_words.cpu().numpy(),
                      lv.cpu().numpy())
    total = mism_total = 0
    for i in range(wl.n_streams):
        d = doms[wl.domains[i]]
        S = int(wl.lengths[i])
        xs = flat[int(offs[i]):int(offs[i]) + S]
        w_h, s_h, l_h = codec.encode_stream(pd[wl.domains[i]], xs)
        l_g = lh[int(enc.level_offsets[i]):int(enc.level_offsets[i]) + l_h.size]
        np.testing.assert_array_equal(l_g, l_h, err_msg=f"levels of stream {i} vs the FP64 host encoder")
        w_g, s_g = _room_words(enc, wh, sh, nh, i)
        np.testing.assert_array_equal(w_g, w_h, err_msg=f"words of stream {i}")
        np.testing.assert_array_equal(s_g, s_h, err_msg=f"symlen of stream {i}")
        w_o, s_o, l_o = _oracle_stream(xs, d)
        mism = np.flatnonzero(l_g != l_o)
        total += l_o.size
        mism_total += mism.size
        for m in mism:
            w, k = divmod(int(m), d.E)
            xw = np.zeros(d.N, np.float64)
            seg = xs[w * d.N:min(S, (w + 1) * d.N)].astype(np.float64)
            xw[:seg.size] = seg
            assert near_level_boundary(d, xw, k, int(l_g[m])), f"stream {i} bin {m}: {l_g[m]} vs {l_o[m]}"
        if mism.size == 0:
            np.testing.assert_array_equal(w_g, w_o)
            np.testing.assert_array_equal(s_g, s_o)
    assert mism_total <= max(2, total // 100000)
    # the decoder reads the GPU-encoded streams: levels and samples against the oracle's
    # decode of those same words
    segs = enc.segments(n_words, codec.packed_out_offsets(wl.lengths, 32))
    plan = Plan([product_domain(d) for d in doms], segs)
    out = plan.empty_out()
    lv2 = torch.empty(plan.info["n_levels_total"], dtype=torch.uint8, device=plan.device)
    plan.decode(words, symlen, out=out, levels=lv2)
    assert plan.device_status()[0] == 0
    b = oracle.EncodedBatch(wh, sh, np.ascontiguousarray(enc.room_offsets), nh[:wl.n_streams].astype(np.uint64),
                            np.asarray(wl.lengths, np.uint64), np.asarray(wl.domains, np.int32), doms)
    compare_with_oracle(plan, b, out, lv2)


def test_room_and_code_flags():
    from paper_2605_01086_gb300 import Encoder, _lib
    doms = oracle_domains()
    wl = siggen.mixed_10000_logu(n=6, lo=5000, hi=9000)
    flat, _ = siggen.signals(wl.domains, wl.seeds, wl.lengths)
    from paper_2605_01086_gb300.codec import word_capacity
    pd = [product_domain(d) for d in doms]
    room = [word_capacity(pd[wl.domains[i]], int(wl.lengths[i])) for i in range(6)]
    room[3] = 2
    enc = Encoder(pd, wl.lengths, wl.domains, room=room)
    enc.encode(torch.from_numpy(flat).to(enc.device))
    st, flags, first = enc.status()
    assert st == _lib.CORRUPT_STREAM and flags & _lib.ENC_FLAG_ROOM and first == 3
    assert enc.status()[0] == 0   # cleared
    # a level whose domain has no codeword for it
    cl = np.zeros(256, np.uint8)
    cl[128], cl[10] = 1, 1
    d = oracle.Domain(32, 16, 2, 16, 50.0, 0.004, (1.0, 1.0, 0.0), 8, cl)
    enc2 = Encoder([product_domain(d)], [320], [0])
    lv = np.full(enc2.n_levels, 128, np.uint8)
    lv[37] = 11
    enc2.pack(torch.from_numpy(lv).to(enc2.device))
    st, flags, first = enc2.status()
    assert st == _lib.CORRUPT_STREAM and flags & _lib.ENC_FLAG_NO_CODE and first == 0


@pytest.mark.parametrize("alpha1", [1.0, 1.0 - 2.0 ** -20, 0.999, 0.3])
def test_encode_zone1_narrow_linear_part(alpha1):
    """Zone 1 with a linear part from empty (alpha1 = 1: every bin level 128) to
    far narrower than the FP32 roundings of A1 and d1 can resolve, and A1 small
    enough that many bins lie beyond it (the map's top): levels equal the FP64
    host encoder's in every bin."""
    from paper_2605_01086_gb300 import Encoder, codec
    base = oracle_domains()[0]
    A = (base.A[0], base.A[1] * 0.05, 0.0)
    d = oracle.Domain(base.N, base.E, base.B1, base.B2, base.mu, alpha1, A, base.lmax, base.code_len.copy())
    pd = product_domain(d)
    wl = siggen.mixed_10000_logu(n=8, lo=1000, hi=40000)
    flat, offs = siggen.signals(np.zeros(8, np.int64), wl.seeds, wl.lengths)
    enc = Encoder([pd], wl.lengths, np.zeros(8, np.int64))
    lv = torch.empty(max(1, enc.n_levels), dtype=torch.uint8, device=enc.device)
    enc.encode(torch.from_numpy(flat).to(enc.device), levels=lv)
    assert enc.status()[0] == 0
    lh = lv.cpu().numpy()
    beyond = 0
    for i in range(8):
        S = int(wl.lengths[i])
        _, _, l_h = codec.encode_stream(pd, flat[int(offs[i]):int(offs[i]) + S])
        l_g = lh[int(enc.level_offsets[i]):int(enc.level_offsets[i]) + l_h.size]
        np.testing.assert_array_equal(l_g, l_h, err_msg=f"levels of stream {i}")
        beyond += int(np.sum((l_h == 255) | (l_h == 0)))
    if alpha1 < 1.0:
        assert beyond > 0   # the map's top is reached
    else:
        z1 = lh[:enc.n_levels].reshape(-1, d.E)[:, d.B1:d.B2]
        assert np.all(z1 == 128)
