"""Pins of the oracle's whole encode/decode path and of its gradient: symbol
round trip, partial windows, exhaustive 16-sample reconstruction against an
independent high-precision evaluation, and central finite differences of the
(exactly quadratic) MSE loss."""
import numpy as np
import pytest

import oracle
import siggen


@pytest.fixture(scope="module")
def eeg_domain():
    return oracle.trained_domain(siggen.EEG)


@pytest.mark.parametrize("S", [0, 1, 5, 31, 32, 33, 1000, 65536])
@pytest.mark.parametrize("domain_id", [0, 1, 2, 3])
def test_round_trip_levels(S, domain_id):
    d = oracle.trained_domain(domain_id)
    x = siggen.signal(domain_id, siggen.stream_seed(2, 12345 + S), S)
    words, symlen, lv = oracle.encode_stream(x, d)
    assert lv.size == d.windows(S) * d.E
    assert int(symlen.sum()) == lv.size
    xh, lv2 = oracle.decode_stream(words, symlen, S, d)
    assert np.array_equal(lv, lv2)
    assert xh.shape == (S,)
    # decoding equals dequantize + inverse transform of the encoder's own levels
    np.testing.assert_array_equal(xh, oracle.reconstruct(lv, S, d))


def test_partial_window_matches_padded(eeg_domain):
    d = eeg_domain
    x = siggen.signal(0, 99, 100)  # 100 = 3 full windows + 4 samples
    pad = np.zeros(128, np.float32)
    pad[:100] = x
    _, _, lv = oracle.encode_stream(x, d)
    _, _, lvp = oracle.encode_stream(pad, d)
    assert np.array_equal(lv, lvp)
    np.testing.assert_array_equal(oracle.reconstruct(lv, 100, d), oracle.reconstruct(lvp, 128, d)[:100])


def test_exhaustive_sixteen_samples():
    # N = 16, S = 16, E = 2: all 65,536 level pairs, against an independent
    # evaluation in mpmath (40 digits) of the DCT-III sum of scipy's definition.
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    d = oracle.Domain(16, 2, 1, 2, 50.0, 0.004, (3.0, 2.0, 0.0), 12)
    cosv = [mpmath.cos(mpmath.pi * (2 * n + 1) / 32) for n in range(16)]
    deq0 = [mpmath.mpf(oracle.dequantize(d, 0, L)) for L in range(256)]
    deq1 = [mpmath.mpf(oracle.dequantize(d, 1, L)) for L in range(256)]
    worst = 0.0
    for L0 in range(256):
        lv = np.empty(2 * 256, np.uint8)
        lv[0::2] = L0
        lv[1::2] = np.arange(256)
        # 256 windows of 16 samples, one per L1 value
        x = oracle.reconstruct(lv, 16 * 256, oracle.Domain(16, 2, 1, 2, 50.0, 0.004, (3.0, 2.0, 0.0), 12))
        x = x.reshape(256, 16)
        for L1 in range(0, 256, 17):
            ref = [deq0[L0] / 2 + deq1[L1] * cosv[n] for n in range(16)]
            err = max(abs(float(ref[n]) - x[L1, n]) for n in range(16))
            worst = max(worst, err)
        # all L1 at once against float64 of the same independent sum
        c1 = np.array([float(v) for v in deq1])
        refm = float(deq0[L0]) / 2 + c1[:, None] * np.array([float(c) for c in cosv])[None, :]
        worst = max(worst, float(np.max(np.abs(refm - x))))
    assert worst < 1e-13


@pytest.mark.parametrize("N", [4, 8, 16])
def test_sixteen_samples_multi_window(N):
    # S = 16 split into 16/N windows: each window reconstructs on its own
    import scipy.fft
    E = 2
    d = oracle.Domain(N, E, 1, 2, 50.0, 0.004, (3.0, 2.0, 0.0), 12)
    rng = np.random.default_rng(N)
    for _ in range(200):
        lv = rng.integers(0, 256, size=(16 // N) * E).astype(np.uint8)
        x = oracle.reconstruct(lv, 16, d)
        for w in range(16 // N):
            c = np.zeros(N)
            c[0] = oracle.dequantize(d, 0, int(lv[w * E]))
            c[1] = oracle.dequantize(d, 1, int(lv[w * E + 1]))
            np.testing.assert_allclose(x[w * N:(w + 1) * N], scipy.fft.dct(c, type=3) / 2, atol=1e-13)


def test_prd_sanity_eeg(eeg_domain):
    # Not a pin: with Table 1 parameters the EEG-like workload reconstructs in
    # the low single-digit PRD band the paper calls high fidelity (Sec. 6.1.3).
    wl = siggen.eeg_1x65536()
    x = siggen.signal(0, int(wl.seeds[0]), 65536)
    words, symlen, _ = oracle.encode_stream(x, eeg_domain)
    xh, _ = oracle.decode_stream(words, symlen, x.size, eeg_domain)
    assert oracle.prd(x, xh) < 10.0
    assert oracle.compression_ratio(x.size, words.size) > 4.0


def _loss(x, d, lv):
    xh = oracle.reconstruct(lv, x.size, d)
    return np.mean((xh - x) ** 2), xh


@pytest.mark.parametrize("domain_id", [2, 0])
def test_gradient_scale_finite_difference(domain_id):
    d = oracle.trained_domain(domain_id)
    S = 4000
    x = siggen.signal(domain_id, 777, S).astype(np.float64)
    _, _, lv = oracle.encode_stream(x.astype(np.float32), d)
    L0, xh = _loss(x, d, lv)
    gx = 2.0 * (xh - x) / S
    gC, gA = oracle.backward_stream(lv, S, d, gx)
    for z in (0, 1):
        h = 1e-6 * d.A[z]
        Ap, Am = list(d.A), list(d.A)
        Ap[z] += h
        Am[z] -= h
        dp = oracle.Domain(d.N, d.E, d.B1, d.B2, d.mu, d.alpha1, tuple(Ap), d.lmax, d.code_len)
        dm = oracle.Domain(d.N, d.E, d.B1, d.B2, d.mu, d.alpha1, tuple(Am), d.lmax, d.code_len)
        fd = (_loss(x, dp, lv)[0] - _loss(x, dm, lv)[0]) / (2 * h)
        assert gA[z] == pytest.approx(fd, rel=1e-6, abs=1e-12 * abs(L0) / d.A[z])
    assert gA[2] == 0.0


def test_gradient_coefficient_finite_difference():
    d = oracle.trained_domain(2)
    S = 1000
    x = siggen.signal(2, 4242, S).astype(np.float64)
    _, _, lv = oracle.encode_stream(x.astype(np.float32), d)
    _, xh = _loss(x, d, lv)
    gx = 2.0 * (xh - x) / S
    gC, _ = oracle.backward_stream(lv, S, d, gx)
    rng = np.random.default_rng(0)
    W = d.windows(S)
    import scipy.fft
    for _ in range(40):
        w = int(rng.integers(0, W))
        k = int(rng.integers(0, d.E))
        # the loss is exactly quadratic in C, so any step is exact up to rounding;
        # 1e-3 keeps the cancellation error of the difference below 1e-9 relative
        h = 1e-3
        n0, n1 = w * d.N, min(S, (w + 1) * d.N)
        e = np.zeros(d.N)
        e[k] = 1.0
        dx = (scipy.fft.dct(e, type=3) / 2)[: n1 - n0]  # d x_window / d C[k]
        seg = xh[n0:n1] - x[n0:n1]
        fd = (np.sum((seg + h * dx) ** 2) - np.sum((seg - h * dx) ** 2)) / (2 * h) / S
        assert gC[w * d.E + k] == pytest.approx(fd, rel=1e-8, abs=1e-15)


def test_batch_encode_decode_matches_single():
    wl = siggen.mixed_10000_logu(n=8, lo=100, hi=5000)
    flat, offs = siggen.signals(wl.domains, wl.seeds, wl.lengths)
    doms = [oracle.trained_domain(i) for i in range(4)]
    b = oracle.encode_many(flat, offs, wl.lengths, wl.domains, doms)
    xs, out_off, lv, lv_off = oracle.decode_many(b, want_levels=True)
    for i in range(8):
        S = int(wl.lengths[i])
        x = flat[int(offs[i]):int(offs[i]) + S]
        w1, s1, l1 = oracle.encode_stream(x, doms[wl.domains[i]])
        a, n = int(b.word_off[i]), int(b.n_words[i])
        assert np.array_equal(b.words[a:a + n], w1) and np.array_equal(b.symlen[a:a + n], s1)
        np.testing.assert_array_equal(xs[int(out_off[i]):int(out_off[i]) + S],
                                      oracle.decode_stream(w1, s1, S, doms[wl.domains[i]])[0])
        assert np.array_equal(lv[int(lv_off[i]):int(lv_off[i]) + l1.size], l1)
