"""Pins of the oracle's trainer (Sec. 3.2.1 per-zone clipped percentile of |c|,
Sec. 3.3 symbol histogram and length-limited codes) and of the zone-2 branch of
the quantizer (Sec. 3.2.3: bins k >= B2 carry level 128 and reconstruct to 0),
on inputs whose answers follow by hand.

The training windows are built from chosen coefficients through the closed-form
inverse of Eq. 1 (a cosine at bin k of amplitude a has Eq. 1 coefficient a at
k, a constant v has C[0] = 2 v), so the pools of |c| per zone, their
nearest-rank percentile and the level histogram are known before the trainer
runs.  The domain has B2 < E, so zone 2 is not empty, and the signals carry
energy above E, so truncation is exercised too."""
import math

import numpy as np
import pytest

import oracle

N, E, B1, B2 = 8, 6, 2, 4
PCT = 90.0


def synth_window(C):
    """Samples of one window with Eq. 1 coefficients C[0..N) (inverse of Eq. 1 written out)."""
    n = np.arange(N)
    x = np.full(N, C[0] / 2.0)
    for k in range(1, N):
        x += C[k] * np.cos(math.pi / N * (n + 0.5) * k)
    return x


def hand_windows():
    """Ten windows: bins 0, 1 (zone 0) and 2, 3 (zone 1) take distinct magnitudes
    with mixed signs, bins 4, 5 (zone 2) +-30, bins 6, 7 (dropped, k >= E) +-20."""
    rng = np.random.default_rng(7)
    z0 = 0.25 * np.arange(1, 21)          # 20 magnitudes for bins 0, 1
    z1 = 0.1 * np.arange(1, 21) + 0.03    # 20 magnitudes for bins 2, 3
    s0 = np.where(rng.random(20) < 0.5, -1.0, 1.0)
    s1 = np.where(rng.random(20) < 0.5, -1.0, 1.0)
    s0[-3:] = -1.0  # the largest zone-0 magnitudes negative: a signed percentile would differ
    z0 = (z0 * s0)[rng.permutation(20)]
    z1 = (z1 * s1)[rng.permutation(20)]
    C = np.zeros((10, N))
    C[:, 0:2] = z0.reshape(10, 2)
    C[:, 2:4] = z1.reshape(10, 2)
    C[:, 4:6] = 30.0 * np.where(rng.random((10, 2)) < 0.5, -1.0, 1.0)
    C[:, 6:8] = 20.0 * np.where(rng.random((10, 2)) < 0.5, -1.0, 1.0)
    return C


def nearest_rank(values, p):
    """Nearest rank ceil(p n / 100) (1-based) of the sorted values; p a whole percent."""
    v = np.sort(np.asarray(values, dtype=np.float64).ravel())
    return float(v[-(-int(p) * v.size // 100) - 1])


def train(C, lmax=12):
    """Two signals of five windows each, at offsets 0 and 50 of one flat array whose
    gap holds values that would show if the trainer read outside a signal."""
    x = np.array([synth_window(c) for c in C])  # 10 x N
    flat = np.full(100, 1.0e4, np.float32)
    flat[0:40] = x[:5].reshape(-1)
    flat[50:90] = x[5:].reshape(-1)
    tmpl = oracle.Domain(N, E, B1, B2, 50.0, 0.004, (0.0, 0.0, 0.0), lmax)
    return oracle.train_domain(flat, np.array([0, 50], np.uint64), np.array([40, 40], np.uint64), tmpl, PCT)


def test_train_scales_are_zone_percentiles_of_abs_coefficients():
    C = hand_windows()
    d = train(C)
    want0 = nearest_rank(np.abs(C[:, 0:B1]), PCT)
    want1 = nearest_rank(np.abs(C[:, B1:B2]), PCT)
    # by hand: 20 values per pool, rank ceil(0.9 * 20) = 18 -> the 18th smallest
    assert want0 == pytest.approx(0.25 * 18) and want1 == pytest.approx(0.1 * 18 + 0.03)
    # the plausible mistakes give other values, so this test separates them
    wrong = {
        "zone 1 pooled over [B1, E)": nearest_rank(np.abs(C[:, B1:E]), PCT),
        "zone 0 pooled over [0, B1]": nearest_rank(np.abs(C[:, 0:B1 + 1]), PCT),
        "signed zone-0 coefficients": nearest_rank(C[:, 0:B1], PCT),
        "signed zone-1 coefficients": nearest_rank(C[:, B1:B2], PCT),
        "rank one too high": float(np.sort(np.abs(C[:, 0:B1]).ravel())[18]),
    }
    for what, v in wrong.items():
        assert abs(v - want0) > 0.05 and abs(v - want1) > 0.05, what
    assert d.A[0] == pytest.approx(want0, abs=1e-4)
    assert d.A[1] == pytest.approx(want1, abs=1e-4)
    assert d.A[2] == 0.0


def test_train_histogram_counts_every_kept_bin_with_smoothing():
    C = hand_windows()
    d = train(C)
    # the levels of the designed coefficients under the trained scales: each is
    # checked to sit well inside its quantizer cell, so float32 samples cannot move it
    hist = np.ones(256, np.uint64)  # +1 on every level (Sec. 3.3 reading: every level gets a code)
    for w in range(C.shape[0]):
        for k in range(E):
            z = d.zone(k)
            L = oracle.quantize(d, z, C[w, k])
            assert oracle.quantize(d, z, C[w, k] - 1e-4) == L == oracle.quantize(d, z, C[w, k] + 1e-4)
            hist[L] += 1
    # zone-2 bins are counted, as level 128
    assert hist[128] >= 1 + 2 * C.shape[0]
    np.testing.assert_array_equal(d.code_len, oracle.package_merge(hist, d.lmax))


def test_train_all_zero_signals_smoothed_code():
    # All-zero training signals: every coefficient is 0, both scales 0 (zones
    # switched off), every symbol is level 128.  With +1 on all 256 counts the
    # optimal code gives level 128 one bit and splits the other half of the code
    # space as evenly as possible over the 255 equally likely other levels:
    # a * 2^-8 + b * 2^-9 = 1/2 with a + b = 255 -> one level of 8 bits, 254 of 9.
    n_sig, S = 4, 512
    flat = np.zeros(n_sig * S, np.float32)
    offs = np.arange(n_sig, dtype=np.uint64) * S
    lens = np.full(n_sig, S, np.uint64)
    d = oracle.train_domain(flat, offs, lens, oracle.Domain(N, E, B1, B2, 50.0, 0.004, (0, 0, 0), 12), PCT)
    assert d.A[0] == 0.0 and d.A[1] == 0.0
    cl = d.code_len.astype(int)
    assert cl[128] == 1
    others = np.delete(cl, 128)
    assert sorted(np.unique(others).tolist()) == [8, 9]
    assert int((others == 8).sum()) == 1 and int((others == 9).sum()) == 254
    # without the smoothing the 255 unseen levels would have no code at all
    assert int((cl == 0).sum()) == 0


def test_zone2_bins_reconstruct_zero_exhaustive():
    # N = 16, E = 3, B1 = 1, B2 = 2: bin 2 is zone 2.  For every level of bin 2
    # and every level of bin 1 (a spread of bin-0 levels), the reconstruction
    # through the quantizer's zone map equals the 40-digit mpmath sum over bins
    # 0 and 1 alone: zone-2 levels carry no value.
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    d = oracle.Domain(16, 3, 1, 2, 50.0, 0.004, (3.0, 2.0, 0.0), 12)
    cosv = np.array([float(mpmath.cos(mpmath.pi * (2 * n + 1) / 32)) for n in range(16)])
    deq0 = [oracle.dequantize(d, 0, L) for L in range(256)]
    deq1 = np.array([oracle.dequantize(d, 1, L) for L in range(256)])
    L1, L2 = np.meshgrid(np.arange(256), np.arange(256), indexing="ij")
    worst = 0.0
    for L0 in (0, 1, 64, 127, 128, 129, 200, 255):
        lv = np.empty((256 * 256, 3), np.uint8)
        lv[:, 0] = L0
        lv[:, 1] = L1.ravel()
        lv[:, 2] = L2.ravel()
        x = oracle.reconstruct(lv.ravel(), 16 * 256 * 256, d).reshape(256, 256, 16)
        ref = deq0[L0] / 2 + deq1[:, None] * cosv[None, :]  # [L1, n]
        worst = max(worst, float(np.max(np.abs(x - ref[:, None, :]))))
    assert worst < 1e-13


def test_zone2_bins_quantize_to_128():
    # A signal with all its energy in bin 2 (zone 2 of this domain) and bin 1:
    # the encoder's levels at bin 2 are 128 in every window, bin 1 is not.
    d = oracle.Domain(16, 3, 1, 2, 50.0, 0.004, (3.0, 2.0, 0.0), 12)
    C = np.zeros(16)
    C[1], C[2] = 1.5, 2.5
    n = np.arange(16)
    win = sum(C[k] * np.cos(math.pi / 16 * (n + 0.5) * k) for k in (1, 2))
    x = np.tile(win, 8).astype(np.float32)
    lv = oracle.quantize_stream(x, d).reshape(8, 3)
    assert np.all(lv[:, 2] == 128)
    assert np.all(lv[:, 1] == oracle.quantize(d, 1, 1.5)) and oracle.quantize(d, 1, 1.5) > 128
    assert np.all(lv[:, 0] == 128)
