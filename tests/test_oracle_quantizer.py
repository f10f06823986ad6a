"""Pins of the oracle's three-zone quantizer (Sec. 3.2, Eq. 2, Eq. 3): level
layout stated by the paper, saturation, monotonicity, lattice idempotence and
the error bound of a uniform / companded quantizer."""
import numpy as np
import pytest

import oracle


def dom(A0=2.0, A1=3.0, mu=50.0, alpha1=0.004):
    return oracle.Domain(32, 16, 2, 16, mu, alpha1, (A0, A1, 0.0), 12)


def test_level_layout_from_paper(golden):
    g = golden("zone_levels.txt")
    d = dom()
    assert oracle.quantize(d, 0, 0.0) == int(g["zero_level"])
    lo, hi = map(int, g["positive_levels"].split())
    nlo, nhi = map(int, g["negative_levels"].split())
    cs = np.linspace(-1.2 * d.A[0], 1.2 * d.A[0], 40001)
    levels = np.array([oracle.quantize(d, 0, c) for c in cs])
    assert set(levels[cs > 1e-3].tolist()) <= set(range(lo, hi + 1)) | {128}
    assert set(levels[cs < -1e-3].tolist()) <= set(range(nlo, nhi + 1)) | {128}
    # every level is reached by a dense sweep
    assert set(levels.tolist()) == set(range(256))
    assert oracle.quantize(d, 1, d.A[1]) == int(g["zone1_at_plus_A1"])
    assert oracle.quantize(d, 1, -d.A[1]) == int(g["zone1_at_minus_A1"])
    for c in (-1e9, -1.0, 0.0, 1.0, 1e9):
        assert oracle.quantize(d, 2, c) == int(g["zone2_level"])
        assert oracle.dequantize(d, 2, oracle.quantize(d, 2, c)) == 0.0


@pytest.mark.parametrize("zone", [0, 1])
def test_monotone_and_saturating(zone):
    d = dom()
    A = d.A[zone]
    cs = np.linspace(-2 * A, 2 * A, 20001)
    levels = np.array([oracle.quantize(d, zone, c) for c in cs])
    assert np.all(np.diff(levels) >= 0)
    assert levels[0] == 0 and levels[-1] == 255
    assert oracle.quantize(d, zone, A) == 255 and oracle.quantize(d, zone, -A) == 0
    deq = np.array([oracle.dequantize(d, zone, L) for L in range(256)])
    assert np.all(np.diff(deq) > 0)
    assert deq[128] == 0.0
    assert deq[255] == pytest.approx(A, rel=1e-14) and deq[0] == pytest.approx(-A, rel=1e-14)


def test_zone0_lattice_idempotence():
    for mu in (1.0, 50.0, 500.0):
        d = dom(mu=mu)
        for L in range(256):
            assert oracle.quantize(d, 0, oracle.dequantize(d, 0, L)) == L


def test_zone0_companded_error_bound():
    # Textbook mu-law compander F(u) = ln(1 + mu|u|)/ln(1 + mu): the reconstruction
    # lies within half a level of the input in the companded domain.
    for mu in (1.0, 50.0, 500.0):
        d = dom(mu=mu)
        A = d.A[0]
        F = lambda u: np.log1p(mu * abs(u)) / np.log1p(mu)
        for c in np.linspace(-A, A, 4001):
            L = oracle.quantize(d, 0, c)
            ch = oracle.dequantize(d, 0, L)
            assert np.sign(ch) in (np.sign(c), 0.0)
            step = 1 / 127 if c >= 0 else 1 / 128
            assert abs(F(c / A) - F(ch / A)) <= step / 2 + 1e-12


def test_zone1_deadzone_and_lattice():
    for alpha in (0.0, 0.004, 0.3):
        d = dom(alpha1=alpha)
        A = d.A[1]
        d1 = alpha * A
        assert oracle.quantize(d, 1, d1) == 128
        assert oracle.quantize(d, 1, -d1) == 128
        assert oracle.quantize(d, 1, 0.5 * d1) == 128
        for L in range(256):
            ch = oracle.dequantize(d, 1, L)
            if L in (127, 129):
                # the first level on each side is reconstructed at the deadzone edge,
                # which belongs to the deadzone itself (Eq. 3 uses strict inequalities)
                assert ch == pytest.approx(d1 if L == 129 else -d1, abs=1e-15)
                if alpha > 0:
                    assert oracle.quantize(d, 1, ch * (1 + 1e-9)) == L
                continue
            assert oracle.quantize(d, 1, ch) == L


def test_zone1_uniform_error_bound():
    d = dom(alpha1=0.004)
    A = d.A[1]
    d1 = 0.004 * A
    for c in np.linspace(-A, A, 8001):
        ch = oracle.dequantize(d, 1, oracle.quantize(d, 1, c))
        if abs(c) <= d1:
            assert ch == 0.0
        else:
            step = (A - d1) / (126 if c > 0 else 127)
            assert abs(c - ch) <= step / 2 + 1e-12


def test_switched_off_zone():
    d = dom(A0=0.0, A1=1e-31)
    for c in (-5.0, 0.0, 5.0):
        assert oracle.quantize(d, 0, c) == 128
        assert oracle.quantize(d, 1, c) == 128
    assert all(oracle.dequantize(d, z, L) == 0.0 for z in (0, 1) for L in range(256))


@pytest.mark.parametrize("zone", [0, 1])
def test_dequant_linear_in_scale(zone):
    # d c_hat / d A_z = reconstruction at A_z = 1 (both maps scale linearly)
    d = dom()
    for L in (0, 17, 127, 128, 129, 200, 255):
        unit = oracle.dequantize_unit(d, zone, L)
        d2 = dom(A0=d.A[0] * 3, A1=d.A[1] * 3)
        assert oracle.dequantize(d2, zone, L) == pytest.approx(3 * oracle.dequantize(d, zone, L), rel=1e-13, abs=1e-300)
        assert oracle.dequantize(d, zone, L) == pytest.approx(d.A[zone] * unit, rel=1e-13, abs=1e-300)


def test_percentile_nearest_rank():
    v = np.arange(1, 1001, dtype=float)[::-1]
    assert oracle.percentile(v, 99.9) == 999.0
    assert oracle.percentile(v, 100.0) == 1000.0
    assert oracle.percentile(v, 50.0) == 500.0
    assert oracle.percentile([7.0], 90.0) == 7.0
