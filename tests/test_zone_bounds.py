"""The host encoder's zone maps as boundary tables (include/fptc_codec.h
fptc_zone_bounds, which the GPU encoder's exact tiers use).  Exactness against
the host encoder: a window of 32 equal samples v has the FP64 bin-0
coefficient 2 v exactly, so fptc_encode_stream's level for bin 0 (zone 0 with
B1 = 2, zone 1 with B1 = 0) is its map at 2 v; at the float32 points nearest
every boundary that level equals the number of boundaries <= 2 v.  Against the
paper's formulas: the oracle's quantizer (Eq. 2, Eq. 3, written on its own,
log(1 + x) where the library uses log1p) gives the same level on random and
special coefficients except within FP64 rounding of a boundary, for several
scales, mu and alpha1 (alpha1 = 1: zone 1 all deadzone; a zone scale <= 1e-30:
the zone is off), at +-inf too."""
import math

import numpy as np
import pytest

import oracle

CASES = [(2.2589, 86.4, 50.0, 0.004), (0.93, 1e-3, 255.0, 0.3), (3e5, 2.0, 8.0, 1.0), (0.0, 0.0, 50.0, 0.004),
         (7.5, 7.5, 50.0, 1.0 - 2.0 ** -20)]


def _domains(A0, A1, mu, alpha1, B1=2):
    from paper_2605_01086_gb300 import codec
    cl = np.full(256, 8, np.uint8)
    return (codec.Domain(32, 16, B1, 16, mu, alpha1, (A0, A1, 0.0), 8, cl),
            oracle.Domain(32, 16, B1, 16, mu, alpha1, (A0, A1, 0.0), 8, cl))


@pytest.mark.parametrize("A0,A1,mu,alpha1", CASES)
def test_bounds_are_the_host_encoders_map(A0, A1, mu, alpha1):
    from paper_2605_01086_gb300 import codec
    for zone, B1 in ((0, 2), (1, 0)):
        pd, _ = _domains(A0, A1, mu, alpha1, B1)
        b = codec.zone_bounds(pd, zone)
        n = int(np.sum(~np.isnan(b)))
        assert np.all(np.isnan(b[n:])) and np.all(b[1:n] >= b[:n - 1])  # unreachable levels last
        vs = []
        for t in b[np.isfinite(b)]:
            v0 = np.float32(t / 2.0)
            for step in range(-2, 3):
                v = v0
                for _ in range(abs(step)):
                    v = np.nextafter(v, np.float32(math.copysign(math.inf, step)))
                vs.append(v)
        vs += [np.float32(0.0), np.float32(3e38), np.float32(-3e38)]
        x = np.repeat(np.array(vs, np.float32), 32)
        _, _, lv = codec.encode_stream(pd, x)
        got = lv.reshape(-1, 16)[:, 0]
        want = np.array([int(np.sum(b <= 2.0 * float(v))) for v in vs])
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("A0,A1,mu,alpha1", CASES)
def test_bounds_follow_the_oracle_quantizer(A0, A1, mu, alpha1):
    from paper_2605_01086_gb300 import codec
    pd, od = _domains(A0, A1, mu, alpha1)
    rng = np.random.default_rng(0)
    for zone in (0, 1):
        b = codec.zone_bounds(pd, zone)
        A = max(A0 if zone == 0 else A1, 1e-3)
        cs = list(rng.uniform(-1.3 * A, 1.3 * A, 4000)) + [0.0, -0.0, A, -A, 1e300, -1e300, math.inf, -math.inf]
        fin = b[np.isfinite(b)]
        for c in cs:
            got, want = int(np.sum(b <= c)), oracle.quantize(od, zone, c)
            if got != want:  # only where c is within FP64 rounding of a boundary
                assert np.min(np.abs(fin - c)) <= 1e-12 * max(abs(c), 1e-300), (zone, c, got, want)
        if A0 <= 1e-30 and zone == 0 or A1 <= 1e-30 and zone == 1 or alpha1 == 1.0 and zone == 1:
            assert np.all(b[:128] == -math.inf) and np.all(np.isnan(b[128:]))  # every level 128
