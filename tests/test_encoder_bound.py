"""CPU check of the error bound the GPU encoder's level kernel relies on: the
compensated FP32 bin of Eq. 1 (exact products by FMA, exact two-sums, hi/lo
cosines, in the kernel's order of operations, emulated here with numpy float32
arithmetic, which rounds each operation as the GPU does, and the FMA's exact
product error formed in float64) lies within the kernel's bound of the FP64 bin
the host encoder computes (products and sums rounded separately, in sample
order).  Adversarial windows: large offsets with small variations, mixed signs,
magnitudes from 1e-20 to 1e6, N from 4 to 128."""
import numpy as np
import pytest

f32 = np.float32


def _emulate(x, ch, cl):
    """hi, lo, s1 of the kernel's loop for one bin (x, ch, cl float32 arrays)."""
    hi = lo = s1 = f32(0.0)
    for xv, c_h, c_l in zip(x, ch, cl):
        pr = f32(xv * c_h)
        fma = f32(np.float64(xv) * np.float64(c_h) - np.float64(pr))  # exact product error, rounded once
        pe = f32(fma + f32(xv * c_l))
        t = f32(hi + pr)
        bp = f32(t - hi)
        lo = f32(lo + f32(f32(f32(hi - f32(t - bp)) + f32(pr - bp)) + pe))
        hi = t
        s1 = f32(s1 + abs(xv))
    return hi, lo, s1


def _fp64_bin(x, cos64, N):
    acc = 0.0
    for xv, c in zip(x, cos64):
        acc = acc + float(xv) * float(c)   # Python floats: each operation rounded separately
    return acc * (2.0 / N)


@pytest.mark.parametrize("N", [4, 16, 32, 128])
def test_compensated_bin_within_bound(N):
    rng = np.random.default_rng(N)
    E = min(N, 16)
    cos64 = np.array([[np.cos(np.pi * (2 * n + 1) * k / (2 * N)) for n in range(N)] for k in range(E)])
    ch = cos64.astype(f32)
    cl = (cos64 - ch.astype(np.float64)).astype(f32)
    worst = 0.0
    for trial in range(300):
        kind = trial % 5
        if kind == 0:
            x = rng.normal(0, 1, N)
        elif kind == 1:
            x = 1e4 + rng.normal(0, 1e-2, N)              # large offset, small variation
        elif kind == 2:
            x = rng.choice([-1, 1], N) * 10.0 ** rng.uniform(-20, 6, N)
        elif kind == 3:
            x = np.full(N, 3.0) + rng.integers(-1, 2, N) * 2.0 ** -20
        else:
            x = rng.normal(100, 5, N) * rng.choice([1, -1], N)
        x = x.astype(f32)
        for k in range(E):
            hi, lo, s1 = _emulate(x, ch[k], cl[k])
            c64 = _fp64_bin(x, cos64[k], N)
            cd = (float(hi) + float(lo)) * (2.0 / N)
            err = float(s1) * (2.0 / N) * 2.0 ** -34 + 1e-30
            gap = abs(cd - c64)
            assert gap <= 2.0 * err, (N, trial, k, gap, err)   # the zone-1 deadzone test's margin
            c = float(f32(f32(hi + lo) * f32(2.0 / N)))
            assert abs(c - c64) <= err + abs(c) * 2.0 ** -21, (N, trial, k)   # the bracket's margin
            worst = max(worst, gap / err if err > 1e-29 else 0.0)
    assert worst < 1.0


def test_plain_fp32_sum_would_break_the_bound():
    """The bound is tight enough to matter: an uncompensated FP32 dot product of
    an offset window misses it by orders of magnitude."""
    N = 32
    rng = np.random.default_rng(1)
    cos64 = np.array([[np.cos(np.pi * (2 * n + 1) * k / (2 * N)) for n in range(N)] for k in range(16)])
    ch = cos64.astype(f32)
    worst = 0.0
    for _ in range(20):
        x = (1e4 + rng.normal(0, 1e-2, N)).astype(f32)
        s1 = float(np.abs(x.astype(np.float64)).sum())
        for k in range(1, 16):
            acc = f32(0.0)
            for xv, c in zip(x, ch[k]):
                acc = f32(acc + f32(xv * c))
            err = s1 * (2.0 / N) * 2.0 ** -34
            worst = max(worst, abs(float(acc) * (2.0 / N) - _fp64_bin(x, cos64[k], N)) / err)
    assert worst > 100.0


def _zone0_64(c, A0, mu):
    a = min(abs(c), A0)
    q = np.log1p(mu * (a / A0)) / np.log1p(mu)
    v = 128 + int(np.floor(127.0 * q + 0.5)) if c >= 0 else 128 - int(np.floor(128.0 * q + 0.5))
    return min(max(v, 0), 255)


def _zone0_32(c, A0, mu):
    c = f32(c)
    a = min(f32(abs(c)), f32(A0))
    q = f32(np.log1p(f32(f32(mu) * f32(a * f32(1.0 / A0))))) * f32(1.0 / np.log1p(mu))
    q = f32(q)
    v = 128 + int(np.floor(f32(f32(127.0) * q + f32(0.5)))) if c >= 0 else 128 - int(np.floor(f32(f32(128.0) * q + f32(0.5))))
    return min(max(v, 0), 255)


@pytest.mark.parametrize("A0", [2.2589, 65.02, 305.3, 1e-3])
def test_zone0_slack_brackets_the_fp64_map(A0):
    """Levels of the FP32 evaluation at c - slack and c + slack bracket the FP64
    level at c (slack = 2^-18 A0), densely around every level boundary."""
    mu = 50.0
    slack = A0 * 2.0 ** -18
    # coefficients at every level boundary of the FP64 map, and just around them
    cs = []
    for L in range(1, 128):
        q = (L - 0.5) / 127.0
        b = A0 / mu * ((1.0 + mu) ** q - 1.0)
        cs += [b * (1 + e) for e in (-1e-6, -1e-9, 0.0, 1e-9, 1e-6)]
        q = (L - 0.5) / 128.0
        b = A0 / mu * ((1.0 + mu) ** q - 1.0)
        cs += [-b * (1 + e) for e in (-1e-6, 0.0, 1e-6)]
    cs += list(np.random.default_rng(0).uniform(-1.2 * A0, 1.2 * A0, 2000))
    for c in cs:
        lo, hi = _zone0_32(c - slack, A0, mu), _zone0_32(c + slack, A0, mu)
        assert lo <= _zone0_64(c, A0, mu) <= hi, (c, lo, hi)


# ---- the window kernel's first tier: the DCT-II butterfly with per-bin bounds ----

def _round_f32(fr):
    """float32 nearest to the exact rational fr (ties to even), as one rounding."""
    from fractions import Fraction
    y = np.float32(float(fr))
    best = None
    for c in (np.nextafter(y, np.float32(-np.inf)), y, np.nextafter(y, np.float32(np.inf))):
        dist = abs(Fraction(float(c)) - fr)
        key = (dist, int(np.array(c, np.float32).view(np.uint32)) & 1)
        if best is None or key < best[0]:
            best = (key, c)
    return np.float32(best[1])


def _fma(a, b, c):
    from fractions import Fraction
    return _round_f32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def _cos32(num, den):
    return f32(np.cos(np.pi * num / den))


def _butterfly_bounded(x):
    """The device's dct2_16_bounded in float32, operation by operation: outputs and bounds."""
    u = 2.0 ** -24 * 1.02
    uu_ = [f32(x[n] + x[31 - n]) for n in range(16)]
    v = [f32(x[n] - x[31 - n]) for n in range(16)]
    su, sv = sum(abs(float(t)) for t in uu_), sum(abs(float(t)) for t in v)
    a, e = [0.0] * 16, [0.0] * 16
    for j in range(8):
        acc = f32(v[0] * _cos32(2 * j + 1, 64))
        for n in range(1, 16):
            acc = _fma(v[n], _cos32((2 * n + 1) * (2 * j + 1), 64), acc)
        a[2 * j + 1], e[2 * j + 1] = acc, 18.1 * u * sv
    uu = [f32(uu_[n] + uu_[15 - n]) for n in range(8)]
    uv = [f32(uu_[n] - uu_[15 - n]) for n in range(8)]
    suu, suv = sum(abs(float(t)) for t in uu), sum(abs(float(t)) for t in uv)
    for j in range(4):
        acc = f32(uv[0] * _cos32(2 * j + 1, 32))
        for n in range(1, 8):
            acc = _fma(uv[n], _cos32((2 * n + 1) * (2 * j + 1), 32), acc)
        a[4 * j + 2], e[4 * j + 2] = acc, u * (9.6 * suv + su)
    uuu = [f32(uu[n] + uu[7 - n]) for n in range(4)]
    uuv = [f32(uu[n] - uu[7 - n]) for n in range(4)]
    suuu, suuv = sum(abs(float(t)) for t in uuu), sum(abs(float(t)) for t in uuv)
    a[0] = f32(f32(0.5) * f32(f32(uuu[0] + uuu[1]) + f32(uuu[2] + uuu[3])))
    e[0] = 0.5 * u * (3 * suuu + suu + su)
    acc = f32(uuu[0] * _cos32(1, 8))
    for n in range(1, 4):
        acc = _fma(uuu[n], _cos32(2 * n + 1, 8), acc)
    a[8], e[8] = acc, u * (5.6 * suuu + suu + su)
    for j in range(2):
        acc = f32(uuv[0] * _cos32(2 * j + 1, 16))
        for n in range(1, 4):
            acc = _fma(uuv[n], _cos32((2 * n + 1) * (2 * j + 1), 16), acc)
        a[8 * j + 4], e[8 * j + 4] = acc, u * (5.6 * suuv + suu + su)
    return a, e


def test_butterfly_bins_within_their_bounds():
    import math
    rng = np.random.default_rng(11)
    worst = 0.0
    tighter = []
    for trial in range(120):
        kind = trial % 6
        if kind == 0:
            x = rng.normal(0, 1, 32)
        elif kind == 1:
            x = 1e4 + rng.normal(0, 1e-2, 32)              # large offset, small variation
        elif kind == 2:
            x = rng.choice([-1, 1], 32) * 10.0 ** rng.uniform(-20, 6, 32)
        elif kind == 3:
            x = np.full(32, 3.0) + rng.integers(-1, 2, 32) * 2.0 ** -20
        elif kind == 4:
            x = rng.normal(100, 5, 32) * rng.choice([1, -1], 32)
        else:
            x = 100.0 + 30 * np.sin(np.arange(32) / 9.0) + rng.normal(0, 2, 32)   # power-like
        x = x.astype(f32)
        a, e = _butterfly_bounded(x)
        s1 = float(np.sum(np.abs(x.astype(np.float64))))
        for k in range(16):
            exact = math.fsum(float(x[n]) * (0.5 if k == 0 else math.cos(math.pi / 32 * (n + 0.5) * k))
                              for n in range(32))
            err = abs(float(a[k]) - exact)
            assert err <= e[k] + 1e-30, (trial, k, err, e[k])
            worst = max(worst, err / (e[k] + 1e-300))
            tighter.append(e[k] / (2.0 ** -19.5 * s1 + 1e-300))
    assert worst < 1.0
    # on the offset windows the bounds are far below the uniform 2^-19.5 sum |x|
    assert np.median(tighter) < 0.5


# ---- the window kernel's branch-free zone-1 map (units of the unscaled sum) ----

def _zone1_64(c, A1, alpha1):
    """The FP64 host encoder's zone-1 map (Eq. 3, |c| clamped to A1)."""
    d1 = alpha1 * A1
    m = min(abs(c), A1)
    if m <= d1:
        return 128
    r = (m - d1) / (A1 - d1)
    return 129 + int(np.floor(r * 126.0 + 0.5)) if c > 0 else 127 - int(np.floor(r * 127.0 + 0.5))


def _zone1_fast32(y, A1, alpha1, form="fast"):
    """Level indices (positive, negative side) of the FP32 zone-1 map at the
    bracket end y = |c| N / 2 (N = 32), operation by operation in float32 with
    the constants the encoder uploads.  form "fast": the window kernel's first
    tier in units of y (fminf, subtraction, one FMA with 126 / span scaled,
    round down); "c": the other tiers in units of c (fminf, subtraction,
    product with 1 / span, then an FMA with 126 or 127)."""
    h = 16.0
    d1 = alpha1 * A1
    span = A1 - d1
    out = []
    if form == "fast":
        u1_d1, u1_A1 = f32(d1 * h), f32(A1 * h)
        for k in (f32(126.0 / span / h), f32(127.0 / span / h)):
            t = _fma(f32(min(f32(y), u1_A1) - u1_d1), k, f32(0.5))
            out.append(int(np.floor(float(t))))
    else:
        a = f32(f32(y) * f32(1.0 / h))
        r = max(f32(f32(min(a, f32(A1)) - f32(d1)) * f32(1.0 / span)), f32(0.0))
        for k in (f32(126.0), f32(127.0)):
            out.append(int(np.floor(float(_fma(r, k, f32(0.5))))))
    return out


@pytest.mark.parametrize("form", ["fast", "c"])
@pytest.mark.parametrize("A1,alpha1", [(86.4, 0.004), (0.933, 0.004), (6.02, 0.2), (1e-3, 0.9),
                                       (3.0, 1.0 - 2.0 ** -12), (2.5e5, 0.5)])
def test_zone1_fp32_slack_brackets_the_fp64_map(A1, alpha1, form):
    """Away from the deadzone edge, the FP32 zone-1 map at y - slack and
    y + slack (slack = 2^-20 A1, in units of y = |c| N / 2) brackets the FP64
    level at c: densely around every level boundary, at the clamp A1 and past
    it, for linear parts down to the narrowest the encoder maps in FP32
    (A1 - d1 = 2^-12 A1).  (It fails with slack 2^-23 A1: the margin is 8x.)"""
    d1 = alpha1 * A1
    span = A1 - d1
    slack = 16.0 * A1 * 2.0 ** -20
    cs = []
    for j in range(0, 127):
        for den in (126.0, 127.0):
            b = d1 + (j + 0.5) / den * span
            cs += [b * (1 + e) for e in (-1e-6, -1e-9, 0.0, 1e-9, 1e-6)]
    cs += [A1 * (1 + e) for e in (-1e-7, 0.0, 1e-7, 1e-3, 0.5, 10.0)]
    cs += list(np.random.default_rng(1).uniform(d1, 1.3 * A1, 1500))
    for c in cs:
        for sgn in (1.0, -1.0):
            cc = sgn * c
            y = abs(cc) * 16.0
            if y - slack <= d1 * 16.0:
                continue  # the deadzone edge is inside the bracket: not decided by the map
            lo, hi = _zone1_fast32(y - slack, A1, alpha1, form), _zone1_fast32(y + slack, A1, alpha1, form)
            lv = [129 + lo[0], 129 + hi[0]] if sgn > 0 else [127 - hi[1], 127 - lo[1]]
            assert lv[0] <= _zone1_64(cc, A1, alpha1) <= lv[1], (cc, lv)
