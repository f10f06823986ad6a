"""Pins of the oracle's decoder-side scale fit (the minimiser of the squared
error over the zone scales A_z with the levels fixed): the gradient of the
loss vanishes there, by the analytic adjoint and by central finite differences
of the loss itself; moving any scale either way raises the loss; the fit never
does worse than the trained scales; a zone without bins keeps its scale."""
import numpy as np

import oracle
import siggen


def _streams(n=6, seed_domain=1, N=32, E=16, B1=2, B2=16):
    d = oracle.trained_domain(seed_domain, N=N, E=E, B1=B1, B2=B2)
    wl = siggen.mixed_10000_logu(n=24, lo=500, hi=6000)
    sel = np.flatnonzero(wl.domains == seed_domain)[:n]
    sub = wl.subset(sel)
    flat, offs = siggen.signals(sub.domains, sub.seeds, sub.lengths)
    xs, lvs = [], []
    for i in range(sub.n_streams):
        x = flat[int(offs[i]):int(offs[i]) + int(sub.lengths[i])].astype(np.float64)
        _, _, lv = oracle.encode_stream(x, d)
        xs.append(x)
        lvs.append(lv)
    return d, xs, lvs


def _loss(d, A, xs, lvs):
    dd = oracle.Domain(d.N, d.E, d.B1, d.B2, d.mu, d.alpha1, tuple(A), d.lmax, d.code_len)
    return sum(float(np.sum((oracle.reconstruct(lv, x.size, dd) - x) ** 2)) for x, lv in zip(xs, lvs))


def test_fit_is_the_minimiser():
    d, xs, lvs = _streams()
    A = oracle.fit_zone_scales(lvs, [x.size for x in xs], [0] * len(xs), [d], xs)[0]
    # analytic gradient (the oracle adjoint) at the fit, against its size at the trained scales
    def grad(a):
        dd = oracle.Domain(d.N, d.E, d.B1, d.B2, d.mu, d.alpha1, tuple(a), d.lmax, d.code_len)
        g = np.zeros(3)
        for x, lv in zip(xs, lvs):
            xh = oracle.reconstruct(lv, x.size, dd)
            g += oracle.backward_stream(lv, x.size, dd, 2.0 * (xh - x))[1]
        return g
    g_fit, g_trained = grad(A), grad(np.asarray(d.A))
    assert np.all(np.abs(g_fit[:2]) <= 1e-9 * np.abs(g_trained[:2]).max())
    # central differences of the loss itself
    L0 = _loss(d, A, xs, lvs)
    for z in (0, 1):
        h = 1e-4 * abs(A[z])
        e = np.zeros(3)
        e[z] = h
        Lp, Lm = _loss(d, A + e, xs, lvs), _loss(d, A - e, xs, lvs)
        assert abs(Lp - Lm) / (2 * h) <= 1e-6 * L0 / abs(A[z])
        assert Lp >= L0 and Lm >= L0
    assert L0 <= _loss(d, d.A, xs, lvs)


def test_fit_improves_prd_and_keeps_unused_zone():
    d, xs, lvs = _streams(seed_domain=2, N=16, E=8, B1=0, B2=8)   # no zone-0 bin
    A = oracle.fit_zone_scales(lvs, [x.size for x in xs], [0] * len(xs), [d], xs)[0]
    assert A[0] == d.A[0]
    dd = oracle.Domain(d.N, d.E, d.B1, d.B2, d.mu, d.alpha1, tuple(A), d.lmax, d.code_len)
    x = np.concatenate(xs)
    p0 = oracle.prd(x, np.concatenate([oracle.reconstruct(lv, xx.size, d) for xx, lv in zip(xs, lvs)]))
    p1 = oracle.prd(x, np.concatenate([oracle.reconstruct(lv, xx.size, dd) for xx, lv in zip(xs, lvs)]))
    assert p1 <= p0
