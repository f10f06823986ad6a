"""Pins of the oracle's transform (Sec. 3.1, Eq. 1) against closed forms and a
textbook routine (scipy's DCT-II / DCT-III), not against itself."""
import numpy as np
import pytest
import scipy.fft

import oracle


def basis_matrix(N):
    return np.array([[oracle.basis(N, n, k) for n in range(N)] for k in range(N)])


@pytest.mark.parametrize("N", [4, 8, 13, 32, 128])
def test_basis_orthogonality(N):
    # rows of the Eq. 1 kernel are orthogonal: M M^T = diag(N, N/2, ..., N/2)
    M = basis_matrix(N)
    G = M @ M.T
    expect = np.diag([N] + [N / 2] * (N - 1))
    np.testing.assert_allclose(G, expect, atol=1e-10 * N)


@pytest.mark.parametrize("N", [4, 8, 32, 128])
def test_dct2_matches_scipy(N):
    # scipy's unnormalised DCT-II is y[k] = 2 sum x[n] cos(pi k (2n+1) / 2N),
    # so Eq. 1 is y / N.
    rng = np.random.default_rng(N)
    x = rng.standard_normal(N)
    for E in sorted({1, N // 2, N}):
        C = oracle.dct2(x, N, E)
        ref = scipy.fft.dct(x, type=2)[:E] / N
        np.testing.assert_allclose(C, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("N", [4, 8, 32, 128])
def test_idct3_matches_scipy(N):
    # scipy's unnormalised DCT-III is y[n] = c[0] + 2 sum_{k>=1} c[k] cos(pi k (2n+1) / 2N);
    # the inverse of Eq. 1 is y / 2, with bins >= E zero.
    rng = np.random.default_rng(100 + N)
    for E in sorted({1, 3, N // 2, N}):
        C = rng.standard_normal(E)
        full = np.zeros(N)
        full[:E] = C
        ref = scipy.fft.dct(full, type=3) / 2
        np.testing.assert_allclose(oracle.idct3(C, N), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("N", [4, 8, 16, 32, 64, 128])
def test_perfect_reconstruction_without_truncation(N):
    rng = np.random.default_rng(7 * N)
    for _ in range(5):
        x = rng.standard_normal(N) * 100
        assert np.max(np.abs(oracle.idct3(oracle.dct2(x, N, N), N) - x)) < 1e-12 * 100


@pytest.mark.parametrize("N", [8, 32])
def test_pure_cosine_and_constant(N):
    for k0 in range(1, N):
        x = np.array([np.cos(np.pi / N * (n + 0.5) * k0) for n in range(N)])
        C = oracle.dct2(x, N, N)
        e = np.zeros(N)
        e[k0] = 1.0
        np.testing.assert_allclose(C, e, atol=1e-13)
    C = oracle.dct2(np.full(N, 3.25), N, N)
    e = np.zeros(N)
    e[0] = 6.5
    np.testing.assert_allclose(C, e, atol=1e-13)


def test_truncation_is_projection():
    # keeping E bins = orthogonal projection onto the first E basis vectors:
    # the residual is orthogonal to each kept basis row
    N, E = 32, 16
    rng = np.random.default_rng(3)
    x = rng.standard_normal(N)
    xr = oracle.idct3(oracle.dct2(x, N, E), N)
    M = basis_matrix(N)
    np.testing.assert_allclose(M[:E] @ (x - xr), 0, atol=1e-12)
