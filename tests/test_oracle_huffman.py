"""Pins of the oracle's codebook (Sec. 3.3): Kraft equality, prefix-freeness,
length limit, optimality against brute force and against plain Huffman, and the
canonical assignment against the RFC 1951 worked example."""
import heapq
import itertools

import numpy as np
import pytest

import oracle


def huffman_cost(freq):
    h = list(freq)
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a = heapq.heappop(h)
        b = heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


def huffman_max_depth(freq):
    h = [(f, i, 0) for i, f in enumerate(freq)]
    heapq.heapify(h)
    uid = len(freq)
    while len(h) > 1:
        a = heapq.heappop(h)
        b = heapq.heappop(h)
        heapq.heappush(h, (a[0] + b[0], uid, max(a[2], b[2]) + 1))
        uid += 1
    return h[0][2]


def brute_force_limited(freq, lmax):
    best = None
    n = len(freq)
    for ls in itertools.product(range(1, lmax + 1), repeat=n):
        if sum(2.0 ** -l for l in ls) <= 1.0 + 1e-12:
            c = sum(f * l for f, l in zip(freq, ls))
            best = c if best is None else min(best, c)
    return best


def kraft_sum(lengths, lmax):
    return sum(1 << (lmax - int(l)) for l in lengths if l)


def test_clrs_example(golden):
    g = golden("clrs_huffman.txt")
    freq = list(map(int, g["freq"].split()))
    lens = oracle.package_merge(freq, 8)
    assert sum(f * int(l) for f, l in zip(freq, lens)) == int(g["cost"])
    assert list(map(int, lens)) == list(map(int, g["lengths"].split()))


@pytest.mark.parametrize("seed", range(6))
def test_package_merge_optimal_vs_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = 6
    freq = rng.integers(1, 1000, size=n)
    if seed % 2:
        freq = np.array([1, 1, 2, 3, 5, 8]) * (seed + 1)  # Fibonacci weights: deep optimal tree
    for lmax in (3, 4, 5):
        lens = oracle.package_merge(freq, lmax)
        assert lens.max() <= lmax
        assert kraft_sum(lens, lmax) == 1 << lmax
        assert int(np.dot(freq, lens)) == brute_force_limited(list(freq), lmax)


@pytest.mark.parametrize("seed", range(5))
def test_package_merge_equals_huffman_when_unconstrained(seed):
    rng = np.random.default_rng(100 + seed)
    freq = rng.integers(1, 10 ** 6, size=256) ** 2 // 10 ** 6 + 1
    depth = huffman_max_depth(list(freq))
    lmax = max(depth, 8)
    lens = oracle.package_merge(freq, lmax)
    assert int(np.dot(freq, lens)) == huffman_cost(list(freq))


@pytest.mark.parametrize("lmax", [8, 10, 12, 16])
def test_kraft_and_prefix_free_256(lmax):
    rng = np.random.default_rng(lmax)
    freq = (rng.pareto(1.2, size=256) * 100).astype(np.uint64) + 1
    lens = oracle.package_merge(freq, lmax)
    assert lens.min() >= 1 and lens.max() <= lmax
    assert kraft_sum(lens, lmax) == 1 << lmax
    codes = oracle.canonical_codes(lens, lmax)
    strs = [format(int(c), f"0{int(l)}b") for c, l in zip(codes, lens)]
    assert len(set(strs)) == 256
    srt = sorted(strs)
    for a, b in zip(srt, srt[1:]):
        assert not b.startswith(a)


def test_canonical_rfc1951(golden):
    g = golden("rfc1951_canonical.txt")
    lens = list(map(int, g["lengths"].split()))
    codes = oracle.canonical_codes(lens, 4)
    got = [format(int(c), f"0{l}b") for c, l in zip(codes, lens)]
    assert got == g["codes"].split()


def test_kraft_violation_rejected():
    with pytest.raises(oracle.OracleError):
        oracle.canonical_codes([1, 1, 1], 4)
    with pytest.raises(oracle.OracleError):
        oracle.package_merge(np.ones(300, np.uint64), 8)


def test_single_symbol():
    f = np.zeros(256, np.uint64)
    f[5] = 10
    lens = oracle.package_merge(f, 12)
    assert lens[5] == 1 and lens.sum() == 1
