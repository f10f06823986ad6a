"""Pins of the oracle's SymLen packing (Sec. 4.1, Alg. 1) and its bit-serial
decoder: the hand-worked Alg. 1 example, greedy-closure invariants, round trips
and adversarial streams."""
import numpy as np
import pytest

import oracle


def _codebook(lens):
    lens = np.asarray(lens, np.uint8)
    return oracle.canonical_codes(lens, int(lens.max())), lens


def test_alg1_worked_example(golden):
    g = golden("alg1_worked_example.txt")
    for pre in ("", "fit_"):
        codes = np.zeros(256, np.uint32)
        lens = np.zeros(256, np.uint8)
        for i in range(3):
            codes[i] = int(g[f"{pre}code{i}"], 16)
            lens[i] = int(g[f"{pre}len{i}"])
        words, symlen = oracle.pack_symlen([0, 1, 2], codes, lens)
        assert [hex(int(w)) for w in words] == [hex(int(v, 16)) for v in g[f"{pre}words"].split()]
        assert list(map(int, symlen)) == list(map(int, g[f"{pre}symlen"].split()))


def check_invariants(X, words, symlen, lens):
    X = np.asarray(X)
    assert int(symlen.sum()) == X.size
    pos = 0
    for w in range(words.size):
        n = int(symlen[w])
        used = int(lens[X[pos:pos + n]].sum())
        assert used <= 64
        # padding bits are zero
        assert (int(words[w]) & ((1 << (64 - used)) - 1)) == 0
        if w + 1 < words.size:
            assert used + int(lens[X[pos + n]]) > 64  # greedy: next codeword did not fit
        pos += n


@pytest.mark.parametrize("lmax", [8, 12, 16])
@pytest.mark.parametrize("seed", range(3))
def test_random_round_trip(lmax, seed):
    rng = np.random.default_rng(seed * 31 + lmax)
    freq = (rng.pareto(1.0, size=256) * 50).astype(np.uint64) + 1
    lens = oracle.package_merge(freq, lmax)
    codes = oracle.canonical_codes(lens, lmax)
    p = freq / freq.sum()
    X = rng.choice(256, size=20000, p=p).astype(np.uint8)
    words, symlen = oracle.pack_symlen(X, codes, lens)
    check_invariants(X, words, symlen, lens)
    Y = oracle.unpack_symlen(words, symlen, lens, lmax, X.size)
    assert np.array_equal(X, Y)


def test_all_max_length_codes():
    lens = np.full(256, 8, np.uint8)  # complete code, all 8 bits
    codes, _ = _codebook(lens)
    X = np.arange(256, dtype=np.uint8).repeat(3)
    words, symlen = oracle.pack_symlen(X, codes, lens)
    assert np.all(symlen[:-1] == 8)
    check_invariants(X, words, symlen, lens)
    assert np.array_equal(oracle.unpack_symlen(words, symlen, lens, 8, X.size), X)


def test_sixty_four_one_bit_codes_per_word():
    lens = np.zeros(256, np.uint8)
    lens[128] = 1  # the zero bin gets a 1-bit code
    lens[0] = 2
    lens[255] = 2
    codes, _ = _codebook(lens)
    X = np.full(64 * 5 + 3, 128, np.uint8)
    words, symlen = oracle.pack_symlen(X, codes, lens)
    assert list(symlen) == [64] * 5 + [3]
    assert np.array_equal(oracle.unpack_symlen(words, symlen, lens, 2, X.size), X)


def test_corruption_detected():
    lens = np.full(256, 8, np.uint8)
    codes, _ = _codebook(lens)
    X = np.arange(64, dtype=np.uint8)
    words, symlen = oracle.pack_symlen(X, codes, lens)
    bad = symlen.copy()
    bad[0] = 9  # 9 codes of 8 bits cannot fit 64 bits
    with pytest.raises(oracle.OracleError, match="overrun"):
        oracle.unpack_symlen(words, bad, lens, 8, X.size + 1)
    with pytest.raises(oracle.OracleError, match="count"):
        oracle.unpack_symlen(words, symlen, lens, 8, X.size + 5)
    # an incomplete code has invalid patterns
    inc = np.zeros(256, np.uint8)
    inc[1] = 1
    with pytest.raises(oracle.OracleError, match="invalid"):
        oracle.unpack_symlen(np.array([0xFFFFFFFFFFFFFFFF], np.uint64), np.array([1], np.uint8), inc, 1, 1)


def test_symbol_without_code_rejected():
    lens = np.zeros(256, np.uint8)
    lens[0] = 1
    codes, _ = _codebook(lens)
    with pytest.raises(oracle.OracleError):
        oracle.pack_symlen([0, 1], codes, lens)
