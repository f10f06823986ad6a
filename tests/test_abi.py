"""CPU tests of the C ABI library: it loads, exports every symbol the headers
declare, its struct layouts match the binding, and its host-side logic
(validation, decode table, trainer, encoder) agrees with the oracle.  No GPU
compute is called."""
import os
import re

import numpy as np
import pytest

import oracle
import siggen
from paper_2605_01086_gb300 import _lib, codec
from paper_2605_01086_gb300.build import INCLUDE, build

from gpu_util import near_level_boundary


@pytest.fixture(scope="module")
def L():
    build()
    return _lib.lib()


def declared_functions():
    names = set()
    for h in os.listdir(INCLUDE):
        txt = open(os.path.join(INCLUDE, h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(fptc_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), f"{n} declared but not exported"
    assert set(_lib.SIGNATURES) == names


def test_struct_sizes(L):
    for i, cls in enumerate((_lib.CDomain, _lib.CSegment, _lib.CPlanOptions, _lib.CPlanInfo)):
        assert L.fptc_struct_size(i) == __import__("ctypes").sizeof(cls)
    assert L.fptc_abi_version() == 1


def od(domain_id=0):
    o = oracle.trained_domain(domain_id)
    return o, codec.Domain(o.N, o.E, o.B1, o.B2, o.mu, o.alpha1, o.A, o.lmax, o.code_len)


def test_validate_domain_rejects_bad_parameters(L):
    _, d = od()
    codec.validate_domain(d)
    bad = [dict(N=3), dict(N=129), dict(E=0), dict(E=40), dict(B1=5, B2=4), dict(B2=17), dict(mu=0.0),
           dict(alpha1=1.5), dict(lmax=0), dict(lmax=17), dict(scale=(-1.0, 1.0, 0.0))]
    for kw in bad:
        dd = codec.Domain(**{**d.__dict__, **kw})
        with pytest.raises(_lib.FptcError):
            codec.validate_domain(dd)
    cl = d.code_len.copy()
    cl[:] = 1  # Kraft sum 128 > 1
    with pytest.raises(_lib.FptcError, match="Kraft"):
        codec.validate_domain(codec.Domain(**{**d.__dict__, "code_len": cl}))
    with pytest.raises(_lib.FptcError):
        codec.validate_domain(codec.Domain(**{**d.__dict__, "code_len": np.zeros(256, np.uint8)}))


@pytest.mark.parametrize("domain_id", [0, 1, 2, 3])
def test_decode_table_matches_oracle_codes(L, domain_id):
    o, d = od(domain_id)
    codes = oracle.canonical_codes(o.code_len, o.lmax)
    np.testing.assert_array_equal(codec.canonical_codes(d), codes)
    t = codec.decode_table(d)
    for s in range(256):
        l = int(o.code_len[s])
        if not l:
            continue
        lo = int(codes[s]) << (o.lmax - l)
        hi = (int(codes[s]) + 1) << (o.lmax - l)
        assert np.all(t[lo:hi] == (s | (l << 8)))
    assert np.all(t != 0)  # complete code: every prefix decodes


def test_incomplete_code_table_has_holes(L):
    _, d = od()
    cl = np.zeros(256, np.uint8)
    cl[128], cl[0] = 1, 2
    t = codec.decode_table(codec.Domain(**{**d.__dict__, "code_len": cl, "lmax": 4}))
    assert (t == 0).sum() == 4 and t[0] == (128 | 1 << 8)


@pytest.mark.parametrize("domain_id", [0, 1, 2, 3])
def test_trainer_matches_oracle(L, domain_id):
    ts = siggen.training_set(domain_id)
    flat, offs = siggen.signals(ts.domains, ts.seeds, ts.lengths)
    d = codec.train_domain(flat, offs, ts.lengths)
    o = oracle.trained_domain(domain_id)
    assert d.scale[0] == pytest.approx(o.A[0], rel=1e-12) and d.scale[1] == pytest.approx(o.A[1], rel=1e-12)
    np.testing.assert_array_equal(d.code_len, o.code_len)


def test_encoder_matches_oracle(L):
    # both sides quantize in FP64 with their own cosine arguments and summation
    # order; a level may differ only where the oracle's coefficient lies within
    # FP64 rounding of a level boundary
    wl = siggen.mixed_10000_logu(n=12, lo=1, hi=20000)
    for i in range(12):
        dom = int(wl.domains[i])
        o, d = od(dom)
        S = int(wl.lengths[i])
        x = siggen.signal(dom, int(wl.seeds[i]), S)
        w1, s1, l1 = codec.encode_stream(d, x)
        w2, s2, l2 = oracle.encode_stream(x, o)
        mism = np.flatnonzero(l1 != l2)
        assert mism.size <= max(1, l1.size // 100000)
        for m in mism:
            w, k = divmod(int(m), o.E)
            xw = np.zeros(o.N)
            seg = x[w * o.N:min(S, (w + 1) * o.N)].astype(np.float64)
            xw[:seg.size] = seg
            assert near_level_boundary(o, xw, k, int(l1[m])), (i, m)
        if mism.size == 0:
            np.testing.assert_array_equal(w1, w2)
            np.testing.assert_array_equal(s1, s2)


def test_encode_batch_matches_single(L):
    wl = siggen.mixed_10000_logu(n=20, lo=10, hi=30000)
    flat, offs = siggen.signals(wl.domains, wl.seeds, wl.lengths)
    doms = [od(i)[1] for i in range(4)]
    b = codec.encode_batch(doms, flat, offs, wl.lengths, wl.domains, n_threads=4)
    for i in range(20):
        x = flat[int(offs[i]):int(offs[i]) + int(wl.lengths[i])]
        w, s, _ = codec.encode_stream(doms[wl.domains[i]], x)
        sg = b.segments[i]
        a, n = int(sg["word_offset"]), int(sg["n_words"])
        np.testing.assert_array_equal(b.words[a:a + n], w)
        np.testing.assert_array_equal(b.symlen[a:a + n], s)
        assert int(sg["out_offset"]) % 4 == 0


def test_plan_rejects_bad_metadata_before_touching_a_gpu(L):
    import ctypes
    _, d = od()
    cds = codec.c_domains([d])
    h = ctypes.c_void_p()
    # too few words for the symbols (W*E = 2048*16 needs >= 512 words)
    segs = codec.segments_array([0], [10], [65536], [0], [0])
    st = L.fptc_plan_create(ctypes.byref(h), 0, cds, 1, segs.ctypes.data, 1, None)
    assert st == _lib.INVALID_ARGUMENT and not h.value
    # domain index out of range
    segs = codec.segments_array([0], [1000], [65536], [0], [3])
    assert L.fptc_plan_create(ctypes.byref(h), 0, cds, 1, segs.ctypes.data, 1, None) == _lib.INVALID_ARGUMENT
    # overlapping outputs
    segs = codec.segments_array([0, 1000], [1000, 1000], [65536, 65536], [0, 100], [0, 0])
    assert L.fptc_plan_create(ctypes.byref(h), 0, cds, 1, segs.ctypes.data, 2, None) == _lib.INVALID_ARGUMENT
    assert b"overlap" in L.fptc_last_error_message()
    # NULL plan handles are rejected, not dereferenced
    assert L.fptc_decode_batch(None, None, None, None, None, None, None) == _lib.INVALID_ARGUMENT


def test_encoder_rejects_bad_arguments_before_touching_a_gpu(L):
    import ctypes
    _, d = od()
    cds = codec.c_domains([d])
    h = ctypes.c_void_p()
    # rooms of two streams overlap
    segs = codec.segments_array([0, 5], [10, 10], [320, 320], [0, 320], [0, 0])
    assert L.fptc_encoder_create(ctypes.byref(h), 0, cds, 1, segs.ctypes.data, 2) == _lib.INVALID_ARGUMENT
    assert not h.value and b"overlap" in L.fptc_last_error_message()
    # domain index out of range
    segs = codec.segments_array([0], [10], [320], [0], [1])
    assert L.fptc_encoder_create(ctypes.byref(h), 0, cds, 1, segs.ctypes.data, 1) == _lib.INVALID_ARGUMENT
    assert b"domain" in L.fptc_last_error_message()
    # an invalid domain (E > N) is rejected by the domain validation
    bad = codec.Domain(8, 9, 1, 2, 50.0, 0.004, (1.0, 1.0, 0.0), 12, d.code_len.copy())
    segs = codec.segments_array([0], [10], [320], [0], [0])
    assert L.fptc_encoder_create(ctypes.byref(h), 0, codec.c_domains([bad]), 1, segs.ctypes.data, 1) \
        == _lib.INVALID_ARGUMENT
    # no handle pointer, no domains
    assert L.fptc_encoder_create(None, 0, cds, 1, segs.ctypes.data, 1) == _lib.INVALID_ARGUMENT
    assert L.fptc_encoder_create(ctypes.byref(h), 0, None, 0, segs.ctypes.data, 1) == _lib.INVALID_ARGUMENT
    # NULL encoders are rejected, not dereferenced
    assert L.fptc_encoder_levels(None) == 0
    assert L.fptc_encoder_level_offsets(None, None) == _lib.INVALID_ARGUMENT
    assert L.fptc_encode_device(None, None, None, None, None, None, None) == _lib.INVALID_ARGUMENT
    assert L.fptc_pack_device(None, None, None, None, None, None) == _lib.INVALID_ARGUMENT
    assert L.fptc_encoder_status(None, None, None) == _lib.INVALID_ARGUMENT
    L.fptc_encoder_destroy(None)


@pytest.mark.parametrize("lmax,lengths", [(16, "max"), (8, "uniform"), (12, "trained"), (4, "one_bit")])
def test_word_capacity_bounds_alg1(L, lmax, lengths):
    """fptc_word_capacity (the room the encoders reserve) is at least the number
    of words Alg. 1 produces, for the worst code lengths (every codeword lmax
    bits) and for ordinary ones, at ragged stream lengths."""
    rng = np.random.default_rng(lmax)
    cl = np.zeros(256, np.uint8)
    if lengths == "max":
        cl[:128], cl[128:] = 8, lmax
        pool = np.arange(128, 256)
    elif lengths == "uniform":
        cl[:] = 8
        pool = np.arange(256)
    elif lengths == "trained":
        cl = od(1)[0].code_len.copy()
        pool = np.flatnonzero(cl)
    else:
        cl[128], cl[0] = 1, 1
        pool = np.array([0, 128])
    o = oracle.Domain(32, 16, 2, 16, 50.0, 0.004, (1.0, 1.0, 0.0), lmax, cl)
    d = codec.Domain(o.N, o.E, o.B1, o.B2, o.mu, o.alpha1, o.A, o.lmax, o.code_len)
    codes = oracle.canonical_codes(cl, lmax)
    for S in (1, 31, 32, 33, 1000, 4097, 65536):
        X = rng.choice(pool, size=o.windows(S) * o.E).astype(np.uint8)
        words, _ = oracle.pack_symlen(X, codes, cl)
        assert words.size <= codec.word_capacity(d, S), (S, words.size)


def test_near_level_boundary_helper():
    # The rule the encoder tests apply to a level that differs from the oracle's:
    # a window whose bin-3 (zone 1) coefficient sits exactly on the boundary
    # between levels 150 and 151 passes for both; the same window moved to the
    # middle of level 150's cell passes for neither, nor does a level two away.
    o = oracle.Domain(32, 16, 2, 16, 50.0, 0.004, (3.0, 2.0, 0.0), 12)
    A1, d1 = 2.0, 0.004 * 2.0
    n = np.arange(32)
    basis3 = np.cos(np.pi / 32 * (n + 0.5) * 3)
    # Eq. 3: L = 129 + floor((c - d1) / (A1 - d1) * 126 + 1/2) for c > d1
    x_edge = (d1 + 21.5 / 126 * (A1 - d1)) * basis3
    assert oracle.quantize(o, 1, float(oracle.dct2(x_edge, 32, 16)[3])) in (150, 151)
    assert near_level_boundary(o, x_edge, 3, 150) and near_level_boundary(o, x_edge, 3, 151)
    x_mid = (d1 + 21.0 / 126 * (A1 - d1)) * basis3
    assert oracle.quantize(o, 1, float(oracle.dct2(x_mid, 32, 16)[3])) == 150
    assert not near_level_boundary(o, x_mid, 3, 150)
    assert not near_level_boundary(o, x_mid, 3, 151)
    assert not near_level_boundary(o, x_edge, 3, 152)
