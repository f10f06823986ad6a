"""FP64 CPU oracle of the FPTC codec -- TEST INFRASTRUCTURE, not the product.

Python binding (ctypes) of ``fptc_oracle.c``: the sequential encoder (Sec. 3.1-3.3,
Sec. 4.1, Alg. 1) and a plain decoder (bit-serial canonical Huffman, FP64
inverse transform), plus the analytic adjoint used to check the decoder's
gradients.  It shares no code with the CUDA path.  Only ``tests/``,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may use it.
"""
from __future__ import annotations

import ctypes
import functools
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fptc_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")

_u64, _i64, _i32, _p, _d = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_double

ERRORS = {0: "ok", -1: "bad argument", -2: "symbol without code", -3: "capacity", -4: "bit overrun",
          -5: "invalid code", -6: "symbol count mismatch", -7: "out of memory"}


class OracleError(RuntimeError):
    pass


class COrDomain(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("E", ctypes.c_int32), ("B1", ctypes.c_int32), ("B2", ctypes.c_int32),
                ("mu", ctypes.c_double), ("alpha1", ctypes.c_double), ("A", ctypes.c_double * 3),
                ("lmax", ctypes.c_int32), ("code_len", ctypes.c_uint8 * 256)]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (plain gcc, OpenMP over streams)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


@functools.lru_cache(maxsize=None)
def lib():
    build()
    L = ctypes.CDLL(_SO)
    sig = {
        "or_basis": (_d, [_i32, _i32, _i32]),
        "or_dct2": (None, [_p, _i32, _i32, _p]),
        "or_idct3": (None, [_p, _i32, _i32, _p]),
        "or_zone": (_i32, [_p, _i32]),
        "or_quantize": (_i32, [_p, _i32, _d]),
        "or_dequantize": (_d, [_p, _i32, _i32]),
        "or_dequantize_unit": (_d, [_p, _i32, _i32]),
        "or_percentile": (_d, [_p, _u64, _d]),
        "or_package_merge": (_i32, [_p, _i32, _i32, _p]),
        "or_canonical_codes": (_i32, [_p, _i32, _i32, _p]),
        "or_pack_symlen": (_i64, [_p, _u64, _p, _p, _p, _p, _u64]),
        "or_unpack_symlen": (_i32, [_p, _p, _u64, _p, _i32, _p, _u64]),
        "or_quantize_stream": (_i32, [_p, _u64, _p, _p]),
        "or_encode_stream": (_i32, [_p, _u64, _p, _p, _p, _u64, _p, _p]),
        "or_reconstruct": (_i32, [_p, _u64, _p, _p]),
        "or_decode_stream": (_i32, [_p, _p, _u64, _u64, _p, _p, _p]),
        "or_backward_stream": (_i32, [_p, _u64, _p, _p, _p, _p]),
        "or_train_domain": (_i32, [_p, _p, _p, _i32, _d, _p]),
        "or_encode_many": (_i32, [_p, _p, _p, _p, _p, _u64, _p, _p, _p, _p, _p, _i32]),
        "or_decode_many": (_i32, [_p, _p, _p, _p, _p, _p, _p, _u64, _p, _p, _p, _p, _i32]),
        "or_domain_size": (_u64, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    assert L.or_domain_size() == ctypes.sizeof(COrDomain), "or_domain layout mismatch"
    return L


def _check(rc):
    if rc != 0:
        raise OracleError(ERRORS.get(int(rc), str(rc)))


def _ptr(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data


# Table 1 typical values (DCT_SIZE, ENCODED_COEFFS, HYBRID_BOUNDARY_1/2, MU_COMPANDING,
# DEAD_RATIO_ZONE1, ZONE_PERCENTILE); L_max is not given by the paper: 12 is this codec's default.
TABLE1 = dict(N=32, E=16, B1=2, B2=16, mu=50.0, alpha1=0.004, percentile=99.9, lmax=12)


@dataclass
class Domain:
    """Per-domain parameters and prebuilt structures (Table 1; Fig. 4)."""
    N: int = 32
    E: int = 16
    B1: int = 2
    B2: int = 16
    mu: float = 50.0
    alpha1: float = 0.004
    A: tuple = (0.0, 0.0, 0.0)
    lmax: int = 12
    code_len: np.ndarray = field(default_factory=lambda: np.zeros(256, np.uint8))

    def c(self) -> COrDomain:
        d = COrDomain()
        d.N, d.E, d.B1, d.B2 = self.N, self.E, self.B1, self.B2
        d.mu, d.alpha1, d.lmax = self.mu, self.alpha1, self.lmax
        for i in range(3):
            d.A[i] = float(self.A[i])
        cl = np.ascontiguousarray(self.code_len, dtype=np.uint8)
        ctypes.memmove(d.code_len, cl.ctypes.data, 256)
        return d

    @staticmethod
    def from_c(d: COrDomain) -> "Domain":
        return Domain(d.N, d.E, d.B1, d.B2, d.mu, d.alpha1, tuple(d.A), d.lmax,
                      np.frombuffer(bytes(d.code_len), dtype=np.uint8).copy())

    def windows(self, S: int) -> int:
        return (S + self.N - 1) // self.N

    def zone(self, k: int) -> int:
        return 0 if k < self.B1 else (1 if k < self.B2 else 2)


# ---- Eq. 1 and its inverse -------------------------------------------------

def basis(N: int, n: int, k: int) -> float:
    return lib().or_basis(N, n, k)


def dct2(x, N: int, E: int) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    assert x.size == N
    C = np.empty(E, np.float64)
    lib().or_dct2(_ptr(x), N, E, _ptr(C))
    return C


def idct3(C, N: int) -> np.ndarray:
    C = np.ascontiguousarray(C, dtype=np.float64)
    x = np.empty(N, np.float64)
    lib().or_idct3(_ptr(C), C.size, N, _ptr(x))
    return x


# ---- Sec. 3.2 quantizer --------------------------------------------------------

def quantize(d: Domain, zone: int, c: float) -> int:
    cd = d.c()
    return int(lib().or_quantize(ctypes.byref(cd), zone, float(c)))


def dequantize(d: Domain, zone: int, L: int) -> float:
    cd = d.c()
    return float(lib().or_dequantize(ctypes.byref(cd), zone, int(L)))


def dequantize_unit(d: Domain, zone: int, L: int) -> float:
    cd = d.c()
    return float(lib().or_dequantize_unit(ctypes.byref(cd), zone, int(L)))


def percentile(values, p: float) -> float:
    v = np.array(values, dtype=np.float64, copy=True)
    return float(lib().or_percentile(_ptr(v), v.size, p))


# ---- Sec. 3.3 codebook ----------------------------------------------------------

def package_merge(freq, lmax: int) -> np.ndarray:
    f = np.ascontiguousarray(freq, dtype=np.uint64)
    out = np.zeros(f.size, np.uint8)
    _check(lib().or_package_merge(_ptr(f), f.size, lmax, _ptr(out)))
    return out


def canonical_codes(lengths, lmax: int) -> np.ndarray:
    ln = np.ascontiguousarray(lengths, dtype=np.uint8)
    out = np.zeros(ln.size, np.uint32)
    _check(lib().or_canonical_codes(_ptr(ln), ln.size, lmax, _ptr(out)))
    return out


# ---- Alg. 1 ----------------------------------------------------------------------

def pack_symlen(X, codes, lengths):
    X = np.ascontiguousarray(X, dtype=np.uint8)
    codes = np.ascontiguousarray(codes, dtype=np.uint32)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
    cap = max(1, X.size)
    words = np.zeros(cap, np.uint64)
    symlen = np.zeros(cap, np.uint8)
    n = lib().or_pack_symlen(_ptr(X), X.size, _ptr(codes), _ptr(lengths), _ptr(words), _ptr(symlen), cap)
    if n < 0:
        _check(n)
    return words[:n].copy(), symlen[:n].copy()


def unpack_symlen(words, symlen, lengths, lmax: int, L: int) -> np.ndarray:
    words = np.ascontiguousarray(words, dtype=np.uint64)
    symlen = np.ascontiguousarray(symlen, dtype=np.uint8)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
    X = np.zeros(max(L, 1), np.uint8)
    _check(lib().or_unpack_symlen(_ptr(words), _ptr(symlen), words.size, _ptr(lengths), lmax, _ptr(X), L))
    return X[:L]


# ---- streams ------------------------------------------------------------------------

def word_capacity(d: Domain, S: int) -> int:
    """Upper bound on words per stream: every word but the last holds at least
    ceil((65 - lmax) / lmax) codewords (Alg. 1 closes a word only when the next
    codeword does not fit)."""
    L = d.windows(S) * d.E
    per = max(1, -(-(65 - d.lmax) // d.lmax))
    return L // per + 2


def quantize_stream(x, d: Domain) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    lv = np.zeros(max(1, d.windows(x.size) * d.E), np.uint8)
    cd = d.c()
    _check(lib().or_quantize_stream(_ptr(x), x.size, ctypes.byref(cd), _ptr(lv)))
    return lv[:d.windows(x.size) * d.E]


def encode_stream(x, d: Domain):
    """Returns (words uint64, symlen uint8, levels uint8[W*E])."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    cap = word_capacity(d, x.size)
    words = np.zeros(cap, np.uint64)
    symlen = np.zeros(cap, np.uint8)
    lv = np.zeros(max(1, d.windows(x.size) * d.E), np.uint8)
    nw = ctypes.c_uint64(0)
    cd = d.c()
    _check(lib().or_encode_stream(_ptr(x), x.size, ctypes.byref(cd), _ptr(words), _ptr(symlen), cap,
                                  ctypes.byref(nw), _ptr(lv)))
    n = nw.value
    return words[:n].copy(), symlen[:n].copy(), lv[:d.windows(x.size) * d.E]


def reconstruct(levels, S: int, d: Domain) -> np.ndarray:
    levels = np.ascontiguousarray(levels, dtype=np.uint8)
    out = np.zeros(S, np.float64)
    cd = d.c()
    _check(lib().or_reconstruct(_ptr(levels), S, ctypes.byref(cd), _ptr(out)))
    return out


def decode_stream(words, symlen, S: int, d: Domain):
    """Returns (samples float64[S], levels uint8[W*E])."""
    words = np.ascontiguousarray(words, dtype=np.uint64)
    symlen = np.ascontiguousarray(symlen, dtype=np.uint8)
    out = np.zeros(max(S, 1), np.float64)
    lv = np.zeros(max(1, d.windows(S) * d.E), np.uint8)
    cd = d.c()
    _check(lib().or_decode_stream(_ptr(words), _ptr(symlen), words.size, S, ctypes.byref(cd), _ptr(out), _ptr(lv)))
    return out[:S], lv[:d.windows(S) * d.E]


def backward_stream(levels, S: int, d: Domain, g_x):
    """Adjoint of the reconstruction: returns (g_C float64[W*E], grad_A float64[3])."""
    levels = np.ascontiguousarray(levels, dtype=np.uint8)
    g_x = np.ascontiguousarray(g_x, dtype=np.float64)
    assert g_x.size == S
    gC = np.zeros(max(1, d.windows(S) * d.E), np.float64)
    gA = np.zeros(3, np.float64)
    cd = d.c()
    _check(lib().or_backward_stream(_ptr(levels), S, ctypes.byref(cd), _ptr(g_x), _ptr(gC), _ptr(gA)))
    return gC[:d.windows(S) * d.E], gA


def train_domain(signals_flat, offsets, lengths, template: Domain, percentile_: float = 99.9) -> Domain:
    x = np.ascontiguousarray(signals_flat, dtype=np.float32)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint64)
    cd = template.c()
    _check(lib().or_train_domain(_ptr(x), _ptr(offsets), _ptr(lengths), len(lengths), percentile_, ctypes.byref(cd)))
    return Domain.from_c(cd)


@functools.lru_cache(maxsize=None)
def trained_domain(domain_id: int, N: int = 32, E: int = 16, B1: int = 2, B2: int = 16, mu: float = 50.0,
                   alpha1: float = 0.004, lmax: int = 12, percentile_: float = 99.9) -> Domain:
    """Prebuilt structures of one signal domain, trained on its disjoint training set."""
    import siggen
    ts = siggen.training_set(domain_id)
    flat, offs = siggen.signals(ts.domains, ts.seeds, ts.lengths)
    return train_domain(flat, offs, ts.lengths, Domain(N, E, B1, B2, mu, alpha1, (0, 0, 0), lmax), percentile_)


# ---- batches -------------------------------------------------------------------------

@dataclass
class EncodedBatch:
    """Concatenated words/symlen of many streams plus per-stream metadata."""
    words: np.ndarray      # uint64 [total_words]
    symlen: np.ndarray     # uint8  [total_words]
    word_off: np.ndarray   # uint64 [n]
    n_words: np.ndarray    # uint64 [n]
    lengths: np.ndarray    # uint64 [n]  samples per stream
    domain_idx: np.ndarray  # int32 [n] index into domains
    domains: list          # list[Domain]

    @property
    def n_streams(self):
        return len(self.lengths)


def _cdomains(domains):
    arr = (COrDomain * max(1, len(domains)))()
    for i, d in enumerate(domains):
        arr[i] = d.c()
    return arr


def encode_many(x_flat, x_off, lengths, domain_idx, domains, n_threads: int = 0) -> EncodedBatch:
    x_flat = np.ascontiguousarray(x_flat, dtype=np.float32)
    x_off = np.ascontiguousarray(x_off, dtype=np.uint64)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint64)
    domain_idx = np.ascontiguousarray(domain_idx, dtype=np.int32)
    n = len(lengths)
    cap = np.array([word_capacity(domains[domain_idx[i]], int(lengths[i])) for i in range(n)], dtype=np.uint64)
    cap_off = np.zeros(n, np.uint64)
    if n > 1:
        cap_off[1:] = np.cumsum(cap[:-1])
    total = int(cap.sum()) if n else 0
    words = np.zeros(max(total, 1), np.uint64)
    symlen = np.zeros(max(total, 1), np.uint8)
    nw = np.zeros(max(n, 1), np.uint64)
    if n_threads <= 0:
        n_threads = os.cpu_count() or 1
    cd = _cdomains(domains)
    _check(lib().or_encode_many(_ptr(x_flat), _ptr(x_off), _ptr(lengths), _ptr(domain_idx), cd, n, _ptr(words),
                                _ptr(symlen), _ptr(cap_off), _ptr(cap), _ptr(nw), n_threads))
    nw = nw[:n]
    word_off = np.zeros(n, np.uint64)
    if n > 1:
        word_off[1:] = np.cumsum(nw[:-1])
    tot = int(nw.sum()) if n else 0
    out_w = np.empty(tot, np.uint64)
    out_s = np.empty(tot, np.uint8)
    for i in range(n):
        a, b, c = int(cap_off[i]), int(nw[i]), int(word_off[i])
        out_w[c:c + b] = words[a:a + b]
        out_s[c:c + b] = symlen[a:a + b]
    return EncodedBatch(out_w, out_s, word_off, nw.copy(), lengths.copy(), domain_idx.copy(), list(domains))


def decode_many(batch: EncodedBatch, idx=None, n_threads: int = 0, want_levels: bool = False):
    """Decode the streams ``idx`` (default all).  Returns (samples float64 flat, out_off, levels, lv_off)."""
    if idx is None:
        idx = np.arange(batch.n_streams)
    idx = np.asarray(idx, dtype=np.int64)
    S = np.ascontiguousarray(batch.lengths[idx], dtype=np.uint64)
    w_off = np.ascontiguousarray(batch.word_off[idx], dtype=np.uint64)
    n_words = np.ascontiguousarray(batch.n_words[idx], dtype=np.uint64)
    dom = np.ascontiguousarray(batch.domain_idx[idx], dtype=np.int32)
    out_off = np.zeros(len(idx), np.uint64)
    if len(idx) > 1:
        out_off[1:] = np.cumsum(S[:-1])
    x = np.zeros(max(1, int(S.sum())), np.float64)
    W = np.array([batch.domains[dom[i]].windows(int(S[i])) * batch.domains[dom[i]].E for i in range(len(idx))],
                 dtype=np.uint64)
    lv_off = np.zeros(len(idx), np.uint64)
    if len(idx) > 1:
        lv_off[1:] = np.cumsum(W[:-1])
    lv = np.zeros(max(1, int(W.sum())), np.uint8) if want_levels else None
    if n_threads <= 0:
        n_threads = os.cpu_count() or 1
    cd = _cdomains(batch.domains)
    _check(lib().or_decode_many(_ptr(batch.words), _ptr(batch.symlen), _ptr(w_off), _ptr(n_words), _ptr(S), _ptr(dom),
                                cd, len(idx), _ptr(x), _ptr(out_off), _ptr(lv) if lv is not None else None,
                                _ptr(lv_off), n_threads))
    return x, out_off, lv, lv_off


# ---- decoder-side scales at a fixed rate ---------------------------------------------

def fit_zone_scales(levels_list, lengths, domain_idx, domains, x_list) -> np.ndarray:
    """The per-zone scales A_z of every domain that minimise the squared error
    sum_i ||x_i - x_hat_i(A)||^2 over the given streams, their levels (hence
    their bit rate) fixed.  Every dequantized coefficient is A_z times a
    function of its level (Sec. 3.2, Eq. 2 and Eq. 3 inverted), so x_hat is
    linear in A: x_hat = sum_z A_z u_z, u_z the reconstruction with A_z = 1 and
    the other zones 0, and the minimiser solves the normal equations
    G A = b, G_yz = sum <u_y, u_z>, b_z = sum <u_z, x>, per domain (FP64).
    Zones a domain does not use (no bin in them) keep their scale.  Returns
    float64 [n_domains, 3]."""
    out = np.array([np.asarray(d.A, np.float64) for d in domains])
    for di, d in enumerate(domains):
        zones = [z for z in (0, 1) if (z == 0 and d.B1 > 0) or (z == 1 and d.B2 > d.B1)]
        if not zones:
            continue
        units = [Domain(d.N, d.E, d.B1, d.B2, d.mu, d.alpha1, tuple(1.0 if q == z else 0.0 for q in range(3)),
                        d.lmax, d.code_len) for z in zones]
        G = np.zeros((len(zones), len(zones)))
        b = np.zeros(len(zones))
        seen = False
        for lv, S, k, x in zip(levels_list, lengths, domain_idx, x_list):
            if k != di or S == 0:
                continue
            seen = True
            u = [reconstruct(lv, int(S), ud) for ud in units]
            xx = np.asarray(x, np.float64)
            for i in range(len(zones)):
                b[i] += float(np.dot(u[i], xx))
                for j in range(len(zones)):
                    G[i, j] += float(np.dot(u[i], u[j]))
        if not seen:
            continue
        sol = np.linalg.solve(G, b)
        for i, z in enumerate(zones):
            out[di, z] = sol[i]
    return out


# ---- metrics (Sec. 5.1) ---------------------------------------------------------------

def prd(x, x_hat) -> float:
    """Eq. 5: 100 * sqrt(sum (x - x_hat)^2 / sum x^2)."""
    x = np.asarray(x, np.float64)
    x_hat = np.asarray(x_hat, np.float64)
    return float(100.0 * np.sqrt(np.sum((x - x_hat) ** 2) / np.sum(x ** 2)))


STREAM_HEADER_BYTES = 16  # per-stream header (sample count, word count) counted in S_comp


def compression_ratio(n_samples: int, n_words: int) -> float:
    """Eq. 4 with S_orig = 4 bytes per sample and S_comp = 8 B per word + 1 B symlen + header."""
    return 4.0 * n_samples / (9.0 * n_words + STREAM_HEADER_BYTES)
