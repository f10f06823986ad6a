"""Host-side codec calls of libfptc (include/fptc_codec.h): per-domain prebuilt
structures (Sec. 3.3, Fig. 4) and the sequential encoder (Sec. 4.1, Alg. 1)."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np

from . import _lib
from ._lib import CDomain, CSegment, check, lib


def _ptr(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data


@dataclass
class Domain:
    """Table 1 parameters of one signal domain plus its prebuilt structures."""
    N: int = 32
    E: int = 16
    B1: int = 2
    B2: int = 16
    mu: float = 50.0
    alpha1: float = 0.004
    scale: tuple = (0.0, 0.0, 0.0)  # A_0, A_1, A_2
    lmax: int = 12
    code_len: np.ndarray = field(default_factory=lambda: np.zeros(256, np.uint8))

    def c(self) -> CDomain:
        d = CDomain()
        d.N, d.E, d.B1, d.B2, d.lmax = self.N, self.E, self.B1, self.B2, self.lmax
        d.mu, d.alpha1 = float(self.mu), float(self.alpha1)
        for i in range(3):
            d.scale[i] = float(self.scale[i])
        cl = np.ascontiguousarray(self.code_len, dtype=np.uint8)
        assert cl.size == 256
        ctypes.memmove(d.code_len, cl.ctypes.data, 256)
        return d

    @staticmethod
    def from_c(d: CDomain) -> "Domain":
        return Domain(d.N, d.E, d.B1, d.B2, d.mu, d.alpha1, tuple(d.scale), d.lmax,
                      np.frombuffer(bytes(d.code_len), dtype=np.uint8).copy())

    def windows(self, n_samples: int) -> int:
        return (int(n_samples) + self.N - 1) // self.N


def c_domains(domains):
    arr = (CDomain * max(1, len(domains)))()
    for i, d in enumerate(domains):
        arr[i] = d.c()
    return arr


def validate_domain(d: Domain) -> None:
    cd = d.c()
    check(lib().fptc_validate_domain(ctypes.byref(cd)))


def decode_table(d: Domain) -> np.ndarray:
    """2^lmax uint16 entries: level | code length << 8 (0 where no codeword matches)."""
    cd = d.c()
    t = np.zeros(1 << d.lmax, np.uint16)
    check(lib().fptc_build_decode_table(ctypes.byref(cd), _ptr(t)))
    return t


def canonical_codes(d: Domain) -> np.ndarray:
    cd = d.c()
    c = np.zeros(256, np.uint32)
    check(lib().fptc_canonical_codes(ctypes.byref(cd), _ptr(c)))
    return c


def train_domain(x_flat, offsets, lengths, N=32, E=16, B1=2, B2=16, mu=50.0, alpha1=0.004, lmax=12,
                 percentile=99.9) -> Domain:
    x = np.ascontiguousarray(x_flat, dtype=np.float32)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint64)
    cd = Domain(N, E, B1, B2, mu, alpha1, (0.0, 0.0, 0.0), lmax).c()
    check(lib().fptc_train_domain(_ptr(x), _ptr(offsets), _ptr(lengths), len(lengths), float(percentile),
                                  ctypes.byref(cd)))
    return Domain.from_c(cd)


def zone_bounds(d: Domain, zone: int) -> np.ndarray:
    """The host encoder's level map of zone 0 or 1 as its 255 boundaries
    (include/fptc_codec.h fptc_zone_bounds): level(c) = #{bounds <= c}."""
    cd = d.c()
    b = np.zeros(255, np.float64)
    check(lib().fptc_zone_bounds(ctypes.byref(cd), int(zone), _ptr(b)))
    return b


def word_capacity(d: Domain, n_samples: int) -> int:
    cd = d.c()
    return int(lib().fptc_word_capacity(ctypes.byref(cd), int(n_samples)))


def encode_stream(d: Domain, x):
    """Returns (words uint64, symlen uint8, levels uint8[W*E])."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    cap = word_capacity(d, x.size)
    words = np.zeros(max(cap, 1), np.uint64)
    symlen = np.zeros(max(cap, 1), np.uint8)
    lv = np.zeros(max(1, d.windows(x.size) * d.E), np.uint8)
    n = ctypes.c_uint64(0)
    cd = d.c()
    check(lib().fptc_encode_stream(ctypes.byref(cd), _ptr(x), x.size, _ptr(words), _ptr(symlen), cap,
                                   ctypes.byref(n), _ptr(lv)))
    k = n.value
    return words[:k].copy(), symlen[:k].copy(), lv[:d.windows(x.size) * d.E]


@dataclass
class Batch:
    """Concatenated compressed streams plus their segment table (host memory)."""
    words: np.ndarray        # uint64 [total words]
    symlen: np.ndarray       # uint8  [total words]
    segments: np.ndarray     # structured: word_offset, n_words, n_samples, out_offset, domain
    domains: list

    @property
    def n_samples(self) -> int:
        return int(self.segments["n_samples"].sum())


SEGMENT_DTYPE = np.dtype([("word_offset", "<u8"), ("n_words", "<u8"), ("n_samples", "<u8"), ("out_offset", "<u8"),
                          ("domain", "<u4"), ("reserved", "<u4")])
assert SEGMENT_DTYPE.itemsize == ctypes.sizeof(CSegment)


def segments_array(word_offset, n_words, n_samples, out_offset, domain) -> np.ndarray:
    n = len(n_words)
    s = np.zeros(n, SEGMENT_DTYPE)
    s["word_offset"], s["n_words"], s["n_samples"] = word_offset, n_words, n_samples
    s["out_offset"], s["domain"] = out_offset, domain
    return s


def packed_out_offsets(n_samples, align: int = 32) -> np.ndarray:
    """Output offsets of consecutive segments, each rounded up to `align` floats (32: 128 bytes,
    the alignment at which the warp-tile kernel stores whole 32-window tiles with the TMA unit;
    8 floats still allow its 32-byte stores)."""
    n_samples = np.asarray(n_samples, dtype=np.uint64)
    padded = (n_samples + np.uint64(align - 1)) // np.uint64(align) * np.uint64(align)
    off = np.zeros(len(n_samples), np.uint64)
    if len(n_samples) > 1:
        off[1:] = np.cumsum(padded[:-1])
    return off


def encode_batch(domains, x_flat, x_offsets, lengths, domain_idx, n_threads: int = 0, out_align: int = 32) -> Batch:
    """Encodes many signals on the host threads; output offsets packed with `out_align` floats alignment."""
    x = np.ascontiguousarray(x_flat, dtype=np.float32)
    x_offsets = np.ascontiguousarray(x_offsets, dtype=np.uint64)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint64)
    domain_idx = np.ascontiguousarray(domain_idx, dtype=np.uint32)
    n = len(lengths)
    cap = np.array([word_capacity(domains[domain_idx[i]], int(lengths[i])) for i in range(n)], dtype=np.uint64)
    cap_off = np.zeros(n, np.uint64)
    if n > 1:
        cap_off[1:] = np.cumsum(cap[:-1])
    tot = int(cap.sum()) if n else 0
    words = np.zeros(max(tot, 1), np.uint64)
    symlen = np.zeros(max(tot, 1), np.uint8)
    nw = np.zeros(max(n, 1), np.uint64)
    cds = c_domains(domains)
    check(lib().fptc_encode_batch(cds, len(domains), _ptr(x), _ptr(x_offsets), _ptr(lengths), _ptr(domain_idx), n,
                                  _ptr(words), _ptr(symlen), _ptr(cap_off), _ptr(nw), int(n_threads)))
    nw = nw[:n]
    woff = np.zeros(n, np.uint64)
    if n > 1:
        woff[1:] = np.cumsum(nw[:-1])
    total = int(nw.sum()) if n else 0
    # compact: gather each stream's words (vectorised index build)
    if total:
        idx = np.repeat(cap_off - woff, nw.astype(np.int64)) + np.arange(total, dtype=np.uint64)
        out_w = words[idx]
        out_s = symlen[idx]
    else:
        out_w = np.zeros(0, np.uint64)
        out_s = np.zeros(0, np.uint8)
    segs = segments_array(woff, nw, lengths, packed_out_offsets(lengths, out_align), domain_idx)
    return Batch(out_w, out_s, segs, list(domains))
