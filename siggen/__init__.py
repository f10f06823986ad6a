"""Seeded synthetic signals standing in for the paper's four signal domains.

The paper evaluates on ten real datasets in four domains (Sec. 5.2, Table 2):
biomedical (ECG/EEG), seismic traces, power-grid telemetry and meteorological
series.  None of them is available here, so every input is generated from a
seed by ``siggen.c`` with the shapes the paper describes.  This module holds
none of the codec's arithmetic; it is the one piece of code shared by the FP64
oracle (tests) and the benchmark.

Workloads (all float32 samples):

* ``eeg_1x65536``        -- one EEG-like channel, 65,536 samples (id 0)
* ``eeg_2048x1m``        -- 2048 EEG-like channels x 1,048,576 samples (id 1)
* ``mixed_10000_logu``   -- 10,000 signals, lengths log-uniform in [4096, 4194304],
                            2,500 per domain in shuffled order (id 2)
* ``seismic_16384x4096`` -- 16,384 seismic traces x 4,096 samples (id 3)
* ``power_1024x65536``   -- 1,024 power-grid series x 65,536 samples (id 4)
* training sets          -- per domain d, 32 signals x 65,536 samples (id 100+d),
                            disjoint from every evaluation seed
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "siggen.c")
_SO = os.path.join(_HERE, "libsiggen.so")

EEG, SEISMIC, POWER, MET = 0, 1, 2, 3
DOMAIN_NAMES = ("eeg", "seismic", "power", "met")

_u64 = ctypes.c_uint64
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile libsiggen.so next to its source (plain gcc, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib_handle = None


def _lib():
    global _lib_handle
    if _lib_handle is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.sg_splitmix64.restype = _u64
        lib.sg_splitmix64.argtypes = [_u64]
        lib.sg_stream_seed.restype = _u64
        lib.sg_stream_seed.argtypes = [ctypes.c_uint32, _u64]
        lib.sg_signal.restype = ctypes.c_int
        lib.sg_signal.argtypes = [ctypes.c_int, _u64, _p, _u64]
        lib.sg_signal_many.restype = ctypes.c_int
        lib.sg_signal_many.argtypes = [_p, _p, _p, _p, _u64, _p, ctypes.c_int]
        lib.sg_mixed_layout.restype = None
        lib.sg_mixed_layout.argtypes = [_u64, _u64, _u64, _u64, _p, _p]
        lib.sg_rng_fill_u64.restype = None
        lib.sg_rng_fill_u64.argtypes = [_u64, _p, _u64]
        lib.sg_rng_fill_normal.restype = None
        lib.sg_rng_fill_normal.argtypes = [_u64, _p, _u64]
        _lib_handle = lib
    return _lib_handle


def splitmix64(x: int) -> int:
    return int(_lib().sg_splitmix64(x))


def stream_seed(workload_id: int, index: int) -> int:
    """Seed of stream ``index`` of workload ``workload_id``: splitmix64(0xF97C0000 + 1000003*id + index)."""
    return int(_lib().sg_stream_seed(workload_id, index))


def rng_u64(seed: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint64)
    _lib().sg_rng_fill_u64(seed, out.ctypes.data, n)
    return out


def rng_normal(seed: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _lib().sg_rng_fill_normal(seed, out.ctypes.data, n)
    return out


def signal(domain: int, seed: int, n_samples: int) -> np.ndarray:
    x = np.empty(n_samples, dtype=np.float32)
    if _lib().sg_signal(domain, seed, x.ctypes.data, n_samples) != 0:
        raise ValueError(f"unknown domain {domain}")
    return x


def signals_into(out: np.ndarray, offsets, domains, seeds, lengths, n_threads: int = 0) -> None:
    """Generate many signals in parallel into ``out`` (float32) at ``offsets``."""
    domains = np.ascontiguousarray(domains, dtype=np.int32)
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint64)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    assert out.dtype == np.float32 and out.flags.c_contiguous
    if len(lengths) and int((offsets + lengths).max()) > out.size:
        raise ValueError("output buffer too small")
    if n_threads <= 0:
        n_threads = os.cpu_count() or 1
    rc = _lib().sg_signal_many(domains.ctypes.data, seeds.ctypes.data, lengths.ctypes.data,
                               offsets.ctypes.data, len(lengths), out.ctypes.data, n_threads)
    if rc != 0:
        raise ValueError("unknown domain id in batch")


def signals(domains, seeds, lengths, n_threads: int = 0):
    """Generate a batch; returns (flat float32 array, offsets)."""
    lengths = np.ascontiguousarray(lengths, dtype=np.uint64)
    offsets = np.zeros(len(lengths), dtype=np.uint64)
    if len(lengths) > 1:
        offsets[1:] = np.cumsum(lengths[:-1])
    out = np.empty(int(lengths.sum()), dtype=np.float32)
    signals_into(out, offsets, domains, seeds, lengths, n_threads)
    return out, offsets


def mixed_layout(seed: int, n: int, lo: int, hi: int):
    lengths = np.empty(n, dtype=np.uint64)
    domains = np.empty(n, dtype=np.int32)
    _lib().sg_mixed_layout(seed, n, lo, hi, lengths.ctypes.data, domains.ctypes.data)
    return lengths, domains


@dataclass
class Workload:
    name: str
    workload_id: int
    domains: np.ndarray  # int32 [n]
    seeds: np.ndarray    # uint64 [n]
    lengths: np.ndarray  # uint64 [n]

    @property
    def n_streams(self) -> int:
        return len(self.lengths)

    @property
    def n_samples(self) -> int:
        return int(self.lengths.sum())

    def subset(self, idx) -> "Workload":
        idx = np.asarray(idx)
        return Workload(self.name + "[subset]", self.workload_id, self.domains[idx], self.seeds[idx],
                        self.lengths[idx])


def _uniform(name, wid, domain, n, S):
    seeds = np.array([stream_seed(wid, i) for i in range(n)], dtype=np.uint64)
    return Workload(name, wid, np.full(n, domain, np.int32), seeds, np.full(n, S, np.uint64))


def eeg_1x65536() -> Workload:
    return _uniform("eeg_1x65536", 0, EEG, 1, 65536)


def eeg_2048x1m(n: int = 2048, S: int = 1 << 20) -> Workload:
    return _uniform(f"eeg_{n}x{S}", 1, EEG, n, S)


MIXED_LAYOUT_INDEX = 1_000_000  # seed index of the layout draw, disjoint from stream indices


def mixed_10000_logu(n: int = 10000, lo: int = 4096, hi: int = 4194304) -> Workload:
    lengths, domains = mixed_layout(stream_seed(2, MIXED_LAYOUT_INDEX), n, lo, hi)
    seeds = np.array([stream_seed(2, i) for i in range(n)], dtype=np.uint64)
    return Workload(f"mixed_{n}_logu_{lo}_{hi}", 2, domains, seeds, lengths)


def seismic_16384x4096(n: int = 16384, S: int = 4096) -> Workload:
    return _uniform(f"seismic_{n}x{S}", 3, SEISMIC, n, S)


def power_1024x65536(n: int = 1024, S: int = 65536) -> Workload:
    return _uniform(f"power_{n}x{S}", 4, POWER, n, S)


def training_set(domain: int, n: int = 32, S: int = 65536) -> Workload:
    return _uniform(f"train_{DOMAIN_NAMES[domain]}_{n}x{S}", 100 + domain, domain, n, S)
