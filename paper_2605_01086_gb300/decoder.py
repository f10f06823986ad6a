"""The GPU batch decoder (include/fptc.h) as a PyTorch-facing API.

PyTorch supplies device memory, the current CUDA stream and autograd; every
step of the decode runs in libfptc's CUDA kernels.  There is no CPU path: if
the library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import CPlanInfo, CPlanOptions, check, lib
from .codec import SEGMENT_DTYPE, Domain, c_domains


def _dptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream, device):
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return ctypes.c_void_p(s.cuda_stream)


def _require(t, dtype, device, name, numel=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.device != device:
        raise ValueError(f"{name} must be on {device}, got {t.device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} needs at least {numel} elements, has {t.numel()}")


class Plan:
    """A decode plan: domains + segment table, validated and uploaded once.

    ``segments`` is a structured array with fields word_offset, n_words,
    n_samples, out_offset, domain (see ``codec.segments_array``)."""

    def __init__(self, domains, segments, device=None, idct: str = "fp32", schedule: str = "persistent",
                 tile_samples: int = 0, threads: int = 0, ctas_per_sm: int = 0, kernel: str = "auto"):
        if not torch.cuda.is_available():
            raise RuntimeError("the FPTC decoder needs a CUDA GPU")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else int(device))
        self.domains = list(domains)
        segs = np.ascontiguousarray(segments, dtype=SEGMENT_DTYPE)
        self.segments = segs
        o = CPlanOptions()
        o.idct = _lib.IDCT[idct]
        o.schedule = _lib.SCHEDULE[schedule]
        o.tile_samples, o.threads, o.ctas_per_sm = tile_samples, threads, ctas_per_sm
        o.kernel = _lib.KERNEL[kernel]
        cds = c_domains(self.domains)
        h = ctypes.c_void_p()
        check(lib().fptc_plan_create(ctypes.byref(h), self.device.index, cds, len(self.domains),
                                     segs.ctypes.data if len(segs) else None, len(segs), ctypes.byref(o)))
        self._h = h
        self.info = self._info()
        offs = np.zeros(max(1, len(segs)), np.uint64)
        check(lib().fptc_plan_level_offsets(self._h, offs.ctypes.data))
        self.level_offsets = offs[:len(segs)]

    def _info(self):
        inf = CPlanInfo()
        check(lib().fptc_plan_get_info(self._h, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in CPlanInfo._fields_}

    @property
    def handle(self):
        return self._h

    @property
    def launches_per_decode(self) -> int:
        return int(lib().fptc_plan_launches_per_decode(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib().fptc_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- buffers
    def empty_out(self):
        return torch.empty(max(1, self.info["out_extent"]), dtype=torch.float32, device=self.device)

    def to_device(self, words: np.ndarray, symlen: np.ndarray):
        w = torch.from_numpy(np.ascontiguousarray(words, np.uint64).view(np.int64)).to(self.device)
        s = torch.from_numpy(np.ascontiguousarray(symlen, np.uint8)).to(self.device)
        return w, s

    def _check_inputs(self, words, symlen):
        n = self.info["words_extent"]
        _require(words, torch.int64, self.device, "words", n)
        _require(symlen, torch.uint8, self.device, "symlen", n)

    # ---- calls
    def decode(self, words, symlen, out=None, levels=None, scale=None, stream=None):
        """fptc_decode_batch: words (int64 view of the uint64 words) and symlen on the GPU."""
        self._check_inputs(words, symlen)
        if out is None:
            out = self.empty_out()
        _require(out, torch.float32, self.device, "out", self.info["out_extent"])
        if levels is not None:
            _require(levels, torch.uint8, self.device, "levels", self.info["n_levels_total"])
        if scale is not None:
            _require(scale, torch.float32, self.device, "scale", 3 * len(self.domains))
        check(lib().fptc_decode_batch(self._h, _dptr(words), _dptr(symlen), _dptr(out), _dptr(levels), _dptr(scale),
                                      _stream(stream, self.device)))
        return out

    def decode_stages(self, words, symlen, out, stages: int, levels=None, scale=None, stream=None):
        """fptc_decode_stages: stages = STAGE_INDEX (1) | STAGE_DECODE (2); the three-kernel schedule also
        takes STAGE_LOSSLESS (4) and STAGE_LOSSY (8), the decode stage's two kernels on their own."""
        self._check_inputs(words, symlen)
        _require(out, torch.float32, self.device, "out", self.info["out_extent"])
        check(lib().fptc_decode_stages(self._h, _dptr(words), _dptr(symlen), _dptr(out), _dptr(levels), _dptr(scale),
                                       int(stages), _stream(stream, self.device)))
        return out

    def backward(self, grad_out, words=None, symlen=None, levels=None, scale=None, grad_coeffs=None,
                 grad_scale=None, stream=None):
        """fptc_decode_backward; returns (grad_scale float64 [n_domains, 3], grad_coeffs or None)."""
        _require(grad_out, torch.float32, self.device, "grad_out", self.info["out_extent"])
        if levels is None:
            self._check_inputs(words, symlen)
        else:
            _require(levels, torch.uint8, self.device, "levels", self.info["n_levels_total"])
        if grad_coeffs is not None:
            _require(grad_coeffs, torch.float32, self.device, "grad_coeffs", self.info["n_levels_total"])
        if grad_scale is None:
            grad_scale = torch.empty(len(self.domains), 3, dtype=torch.float64, device=self.device)
        _require(grad_scale, torch.float64, self.device, "grad_scale", 3 * len(self.domains))
        if scale is not None:
            _require(scale, torch.float32, self.device, "scale", 3 * len(self.domains))
        check(lib().fptc_decode_backward(self._h, _dptr(words), _dptr(symlen), _dptr(levels), _dptr(scale),
                                         _dptr(grad_out), _dptr(grad_coeffs), _dptr(grad_scale),
                                         _stream(stream, self.device)))
        return grad_scale, grad_coeffs

    def decode_host(self, h_words, h_symlen, h_out, d_words, d_symlen, d_out, stream=None):
        """fptc_decode_host: host (ideally pinned) buffers in and out, staged through the device buffers."""
        for t, dt, nm in ((h_words, torch.int64, "h_words"), (h_symlen, torch.uint8, "h_symlen"),
                          (h_out, torch.float32, "h_out")):
            if t.device.type != "cpu" or t.dtype != dt or not t.is_contiguous():
                raise ValueError(f"{nm} must be a contiguous CPU {dt} tensor")
        self._check_inputs(d_words, d_symlen)
        _require(d_out, torch.float32, self.device, "d_out", self.info["out_extent"])
        check(lib().fptc_decode_host(self._h, _dptr(h_words), _dptr(h_symlen), _dptr(h_out), _dptr(d_words),
                                     _dptr(d_symlen), _dptr(d_out), _stream(stream, self.device)))
        return h_out

    def device_status(self):
        """(status, flags, first_bad_segment); synchronizes and clears the sticky status."""
        flags = ctypes.c_uint32(0)
        first = ctypes.c_uint64(0)
        st = lib().fptc_plan_device_status(self._h, ctypes.byref(flags), ctypes.byref(first))
        if st not in (_lib.OK, _lib.CORRUPT_STREAM):
            check(st)
        return int(st), int(flags.value), int(first.value)

    def autotune(self, words, symlen, out, trials: int = 3, stream=None):
        self._check_inputs(words, symlen)
        best = CPlanOptions()
        ms = ctypes.c_float(0)
        check(lib().fptc_plan_autotune(self._h, _dptr(words), _dptr(symlen), _dptr(out), trials,
                                       _stream(stream, self.device), ctypes.byref(best), ctypes.byref(ms)))
        self.info = self._info()
        return {k: getattr(best, k) for k, _ in CPlanOptions._fields_ if k != "reserved"}, float(ms.value)

    def segment_view(self, out, i: int):
        s = self.segments[i]
        return out[int(s["out_offset"]):int(s["out_offset"]) + int(s["n_samples"])]


class FPTCDecode(torch.autograd.Function):
    """Differentiable decode: x_hat = decode(words, symlen; A), A = scale [n_domains, 3].

    backward gives dL/dA (FP64 reduction on the GPU, cast to scale's dtype) and,
    when ``coeff_probe`` requires grad, dL/dC for every dequantized coefficient
    (level layout of the plan).  The probe's values are not read: it only
    receives the coefficient gradient."""

    @staticmethod
    def forward(ctx, scale, coeff_probe, plan: Plan, words, symlen):
        sc = scale.detach().to(torch.float32).contiguous()
        levels = torch.empty(max(1, plan.info["n_levels_total"]), dtype=torch.uint8, device=plan.device)
        out = plan.decode(words, symlen, levels=levels, scale=sc)
        ctx.plan = plan
        ctx.scale_dtype = scale.dtype
        ctx.save_for_backward(sc, levels)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        sc, levels = ctx.saved_tensors
        plan = ctx.plan
        want_c = ctx.needs_input_grad[1]
        gco = torch.empty(max(1, plan.info["n_levels_total"]), dtype=torch.float32,
                          device=plan.device) if want_c else None
        gsc, _ = plan.backward(grad_out.contiguous().to(torch.float32), levels=levels, scale=sc, grad_coeffs=gco)
        g_scale = gsc.to(ctx.scale_dtype).reshape(sc.shape) if ctx.needs_input_grad[0] else None
        return g_scale, gco, None, None, None


def decode_differentiable(plan: Plan, words, symlen, scale, coeff_probe=None):
    if coeff_probe is None:
        coeff_probe = torch.zeros(1, device=plan.device)
    return FPTCDecode.apply(scale, coeff_probe, plan, words, symlen)


def check_bounded_wait(device: int = 0, arrive: bool = False) -> int:
    """Runs the decode kernels' bounded completion wait on its own
    (include/fptc.h fptc_check_bounded_wait); returns the status flags it set:
    FLAG_TIMEOUT when nothing arrived (after about 1 s), 0 when it did."""
    flags = ctypes.c_uint32(0)
    check(lib().fptc_check_bounded_wait(int(device), 1 if arrive else 0, ctypes.byref(flags)))
    return int(flags.value)
