"""Binding of the GPU encoder (include/fptc_encoder.h): argument marshalling only.

``Encoder(domains, lengths, domain_idx)`` lays out one room of
``word_capacity(domain, S)`` words per stream and the input offsets of the
streams packed back to back; ``encode`` runs Eq. 1, the zone quantizer and
Alg. 1 on the GPU and returns the words, symbol counts and word counts, from
which ``segments`` gives the segment table a decode ``Plan`` takes.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import check, lib
from .codec import c_domains, segments_array, word_capacity
from .decoder import _dptr, _require, _stream


class Encoder:
    def __init__(self, domains, lengths, domain_idx, device=None, in_offsets=None, room=None):
        if not torch.cuda.is_available():
            raise RuntimeError("the FPTC encoder needs a CUDA GPU")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else int(device))
        self.domains = list(domains)
        self.lengths = np.ascontiguousarray(lengths, np.uint64)
        self.domain_idx = np.ascontiguousarray(domain_idx, np.uint32)
        n = len(self.lengths)
        if in_offsets is None:
            in_offsets = np.zeros(n, np.uint64)
            if n > 1:
                in_offsets[1:] = np.cumsum(self.lengths[:-1])
        self.in_offsets = np.ascontiguousarray(in_offsets, np.uint64)
        if room is None:
            room = [word_capacity(self.domains[self.domain_idx[i]], int(self.lengths[i])) for i in range(n)]
        self.room = np.ascontiguousarray(room, np.uint64)
        self.room_offsets = np.zeros(n, np.uint64)
        if n > 1:
            self.room_offsets[1:] = np.cumsum(self.room[:-1])
        self.words_extent = int(self.room.sum()) if n else 0
        segs = segments_array(self.room_offsets, self.room, self.lengths, self.in_offsets, self.domain_idx)
        h = ctypes.c_void_p()
        check(lib().fptc_encoder_create(ctypes.byref(h), self.device.index, c_domains(self.domains), len(self.domains),
                                        segs.ctypes.data if n else None, n))
        self._h = h
        self.n_levels = int(lib().fptc_encoder_levels(self._h))
        offs = np.zeros(max(1, n), np.uint64)
        check(lib().fptc_encoder_level_offsets(self._h, offs.ctypes.data))
        self.level_offsets = offs[:n]

    def close(self):
        if getattr(self, "_h", None):
            lib().fptc_encoder_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def buffers(self):
        """Device rooms: words (int64 view of uint64), symlen, word counts."""
        w = torch.zeros(max(1, self.words_extent), dtype=torch.int64, device=self.device)
        s = torch.zeros(max(1, self.words_extent), dtype=torch.uint8, device=self.device)
        nw = torch.zeros(max(1, len(self.lengths)), dtype=torch.int64, device=self.device)
        return w, s, nw

    def encode(self, x, words=None, symlen=None, n_words=None, levels=None, stream=None):
        """x: float32 samples on the GPU at ``in_offsets``.  Returns (words, symlen, n_words)."""
        _require(x, torch.float32, self.device, "x",
                 int((self.in_offsets + self.lengths).max()) if len(self.lengths) else 0)
        if words is None:
            words, symlen, n_words = self.buffers()
        if levels is not None:
            _require(levels, torch.uint8, self.device, "levels", self.n_levels)
        check(lib().fptc_encode_device(self._h, _dptr(x), _dptr(words), _dptr(symlen), _dptr(n_words),
                                       _dptr(levels), _stream(stream, self.device)))
        return words, symlen, n_words

    def pack(self, levels, words=None, symlen=None, n_words=None, stream=None):
        """SymLen packing of given levels (the ``level_offsets`` layout)."""
        _require(levels, torch.uint8, self.device, "levels", self.n_levels)
        if words is None:
            words, symlen, n_words = self.buffers()
        check(lib().fptc_pack_device(self._h, _dptr(levels), _dptr(words), _dptr(symlen), _dptr(n_words),
                                     _stream(stream, self.device)))
        return words, symlen, n_words

    def status(self):
        """(status, flags, first_bad_segment); synchronizes and clears the status."""
        flags = ctypes.c_uint32(0)
        first = ctypes.c_uint64(0)
        st = lib().fptc_encoder_status(self._h, ctypes.byref(flags), ctypes.byref(first))
        if st not in (_lib.OK, _lib.CORRUPT_STREAM):
            check(st)
        return int(st), int(flags.value), int(first.value)

    def segments(self, n_words, out_offsets):
        """Decode segment table of the encoded streams (rooms at room_offsets,
        n_words from the encode, outputs at out_offsets)."""
        nw = n_words.cpu().numpy().astype(np.uint64)[:len(self.lengths)]
        return segments_array(self.room_offsets, nw, self.lengths, np.asarray(out_offsets, np.uint64),
                              self.domain_idx)
