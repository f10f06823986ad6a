"""ctypes binding of libfptc (include/fptc.h, include/fptc_codec.h, include/fptc_encoder.h): struct mirrors,
argument types and status checking.  Argument marshalling only."""
from __future__ import annotations

import ctypes
import functools
import os

from .build import LIB

_u8, _u16, _u32, _u64, _i32 = ctypes.c_uint8, ctypes.c_uint16, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
_d, _f, _p = ctypes.c_double, ctypes.c_float, ctypes.c_void_p

OK, INVALID_ARGUMENT, UNSUPPORTED, OUT_OF_MEMORY, CUDA_ERROR, CORRUPT_STREAM = range(6)
FLAG_SYMLEN_RANGE, FLAG_BIT_OVERRUN, FLAG_INVALID_CODE, FLAG_SYMBOL_COUNT, FLAG_TIMEOUT = 1, 2, 4, 8, 16
ENC_FLAG_NO_CODE, ENC_FLAG_ROOM = 1, 2
STAGE_INDEX, STAGE_DECODE = 1, 2
STAGE_LOSSLESS, STAGE_LOSSY = 4, 8  # three-kernel schedule only: the decode stage's two kernels
IDCT = {"fp32": 0, "tf32": 1, "bf16x3": 2, "tf32x3": 3}
SCHEDULE = {"persistent": 0, "per_segment": 1, "three_kernel": 2}
KERNEL = {"auto": 0, "generic": 1, "block_tile": 2, "warp_tile": 3, "tensor": 4}


class CDomain(ctypes.Structure):
    _fields_ = [("N", _u32), ("E", _u32), ("B1", _u32), ("B2", _u32), ("mu", _d), ("alpha1", _d),
                ("scale", _d * 3), ("lmax", _u32), ("code_len", _u8 * 256)]


class CSegment(ctypes.Structure):
    _fields_ = [("word_offset", _u64), ("n_words", _u64), ("n_samples", _u64), ("out_offset", _u64),
                ("domain", _u32), ("reserved", _u32)]


class CPlanOptions(ctypes.Structure):
    _fields_ = [("idct", _u32), ("schedule", _u32), ("tile_samples", _u32), ("threads", _u32),
                ("ctas_per_sm", _u32), ("kernel", _u32), ("reserved", _u32 * 2)]


class CPlanInfo(ctypes.Structure):
    _fields_ = [("n_segments", _u64), ("n_tiles", _u64), ("n_chunks", _u64), ("words_extent", _u64),
                ("out_extent", _u64), ("n_samples_total", _u64), ("n_words_total", _u64),
                ("n_levels_total", _u64), ("device_bytes", _u64), ("n_domains", _u32), ("device", _u32),
                ("sm_count", _u32), ("threads", _u32), ("grid", _u32), ("ctas_per_sm", _u32), ("idct", _u32),
                ("schedule", _u32), ("kernel", _u32), ("smem_bytes", _u32)]


class FptcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


# name -> (restype, argtypes); every symbol the headers declare
SIGNATURES = {
    "fptc_plan_create": (_i32, [ctypes.POINTER(_p), _i32, _p, _u32, _p, _u64, _p]),
    "fptc_plan_destroy": (None, [_p]),
    "fptc_plan_get_info": (_i32, [_p, _p]),
    "fptc_plan_level_offsets": (_i32, [_p, _p]),
    "fptc_decode_batch": (_i32, [_p, _p, _p, _p, _p, _p, _p]),
    "fptc_decode_stages": (_i32, [_p, _p, _p, _p, _p, _p, _u32, _p]),
    "fptc_decode_backward": (_i32, [_p, _p, _p, _p, _p, _p, _p, _p, _p]),
    "fptc_decode_host": (_i32, [_p, _p, _p, _p, _p, _p, _p, _p]),
    "fptc_decode_stream_noalloc": (_i32, [_p, _p, _p, _u64, _u64, _p, _p]),
    "fptc_plan_device_status": (_i32, [_p, ctypes.POINTER(_u32), ctypes.POINTER(_u64)]),
    "fptc_plan_autotune": (_i32, [_p, _p, _p, _p, _u32, _p, _p, ctypes.POINTER(_f)]),
    "fptc_plan_launches_per_decode": (_u32, [_p]),
    "fptc_check_bounded_wait": (_i32, [_i32, _i32, ctypes.POINTER(_u32)]),
    "fptc_struct_size": (_u64, [_u32]),
    "fptc_status_string": (ctypes.c_char_p, [_i32]),
    "fptc_last_error_message": (ctypes.c_char_p, []),
    "fptc_abi_version": (_u32, []),
    "fptc_validate_domain": (_i32, [_p]),
    "fptc_build_decode_table": (_i32, [_p, _p]),
    "fptc_canonical_codes": (_i32, [_p, _p]),
    "fptc_train_domain": (_i32, [_p, _p, _p, _u64, _d, _p]),
    "fptc_word_capacity": (_u64, [_p, _u64]),
    "fptc_zone_bounds": (_i32, [_p, _u32, _p]),
    "fptc_encode_stream": (_i32, [_p, _p, _u64, _p, _p, _u64, _p, _p]),
    "fptc_encode_batch": (_i32, [_p, _u32, _p, _p, _p, _p, _u64, _p, _p, _p, _p, _i32]),
    "fptc_encoder_create": (_i32, [ctypes.POINTER(_p), _i32, _p, _u32, _p, _u64]),
    "fptc_encoder_destroy": (None, [_p]),
    "fptc_encoder_levels": (_u64, [_p]),
    "fptc_encoder_level_offsets": (_i32, [_p, _p]),
    "fptc_encode_device": (_i32, [_p, _p, _p, _p, _p, _p, _p]),
    "fptc_pack_device": (_i32, [_p, _p, _p, _p, _p, _p]),
    "fptc_encoder_status": (_i32, [_p, ctypes.POINTER(_u32), ctypes.POINTER(_u64)]),
}


@functools.lru_cache(maxsize=None)
def lib():
    """Loads the in-tree libfptc.so; raises if it has not been built."""
    if not os.path.exists(LIB):
        raise RuntimeError(f"{LIB} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(LIB)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    for i, cls in enumerate((CDomain, CSegment, CPlanOptions, CPlanInfo)):
        if L.fptc_struct_size(i) != ctypes.sizeof(cls):
            raise RuntimeError(f"ABI mismatch: {cls.__name__} is {ctypes.sizeof(cls)} bytes here, "
                               f"{L.fptc_struct_size(i)} in libfptc")
    return L


def check(status: int):
    if status != OK:
        msg = lib().fptc_last_error_message().decode() or lib().fptc_status_string(status).decode()
        raise FptcError(int(status), msg)
