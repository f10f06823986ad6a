"""FPTC server-side batch decoder for one GB300 GPU (sm_103a).

Implements the decompression side of FPTC (arXiv 2605.01086, Sec. 4.2): SymLen
segment indexing, table-driven Huffman decoding, inverse three-zone
quantization and the inverse windowed DCT with window reassembly, all in
hand-written CUDA kernels behind the C ABI of include/fptc.h.  The host-side
encoder and trainer of the prebuilt structures (Sec. 3, Sec. 4.1) are in
``codec``; ``Encoder`` runs the same encoder on the GPU.
"""
from ._lib import STAGE_DECODE, STAGE_INDEX, STAGE_LOSSLESS, STAGE_LOSSY, FptcError, lib  # noqa: F401
from .build import build  # noqa: F401
from .codec import (Batch, Domain, canonical_codes, decode_table, encode_batch, encode_stream,  # noqa: F401
                    packed_out_offsets, segments_array, train_domain, validate_domain, word_capacity)
from .decoder import FPTCDecode, Plan, check_bounded_wait, decode_differentiable  # noqa: F401
from .encoder import Encoder  # noqa: F401
from .tuning import fit_zone_scales  # noqa: F401
