"""The product path has no CPU fallback: without a CUDA device the decoder and
the encoder refuse to start, and a missing shared library is an error, not a
silent substitute (CPU only)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_01086_gb300 import Encoder, Plan, _lib, codec  # noqa: E402


def _one():
    d = codec.Domain(32, 16, 2, 16, 50.0, 0.004, (1.0, 1.0, 0.0), 12, np.full(256, 8, np.uint8))
    return [d], codec.segments_array([0], [100], [1000], [0], [0])


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a CUDA device")
def test_decoder_and_encoder_refuse_without_a_gpu():
    doms, segs = _one()
    with pytest.raises(RuntimeError, match="CUDA"):
        Plan(doms, segs)
    with pytest.raises(RuntimeError, match="CUDA"):
        Encoder(doms, [1000], [0])


def test_missing_library_is_an_error(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "LIB", str(tmp_path / "absent.so"))
    _lib.lib.cache_clear()
    try:
        with pytest.raises(RuntimeError, match="missing"):
            _lib.lib()
    finally:
        monkeypatch.undo()
        _lib.lib.cache_clear()
