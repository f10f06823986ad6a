"""GPU test of fptc_decode_stream_noalloc, the allocation-free single-stream decode.

That entry point serves callers that cannot allocate device memory at decode
time (inside a framework's memory pool or allocator callback, serving paths that
forbid allocation after start-up): all of its working memory is one file-scope
device array.  Here it is called through the C ABI and its samples are compared
with those of the plan entry point (fptc_decode_batch) on the same stream, and
with the FP64 oracle's decode, within the FP32 tolerance of the other tests, on
two calls in a row; the second stream
is shorter and of another domain, so anything left over from the first call in
the shared array would show.  This file sorts last so that a run that stops at
the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

import oracle
import siggen

from gpu_util import FP32_REL_L2, make_plan, product_domain

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_01086_gb300 import build
    build()


def _one_stream(domain_id, seed, S):
    d = oracle.trained_domain(domain_id)
    x = siggen.signal(domain_id, seed, S)
    words, symlen, _ = oracle.encode_stream(x, d)
    b = oracle.EncodedBatch(words, symlen, np.zeros(1, np.uint64), np.array([words.size], np.uint64),
                            np.array([S], np.uint64), np.zeros(1, np.int32), [d])
    return b


def _plan_reference(b):
    plan = make_plan(b)
    w, s = plan.to_device(b.words, b.symlen)
    out = plan.decode(w, s)
    torch.cuda.synchronize()
    ref = out[:int(b.lengths[0])].double().cpu().numpy()
    plan.close()
    return ref


def _noalloc(b):
    from paper_2605_01086_gb300 import _lib
    L = _lib.lib()
    dev = torch.device("cuda", torch.cuda.current_device())
    S = int(b.lengths[0])
    w = torch.from_numpy(b.words.view(np.int64)).to(dev)
    s = torch.from_numpy(b.symlen).to(dev)
    out = torch.full((S,), float("nan"), dtype=torch.float32, device=dev)
    cd = product_domain(b.domains[0]).c()
    st = L.fptc_decode_stream_noalloc(ctypes.byref(cd), ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(s.data_ptr()),
                                      int(b.n_words[0]), S, ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
    assert st == _lib.OK, L.fptc_last_error_message()
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


def test_noalloc_matches_plan_on_two_calls():
    first = _one_stream(0, siggen.stream_seed(0, 0), 65536)
    second = _one_stream(1, siggen.stream_seed(3, 5), 20001)
    for b in (first, second):
        ref = _plan_reference(b)
        got = _noalloc(b)
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= FP32_REL_L2, rel
        # and against the FP64 oracle's decode of the same stream
        x64, _ = oracle.decode_stream(b.words, b.symlen, int(b.lengths[0]), b.domains[0])
        rel64 = np.linalg.norm(got - x64) / np.linalg.norm(x64)
        assert rel64 <= FP32_REL_L2, rel64


def test_noalloc_rejects_oversize():
    from paper_2605_01086_gb300 import _lib
    L = _lib.lib()
    b = _one_stream(2, 7, 1000)
    cd = product_domain(b.domains[0]).c()
    S = (1 << 26) + 1
    st = L.fptc_decode_stream_noalloc(ctypes.byref(cd), None, None, S // 2, S, None, None)
    assert st == _lib.UNSUPPORTED
    assert b"at most" in L.fptc_last_error_message()
