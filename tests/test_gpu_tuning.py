"""Decoder-side scale fit through the GPU adjoint (rate-distortion tuning at a
fixed rate): the scales equal the oracle's FP64 normal-equation solution, and
the PRD of the same streams does not rise."""
import numpy as np
import pytest

import oracle
import siggen

from gpu_util import encode_workload, make_plan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_01086_gb300 import build
    build()


def _reference(plan, wl):
    flat, offs = siggen.signals(wl.domains, wl.seeds, wl.lengths)
    x = np.zeros(plan.info["out_extent"], np.float32)
    xs = []
    for i, sg in enumerate(plan.segments):
        n = int(sg["n_samples"])
        xi = flat[int(offs[i]):int(offs[i]) + n]
        x[int(sg["out_offset"]):int(sg["out_offset"]) + n] = xi
        xs.append(xi.astype(np.float64))
    return torch.from_numpy(x).to(plan.device), xs


@pytest.mark.parametrize("kernel", ["warp_tile", "generic"])
def test_fit_zone_scales_matches_oracle(kernel):
    from paper_2605_01086_gb300 import fit_zone_scales
    wl = siggen.mixed_10000_logu(n=16, lo=1000, hi=60000)
    b = encode_workload(wl)
    plan = make_plan(b, kernel=kernel)
    w, s = plan.to_device(b.words, b.symlen)
    x, xs = _reference(plan, wl)
    sc, rep = fit_zone_scales(plan, w, s, x)
    assert plan.device_status()[0] == 0
    lvs = [oracle.decode_stream(b.words[int(b.word_off[i]):int(b.word_off[i]) + int(b.n_words[i])],
                                b.symlen[int(b.word_off[i]):int(b.word_off[i]) + int(b.n_words[i])],
                                int(b.lengths[i]), b.domains[b.domain_idx[i]])[1] for i in range(b.n_streams)]
    A_orc = oracle.fit_zone_scales(lvs, [int(v) for v in b.lengths], list(b.domain_idx), b.domains, xs)
    A_gpu = sc.double().cpu().numpy().reshape(-1, 3)
    np.testing.assert_allclose(A_gpu[:, :2], A_orc[:, :2], rtol=1e-4)
    assert rep["prd_after"] <= rep["prd_before"]
    # the PRD the GPU reports after the fit is the oracle's at the oracle's scales
    x_all = np.concatenate(xs)
    doms = [oracle.Domain(d.N, d.E, d.B1, d.B2, d.mu, d.alpha1, tuple(A_orc[k]), d.lmax, d.code_len)
            for k, d in enumerate(b.domains)]
    xh = np.concatenate([oracle.reconstruct(lv, xi.size, doms[b.domain_idx[i]])
                         for i, (lv, xi) in enumerate(zip(lvs, xs))])
    assert abs(rep["prd_after"] - oracle.prd(x_all, xh)) <= 1e-4 * oracle.prd(x_all, xh)
