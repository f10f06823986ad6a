"""GPU parity of the hand-written adjoint (fptc_decode_backward) and of the
autograd wrapper against the FP64 oracle gradient, for the MSE loss to the
original signal.  The oracle gradient itself is pinned by central finite
differences in test_oracle_pipeline.py."""
import numpy as np
import pytest

import oracle
import siggen

from gpu_util import encode_workload, gpu_decode, make_plan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRAD_COEFF_REL_L2 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_01086_gb300 import build
    build()


def _signals_on_device(plan, wl):
    """Original signals laid out like the decoder output (0 in the gaps)."""
    x = torch.zeros(plan.info["out_extent"], dtype=torch.float32)
    for i in range(wl.n_streams):
        s = plan.segments[i]
        a = int(s["out_offset"])
        x[a:a + int(s["n_samples"])] = torch.from_numpy(siggen.signal(int(wl.domains[i]), int(wl.seeds[i]),
                                                                      int(wl.lengths[i])))
    return x.to(plan.device)


def _oracle_grads(plan, b, lv_h, gx_h, scale=None):
    n_dom = len(b.domains)
    gA = np.zeros((n_dom, 3))
    absA = np.zeros((n_dom, 3))
    gC = []
    for i in range(b.n_streams):
        d = b.domains[b.domain_idx[i]]
        if scale is not None:
            d = oracle.Domain(d.N, d.E, d.B1, d.B2, d.mu, d.alpha1, tuple(scale[b.domain_idx[i]]), d.lmax, d.code_len)
        S = int(b.lengths[i])
        L = d.windows(S) * d.E
        a = int(plan.level_offsets[i])
        o = int(plan.segments[i]["out_offset"])
        lv = lv_h[a:a + L]
        c, g = oracle.backward_stream(lv, S, d, gx_h[o:o + S])
        gA[b.domain_idx[i]] += g
        gC.append(c)
        # sum of |terms| bounds the rounding error of the FP32 products
        unit = np.array([[oracle.dequantize_unit(d, z, Lv) for Lv in range(256)] for z in (0, 1)])
        zones = np.array([d.zone(k) for k in range(d.E)])
        cc = c.reshape(-1, d.E)
        ll = lv.reshape(-1, d.E)
        for z in (0, 1):
            m = zones == z
            absA[b.domain_idx[i], z] += np.abs(cc[:, m] * unit[z][ll[:, m]]).sum()
    return gA, absA, gC


def _check(plan, b, gsc, gco, gA, absA, gC):
    g = gsc.cpu().numpy()
    # FP32 products g_C * unit: each term carries ~N+2 roundings of 2^-24; FP64 reduction
    tol = 1e-6 * np.abs(gA) + 40 * 2.0 ** -24 * absA
    assert np.all(np.abs(g - gA) <= tol), (g, gA, tol)
    if gco is not None:
        h = gco.cpu().numpy()
        for i, c in enumerate(gC):
            a = int(plan.level_offsets[i])
            seg = h[a:a + c.size].astype(np.float64)
            nr = np.linalg.norm(c)
            assert np.linalg.norm(seg - c) <= GRAD_COEFF_REL_L2 * max(nr, 1e-30), i


@pytest.mark.parametrize("name", ["power", "mixed"])
def test_backward_matches_oracle(name):
    wl = siggen.power_1024x65536(n=12, S=20000) if name == "power" else \
        siggen.mixed_10000_logu(n=16, lo=33, hi=60000)
    b = encode_workload(wl)
    plan = make_plan(b)
    w, s, out, lv = gpu_decode(plan, b)
    x = _signals_on_device(plan, wl)
    M = wl.n_samples
    gx = (2.0 / M) * (out - x)
    mask = torch.zeros_like(gx, dtype=torch.bool)
    for sg in plan.segments:
        mask[int(sg["out_offset"]):int(sg["out_offset"]) + int(sg["n_samples"])] = True
    gx = torch.where(mask, gx, torch.zeros_like(gx)).contiguous()
    gco = torch.empty(plan.info["n_levels_total"], dtype=torch.float32, device=plan.device)
    gsc, _ = plan.backward(gx, levels=lv, grad_coeffs=gco)
    # the same with the levels decoded again from the words
    gco2 = torch.empty_like(gco)
    gsc2, _ = plan.backward(gx, words=w, symlen=s, grad_coeffs=gco2)
    torch.cuda.synchronize()
    assert torch.equal(gco, gco2)
    assert torch.allclose(gsc, gsc2, rtol=1e-12, atol=0)
    gA, absA, gC = _oracle_grads(plan, b, lv.cpu().numpy(), gx.double().cpu().numpy())
    _check(plan, b, gsc, gco, gA, absA, gC)
    assert plan.device_status()[0] == 0


def test_autograd_function():
    from paper_2605_01086_gb300 import decode_differentiable
    wl = siggen.power_1024x65536(n=6, S=30000)
    b = encode_workload(wl)
    plan = make_plan(b)
    w, s = plan.to_device(b.words, b.symlen)
    x = _signals_on_device(plan, wl)
    base = np.array([d.A for d in b.domains])
    scale = torch.tensor(base * 1.1, dtype=torch.float64, device=plan.device, requires_grad=True)
    probe = torch.zeros(plan.info["n_levels_total"], device=plan.device, requires_grad=True)
    out = decode_differentiable(plan, w, s, scale, probe)
    n = int(plan.segments[-1]["out_offset"] + plan.segments[-1]["n_samples"])
    mask = torch.zeros(out.numel(), dtype=torch.bool, device=plan.device)
    for sg in plan.segments:
        mask[int(sg["out_offset"]):int(sg["out_offset"]) + int(sg["n_samples"])] = True
    loss = ((out - x)[mask] ** 2).mean()
    loss.backward()
    assert scale.grad is not None and probe.grad is not None
    # oracle with the same g_x
    gx = torch.where(mask, (2.0 / int(mask.sum())) * (out.detach() - x), torch.zeros_like(x))
    lv = torch.empty(plan.info["n_levels_total"], dtype=torch.uint8, device=plan.device)
    plan.decode(w, s, out=torch.empty_like(out), levels=lv)
    sc32 = (base * 1.1).astype(np.float32).astype(np.float64)
    gA, absA, gC = _oracle_grads(plan, b, lv.cpu().numpy(), gx.double().cpu().numpy(), scale=sc32)
    _check(plan, b, scale.grad, probe.grad, gA, absA, gC)
    assert n <= out.numel()


def test_backward_zone_switched_off():
    # A_1 = 0 at run time: zone 1 reconstructs 0 and has no gradient
    wl = siggen.power_1024x65536(n=3, S=5000)
    b = encode_workload(wl)
    plan = make_plan(b)
    w, s = plan.to_device(b.words, b.symlen)
    sc = torch.tensor(np.array([[d.A[0], 0.0, 0.0] for d in b.domains], np.float32).ravel(), device=plan.device)
    out = plan.decode(w, s, scale=sc)
    gx = torch.ones_like(out) * 1e-3
    gsc, _ = plan.backward(gx, words=w, symlen=s, scale=sc)
    torch.cuda.synchronize()
    g = gsc.cpu().numpy()
    assert np.all(g[:, 1] == 0.0) and np.all(g[:, 2] == 0.0) and np.any(g[:, 0] != 0.0)


@pytest.mark.parametrize("mode", ["levels", "redecode"])
def test_backward_other_shapes_matches_oracle(mode):
    """The adjoint on a plan of other window shapes (N = 64, 128, 16, 32 with E = N/2, N/2, N/2,
    N/4 in one batch; decoded by the shape kernel, differentiated by the block adjoint), from saved
    levels and decoding them again, against the oracle gradient."""
    shapes = [(64, 32), (128, 64), (16, 8), (32, 8)]
    doms = [oracle.trained_domain(i, N=N, E=E, B1=2, B2=E) for i, (N, E) in enumerate(shapes)]
    wl = siggen.mixed_10000_logu(n=12, lo=100, hi=40000)
    b = encode_workload(wl, domains=doms)
    plan = make_plan(b)
    assert plan.info["kernel"] == 3
    w, s, out, lv = gpu_decode(plan, b)
    x = _signals_on_device(plan, wl)
    gx = (2.0 / wl.n_samples) * (out - x)
    mask = torch.zeros_like(gx, dtype=torch.bool)
    for sg in plan.segments:
        mask[int(sg["out_offset"]):int(sg["out_offset"]) + int(sg["n_samples"])] = True
    gx = torch.where(mask, gx, torch.zeros_like(gx)).contiguous()
    gco = torch.empty(plan.info["n_levels_total"], dtype=torch.float32, device=plan.device)
    if mode == "levels":
        gsc, _ = plan.backward(gx, levels=lv, grad_coeffs=gco)
    else:
        gsc, _ = plan.backward(gx, words=w, symlen=s, grad_coeffs=gco)
    torch.cuda.synchronize()
    assert plan.device_status()[0] == 0
    gA, absA, gC = _oracle_grads(plan, b, lv.cpu().numpy(), gx.double().cpu().numpy())
    g = gsc.cpu().numpy()
    # FP32 products of up to N = 128 terms per coefficient, FP64 reduction
    tol = 1e-6 * np.abs(gA) + 136 * 2.0 ** -24 * absA
    assert np.all(np.abs(g - gA) <= tol), (g, gA, tol)
    h = gco.cpu().numpy()
    for i, c in enumerate(gC):
        a = int(plan.level_offsets[i])
        assert np.linalg.norm(h[a:a + c.size] - c) <= GRAD_COEFF_REL_L2 * max(np.linalg.norm(c), 1e-30), i


def test_backward_after_autotune():
    """The adjoint of a plan whose autotuner tried warp-tile candidates and may
    have settled on a block kernel (a single stream of 65,536 samples, where the
    block-tile kernel tends to win): the adjoint serves the configuration the
    autotuner left, and agrees with a plan configured once."""
    wl = siggen.Workload("one", 3, np.zeros(1, np.int32), np.array([siggen.stream_seed(3, 0)], np.uint64),
                         np.array([65536], np.uint64))
    b = encode_workload(wl)
    outs = []
    for tune in (True, False):
        plan = make_plan(b, out_align=32)
        w, s = plan.to_device(b.words, b.symlen)
        out = plan.empty_out().zero_()
        if tune:
            plan.autotune(w, s, out, trials=2)
        n_lev = plan.info["n_levels_total"]
        lv = torch.empty(n_lev, dtype=torch.uint8, device=plan.device)
        gco = torch.empty(n_lev, dtype=torch.float32, device=plan.device)
        plan.decode(w, s, out=out, levels=lv)
        gsc, _ = plan.backward(out, levels=lv, grad_coeffs=gco)
        torch.cuda.synchronize()
        assert plan.device_status()[0] == 0
        outs.append((gsc.cpu().numpy(), gco.cpu().numpy().astype(np.float64)))
    (g1, c1), (g2, c2) = outs
    np.testing.assert_allclose(g1, g2, rtol=1e-6, atol=1e-9)
    assert np.linalg.norm(c1 - c2) <= 1e-6 * np.linalg.norm(c2)
