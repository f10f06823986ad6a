"""Rate-distortion tuning through the differentiable decoder.

For streams whose levels (hence bit rate) stay fixed, the decoder-side zone
scales A_z can still move: every dequantized coefficient is A_z times a function
of its level (Sec. 3.2, Eq. 2 and Eq. 3 inverted), so the reconstruction is
linear in A and the squared error to reference signals is exactly quadratic in
A.  ``fit_zone_scales`` finds its minimiser with the GPU adjoint
(``fptc_decode_backward``): the gradient at the current scales, the columns of
the Hessian from gradients at scales moved one parameter at a time, one Newton
step.  The result is passed to the decoder at run time (``scale``), which is the
distortion the same streams reach at their bit budget when the decoder, not the
encoder, picks the scales (Sec. 5.2's rate-distortion trade-off, at a fixed rate).
"""
from __future__ import annotations

import numpy as np
import torch

from .decoder import Plan


def _valid_mask(plan: Plan) -> torch.Tensor:
    m = torch.zeros(plan.info["out_extent"], dtype=torch.bool, device=plan.device)
    for s in plan.segments:
        o, n = int(s["out_offset"]), int(s["n_samples"])
        m[o:o + n] = True
    return m


def fit_zone_scales(plan: Plan, words, symlen, x, scale=None, stream=None):
    """Zone scales minimising sum over the plan's samples of (x_hat(A) - x)^2.

    words / symlen: the compressed batch on the GPU; x: float32 reference
    samples in the output layout (out_extent floats on the GPU; values outside
    the segments are ignored); scale: the starting scales (float [n_domains*3]),
    default the domains' own.  Zones a domain has no bin in keep their scale.
    Returns (scale float32 [n_domains * 3] on the GPU, report) where report holds
    the squared error and PRD before and after."""
    D = len(plan.domains)
    dev = plan.device
    if scale is None:
        A = np.array([[float(v) for v in d.scale] for d in plan.domains], np.float64)
    else:
        A = scale.detach().double().cpu().numpy().reshape(D, 3).copy()
    mask = _valid_mask(plan)
    xm = torch.where(mask, x, torch.zeros_like(x))
    x64 = xm.double()
    levels = torch.empty(max(1, plan.info["n_levels_total"]), dtype=torch.uint8, device=dev)
    plan.decode(words, symlen, levels=levels, scale=torch.tensor(A.ravel(), dtype=torch.float32, device=dev),
                stream=stream)

    def loss_grad(a):
        sc = torch.tensor(a.ravel(), dtype=torch.float32, device=dev)
        out = plan.decode(words, symlen, scale=sc, stream=stream)
        r = torch.where(mask, out, torch.zeros_like(out)) - xm
        gsc, _ = plan.backward((2.0 * r).contiguous(), levels=levels, scale=sc, stream=stream)
        return float((r.double() ** 2).sum()), gsc.cpu().numpy().reshape(D, 3)

    params = [(d, z) for d, dom in enumerate(plan.domains) for z in (0, 1)
              if (z == 0 and dom.B1 > 0) or (z == 1 and dom.B2 > dom.B1)]
    L0, g0 = loss_grad(A)
    H = np.zeros((len(params), len(params)))
    for j, (d, z) in enumerate(params):
        h = max(abs(A[d, z]), 1.0) * 0.5
        a = A.copy()
        a[d, z] += h
        _, g = loss_grad(a)
        H[:, j] = [(g[dd, zz] - g0[dd, zz]) / h for dd, zz in params]
    gvec = np.array([g0[d, z] for d, z in params])
    # zones whose bins never occur give an empty row: they keep their scale
    live = np.flatnonzero(np.abs(np.diag(H)) > 0)
    A_new = A.copy()
    if live.size:
        step = np.linalg.solve(H[np.ix_(live, live)], -gvec[live])
        for i, s in zip(live, step):
            d, z = params[i]
            A_new[d, z] += s
    L1, _ = loss_grad(A_new)
    energy = float((x64 ** 2).sum())
    report = {"sq_error_before": L0, "sq_error_after": L1,
              "prd_before": 100.0 * np.sqrt(L0 / energy) if energy > 0 else 0.0,
              "prd_after": 100.0 * np.sqrt(L1 / energy) if energy > 0 else 0.0,
              "scale_before": A, "scale_after": A_new}
    return torch.tensor(A_new.ravel(), dtype=torch.float32, device=dev), report
