"""Differentiable path lengths: a torch.autograd.Function over the C ABI.

Forward: enumerate, solve and validate on the GPU (mpt_enumerate /
mpt_solve / mpt_validate) for TX positions, RX positions and per-object
plane offsets d (each plane <n, X> = d moved along its normal by delta_d).
Backward: mpt_grad, the implicit-function-theorem adjoint of the converged
paths (the set of valid paths is held fixed, as for any piecewise-smooth
selection).  Outputs are the lengths and points of the valid paths plus
their candidate indices (integer, not differentiable).
"""
from __future__ import annotations

import numpy as np
import torch

from . import mpt, scenes


def shifted_scene(scene: scenes.Scene, delta_d: np.ndarray | None) -> scenes.Scene:
    """Copy of `scene` with every plane object moved by delta_d[i] along its
    normal (offset d and rectangle corner; its occluder rectangle too)."""
    if delta_d is None or not np.any(delta_d):
        return scene
    s = scenes.Scene(scene.name, scene.scale, scene.obj_kind.copy(), scene.obj_param.copy(),
                     scene.occ_kind.copy(), scene.occ_param.copy(), scene.tx.copy(), scene.rx.copy(),
                     scene.pair_mode, dict(scene.meta))
    L = scenes.OBJ_LAYOUT[scenes.PLANE]
    OL = scenes.OCC_LAYOUT[scenes.OCC_RECT]
    for i in np.nonzero(np.asarray(delta_d))[0]:
        if s.obj_kind[i] != scenes.PLANE:
            continue
        p = s.obj_param[i]
        n = p[L["n"]:L["n"] + 3].copy()
        O0 = p[L["O"]:L["O"] + 3].copy()
        dd = float(delta_d[i])
        # the occluder rectangle of this plane (same corner and axes), if any
        for q in range(s.n_occ):
            if s.occ_kind[q] == scenes.OCC_RECT and np.array_equal(s.occ_param[q, OL["O"]:OL["O"] + 3], O0) and \
                    np.array_equal(s.occ_param[q, OL["u"]:OL["u"] + 3], p[L["u"]:L["u"] + 3]):
                s.occ_param[q, OL["O"]:OL["O"] + 3] += dd * n
        p[L["d"]] += dd
        p[L["O"]:L["O"] + 3] += dd * n
    return s.contiguous()


class _MPTPaths(torch.autograd.Function):
    @staticmethod
    def forward(ctx_, tx, rx, delta_d, state):
        ctxm, scene, max_order, spec, cap = state
        sc = shifted_scene(scene, delta_d.detach().cpu().numpy() if delta_d is not None else None)
        sc = scenes.Scene(sc.name, sc.scale, sc.obj_kind, sc.obj_param, sc.occ_kind, sc.occ_param,
                          tx.detach().cpu().double().numpy(), rx.detach().cpu().double().numpy(),
                          sc.pair_mode, sc.meta).contiguous()
        ds = mpt.DeviceScene(ctxm, sc)
        res = mpt.trace(ds, max_order, spec, path_capacity=cap)
        n = res.paths.n()
        ctx_.saved = (ds, res, n)
        L = res.paths.length[:n].clone()
        X = res.paths.X[:, :n].t().contiguous().clone()
        cand = res.paths.cand[:n].clone()
        ctx_.mark_non_differentiable(cand)
        return L, X, cand

    @staticmethod
    def backward(ctx_, gL, gX, _gc):
        ds, res, n = ctx_.saved
        paths = res.paths
        g_len = torch.zeros(paths.capacity, dtype=torch.float64, device=ds.tx.device)
        g_pts = None
        if gL is not None:
            g_len[:n] = gL.to(torch.float64)
        if gX is not None:
            g_pts = torch.zeros((12, paths.capacity), dtype=torch.float64, device=ds.tx.device)
            g_pts[:, :n] = gX.t().to(torch.float64)
        g_tx, g_rx, g_obj = mpt.grad(ds, res.cands, paths, g_len, g_pts)
        return g_tx, g_rx, g_obj, None


def path_lengths(ctxm: mpt.Context, scene: scenes.Scene, tx: torch.Tensor, rx: torch.Tensor,
                 delta_d: torch.Tensor | None = None, max_order: int = 2, spec=None, capacity: int = 1 << 20):
    """Lengths [P], points [P, 12] and candidate indices [P] of the valid paths;
    lengths and points are differentiable w.r.t. tx [n_tx, 3], rx [n_rx, 3]
    and delta_d [n_obj] (plane offsets)."""
    if spec is None:
        spec = scenes.SequenceSpec(quota=(-1, -1, 0, 0))
    if delta_d is None:
        delta_d = torch.zeros(scene.n_obj, dtype=torch.float64, device=tx.device, requires_grad=False)
    return _MPTPaths.apply(tx, rx, delta_d, (ctxm, scene, max_order, spec, capacity))
