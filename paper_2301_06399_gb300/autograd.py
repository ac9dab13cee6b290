"""Differentiable path lengths: a torch.autograd.Function over the C ABI.

Forward: enumerate, solve and validate on the GPU (mpt_enumerate /
mpt_solve / mpt_validate) for TX positions, RX positions and per-object
plane offsets d (each plane <n, X> = d moved along its normal by delta_d).
Everything stays on the device: the TX/RX tensors are the endpoints the
library reads, and the offsets move the planes of a device copy of the scene
(mpt_scene_shift_planes).  Backward: mpt_grad, the implicit-function-theorem
adjoint of the converged paths (the set of valid paths is held fixed, as for
any piecewise-smooth selection).  Outputs are the lengths and points of the
valid paths plus their candidate indices (integer, not differentiable).  The
forward pass reads one number back: the count of valid paths, which sizes
its outputs.
"""
from __future__ import annotations

import torch

from . import mpt, scenes

# per (context, scene): the scene as uploaded and a second upload that
# receives its plane-shifted copies
_SCENES: dict = {}


def _device_scenes(ctxm: mpt.Context, scene: scenes.Scene):
    key = (id(ctxm), id(scene))
    entry = _SCENES.get(key)
    if entry is None or entry[0] is not ctxm or entry[1] is not scene:
        base = mpt.DeviceScene(ctxm, scene)
        dst = mpt.DeviceScene(ctxm, scene)
        entry = (ctxm, scene, base, dst)
        _SCENES[key] = entry
    return entry[2], entry[3]


class _MPTPaths(torch.autograd.Function):
    @staticmethod
    def forward(ctx_, tx, rx, delta_d, state):
        ctxm, scene, max_order, spec, cap = state
        base, dst = _device_scenes(ctxm, scene)
        stream = torch.cuda.current_stream()
        mpt.shift_planes(base, dst, delta_d, stream=stream)
        ds = mpt.SceneView(ctxm, scene, dst.h, tx.detach().to(torch.float64).contiguous(),
                           rx.detach().to(torch.float64).contiguous())
        res = mpt.trace(ds, max_order, spec, path_capacity=cap, stream=stream)
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
    and delta_d [n_obj] (plane offsets), all device tensors."""
    if spec is None:
        spec = scenes.SequenceSpec(quota=(-1, -1, 0, 0))
    if delta_d is None:
        delta_d = torch.zeros(scene.n_obj, dtype=torch.float64, device=tx.device, requires_grad=False)
    return _MPTPaths.apply(tx, rx, delta_d, (ctxm, scene, max_order, spec, capacity))
