"""torch.autograd.Function over gs_render_fwd / gs_render_bwd.

The function takes post-activation Gaussian parameters (scales > 0, opacities in [0,1],
raw quaternions) so that callers keep their own parameterisation (log-scales, opacity
logits, ...) in PyTorch and autograd chains through it; and a pose twist ``xi`` (6,)
applied on the left of the base world->camera pose, T = Exp(xi) T0.  The gradient
returned for ``xi`` is the twist gradient at the composed pose, which equals dL/dxi at
xi = 0 -- the way pose tracking uses it (compose, step, reset xi).  The pose is composed
on the host; pass ``xi`` as a CPU tensor to keep the forward free of a device
synchronisation (its gradient is returned on the device of ``xi``).

Several renders may share one Rasterizer before a single backward (e.g. the keyframes of
one mapping step, Eq. 3, summed into one loss).  The workspace keeps only the latest
forward's state, so the backward of an earlier render first recomputes its own forward
(projection, tile lists and per-pixel state; deterministic, so identical to the original)
before differentiating.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as L
from .render import Rasterizer


def _hat(w):
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def se3_exp(xi):
    """Exp of the twist (rho, phi) -> 4x4 matrix (Rodrigues; small-angle series)."""
    xi = np.asarray(xi, np.float64)
    rho, phi = xi[:3], xi[3:]
    th = float(np.linalg.norm(phi))
    K = _hat(phi)
    if th < 1e-8:
        Rm = np.eye(3) + K + 0.5 * K @ K
        V = np.eye(3) + 0.5 * K + K @ K / 6.0
    else:
        a = np.sin(th) / th
        b = (1 - np.cos(th)) / th ** 2
        c = (th - np.sin(th)) / th ** 3
        Rm = np.eye(3) + a * K + b * K @ K
        V = np.eye(3) + b * K + c * K @ K
    T = np.eye(4)
    T[:3, :3] = Rm
    T[:3, 3] = V @ rho
    return T


class _Cam:
    def __init__(self, base, R, t):
        self.W, self.H, self.fx, self.fy, self.cx, self.cy = base.W, base.H, base.fx, base.fy, base.cx, base.cy
        self.near = getattr(base, "near", 0.2)
        self.R, self.t = R, t


class GSRenderFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, scales, quats, opacities, sh, feats, xi, cam, rast: Rasterizer):
        T0 = np.eye(4)
        T0[:3, :3], T0[:3, 3] = np.asarray(cam.R, np.float64), np.asarray(cam.t, np.float64)
        T = se3_exp(xi.detach().double().cpu().numpy()) @ T0
        c = _Cam(cam, T[:3, :3], T[:3, 3])
        scene = L.Scene(means.detach(), scales.detach(), quats.detach(), opacities.detach(),
                        sh.detach(), feats.detach() if feats is not None else None)
        want_feat = feats is not None and feats.shape[1] > 0
        out = rast.forward(scene, c, feat=want_feat)
        # saved so that autograd rejects a backward after an in-place change of the parameters
        ctx.save_for_backward(means, scales, quats, opacities, sh, *(() if feats is None else (feats,)))
        ctx.scene, ctx.cam, ctx.rast = scene, c, rast
        ctx.generation, ctx.want_feat = rast.generation, want_feat
        ctx.feat_dtype = None if feats is None else feats.dtype
        ctx.has_feats = feats is not None
        ctx.xi_device = xi.device
        f = out["feat"] if out["feat"] is not None else torch.zeros((0,) + out["depth"].shape,
                                                                    device=means.device)
        return out["rgb"], out["depth"], out["alpha"], f

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_alpha, g_feat):
        ctx.saved_tensors   # raises if a parameter was modified in place since the forward
        if ctx.rast.generation != ctx.generation:
            # another render has used the workspace since: rebuild this render's state
            ctx.rast.forward(ctx.scene, ctx.cam, feat=ctx.want_feat)

        def c(g):
            return None if g is None else g.contiguous().float()
        gr = ctx.rast.backward(ctx.scene, ctx.cam, c(g_rgb), c(g_depth), c(g_alpha),
                               c(g_feat) if ctx.scene.n_feat else None)
        gfe = None
        if ctx.has_feats:
            gfe = gr["feats"] if gr["feats"] is not None else torch.zeros_like(ctx.scene.feats, dtype=torch.float32)
            gfe = gfe.to(ctx.feat_dtype)
        return (gr["means"], gr["scales"], gr["quats"], gr["opacities"], gr["sh"], gfe,
                gr["pose"].to(device=ctx.xi_device, dtype=torch.float32), None, None)


def render(means, scales, quats, opacities, sh, feats, cam, xi=None, rasterizer=None):
    """Differentiable render: returns (rgb [3,H,W], depth [H,W], alpha [H,W], feat [D,H,W])."""
    if rasterizer is None:
        rasterizer = Rasterizer(means.device)
    if xi is None:
        xi = torch.zeros(6, device=means.device, dtype=torch.float32)
    return GSRenderFunction.apply(means, scales, quats, opacities, sh, feats, xi, cam, rasterizer)
