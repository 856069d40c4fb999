"""Convenience layer over the C ABI: allocate outputs with PyTorch and run the four steps
(gs_project -> gs_bin_tiles -> gs_render_fwd -> gs_render_bwd) on one workspace."""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as L


def as_camera(cam, stride=1, off_x=0, off_y=0) -> L.gs_camera:
    """Camera from any object with W, H, fx, fy, cx, cy, R (3x3 world->camera), t, near."""
    if isinstance(cam, L.gs_camera):
        return cam
    return L.make_camera(cam.W, cam.H, cam.fx, cam.fy, cam.cx, cam.cy, np.asarray(cam.R),
                         np.asarray(cam.t), getattr(cam, "near", 0.2), stride, off_x, off_y)


def grid_shape(cam):
    """(rows, cols) of the rendered pixels: the image, or the compact stride-s sample grid
    ceil(H / s) x ceil(W / s)."""
    s = max(int(cam.stride), 1)
    return (cam.H + s - 1) // s, (cam.W + s - 1) // s


class Rasterizer:
    """One workspace on one device.  Not thread-safe; one stream order at a time.

    The workspace holds the state of the most recent forward (projection, tile lists,
    per-pixel transmittance and last-contributor counts), which ``backward`` consumes.
    ``generation`` counts the forwards, so that a caller holding an older forward can tell
    that the workspace has moved on (the autograd function then recomputes its forward)."""

    def __init__(self, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.ws = L.Workspace(self.device.index)
        self.generation = 0

    def reserve(self, n_gauss, n_instances, n_pixels):
        L.gs_workspace_reserve(self.ws, n_gauss, n_instances, n_pixels)

    def forward(self, scene: L.Scene, cam, feat=True, sync=True, stream=None, out=None):
        """Project, bin and render.  Returns dict rgb [3,H,W], depth [H,W], alpha [H,W],
        feat [D,H,W] (float32 device tensors; H, W = grid_shape(cam) for a sample-grid
        camera) and, with ``sync``, the instance count."""
        c = as_camera(cam)
        H, W = grid_shape(c)
        dev = self.device
        if out is None:
            out = dict(rgb=torch.empty((3, H, W), device=dev), depth=torch.empty((H, W), device=dev),
                       alpha=torch.empty((H, W), device=dev),
                       feat=torch.empty((scene.n_feat, H, W), device=dev) if feat and scene.n_feat else None)
        self.generation += 1
        L.gs_project(scene, c, self.ws, stream)
        n_inst = L.gs_bin_tiles(self.ws, sync, stream)
        L.gs_render_fwd(scene, c, self.ws, out["rgb"], out["depth"], out["alpha"], out.get("feat"),
                        stream)
        if sync:
            out["instances"] = n_inst
        return out

    def backward(self, scene: L.Scene, cam, g_rgb=None, g_depth=None, g_alpha=None, g_feat=None,
                 stream=None, grads=None):
        """Gradients of the last forward w.r.t. every Gaussian parameter and the pose twist."""
        c = as_camera(cam)
        n, D, K = scene.n, scene.n_feat, (scene.sh_degree + 1) ** 2
        dev = self.device
        if grads is None:
            grads = dict(means=torch.empty((n, 3), device=dev), scales=torch.empty((n, 3), device=dev),
                         quats=torch.empty((n, 4), device=dev), opacities=torch.empty(n, device=dev),
                         sh=torch.empty((n, K, 3), device=dev),
                         feats=torch.empty((n, D), device=dev) if D else None,
                         pose=torch.empty(6, device=dev))
        L.gs_render_bwd(scene, c, self.ws, g_rgb, g_depth, g_alpha, g_feat if D else None,
                        grads["means"], grads["scales"], grads["quats"], grads["opacities"],
                        grads["sh"], grads.get("feats"), grads["pose"], stream)
        return grads

    def stats(self, stream=None):
        return L.gs_get_stats(self.ws, stream)

    def close(self):
        self.ws.close()
