"""gs_render_fwd_noalloc: the forward render for callers that cannot allocate device memory
(a plugin whose host application owns every allocation, code held to a fixed memory
budget).  It keeps every intermediate in a fixed library-held device array, so it must
give the same images as the allocating path gs_project -> gs_bin_tiles -> gs_render_fwd,
call after call, and refuse requests larger than that array.

This file is collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test."""
import numpy as np
import pytest

from synth import scenes as S
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

TOL = 1e-4   # the forward parity tolerance of the other GPU tests


def _render_alloc(rast, scene, cam):
    out = rast.forward(scene, cam)
    return {k: out[k].cpu().numpy() for k in ("rgb", "depth", "alpha", "feat")}


def _render_noalloc(L, scene, cam):
    import torch
    dev = U.device()
    out = dict(rgb=torch.full((3, cam.H, cam.W), -7.0, device=dev),
               depth=torch.full((cam.H, cam.W), -7.0, device=dev),
               alpha=torch.full((cam.H, cam.W), -7.0, device=dev),
               feat=torch.full((scene.n_feat, cam.H, cam.W), -7.0, device=dev))
    c = L.make_camera(cam.W, cam.H, cam.fx, cam.fy, cam.cx, cam.cy, cam.R, cam.t, cam.near)
    status = L.gs_render_fwd_noalloc(scene, c, out["rgb"], out["depth"], out["alpha"], out["feat"])
    torch.cuda.synchronize()
    return status, {k: v.cpu().numpy() for k, v in out.items()}


def test_noalloc_matches_allocating_path_on_two_calls_in_a_row():
    from paper_2603_09632_gb300 import _lib as L
    from paper_2603_09632_gb300.render import Rasterizer
    rast = Rasterizer(U.device())
    sc_a, (cam_a,) = S.config_tiny()
    sc_b = S.room_scene(12_000, n_feat=8, sh_degree=1, seed=5)
    cam_b = S.room_trajectory(4, 200, 120, 180.0)[2]
    for sc, cam in ((sc_a, cam_a), (sc_b, cam_b)):      # two calls in a row, different inputs
        scene = U.upload(sc)
        ref = _render_alloc(rast, scene, cam)
        status, got = _render_noalloc(L, scene, cam)
        assert status == L.GS_OK, L.status_string(status)
        for k in ref:
            assert np.abs(got[k] - ref[k]).max() <= TOL, k


def test_noalloc_rejects_requests_beyond_its_fixed_scratch():
    from paper_2603_09632_gb300 import _lib as L
    sc, (cam,) = S.config_tiny()
    big_image = S.pinhole(512, 512, 400.0, 400.0, cam.R, cam.t)     # 262144 pixels > 65536
    status, got = _render_noalloc(L, U.upload(sc), big_image)
    assert status == L.GS_ERR_OVER_BUDGET
    assert np.all(got["alpha"] == -7.0)                              # nothing written
    many = S.cube_scene(20_000, n_feat=2)                            # > 16384 Gaussians
    status, _ = _render_noalloc(L, U.upload(many), cam)
    assert status == L.GS_ERR_OVER_BUDGET
