"""gs_render_fwd_noalloc: the forward render for callers that cannot allocate device memory
(a plugin whose host application owns every allocation, code held to a fixed memory
budget).  It keeps every intermediate in a fixed library-held device array, so it must
give the same images as the allocating path gs_project -> gs_bin_tiles -> gs_render_fwd,
call after call (bit for bit: the same kernels on the same inputs), and refuse requests
larger than that array without writing any output.

This file is collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test."""
import numpy as np
import pytest

from synth import scenes as S
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

def _render_alloc(rast, scene, cam):
    out = rast.forward(scene, cam)
    return {k: out[k] for k in ("rgb", "depth", "alpha", "feat")}


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
    return status, out


def _same_as_allocating_path(L, rast, sc, cam):
    import torch
    scene = U.upload(sc)
    ref = _render_alloc(rast, scene, cam)
    status, got = _render_noalloc(L, scene, cam)
    assert status == L.GS_OK, L.status_string(status)
    for k in ref:
        # the same kernels on the same inputs: bit for bit
        assert torch.equal(got[k], ref[k]), k


def _cases():
    small = S.config_tiny()[0], S.config_tiny()[1][0]                     # 48 tiles
    larger = (S.room_scene(12_000, n_feat=8, sh_degree=1, seed=5),
              S.room_trajectory(4, 200, 120, 180.0)[2])                     # 104 tiles
    return small, larger


def test_noalloc_matches_allocating_path_on_two_calls_in_a_row():
    from paper_2603_09632_gb300 import _lib as L
    from paper_2603_09632_gb300.render import Rasterizer
    rast = Rasterizer(U.device())
    small, larger = _cases()
    # two calls in a row with different inputs, in both orders: a larger call's leftovers
    # must not leak into a smaller one, nor the other way round
    for sc, cam in (small, larger, small):
        _same_as_allocating_path(L, rast, sc, cam)


def test_noalloc_rejects_requests_beyond_its_fixed_scratch():
    from paper_2603_09632_gb300 import _lib as L
    from paper_2603_09632_gb300.render import Rasterizer
    sc, (cam,) = S.config_tiny()
    big_image = S.pinhole(512, 512, 400.0, 400.0, cam.R, cam.t)     # 262144 pixels > 65536
    status, got = _render_noalloc(L, U.upload(sc), big_image)
    assert status == L.GS_ERR_OVER_BUDGET
    assert (got["alpha"] == -7.0).all()                              # nothing written
    wide = S.pinhole(1 << 20, 1, 400.0, 400.0, cam.R, cam.t)         # one row, far too wide
    assert _render_noalloc(L, U.upload(sc), wide)[0] == L.GS_ERR_OVER_BUDGET
    many = S.cube_scene(20_000, n_feat=2)                            # > 16384 Gaussians
    status, _ = _render_noalloc(L, U.upload(many), cam)
    assert status == L.GS_ERR_OVER_BUDGET
    # 4000 large Gaussians on a 256 x 256 image: about 200k tile instances > 131072.  The
    # refusal comes after projection has run and left its tile counts in the array; the
    # next call must not see them.
    crowd = S.cube_scene(4000, n_feat=4, seed=8, log_scale_mu=-2.0, log_scale_sd=0.2)
    c256 = S.pinhole(256, 256, 200.0, 200.0, cam.R, cam.t)
    status, got = _render_noalloc(L, U.upload(crowd), c256)
    assert status == L.GS_ERR_OVER_BUDGET
    for k, v in got.items():
        assert (v == -7.0).all(), k
    rast = Rasterizer(U.device())
    small, larger = _cases()
    _same_as_allocating_path(L, rast, *larger)
    _same_as_allocating_path(L, rast, *small)
