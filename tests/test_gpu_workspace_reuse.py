"""One workspace across calls, on the GPU: the binning's tile counts and the forward and
sort queues are put back to zero by the kernels that use them (the scan clears the counts
after reading them, the last CTA to leave a queue resets it), the backward's accumulators
and queue are cleared by the host before each backward, and the host clears the counts
itself when a projection was not followed by a binning.  Calls in any valid order and on
cameras of different sizes must therefore give the results of a fresh workspace.  Checked
against a fresh workspace (bit-exact lists, images and gradients up to the order of float
atomics)."""
import numpy as np
import pytest

from synth import scenes as S
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def _scene():
    return S.room_scene(20_000, n_feat=8, sh_degree=1, seed=5)


def _cams():
    big = S.room_trajectory(6, 160, 112, 150.0)
    small = S.room_trajectory(6, 72, 40, 70.0)
    return [big[1], small[2], big[4], small[5], big[1]]


def _fresh(scene, cam, g):
    from paper_2603_09632_gb300.render import Rasterizer
    import torch
    r = Rasterizer(U.device())
    out = r.forward(scene, cam)
    gt = {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).to(U.device()) for k, v in g.items()}
    grads = r.backward(scene, cam, gt["rgb"], gt["depth"], gt["alpha"], gt["feat"])
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items() if isinstance(v, torch.Tensor)}
    res["grads"] = {k: v.cpu().numpy() for k, v in grads.items() if v is not None}
    r.close()
    return res


def _lists(ws, cam):
    from paper_2603_09632_gb300 import _lib as L
    TX, TY = (cam.W + 15) // 16, (cam.H + 15) // 16
    return L.gs_get_instances(ws, TX * TY)


def test_reused_workspace_matches_fresh_ones():
    import torch
    from paper_2603_09632_gb300 import _lib as L
    from paper_2603_09632_gb300.render import Rasterizer, as_camera
    sc = _scene()
    scene = U.upload(sc)
    rast = Rasterizer(U.device())
    for k, cam in enumerate(_cams()):
        g = S.upstream_grads(cam.H, cam.W, sc.n_feat, seed=40 + k)
        ref = _fresh(scene, cam, g)
        c = as_camera(cam)
        if k == 1:
            # a projection that is never binned: its tile counts must not leak into the next
            L.gs_project(scene, c, rast.ws)
        out = rast.forward(scene, cam)
        if k == 2:
            # binning again for the same projection changes nothing
            before = _lists(rast.ws, cam)
            L.gs_bin_tiles(rast.ws, sync=True)
            after = _lists(rast.ws, cam)
            for a, b in zip(before, after):
                np.testing.assert_array_equal(a, b)
        gt = {n: torch.from_numpy(np.ascontiguousarray(v, np.float32)).to(U.device()) for n, v in g.items()}
        grads = rast.backward(scene, cam, gt["rgb"], gt["depth"], gt["alpha"], gt["feat"])
        if k == 3:
            # a second backward of the same projection (accumulators cleared after use)
            grads = rast.backward(scene, cam, gt["rgb"], gt["depth"], gt["alpha"], gt["feat"])
        torch.cuda.synchronize()
        for n in ("rgb", "depth", "alpha", "feat"):
            np.testing.assert_array_equal(out[n].cpu().numpy(), ref[n], err_msg=f"{n} at camera {k}")
        keys = [n for n, v in grads.items() if v is not None]
        U.assert_grads_close({n: grads[n].cpu().numpy() for n in keys}, ref["grads"], keys,
                             rtol=1e-4, floor=1e-6, norm_tol=1e-5, label=f"reused workspace, camera {k}")
    rast.close()
