"""Phase-specialised backward (NEXT-3): the semantic phase of Sec. 3.2 freezes geometry and
colour, so only the feature gradient is requested (the rasterizer then skips every geometry
term and the projection backward); tracking (Eq. 2) asks for the pose gradient only.  Each
specialised call must equal the same outputs of the full backward, and the oracle."""
import numpy as np
import pytest

from synth import scenes as S
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def _setup(oracle, D=32, bf16=False, stride=1, off=(0, 0)):
    """Scene, camera and upstream gradients, the latter zeroed at the pixels (samples) the
    oracle flags as within rounding distance of a blend threshold."""
    import torch
    from oracle import grid as OG
    from paper_2603_09632_gb300.render import Rasterizer, as_camera, grid_shape
    sc = S.room_scene(40_000, n_feat=D, sh_degree=1, seed=17)
    cam = S.room_trajectory(8, 240, 176, 210.0)[5]
    c = as_camera(cam, stride, *off)
    rast = Rasterizer(U.device())
    scene = U.upload(sc, bf16=bf16)
    rast.forward(scene, c)
    Hs, Ws = grid_shape(c)
    feats = U.bf16_round(sc.feats) if bf16 else None
    flags = (oracle.render(sc, cam, "f32", feats=feats) if stride == 1 else
             OG.render(sc, cam, c.stride, c.off_x, c.off_y, "f32", feats=feats))["flags"]
    g, _ = U.mask_flagged(S.upstream_grads(Hs, Ws, D, seed=31), flags)
    gt = {k: torch.from_numpy(v).to(U.device()) for k, v in g.items()}
    return sc, cam, c, rast, scene, g, gt


@pytest.mark.parametrize("D,bf16,stride", [(32, False, 1), (64, True, 1), (16, False, 3)])
def test_features_only_backward(oracle, D, bf16, stride):
    import torch
    from paper_2603_09632_gb300 import _lib as L
    sc, cam, c, rast, scene, g, gt = _setup(oracle, D, bf16, stride, (1, 2) if stride > 1 else (0, 0))
    n = sc.n
    full = rast.backward(scene, c, gt["rgb"], gt["depth"], gt["alpha"], gt["feat"])
    gf = torch.full((n, D), float("nan"), device=U.device())
    L.gs_render_bwd(scene, c, rast.ws, g_rgb=gt["rgb"], g_depth=gt["depth"], g_alpha=gt["alpha"],
                    g_feat=gt["feat"], g_feats=gf)
    torch.cuda.synchronize()
    assert torch.isfinite(gf).all()
    # same terms, summed in another order by the specialised kernel
    U.assert_grads_close({"feats": gf.cpu().numpy()}, {"feats": full["feats"].cpu().numpy()},
                         ["feats"], rtol=1e-4, floor=1e-6, norm_tol=1e-6,
                         label=f"features-only vs full D={D} s={stride}")
    # and against the oracle (features only depend on the feature upstream gradient)
    feats = U.bf16_round(sc.feats) if bf16 else None
    if stride == 1:
        ref = oracle.backward(sc, cam, {"feat": g["feat"]}, "f32", feats=feats)
        alt = oracle.backward(sc, cam, {"feat": g["feat"]}, "mixed", feats=feats)
    else:
        from oracle import grid as OG
        ref = OG.backward(sc, cam, c.stride, c.off_x, c.off_y, {"feat": g["feat"]}, "f32", feats=feats)
        alt = OG.backward(sc, cam, c.stride, c.off_x, c.off_y, {"feat": g["feat"]}, "mixed", feats=feats)
    U.assert_grads_close({"feats": gf.cpu().numpy()}, ref, ["feats"], ref_alt=alt,
                         label=f"features-only vs oracle D={D} s={stride}")


def test_pose_only_backward(oracle):
    import torch
    from paper_2603_09632_gb300 import _lib as L
    sc, cam, c, rast, scene, g, gt = _setup(oracle, D=16)
    full = rast.backward(scene, c, gt["rgb"], gt["depth"], gt["alpha"], None)
    pose = torch.full((6,), float("nan"), device=U.device())
    L.gs_render_bwd(scene, c, rast.ws, g_rgb=gt["rgb"], g_depth=gt["depth"], g_alpha=gt["alpha"],
                    g_pose6=pose)
    torch.cuda.synchronize()
    U.assert_grads_close({"pose": pose.cpu().numpy()}, {"pose": full["pose"].cpu().numpy()},
                         ["pose"], rtol=1e-4, floor=1e-6, norm_tol=1e-5, label="pose-only vs full")
    gi = {k: g[k] for k in ("rgb", "depth", "alpha")}
    U.assert_grads_close({"pose": pose.cpu().numpy()}, oracle.backward(sc, cam, gi, "f32"), ["pose"],
                         ref_alt=oracle.backward(sc, cam, gi, "mixed"), label="pose-only vs oracle")
