"""The torch.autograd.Function over gs_render_fwd / gs_render_bwd (App. B: the rasterizer is
differentiated for mapping, Eq. 3, and tracking, Eq. 2), with the optimiser's own
parameterisation (log-scales, opacity logits) chained by PyTorch above the C ABI.

Checked against the FP64 oracle's analytic gradient (thresholds on, same function as the
GPU) and against central finite differences of the FP64 oracle on the 500-Gaussian 64x64
scene (step 1e-4)."""
import numpy as np
import pytest

from synth import scenes as S
from tests import gpu_util as U
from tests.test_oracle_backward import fd_camera, fd_scene, layered_scene, loss

pytestmark = pytest.mark.gpu


def _leaves(sc, dev):
    import torch
    t = lambda a: torch.tensor(np.asarray(a, np.float32), device=dev, requires_grad=True)
    return dict(means=t(sc.means), log_scales=t(np.log(sc.scales)), quats=t(sc.quats),
                logits=t(np.log(sc.opacities / (1 - sc.opacities))), sh=t(sc.sh), feats=t(sc.feats),
                xi=t(np.zeros(6)))


def _autograd_grads(sc, cam, g):
    import torch
    from paper_2603_09632_gb300.autograd import render
    dev = U.device()
    p = _leaves(sc, dev)
    rgb, depth, alpha, feat = render(p["means"], torch.exp(p["log_scales"]), p["quats"],
                                     torch.sigmoid(p["logits"]), p["sh"], p["feats"], cam, xi=p["xi"])
    gt = {k: torch.tensor(v, device=dev) for k, v in g.items()}
    L = (rgb * gt["rgb"]).sum() + (depth * gt["depth"]).sum() + (alpha * gt["alpha"]).sum() + \
        (feat * gt["feat"]).sum()
    L.backward()
    return {k: v.grad.detach().cpu().double().numpy() for k, v in p.items()}, float(L)


def _oracle_in_leaf_coords(oracle, sc, cam, g, thresholds=True):
    sc64 = S.Scene(**{k: np.asarray(getattr(sc, k), np.float32).astype(np.float64) for k in
                      ("means", "scales", "quats", "opacities", "sh", "feats")}, sh_degree=sc.sh_degree)
    b = oracle.backward(sc64, cam, {k: v.astype(np.float64) for k, v in g.items()}, "f64",
                        thresholds=thresholds)
    o = sc64.opacities
    return dict(means=b["means"], log_scales=b["scales"] * sc64.scales, quats=b["quats"],
                logits=b["opacities"] * o * (1 - o), sh=b["sh"], feats=b["feats"], xi=b["pose"])


def test_autograd_matches_oracle_analytic_fp64(oracle):
    sc = fd_scene(n=500, deg=3, D=4, seed=21)
    cam = fd_camera()
    g = S.upstream_grads(cam.H, cam.W, sc.n_feat, seed=2)
    got, _ = _autograd_grads(sc, cam, g)
    ref = _oracle_in_leaf_coords(oracle, sc, cam, g)
    for k in ref:
        assert U.rel_err(got[k], ref[k]) <= 1e-3, k


def test_autograd_matches_fp64_finite_differences(oracle):
    # FD of the FP64 oracle with the GPU's thresholds; the loss is only piecewise smooth
    # there, so entries whose FD interval crosses a threshold are counted, not failed.
    cam = fd_camera()
    sc = layered_scene(cam, n=500, deg=3, D=4, seed=33)
    g = {k: v.astype(np.float64) for k, v in S.upstream_grads(cam.H, cam.W, sc.n_feat).items()}
    got, _ = _autograd_grads(sc, cam, g)
    rng = np.random.default_rng(4)
    h = 1e-4
    sc64 = S.Scene(**{k: np.asarray(getattr(sc, k), np.float32).astype(np.float64) for k in
                      ("means", "scales", "quats", "opacities", "sh", "feats")}, sh_degree=3)
    vis = np.nonzero(oracle.project(sc64, cam, "f64")["valid"])[0]
    ok, total = 0, 0
    for name, attr in (("means", "means"), ("quats", "quats"), ("sh", "sh"), ("feats", "feats"),
                       ("log_scales", "scales"), ("logits", "opacities")):
        arr = getattr(sc64, attr)
        for _ in range(6):
            i = int(rng.choice(vis))
            idx = (i,) + tuple(int(rng.integers(s)) for s in arr.shape[1:])
            old = arr[idx]
            if name == "log_scales":
                vals = (old * np.exp(h), old * np.exp(-h))
            elif name == "logits":
                y = np.log(old / (1 - old))
                vals = (1 / (1 + np.exp(-(y + h))), 1 / (1 + np.exp(-(y - h))))
            else:
                vals = (old + h, old - h)
            arr[idx] = vals[0]
            lp = loss(oracle, sc64, cam, g, True)
            arr[idx] = vals[1]
            lm = loss(oracle, sc64, cam, g, True)
            arr[idx] = old
            fd = (lp - lm) / (2 * h)
            a = got[name][idx]
            scale = np.abs(got[name]).max()
            total += 1
            ok += abs(fd - a) <= 1e-2 * abs(a) + 1e-4 * scale
    assert ok / total >= 0.85, (ok, total)


def test_autograd_pose_gradient_tracks(oracle):
    # a few steps of gradient descent on the pose twist alone reduce a photometric L2 loss
    import torch
    from paper_2603_09632_gb300.autograd import render, se3_exp
    from paper_2603_09632_gb300.render import Rasterizer
    sc, (cam,) = S.config_tiny()
    dev = U.device()
    rast = Rasterizer(dev)
    t = lambda a: torch.tensor(np.asarray(a, np.float32), device=dev)
    args = (t(sc.means), t(sc.scales), t(sc.quats), t(sc.opacities), t(sc.sh), t(sc.feats))
    target = render(*args, cam, rasterizer=rast)[0].detach()
    T = np.eye(4)
    T[:3, :3], T[:3, 3] = cam.R, cam.t
    T = se3_exp(np.array([0.02, -0.015, 0.01, 0.01, -0.01, 0.005])) @ T
    cur = cam.copy_with(R=T[:3, :3], t=T[:3, 3])
    losses = []
    for _ in range(30):
        xi = torch.zeros(6, device=dev, requires_grad=True)
        rgb = render(*args, cur, xi=xi, rasterizer=rast)[0]
        L = ((rgb - target) ** 2).sum()
        L.backward()
        losses.append(float(L))
        gx = xi.grad.double().cpu().numpy()
        step = -0.5 * float(L) / max(float(gx @ gx), 1e-30) * gx      # Polyak step (L* = 0)
        Tn = se3_exp(step) @ np.vstack([np.hstack([cur.R, cur.t[:, None]]), [0, 0, 0, 1]])
        cur = cur.copy_with(R=Tn[:3, :3], t=Tn[:3, 3])
    assert losses[-1] < 0.5 * losses[0], losses
