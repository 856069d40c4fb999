"""The torch.autograd.Function over gs_render_fwd / gs_render_bwd (App. B: the rasterizer is
differentiated for mapping, Eq. 3, and tracking, Eq. 2), with the optimiser's own
parameterisation (log-scales, opacity logits) chained by PyTorch above the C ABI.

Checked against the FP64 oracle's analytic gradient (thresholds on, same function as the
GPU) element by element, against central finite differences of the FP64 oracle on the
500-Gaussian 64x64 scene (step 1e-4; threshold crossings counted), and against central
differences of every parameter group and the pose twist in a regime where no blend
threshold is active (step 1e-5; no outliers allowed)."""
import numpy as np
import pytest

from synth import scenes as S
from tests import gpu_util as U
from tests.test_oracle_backward import fd_camera, fd_scene, layered_scene, loss, perturbed_cam

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
    b = oracle.backward(sc64, cam, {k: v.astype(np.float64) for k, v in g.items()},
                        "mixed" if thresholds else "f64", thresholds=thresholds)
    o = sc64.opacities
    return dict(means=b["means"], log_scales=b["scales"] * sc64.scales, quats=b["quats"],
                logits=b["opacities"] * o * (1 - o), sh=b["sh"], feats=b["feats"], xi=b["pose"])


def test_autograd_matches_oracle_analytic_fp64(oracle):
    sc = fd_scene(n=500, deg=3, D=4, seed=21)
    cam = fd_camera()
    sc32 = S.Scene(**{k: np.asarray(getattr(sc, k), np.float32) for k in
                      ("means", "scales", "quats", "opacities", "sh", "feats")}, sh_degree=sc.sh_degree)
    # upstream gradient zeroed where the GPU's FP32 decisions may take the other branch
    g, nflag = U.mask_flagged(S.upstream_grads(cam.H, cam.W, sc.n_feat, seed=2),
                              oracle.render(sc32, cam, "f32")["flags"])
    got, _ = _autograd_grads(sc, cam, g)
    ref = _oracle_in_leaf_coords(oracle, sc, cam, g)
    U.assert_grads_close(got, ref, list(ref), label=f"autograd vs FP64 analytic ({nflag} flagged px)")


LEAF_OF = (("means", "means"), ("quats", "quats"), ("sh", "sh"), ("feats", "feats"),
           ("log_scales", "scales"), ("logits", "opacities"))


def _leaf_fd(oracle, sc64, cam, g, name, attr, idx, h):
    """Central difference of the FP64 oracle's loss in the optimiser's leaf coordinate."""
    arr = getattr(sc64, attr)
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
    return (lp - lm) / (2 * h)


def _pose_fd(oracle, sc64, cam, g, k, h):
    e = np.zeros(6)
    e[k] = h
    return (loss(oracle, sc64, perturbed_cam(cam, e), g, True)
            - loss(oracle, sc64, perturbed_cam(cam, -e), g, True)) / (2 * h)


def test_autograd_matches_fp64_finite_differences(oracle):
    # FD of the FP64 oracle with the GPU's thresholds on a depth-layered 500-Gaussian scene:
    # the loss is only piecewise smooth there (a step can carry a Gaussian's alpha across
    # 1/255 at some pixel), so entries whose FD interval crosses a threshold are counted and
    # reported, not failed.  20 entries per parameter group.  (A pose step moves every
    # Gaussian's 1/255 contour at once, so the pose twist is checked in the smooth regime.)
    cam = fd_camera()
    sc = layered_scene(cam, n=500, deg=3, D=4, seed=33)
    g = {k: v.astype(np.float64) for k, v in S.upstream_grads(cam.H, cam.W, sc.n_feat).items()}
    got, _ = _autograd_grads(sc, cam, g)
    rng = np.random.default_rng(4)
    sc64 = S.Scene(**{k: np.asarray(getattr(sc, k), np.float32).astype(np.float64) for k in
                      ("means", "scales", "quats", "opacities", "sh", "feats")}, sh_degree=3)
    vis = np.nonzero(oracle.project(sc64, cam, "f64")["valid"])[0]
    outliers, total = [], 0
    for name, attr in LEAF_OF:
        arr = getattr(sc64, attr)
        scale = np.abs(got[name]).max()
        for _ in range(20):
            i = int(rng.choice(vis))
            idx = (i,) + tuple(int(rng.integers(s)) for s in arr.shape[1:])
            fd = _leaf_fd(oracle, sc64, cam, g, name, attr, idx, 1e-4)
            a = got[name][idx]
            total += 1
            if abs(fd - a) > 1e-2 * abs(a) + 1e-4 * scale:
                outliers.append((name, idx, float(fd), float(a)))
    U._report("autograd FD, thresholds on (layered 500 Gaussians)",
              {"outliers": (len(outliers), 0.0, total)})
    assert len(outliers) <= 0.1 * total, (len(outliers), total, outliers)


def smooth_scene(cam, n=20, seed=5):
    """Large, semi-transparent Gaussians at distinct depths covering the whole 64 x 64 view:
    at every pixel each Gaussian's alpha lies well inside (1/255, 0.99), sigma >= 0, the
    transmittance stays above 1e-4 after all of them and every 3-sigma rectangle is the
    whole image, so no threshold of the blend is active and the loss is smooth in every
    parameter and in the pose."""
    rng = np.random.default_rng(seed)
    z = 2.2 + np.linspace(-0.6, 0.6, n)[rng.permutation(n)]
    xy = rng.uniform(-0.15, 0.15, size=(n, 2)) * z[:, None]
    pc = np.concatenate([xy, z[:, None]], 1)
    q = rng.normal(size=(n, 4))
    q[:, 0] += 2.0
    sh = rng.normal(0, 0.3, size=(n, 16, 3))
    sh[:, 0, :] = rng.uniform(-1, 1, size=(n, 3))
    sc = S.Scene(means=(pc - cam.t) @ cam.R, scales=np.exp(rng.uniform(np.log(1.2), np.log(2.0), (n, 3))),
                 quats=q, opacities=rng.uniform(0.08, 0.3, n), sh=sh,
                 feats=rng.normal(size=(n, 4)), sh_degree=3)
    return S.Scene(**{k: np.asarray(getattr(sc, k), np.float32).astype(np.float64) for k in
                      ("means", "scales", "quats", "opacities", "sh", "feats")}, sh_degree=3)


def test_autograd_fd_smooth_regime_every_parameter_and_pose(oracle):
    """Where no blend threshold is active the thresholded loss is smooth, so central
    differences of the FP64 oracle (step 1e-5) converge for every parameter and for the
    pose twist xi (perturbed through Exp, T = Exp(xi) T0).  Every sampled entry of the GPU
    gradient (at least 20 per group where the group has them, all six of xi) must lie
    within 1e-3 of FD plus 1e-5 of the group's largest entry: no outliers allowed."""
    cam = fd_camera()
    sc64 = smooth_scene(cam)
    n = sc64.n
    # the regime itself: nothing flagged, every Gaussian blended at every pixel
    r = oracle.render(sc64, cam, "f32")
    assert (r["flags"] == 0).all() and (r["n_contrib"] == n).all()
    assert r["T_final"].min() > 1e-3
    p = oracle.project(sc64, cam, "f64")
    assert p["valid"].all() and (p["rect"] == [0, 0, 4, 4]).all()
    ys, xs = np.mgrid[0:cam.H, 0:cam.W] + 0.5
    for i in range(n):
        (u, v), (a, b, c) = p["mean2d"][i], p["conic"][i]
        sig = 0.5 * (a * (xs - u) ** 2 + c * (ys - v) ** 2) + b * (xs - u) * (ys - v)
        al = sc64.opacities[i] * np.exp(-sig)
        assert sig.min() >= 0 and al.min() > 2 / 255 and al.max() < 0.9

    g = {k: v.astype(np.float64) for k, v in S.upstream_grads(cam.H, cam.W, sc64.n_feat, seed=9).items()}
    got, _ = _autograd_grads(sc64, cam, g)
    rng = np.random.default_rng(6)
    bad, total = [], 0
    for name, attr in LEAF_OF + (("xi", None),):
        if name == "xi":
            idxs = [(k,) for k in range(6)]
        else:
            all_idx = list(np.ndindex(getattr(sc64, attr).shape))
            pick = rng.choice(len(all_idx), size=min(len(all_idx), 24), replace=False)
            idxs = [all_idx[j] for j in pick]
        fds = np.array([_pose_fd(oracle, sc64, cam, g, idx[0], 1e-5) if name == "xi" else
                        _leaf_fd(oracle, sc64, cam, g, name, attr, idx, 1e-5) for idx in idxs])
        a = np.array([got[name][idx] for idx in idxs])
        bound = 1e-3 * np.abs(fds) + 1e-5 * np.abs(fds).max()
        total += len(idxs)
        for j in np.nonzero(np.abs(a - fds) > bound)[0]:
            bad.append((name, idxs[j], float(fds[j]), float(a[j])))
    U._report("autograd FD, smooth regime (20 Gaussians, every group and xi)",
              {"outliers": (len(bad), 0.0, total)})
    assert not bad, bad


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


def test_two_renders_share_a_rasterizer_before_one_backward():
    """Two keyframes rendered through one Rasterizer, their losses summed, one backward (a
    mapping step of Eq. 3): each render's gradient must be that of its own forward, equal
    to the same renders on separate rasterizers."""
    import torch
    from paper_2603_09632_gb300.autograd import render
    from paper_2603_09632_gb300.render import Rasterizer
    sc = S.room_scene(20_000, n_feat=8, sh_degree=1, seed=3)
    cams = S.room_trajectory(8, 160, 120, 150.0)
    dev = U.device()
    g = [S.upstream_grads(120, 160, 8, seed=50 + k) for k in range(2)]

    def run(shared):
        p = {k: torch.tensor(np.asarray(getattr(sc, k), np.float32), device=dev, requires_grad=True)
             for k in ("means", "scales", "quats", "opacities", "sh", "feats")}
        xis = [torch.zeros(6, requires_grad=True) for _ in range(2)]   # host twists: no sync
        rs = [Rasterizer(dev)] * 2 if shared else [Rasterizer(dev), Rasterizer(dev)]
        total = 0
        for k, cam in enumerate((cams[1], cams[4])):
            outs = render(p["means"], p["scales"], p["quats"], p["opacities"], p["sh"], p["feats"],
                          cam, xi=xis[k], rasterizer=rs[k])
            for o, name in zip(outs, ("rgb", "depth", "alpha", "feat")):
                total = total + (o * torch.from_numpy(g[k][name]).to(dev)).sum()
        total.backward()
        res = {k: v.grad.cpu().numpy() for k, v in p.items()}
        for k in range(2):
            assert xis[k].grad.device.type == "cpu"
            res[f"xi{k}"] = xis[k].grad.numpy()
        return res

    sep, shared = run(False), run(True)
    keys = list(sep)
    U.assert_grads_close(shared, sep, keys, rtol=1e-4, floor=1e-6, norm_tol=1e-5,
                         label="two renders on one rasterizer vs separate")
