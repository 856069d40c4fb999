"""Pins of the oracle's analytic gradients (App. B: the rasterizer is differentiated w.r.t.
the Gaussians for mapping, Eq. 3, and w.r.t. the camera pose for tracking, Eq. 2) against
central finite differences of the FP64 oracle, the adjoint identity and a closed form."""
import numpy as np
import pytest
import scipy.linalg

from synth import scenes as S


def fd_scene(n=500, deg=3, D=4, seed=21):
    sc = S.cube_scene(n, n_feat=D, sh_degree=deg, seed=seed, log_scale_mu=-2.6,
                      log_scale_sd=0.3, raw_quats=True)
    # higher-order SH big enough to matter
    rng = np.random.default_rng(seed + 1)
    if deg > 0:
        sc.sh[:, 1:, :] = rng.normal(0, 0.3, size=sc.sh[:, 1:, :].shape).astype(np.float32)
    return _as64(sc)


def _as64(sc):
    return S.Scene(**{k: getattr(sc, k).astype(np.float64) for k in
                      ("means", "scales", "quats", "opacities", "sh", "feats")},
                   sh_degree=sc.sh_degree)


def fd_camera(W=64, H=64):
    R, t = S.look_at(np.array([0.4, -0.3, -2.2]), np.array([0.0, 0.0, 0.0]))
    return S.pinhole(W, H, 60.0, 62.0, R, t)


def loss(oracle, sc, cam, g, thresholds):
    r = oracle.render(sc, cam, "f64", thresholds=thresholds)
    return (np.sum(g["rgb"] * r["rgb"]) + np.sum(g["depth"] * r["depth"])
            + np.sum(g["alpha"] * r["alpha"]) + np.sum(g["feat"] * r["feat"]))


def exp_se3(xi):
    """Exp of the twist (rho, phi) as a 4x4 matrix (scipy.linalg.expm of its hat)."""
    Xi = np.zeros((4, 4))
    rho, phi = xi[:3], xi[3:]
    Xi[:3, :3] = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    Xi[:3, 3] = rho
    return scipy.linalg.expm(Xi)


def perturbed_cam(cam, xi):
    T = np.eye(4)
    T[:3, :3], T[:3, 3] = cam.R, cam.t
    T2 = exp_se3(xi) @ T
    return cam.copy_with(R=T2[:3, :3], t=T2[:3, 3])


PARAMS = ("means", "scales", "quats", "opacities", "sh", "feats")


def _fd_entries(oracle, sc, cam, g, thresholds, picks, h=1e-4):
    out = []
    for name, idx in picks:
        arr = getattr(sc, name)
        old = arr[idx]
        arr[idx] = old + h
        lp = loss(oracle, sc, cam, g, thresholds)
        arr[idx] = old - h
        lm = loss(oracle, sc, cam, g, thresholds)
        arr[idx] = old
        out.append((lp - lm) / (2 * h))
    return np.array(out)


def _picks(sc, valid, rng, per=6):
    picks = []
    vis = np.nonzero(valid)[0]
    for name in PARAMS:
        arr = getattr(sc, name)
        for _ in range(per):
            i = int(rng.choice(vis))
            rest = tuple(int(rng.integers(s)) for s in arr.shape[1:])
            picks.append((name, (i,) + rest))
    return picks


@pytest.fixture(scope="module")
def fd_case(oracle):
    sc = fd_scene()
    cam = fd_camera()
    g = S.upstream_grads(cam.H, cam.W, sc.n_feat, seed=2)
    g = {k: v.astype(np.float64) for k, v in g.items()}
    return sc, cam, g


def test_fd_all_parameters_thresholds_off(oracle, fd_case):
    sc, cam, g = fd_case
    an = oracle.backward(sc, cam, g, "f64", thresholds=False)
    valid = oracle.project(sc, cam, "f64", thresholds=False)["valid"]
    rng = np.random.default_rng(0)
    picks = _picks(sc, valid, rng)
    fd = _fd_entries(oracle, sc, cam, g, False, picks)
    a = np.array([an[name][idx] for name, idx in picks])
    scale = {name: np.abs(an[name]).max() for name in PARAMS}
    floor = np.array([1e-7 * scale[name] for name, _ in picks])
    err = np.abs(fd - a)
    bad = err > 1e-4 * np.abs(a) + floor
    assert not bad.any(), [(picks[i], fd[i], a[i]) for i in np.nonzero(bad)[0]]


def test_fd_log_scale_and_logit_opacity(oracle, fd_case):
    # through the activations used by the optimiser: s = exp(l), o = sigmoid(y)
    sc, cam, g = fd_case
    an = oracle.backward(sc, cam, g, "f64", thresholds=False)
    rng = np.random.default_rng(1)
    h = 1e-4
    for _ in range(6):
        i, k = int(rng.integers(sc.n)), int(rng.integers(3))
        l0 = np.log(sc.scales[i, k])
        sc.scales[i, k] = np.exp(l0 + h); lp = loss(oracle, sc, cam, g, False)
        sc.scales[i, k] = np.exp(l0 - h); lm = loss(oracle, sc, cam, g, False)
        sc.scales[i, k] = np.exp(l0)
        assert (lp - lm) / (2 * h) == pytest.approx(an["scales"][i, k] * sc.scales[i, k], rel=1e-4,
                                                    abs=1e-7 * np.abs(an["scales"]).max())
        o0 = sc.opacities[i]
        y0 = np.log(o0 / (1 - o0))
        sc.opacities[i] = 1 / (1 + np.exp(-(y0 + h))); lp = loss(oracle, sc, cam, g, False)
        sc.opacities[i] = 1 / (1 + np.exp(-(y0 - h))); lm = loss(oracle, sc, cam, g, False)
        sc.opacities[i] = o0
        assert (lp - lm) / (2 * h) == pytest.approx(an["opacities"][i] * o0 * (1 - o0), rel=1e-4,
                                                    abs=1e-7 * np.abs(an["opacities"]).max())


def layered_scene(cam, n=200, deg=3, D=4, seed=31, gap=0.005):
    """Gaussians whose camera-space depths differ by at least ``gap``: a pose step of 1e-5
    cannot swap two of them, which would make rgb and features jump (an order swap changes
    c1 a1 + c2 a2 (1 - a1) by a1 a2 (c2 - c1))."""
    rng = np.random.default_rng(seed)
    z = 1.5 + gap * rng.permutation(n)
    xy = rng.uniform(-0.4, 0.4, size=(n, 2)) * z[:, None]
    pc = np.concatenate([xy, z[:, None]], 1)
    sc = fd_scene(n=n, deg=deg, D=D, seed=seed)
    sc.means = (pc - cam.t) @ cam.R          # R^T (p_c - t), row-wise
    return sc


def test_fd_pose_twist_thresholds_off(oracle):
    cam = fd_camera()
    sc = layered_scene(cam)
    g = {k: v.astype(np.float64) for k, v in S.upstream_grads(cam.H, cam.W, sc.n_feat).items()}
    an = oracle.backward(sc, cam, g, "f64", thresholds=False)["pose"]
    h = 1e-5
    fd = np.zeros(6)
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        fd[k] = (loss(oracle, sc, perturbed_cam(cam, e), g, False)
                 - loss(oracle, sc, perturbed_cam(cam, -e), g, False)) / (2 * h)
    np.testing.assert_allclose(an, fd, rtol=1e-5, atol=1e-7 * np.abs(an).max())


def test_adjoint_identity(oracle):
    # <grad L, v> = dL/de (theta + e v) for a random direction v over all parameters
    # (depth-layered scene so that no two Gaussians swap order under the step).
    cam = fd_camera()
    sc = layered_scene(cam)
    g = {k: v.astype(np.float64) for k, v in S.upstream_grads(cam.H, cam.W, sc.n_feat).items()}
    an = oracle.backward(sc, cam, g, "f64", thresholds=False)
    rng = np.random.default_rng(7)
    vs = {name: rng.normal(size=getattr(sc, name).shape) for name in PARAMS}
    vs["scales"] *= 0.01
    vs["opacities"] *= 0.01
    lin = sum(np.sum(an[name] * vs[name]) for name in PARAMS)
    h = 1e-5
    base = {name: getattr(sc, name).copy() for name in PARAMS}
    for name in PARAMS:
        setattr(sc, name, base[name] + h * vs[name])
    lp = loss(oracle, sc, cam, g, False)
    for name in PARAMS:
        setattr(sc, name, base[name] - h * vs[name])
    lm = loss(oracle, sc, cam, g, False)
    for name in PARAMS:
        setattr(sc, name, base[name])
    assert (lp - lm) / (2 * h) == pytest.approx(lin, rel=1e-6)


def test_pose_translation_closed_form(oracle):
    # One isotropic Gaussian on the optical axis, thresholds off, L = sum_p g(p) alpha(p).
    # Translating the camera by rho_x shifts the image by fx rho_x / z, so
    # dL/drho_x = sum_p g(p) alpha(p) (px - u) / s'^2 * fx / z.
    s, z, f, o = 0.05, 2.0, 70.0, 0.6
    sc = S.Scene(means=np.array([[0.0, 0.0, z]]), scales=np.array([[s, s, s]]),
                 quats=np.array([[1.0, 0, 0, 0]]), opacities=np.array([o]),
                 sh=np.zeros((1, 1, 3)), feats=np.zeros((1, 1)), sh_degree=0)
    cam = S.pinhole(48, 40, f)
    rng = np.random.default_rng(2)
    ga = rng.normal(size=(cam.H, cam.W))
    g = dict(alpha=ga)
    an = oracle.backward(sc, cam, g, "f64", thresholds=False)["pose"]
    var = (f * s / z) ** 2 + 0.3
    ys, xs = np.mgrid[0:cam.H, 0:cam.W]
    dx, dy = xs + 0.5 - cam.cx, ys + 0.5 - cam.cy
    al = o * np.exp(-0.5 * (dx * dx + dy * dy) / var)
    assert an[0] == pytest.approx(np.sum(ga * al * dx / var) * f / z, rel=1e-10)
    assert an[1] == pytest.approx(np.sum(ga * al * dy / var) * f / z, rel=1e-10)


def test_thresholds_on_fd_mostly_agrees(oracle):
    # With thresholds the loss is only piecewise smooth; most entries still match FD.
    sc = fd_scene(n=300, deg=1, D=3, seed=5)
    cam = fd_camera()
    g = {k: v.astype(np.float64) for k, v in S.upstream_grads(cam.H, cam.W, 3, seed=2).items()}
    an = oracle.backward(sc, cam, g, "f64", thresholds=True)
    valid = oracle.project(sc, cam, "f64")["valid"]
    picks = _picks(sc, valid, np.random.default_rng(3), per=8)
    fd = _fd_entries(oracle, sc, cam, g, True, picks, h=1e-6)
    a = np.array([an[name][idx] for name, idx in picks])
    scale = np.array([np.abs(an[name]).max() for name, _ in picks])
    ok = np.abs(fd - a) <= 1e-3 * np.abs(a) + 1e-5 * scale
    assert ok.mean() >= 0.9, ok.mean()


def test_f32_mirror_close_to_f64(oracle):
    sc, (cam,) = S.config_tiny()
    g = S.upstream_grads(cam.H, cam.W, sc.n_feat, seed=2)
    a = oracle.backward(sc, cam, g, "f32")
    b = oracle.backward(sc, cam, g, "f64")
    for name in PARAMS + ("pose",):
        rel = np.linalg.norm(a[name] - b[name]) / np.linalg.norm(b[name])
        assert rel < 1e-3, (name, rel)
