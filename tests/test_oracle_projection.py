"""Pins of the oracle's projection (App. A: Sigma = R S S^T R^T, Sigma' = J W Sigma W^T J^T)
and of its real SH basis, against facts that do not come from the oracle itself."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from synth import scenes as S


def one_gaussian(mu, scale, quat=(1, 0, 0, 0), opac=0.8, sh=None, deg=0, feats=None):
    K = (deg + 1) ** 2
    shv = np.zeros((1, K, 3), np.float32) if sh is None else np.asarray(sh, np.float32).reshape(1, K, 3)
    f = np.zeros((1, 1), np.float32) if feats is None else np.asarray(feats, np.float32).reshape(1, -1)
    return S.Scene(means=np.asarray([mu], np.float32), scales=np.asarray([scale], np.float32),
                   quats=np.asarray([quat], np.float32), opacities=np.asarray([opac], np.float32),
                   sh=shv, feats=f, sh_degree=deg)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_isotropic_on_axis_closed_form(oracle, prec):
    # An isotropic Gaussian of std s on the optical axis at depth z images to an
    # isotropic 2D Gaussian of std f s / z at the principal point; +0.3 px^2 dilation.
    s, z, f = 0.05, 2.0, 100.0
    sc = one_gaussian((0.0, 0.0, z), (s, s, s))
    cam = S.pinhole(128, 96, f)
    p = oracle.project(sc, cam, prec)
    assert p["valid"][0]
    s = float(sc.scales[0, 0])                                # the float32 value passed in
    var = (f * s / z) ** 2 + 0.3
    tol = 1e-6 if prec == "f32" else 1e-12
    np.testing.assert_allclose(p["mean2d"][0], [64.0, 48.0], rtol=tol)
    np.testing.assert_allclose(p["conic"][0], [1 / var, 0.0, 1 / var], rtol=tol, atol=tol)
    assert p["depth"][0] == pytest.approx(z, rel=tol)


def _fd_jacobian_world(cam, mu, h=1e-6):
    """d(u,v)/d(mu) of the exact pinhole map, by central differences."""
    def uv(m):
        pc = cam.R @ m + cam.t
        return np.array([cam.fx * pc[0] / pc[2] + cam.cx, cam.fy * pc[1] / pc[2] + cam.cy])
    J = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        J[:, k] = (uv(mu + e) - uv(mu - e)) / (2 * h)
    return J


def test_general_covariance_matches_linearised_pinhole(oracle):
    # Sigma' - 0.3 I must equal Jw Sigma Jw^T where Jw is the numerical Jacobian of the
    # exact pinhole projection w.r.t. the world position, and Sigma = R diag(s^2) R^T with
    # R from scipy's quaternion convention (scalar last there, scalar first here).
    rng = np.random.default_rng(5)
    R, t = S.look_at(np.array([0.3, -0.2, -2.5]), np.array([0.1, 0.05, 0.0]))
    cam = S.pinhole(200, 150, 180.0, 170.0, R, t)
    for _ in range(20):
        mu = rng.uniform(-0.3, 0.3, 3)
        s = np.exp(rng.normal(-3, 0.4, 3))
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        sc = one_gaussian(mu, s, q)
        mu, s, q = (sc.means[0].astype(np.float64), sc.scales[0].astype(np.float64),
                    sc.quats[0].astype(np.float64))
        q = q / np.linalg.norm(q)
        p = oracle.project(sc, cam, "f64")
        assert p["valid"][0]
        Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        Sig = Rq @ np.diag(s ** 2) @ Rq.T
        Jw = _fd_jacobian_world(cam, mu)
        cov = Jw @ Sig @ Jw.T + 0.3 * np.eye(2)
        conic = np.linalg.inv(cov)
        np.testing.assert_allclose(p["conic"][0], [conic[0, 0], conic[0, 1], conic[1, 1]],
                                   rtol=1e-6, atol=1e-9)
        pc = R @ mu + t
        np.testing.assert_allclose(p["depth"][0], pc[2], rtol=1e-12)
        np.testing.assert_allclose(p["mean2d"][0], [cam.fx * pc[0] / pc[2] + cam.cx,
                                                   cam.fy * pc[1] / pc[2] + cam.cy], rtol=1e-12)


def test_quaternion_scale_invariance(oracle):
    # q and c*q (c != 0, including c < 0) describe the same rotation (powers of two keep
    # the float32 inputs exact).
    sc = one_gaussian((0.1, 0.0, 2.0), (0.02, 0.05, 0.01), (0.8, 0.1, -0.3, 0.5))
    cam = S.pinhole(64, 64, 60.0)
    a = oracle.project(sc, cam, "f64")
    for c in (-4.0, 0.125):
        sc2 = one_gaussian(sc.means[0], sc.scales[0], sc.quats[0] * c)
        b = oracle.project(sc2, cam, "f64")
        np.testing.assert_allclose(a["conic"], b["conic"], rtol=1e-12)


def test_near_plane_and_rect_cull(oracle):
    cam = S.pinhole(64, 64, 60.0)
    behind = one_gaussian((0.0, 0.0, 0.15), (0.01,) * 3)
    assert not oracle.project(behind, cam)["valid"][0]
    off = one_gaussian((50.0, 0.0, 2.0), (0.01,) * 3)       # far outside the image
    assert not oracle.project(off, cam)["valid"][0]
    assert oracle.project(off, cam, thresholds=False)["valid"][0]


def test_rect_contains_three_sigma_ellipse(oracle):
    # Every pixel centre within Mahalanobis distance 3 of the mean lies in the tile rectangle.
    sc = S.cube_scene(300, n_feat=1, seed=11)
    cam = S.pinhole(160, 128, 120.0, 120.0, np.eye(3), np.array([0.0, 0.0, 1.5]))
    p = oracle.project(sc, cam, "f64")
    ys, xs = np.mgrid[0:cam.H, 0:cam.W]
    cxp, cyp = xs + 0.5, ys + 0.5
    for i in np.nonzero(p["valid"])[0]:
        A, B, Cc = p["conic"][i]
        dx, dy = cxp - p["mean2d"][i, 0], cyp - p["mean2d"][i, 1]
        m2 = A * dx * dx + 2 * B * dx * dy + Cc * dy * dy
        inside = m2 <= 9.0
        x0, y0, x1, y1 = p["rect"][i]
        tx, ty = xs // 16, ys // 16
        in_rect = (tx >= x0) & (tx < x1) & (ty >= y0) & (ty < y1)
        assert not np.any(inside & ~in_rect), i


def _sphere_quadrature(nt=64, nphi=128):
    x, w = np.polynomial.legendre.leggauss(nt)          # cos(theta) nodes
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    wts = (w[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    return dirs, wts


def test_sh_basis_orthonormal(oracle):
    dirs, wts = _sphere_quadrature()
    Y = oracle.sh_basis(3, dirs)
    gram = (Y * wts[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)
    # degree l functions are homogeneous harmonic polynomials: Y(-d) = (-1)^l Y(d)
    Ym = oracle.sh_basis(3, -dirs)
    deg = np.array([0] + [1] * 3 + [2] * 5 + [3] * 7)
    np.testing.assert_allclose(Ym, Y * (-1.0) ** deg[None, :], atol=1e-14)
    # degree 1 spans the coordinate functions in the order (y, z, x)
    c1 = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(Y[:, 1:4], c1 * dirs[:, [1, 2, 0]], atol=1e-14)
    assert Y[0, 0] == pytest.approx(1 / math.sqrt(4 * math.pi))


def _real_sh_from_scipy(deg, dirs):
    """Real SH of degree <= deg, ordered (l, m = -l..l), built from SciPy's complex
    spherical harmonics (which carry the Condon-Shortley phase (-1)^m) by the textbook
    construction sqrt(2) (-1)^m Im Y_l^|m| (m < 0), Y_l^0, sqrt(2) (-1)^m Re Y_l^m (m > 0);
    the (-1)^m cancels the phase."""
    from scipy import special
    theta = np.arccos(np.clip(dirs[:, 2], -1.0, 1.0))   # polar angle from +z
    phi = np.arctan2(dirs[:, 1], dirs[:, 0])             # azimuth from +x
    if hasattr(special, "sph_harm_y"):
        Ylm = lambda l, m: special.sph_harm_y(l, m, theta, phi)   # noqa: E731
    else:
        Ylm = lambda l, m: special.sph_harm(m, l, phi, theta)     # noqa: E731
    cols = []
    for l in range(deg + 1):
        for m in range(-l, l + 1):
            if m < 0:
                cols.append(math.sqrt(2) * (-1) ** m * Ylm(l, -m).imag)
            elif m == 0:
                cols.append(Ylm(l, 0).real)
            else:
                cols.append(math.sqrt(2) * (-1) ** m * Ylm(l, m).real)
    return np.stack(cols, -1)


def test_sh_basis_equals_the_textbook_real_harmonics(oracle):
    # orthonormality cannot tell a sign flip or a swap inside a degree; the basis itself can
    pytest.importorskip("scipy.special")
    rng = np.random.default_rng(12)
    d = rng.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    np.testing.assert_allclose(oracle.sh_basis(3, d), _real_sh_from_scipy(3, d), atol=1e-12)


def test_sh_colour_uses_view_direction_from_camera_centre(oracle):
    # Camera centre c placed explicitly (t = -R c); colour = 0.5 + sum_k sh_k Y_k(dir).
    rng = np.random.default_rng(3)
    R = Rotation.from_rotvec([0.2, -0.4, 0.1]).as_matrix()
    c = np.array([0.3, -0.1, -2.0])
    cam = S.pinhole(64, 64, 50.0, 50.0, R, -R @ c)
    mu = R.T @ np.array([0.05, -0.02, 2.2]) + c
    sh = rng.normal(0, 0.3, size=(16, 3))
    sc = one_gaussian(mu, (0.05,) * 3, sh=sh, deg=3)
    mu = sc.means[0].astype(np.float64)
    p = oracle.project(sc, cam, "f64")
    d = (mu - c) / np.linalg.norm(mu - c)
    Y = oracle.sh_basis(3, d[None])[0]
    expect = np.maximum(0.0, Y @ sh.astype(np.float32).astype(np.float64) + 0.5)
    np.testing.assert_allclose(p["rgb"][0], expect, rtol=1e-6, atol=1e-7)
