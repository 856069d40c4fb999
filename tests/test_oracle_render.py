"""Pins of the oracle's forward blending (Eq. 1 / discrete rendering, App. B; feature
substitution, Sec. 3.1) and of its sorted tile lists."""
import math

import numpy as np
import pytest

from synth import scenes as S
from tests.test_oracle_projection import one_gaussian


def _scene_of(gs, deg=0):
    """Concatenate single-Gaussian scenes."""
    return S.Scene(**{k: np.concatenate([getattr(g, k) for g in gs]) for k in
                      ("means", "scales", "quats", "opacities", "sh", "feats")}, sh_degree=deg)


def _dc(rgb):
    # degree-0 coefficient giving colour rgb (Y_00 = 1/sqrt(4 pi), pinned by orthonormality)
    return (np.asarray(rgb, np.float64) - 0.5) * math.sqrt(4 * math.pi)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_single_gaussian_closed_form(oracle, prec):
    s, z, f, o = 0.04, 2.0, 100.0, 0.7
    rgb = np.array([0.9, 0.2, 0.6])
    feat = np.array([1.5, -2.0, 0.25])
    sc = one_gaussian((0.0, 0.0, z), (s, s, s), opac=o, sh=_dc(rgb), feats=feat)
    cam = S.pinhole(64, 48, f)
    r = oracle.render(sc, cam, prec)
    s32, o32 = float(sc.scales[0, 0]), float(sc.opacities[0])
    var = (f * s32 / z) ** 2 + 0.3
    ys, xs = np.mgrid[0:cam.H, 0:cam.W]
    d2 = (xs + 0.5 - 32.0) ** 2 + (ys + 0.5 - 24.0) ** 2
    a = np.minimum(0.99, o32 * np.exp(-0.5 * d2 / var))
    a = np.where(a >= 1 / 255, a, 0.0)
    # only tiles inside the 3-sigma rectangle are rendered
    rect = oracle.project(sc, cam, prec)["rect"][0]
    tx, ty = xs // 16, ys // 16
    a = np.where((tx >= rect[0]) & (tx < rect[2]) & (ty >= rect[1]) & (ty < rect[3]), a, 0.0)
    tol = 2e-6 if prec == "f32" else 1e-12
    rgb32 = sc.sh[0, 0].astype(np.float64) / math.sqrt(4 * math.pi) + 0.5
    np.testing.assert_allclose(r["alpha"], a, atol=tol)
    np.testing.assert_allclose(r["rgb"], rgb32[:, None, None] * a[None], atol=tol)
    np.testing.assert_allclose(r["depth"], z * a, atol=tol * z)
    np.testing.assert_allclose(r["feat"], sc.feats[0].astype(np.float64)[:, None, None] * a[None],
                               atol=tol * 2)
    np.testing.assert_array_equal(r["n_contrib"], (a > 0).astype(np.int32))


def test_two_gaussians_front_to_back(oracle):
    # C = c1 a1 + c2 a2 (1 - a1) with 1 the nearer Gaussian, whatever the input order.
    g_near = one_gaussian((0.0, 0.0, 2.0), (0.05,) * 3, opac=0.6, sh=_dc([0.9, 0.1, 0.2]),
                          feats=[1.0, 0.0])
    g_far = one_gaussian((0.01, 0.0, 3.0), (0.08,) * 3, opac=0.9, sh=_dc([0.2, 0.8, 0.3]),
                         feats=[0.0, 1.0])
    cam = S.pinhole(32, 32, 80.0)
    pix = np.array([16 * 32 + 16])
    for order in ([g_near, g_far], [g_far, g_near]):
        r = oracle.render(_scene_of(order), cam, "f64", pixels=pix)
        a1 = oracle.render(_scene_of([g_near]), cam, "f64", pixels=pix)["alpha"][0]
        a2 = oracle.render(_scene_of([g_far]), cam, "f64", pixels=pix)["alpha"][0]
        c1 = g_near.sh[0, 0].astype(np.float64) / math.sqrt(4 * math.pi) + 0.5
        c2 = g_far.sh[0, 0].astype(np.float64) / math.sqrt(4 * math.pi) + 0.5
        np.testing.assert_allclose(r["rgb"][:, 0], c1 * a1 + c2 * a2 * (1 - a1), rtol=1e-12)
        np.testing.assert_allclose(r["feat"][:, 0], [a1, a2 * (1 - a1)], rtol=1e-12)
        np.testing.assert_allclose(r["depth"][0], 2.0 * a1 + 3.0 * a2 * (1 - a1), rtol=1e-7)
        np.testing.assert_allclose(r["alpha"][0], 1 - (1 - a1) * (1 - a2), rtol=1e-12)


def test_early_stop_is_exclusive(oracle):
    # Three wide opaque Gaussians (alpha capped at 0.99 at the centre pixel): after two,
    # T = 0.01 * 0.01 is not below 1e-4, so the second is included; the third would take
    # T to 1e-6 < 1e-4, so blending stops before it.
    gs = [one_gaussian((0.0, 0.0, z), (2.0,) * 3, opac=1.0, sh=_dc([0.5] * 3), feats=[k])
          for k, z in enumerate((2.0, 2.5, 3.0))]
    cam = S.pinhole(16, 16, 20.0)
    r = oracle.render(_scene_of(gs), cam, "f64", pixels=np.array([8 * 16 + 8]))
    # first: T 1 -> 0.01 ; second: 0.01 * 0.01 = 1e-4 (not < 1e-4): included; third: 1e-6 < 1e-4
    assert r["n_contrib"][0] == 2
    assert r["T_final"][0] == pytest.approx(1e-4, rel=1e-9)
    np.testing.assert_allclose(r["feat"][0, 0], 0 * 0.99 + 1 * 0.99 * 0.01, rtol=1e-12)


@pytest.fixture(scope="module")
def tiny():
    return S.config_tiny()


def test_brute_force_equals_tile_lists(oracle, tiny):
    sc, (cam,) = tiny
    a = oracle.render(sc, cam, "f32", mode=0)
    b = oracle.render(sc, cam, "f32", mode=1)
    for k in ("rgb", "depth", "alpha", "feat", "T_final", "n_contrib"):
        np.testing.assert_array_equal(a[k], b[k])
    room, cams = S.config_slam(n=20_000, n_poses=4)
    cam2 = S.pinhole(160, 120, 150.0, 150.0, cams[1].R, cams[1].t)
    a = oracle.render(room, cam2, "f32", mode=0)
    b = oracle.render(room, cam2, "f32", mode=1)
    np.testing.assert_array_equal(a["rgb"], b["rgb"])
    np.testing.assert_array_equal(a["n_contrib"], b["n_contrib"])


def test_invariants(oracle, tiny):
    sc, (cam,) = tiny
    r = oracle.render(sc, cam, "f32")
    al = r["alpha"]
    assert np.all(al >= 0) and np.all(al <= 1 - 1e-4 + 1e-7)
    assert np.all(r["T_final"] >= 1e-4 * (1 - 1e-6))
    np.testing.assert_allclose(al, 1 - r["T_final"], atol=1e-7)
    assert np.all(r["rgb"] >= 0)
    # colours in [0,1] and weights summing to alpha: rgb <= alpha
    assert np.all(r["rgb"] <= al[None] + 1e-6)
    # depth is a weighted mean of positive depths: min z * alpha <= depth <= max z * alpha
    z = oracle.project(sc, cam)["depth"]
    z = z[z > 0]
    assert np.all(r["depth"] >= z.min() * al - 1e-5) and np.all(r["depth"] <= z.max() * al + 1e-5)
    assert r["n_contrib"].max() > 10 and al.max() > 0.99


def test_feature_linearity_and_substitution(oracle, tiny):
    sc, (cam,) = tiny
    rng = np.random.default_rng(9)
    f, g = sc.feats, rng.normal(size=sc.feats.shape)
    a, b = 0.75, -1.25
    Ff = oracle.render(sc, cam, "f64", feats=f)["feat"]
    Fg = oracle.render(sc, cam, "f64", feats=g)["feat"]
    Fab = oracle.render(sc, cam, "f64", feats=a * f.astype(np.float64) + b * g)["feat"]
    np.testing.assert_allclose(Fab, a * Ff + b * Fg, atol=1e-12)
    # constant features k give k * alpha
    r = oracle.render(sc, cam, "f64", feats=np.full((sc.n, 2), 3.0))
    np.testing.assert_allclose(r["feat"], 3.0 * r["alpha"][None].repeat(2, 0), atol=1e-12)
    # features set to the per-Gaussian colours reproduce the colour image
    cols = oracle.project(sc, cam, "f64")["rgb"]
    r = oracle.render(sc, cam, "f64", feats=cols)
    np.testing.assert_allclose(r["feat"], r["rgb"], atol=1e-12)


def test_permutation_invariance(oracle, tiny):
    sc, (cam,) = tiny
    perm = np.random.default_rng(4).permutation(sc.n)
    sp = S.Scene(means=sc.means[perm], scales=sc.scales[perm], quats=sc.quats[perm],
                 opacities=sc.opacities[perm], sh=sc.sh[perm], feats=sc.feats[perm], sh_degree=0)
    a = oracle.render(sc, cam, "f32")
    b = oracle.render(sp, cam, "f32")
    for k in ("rgb", "depth", "alpha", "feat", "n_contrib"):
        np.testing.assert_array_equal(a[k], b[k])
    ka, ia, ra = oracle.tile_lists(sc, cam)
    kb, ib, rb = oracle.tile_lists(sp, cam)
    np.testing.assert_array_equal(ka, kb)
    np.testing.assert_array_equal(ia, perm[ib])
    np.testing.assert_array_equal(ra, rb)


def test_tile_lists_structure(oracle, tiny):
    sc, (cam,) = tiny
    keys, ids, ranges = oracle.tile_lists(sc, cam)
    p = oracle.project(sc, cam)
    TX, TY = oracle.tiles(cam)
    assert np.all(np.diff(keys.astype(np.float64)) >= 0) or np.all(keys[1:] >= keys[:-1])
    depth_bits = p["depth"].astype(np.float32).view(np.uint32)
    for t in range(TX * TY):
        s, e = ranges[t]
        lst = ids[s:e]
        assert np.all((keys[s:e] >> np.uint64(32)) == t)
        np.testing.assert_array_equal(keys[s:e] & np.uint64(0xFFFFFFFF), depth_bits[lst])
        tx, ty = t % TX, t // TX
        x0, y0, x1, y1 = p["rect"].T
        members = np.nonzero(p["valid"] & (x0 <= tx) & (tx < x1) & (y0 <= ty) & (ty < y1))[0]
        expect = members[np.lexsort((members, p["depth"][members]))]
        np.testing.assert_array_equal(lst, expect)
    assert ranges[:, 1].max() == len(keys)
