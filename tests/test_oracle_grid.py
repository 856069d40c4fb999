"""Pins of the grid-sampling oracle (``oracle/grid.py``; Sec. 3.2 and App. D): hand-worked
sample locations, reassembly of the full image from all s^2 offsets, out-of-image samples,
hand-worked region and continuous targets (exact rational rounding), and the masked
L1 + cosine loss against PyTorch's own L1 / cosine-similarity routines, closed forms and
finite differences."""
from decimal import ROUND_HALF_UP, Decimal
from fractions import Fraction

import numpy as np
import pytest

from synth import scenes as S


@pytest.fixture(scope="module")
def OG(oracle):
    from oracle import grid
    return grid


def small_scene():
    sc = S.cube_scene(300, n_feat=3, sh_degree=1, seed=11, log_scale_mu=-2.6)
    cam = S.pinhole(40, 28, 30.0, 30.0, np.eye(3), np.array([0.0, 0.0, 2.0]))
    return sc, cam


def test_sample_coords_worked_example(OG):
    # H = 5, W = 7, s = 2, (o_h, o_w) = (1, 0): rows 1, 3, 5 (5 is outside), columns 0, 2, 4, 6
    u, v, inb = OG.sample_coords(5, 7, 2, 0, 1)
    assert OG.grid_shape(5, 7, 2) == (3, 4)
    assert list(u) == [1, 3, 5] and list(v) == [0, 2, 4, 6]
    assert inb.tolist() == [[True] * 4, [True] * 4, [False] * 4]
    # rows and columns are not swapped: offsets act on their own axis
    u, v, inb = OG.sample_coords(5, 7, 2, 1, 0)
    assert list(u) == [0, 2, 4] and list(v) == [1, 3, 5, 7]
    assert inb[:, 3].tolist() == [False] * 3 and inb[:, :3].all()
    with pytest.raises(ValueError):
        OG.sample_coords(5, 7, 2, 2, 0)


@pytest.mark.parametrize("stride", [2, 3])
def test_offsets_partition_the_full_image(oracle, OG, stride):
    sc, cam = small_scene()
    full = oracle.render(sc, cam, "f32")
    rec = {k: np.zeros_like(full[k]) for k in ("rgb", "depth", "alpha", "feat", "n_contrib")}
    hits = np.zeros((cam.H, cam.W), np.int32)
    for oy in range(stride):
        for ox in range(stride):
            g = OG.render(sc, cam, stride, ox, oy, "f32")
            u, v, inb = OG.sample_coords(cam.H, cam.W, stride, ox, oy)
            assert g["alpha"].shape == OG.grid_shape(cam.H, cam.W, stride)
            for m in range(len(u)):
                for n in range(len(v)):
                    if inb[m, n]:
                        hits[u[m], v[n]] += 1
                        for k in ("depth", "alpha", "n_contrib"):
                            rec[k][u[m], v[n]] = g[k][m, n]
                        rec["rgb"][:, u[m], v[n]] = g["rgb"][:, m, n]
                        rec["feat"][:, u[m], v[n]] = g["feat"][:, m, n]
    assert (hits == 1).all()
    assert full["alpha"].max() > 0.5
    for k in rec:
        np.testing.assert_array_equal(rec[k], full[k])


def test_out_of_image_samples_render_nothing(OG):
    sc, cam = small_scene()                      # 40 x 28, stride 3: last row 3 + 27 = 30 > 27
    g = OG.render(sc, cam, 3, 2, 2, "f32")
    u, v, inb = OG.sample_coords(cam.H, cam.W, 3, 2, 2)
    assert not inb.all()
    assert (g["alpha"][~inb] == 0).all() and (g["T_final"][~inb] == 1).all()
    assert (g["feat"][:, ~inb] == 0).all() and (g["n_contrib"][~inb] == 0).all()
    assert g["alpha"][inb].max() > 0.5


def test_grid_backward_is_the_full_backward_of_the_sampled_pixels(oracle, OG):
    sc, cam = small_scene()
    s, ox, oy = 3, 1, 2
    Hs, Ws = OG.grid_shape(cam.H, cam.W, s)
    rng = np.random.default_rng(4)
    gc = dict(rgb=rng.normal(size=(3, Hs, Ws)), depth=rng.normal(size=(Hs, Ws)),
              alpha=rng.normal(size=(Hs, Ws)), feat=rng.normal(size=(3, Hs, Ws)))
    g = OG.backward(sc, cam, s, ox, oy, gc, "f64")
    # the same loss written on the full image: upstream gradient scattered to (u, v)
    u, v, inb = OG.sample_coords(cam.H, cam.W, s, ox, oy)
    gf = dict(rgb=np.zeros((3, cam.H, cam.W)), depth=np.zeros((cam.H, cam.W)),
              alpha=np.zeros((cam.H, cam.W)), feat=np.zeros((3, cam.H, cam.W)))
    for m in range(Hs):
        for n in range(Ws):
            if inb[m, n]:
                gf["rgb"][:, u[m], v[n]] = gc["rgb"][:, m, n]
                gf["feat"][:, u[m], v[n]] = gc["feat"][:, m, n]
                gf["depth"][u[m], v[n]] = gc["depth"][m, n]
                gf["alpha"][u[m], v[n]] = gc["alpha"][m, n]
    ref = oracle.backward(sc, cam, gf, "f64")
    for k in ("means", "scales", "quats", "opacities", "sh", "feats", "pose"):
        np.testing.assert_allclose(g[k], ref[k], rtol=1e-10, atol=1e-12 * np.abs(ref[k]).max())
    assert np.abs(ref["means"]).max() > 0


def test_target_region_worked_example(OG):
    seg = np.array([[0, 0, -1, 2, 2],
                    [1, 1, -1, 2, 7],
                    [1, -1, 0, 0, 2],
                    [-1, -1, 0, 0, 2]])
    table = np.array([[1.0, 10.0], [2.0, 20.0], [3.0, 30.0]])
    # s = 2, (o_h, o_w) = (1, 1): rows 1, 3; columns 1, 3, 5 (5 outside)
    G, V = OG.target_region(seg, table, 2, 1, 1)
    # (1,1) -> 1, (1,3) -> 2, (3,1) -> -1, (3,3) -> 0; id 7 is never sampled here
    np.testing.assert_array_equal(V, [[1, 1, 0], [0, 1, 0]])
    np.testing.assert_array_equal(G[0], [[2, 3, 0], [0, 1, 0]])
    np.testing.assert_array_equal(G[1], [[20, 30, 0], [0, 10, 0]])
    # an id outside the table counts as background: (1, 4) is sampled with (o_h, o_w) = (1, 0)
    G, V = OG.target_region(seg, table, 2, 0, 1)
    np.testing.assert_array_equal(V, [[1, 0, 0], [0, 1, 1]])


def test_target_resample_rounding(OG):
    # H = 5, H_f = 4: u * 3/4 = 0, 0.75, 1.5, 2.25, 3 -> 0, 1, 2, 2, 3 (1.5 rounds away)
    # W = 9, W_f = 3: v * 2/8 = 0, 0.5, 1, 1.5, 2 at v = 0, 2, 4, 6, 8 -> 0, 1, 1, 2, 2
    D, Hf, Wf = 2, 4, 3
    P = np.arange(D * Hf * Wf, dtype=np.float64).reshape(D, Hf, Wf)
    G, V = OG.target_resample(P, 5, 9, 1, 0, 0)
    assert V.shape == (5, 9) and (V == 1).all()
    rows, cols = [0, 1, 2, 2, 3], {0: 0, 2: 1, 4: 1, 6: 2, 8: 2}
    for m in range(5):
        for n, c in cols.items():
            np.testing.assert_array_equal(G[:, m, n], P[:, rows[m], c])
    # against exact decimal rounding of the rational coordinate, over many sizes
    for H, Hf in [(480, 30), (680, 43), (7, 7), (2, 5), (1, 4), (1000, 999)]:
        for u in range(H):
            q = Fraction(u * (Hf - 1), max(H - 1, 1))
            ref = int((Decimal(q.numerator) / Decimal(q.denominator)).quantize(Decimal(1), ROUND_HALF_UP))
            assert OG.round_half_away(u * (Hf - 1), max(H - 1, 1)) == ref
    # stride / offset: sample (m, n) reads the map at the rounded (o_h + m s, o_w + n s)
    G2, V2 = OG.target_resample(P, 5, 9, 2, 1, 1)
    assert V2.shape == (3, 5)
    np.testing.assert_array_equal(V2[2], [0] * 5)          # row 5 is outside
    np.testing.assert_array_equal(V2[:, 4], [0] * 3)       # column 9 is outside
    np.testing.assert_array_equal(G2[:, 1, 1], P[:, 2, 1])  # (u, v) = (3, 3) -> (2.25, 0.75)


def _torch_loss(Gh, Gs, V, lam):
    import torch
    import torch.nn.functional as F
    a = torch.tensor(Gh, dtype=torch.float64, requires_grad=True)
    Vt = torch.tensor(V, dtype=torch.float64)[None]
    b = torch.tensor(Gs, dtype=torch.float64) * Vt
    am = a * Vt
    l1 = F.l1_loss(am, b)
    lc = (1.0 - F.cosine_similarity(am, b, dim=0, eps=1e-8)).mean()
    L = lam * (l1 + lc)
    L.backward()
    return L.item(), l1.item(), lc.item(), a.grad.numpy()


def test_loss_against_pytorch_routines(OG):
    rng = np.random.default_rng(9)
    D, Hs, Ws = 16, 9, 13
    Gh = rng.normal(size=(D, Hs, Ws))
    Gs = rng.normal(size=(D, Hs, Ws))
    V = (rng.uniform(size=(Hs, Ws)) < 0.7).astype(np.float64)
    L, l1, lc, g = OG.loss(Gh, Gs, V, lam=0.5)
    tL, tl1, tlc, tg = _torch_loss(Gh, Gs, V, 0.5)
    assert abs(l1 - tl1) < 1e-13 and abs(lc - tlc) < 1e-13 and abs(L - tL) < 1e-13
    np.testing.assert_allclose(g, tg, rtol=1e-10, atol=1e-15)
    assert (g[:, V == 0] == 0).all()


def test_loss_closed_forms_and_finite_differences(OG):
    rng = np.random.default_rng(10)
    D, Hs, Ws = 5, 4, 6
    Gs = rng.normal(size=(D, Hs, Ws))
    ones = np.ones((Hs, Ws))
    L, l1, lc, g = OG.loss(Gs, Gs, ones)
    assert abs(L) < 1e-14 and abs(l1) == 0
    L, l1, lc, _ = OG.loss(-2 * Gs, Gs, ones)              # cos = -1, |a - b| = 3 |b|
    assert abs(lc - 2.0) < 1e-14 and abs(l1 - 3 * np.abs(Gs).mean()) < 1e-14
    L, l1, lc, _ = OG.loss(3 * Gs, Gs, ones)               # cos = 1, |a - b| = 2 |b|
    assert abs(lc) < 1e-14 and abs(l1 - 2 * np.abs(Gs).mean()) < 1e-14
    V = ones.copy()
    V[1, 2] = V[3, 0] = 0.0                                # masked pixels: 1 - 0 each
    _, _, lc, _ = OG.loss(Gs, Gs, V)
    assert abs(lc - 2.0 / (Hs * Ws)) < 1e-14
    # gradient by central differences (away from the kinks of |.|)
    Gh = Gs + rng.normal(size=Gs.shape)
    _, _, _, g = OG.loss(Gh, Gs, V, lam=1.7)
    h = 1e-6
    for idx in [(0, 0, 0), (3, 1, 2), (4, 2, 5), (1, 3, 1), (2, 0, 4)]:
        e = np.zeros_like(Gh)
        e[idx] = h
        fd = (OG.loss(Gh + e, Gs, V, 1.7)[0] - OG.loss(Gh - e, Gs, V, 1.7)[0]) / (2 * h)
        assert abs(fd - g[idx]) < 1e-8, (idx, fd, g[idx])
