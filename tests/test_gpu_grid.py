"""Grid-sampled rendering (Sec. 3.2, App. D) on the GPU against the grid oracle
(``oracle/grid.py``): compact forward within the forward tolerance on unflagged samples,
every sample bit-identical to the full-resolution GPU render at its pixel, backward within
the gradient tolerance, grid targets bit-exact, argument and state errors."""
import numpy as np
import pytest

from synth import scenes as S
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

TOL_FWD = 1e-4
TOL_BWD = 1e-3
GRAD_KEYS = ("means", "scales", "quats", "opacities", "sh", "feats", "pose")
# (stride, off_x, off_y): ragged compact grids, largest offsets (samples past the edge)
GRIDS = [(2, 0, 0), (2, 1, 1), (3, 2, 0), (4, 3, 3), (7, 6, 5), (16, 15, 4), (20, 19, 13)]


@pytest.fixture(scope="module")
def OG(oracle):
    from oracle import grid
    return grid


@pytest.fixture(scope="module")
def room():
    sc = S.room_scene(30_000, n_feat=16, sh_degree=2, seed=7)
    cam = S.room_trajectory(8, 203, 139, 180.0)[3]
    return sc, cam


def _render(rast, scene, cam, s, ox, oy):
    from paper_2603_09632_gb300.render import as_camera
    import torch
    c = as_camera(cam, s, ox, oy)
    out = rast.forward(scene, c)
    torch.cuda.synchronize()
    return c, out


@pytest.mark.parametrize("grid", GRIDS)
def test_grid_forward_matches_oracle_and_full_render(oracle, OG, room, grid):
    import torch
    from paper_2603_09632_gb300 import _lib as L
    from paper_2603_09632_gb300.render import Rasterizer
    s, ox, oy = grid
    sc, cam = room
    rast = Rasterizer(U.device())
    scene = U.upload(sc)
    full = rast.forward(scene, cam)
    full = {k: v.clone() for k, v in full.items() if isinstance(v, torch.Tensor)}
    torch.cuda.synchronize()
    T_full, nc_full = L.gs_get_pixel_state(rast.ws, cam.H, cam.W)
    c, got = _render(rast, scene, cam, s, ox, oy)
    Hs, Ws = OG.grid_shape(cam.H, cam.W, s)
    assert got["alpha"].shape == (Hs, Ws) and got["feat"].shape == (16, Hs, Ws)
    ref = OG.render(sc, cam, s, ox, oy, "f32")
    flags = ref["flags"]
    for k in ("rgb", "depth", "alpha", "feat"):
        err = U.max_abs_unflagged(got[k].cpu().numpy(), ref[k], flags)
        assert err <= TOL_FWD, (k, err)
    # each sample is the full-resolution GPU render at its pixel, bit for bit
    u, v, inb = OG.sample_coords(cam.H, cam.W, s, ox, oy)
    uu = torch.as_tensor(np.broadcast_to(u[:, None], inb.shape)[inb], device=U.device())
    vv = torch.as_tensor(np.broadcast_to(v[None, :], inb.shape)[inb], device=U.device())
    mi = torch.as_tensor(inb, device=U.device())
    for k in ("rgb", "depth", "alpha", "feat"):
        a, b = got[k], full[k]
        if a.dim() == 3:
            assert torch.equal(a[:, mi], b[:, uu, vv]), k
            assert (a[:, ~mi] == 0).all(), k
        else:
            assert torch.equal(a[mi], b[uu, vv]), k
            assert (a[~mi] == 0).all(), k
    # per-sample final transmittance and last-contributor count (the backward's replay
    # bound) of the samples inside the image: the oracle's on unflagged samples, and the
    # full-resolution render's at the sample's pixel, bit for bit
    T_g, nc_g = L.gs_get_pixel_state(rast.ws, Hs, Ws)
    ok = inb & (flags == 0)
    np.testing.assert_array_equal(nc_g[ok], ref["n_contrib"][ok])
    assert np.abs(T_g - ref["T_final"])[ok].max() <= TOL_FWD
    ui = np.broadcast_to(u[:, None], inb.shape)[inb]
    vi = np.broadcast_to(v[None, :], inb.shape)[inb]
    np.testing.assert_array_equal(nc_g[inb], nc_full[ui, vi])
    np.testing.assert_array_equal(T_g[inb], T_full[ui, vi])


@pytest.mark.parametrize("grid", [(2, 1, 0), (3, 2, 2), (16, 15, 4)])
def test_grid_backward_matches_oracle(OG, room, grid):
    import torch
    from paper_2603_09632_gb300.render import Rasterizer
    s, ox, oy = grid
    sc, cam = room
    Hs, Ws = OG.grid_shape(cam.H, cam.W, s)
    # upstream gradient zeroed at the samples the oracle flags as near a blend threshold
    flags = OG.render(sc, cam, s, ox, oy, "f32")["flags"]
    g, nflag = U.mask_flagged(S.upstream_grads(Hs, Ws, sc.n_feat, seed=21), flags)
    rast = Rasterizer(U.device())
    scene = U.upload(sc)
    c, _ = _render(rast, scene, cam, s, ox, oy)
    gt = {k: torch.from_numpy(v).to(U.device()) for k, v in g.items()}
    got = rast.backward(scene, c, gt["rgb"], gt["depth"], gt["alpha"], gt["feat"])
    ref = OG.backward(sc, cam, s, ox, oy, g, "f32")
    U.assert_grads_close({k: v.cpu().numpy() for k, v in got.items()}, ref, GRAD_KEYS,
                         ref_alt=OG.backward(sc, cam, s, ox, oy, g, "mixed"),
                         label=f"grid s={s} off=({ox},{oy}) ({nflag} flagged samples)")


def test_grid_targets_bit_exact(OG):
    import torch
    from paper_2603_09632_gb300 import _lib as L
    dev = U.device()
    rng = np.random.default_rng(3)
    H, W, R, D = 139, 203, 40, 12
    seg = rng.integers(-1, R + 3, size=(H, W)).astype(np.int32)   # includes ids >= R
    table = rng.normal(size=(R, D)).astype(np.float32)
    fmap = rng.normal(size=(D, 30, 43)).astype(np.float32)
    for s, ox, oy in [(1, 0, 0), (3, 2, 1), (8, 7, 7)]:
        Hs, Ws = OG.grid_shape(H, W, s)
        tg = torch.empty((D, Hs, Ws), device=dev)
        mk = torch.empty((Hs, Ws), device=dev)
        L.gs_grid_target_region(torch.from_numpy(seg).to(dev), torch.from_numpy(table).to(dev), s, ox,
                                oy, tg, mk)
        G, V = OG.target_region(seg, table.astype(np.float64), s, ox, oy)
        np.testing.assert_array_equal(tg.cpu().numpy(), G.astype(np.float32))
        np.testing.assert_array_equal(mk.cpu().numpy(), V.astype(np.float32))
        L.gs_grid_target_resample(torch.from_numpy(fmap).to(dev), H, W, s, ox, oy, tg, mk)
        G, V = OG.target_resample(fmap.astype(np.float64), H, W, s, ox, oy)
        np.testing.assert_array_equal(tg.cpu().numpy(), G.astype(np.float32))
        np.testing.assert_array_equal(mk.cpu().numpy(), V.astype(np.float32))


def test_grid_argument_and_state_errors(room):
    import torch
    from paper_2603_09632_gb300 import _lib as L
    from paper_2603_09632_gb300.render import Rasterizer, as_camera
    sc, cam = room
    rast = Rasterizer(U.device())
    scene = U.upload(sc)
    for s, ox, oy in [(0, 0, 0), (2, 2, 0), (2, 0, -1), (257, 0, 0)]:
        with pytest.raises(L.GSError) as e:
            L.gs_project(scene, as_camera(cam, s, ox, oy), rast.ws)
        assert e.value.status == L.GS_ERR_ARG
    # a render must use the grid its projection used
    L.gs_project(scene, as_camera(cam, 2, 1, 0), rast.ws)
    L.gs_bin_tiles(rast.ws, sync=True)
    out = torch.empty((3, cam.H, cam.W), device=U.device())
    with pytest.raises(L.GSError) as e:
        L.gs_render_fwd(scene, as_camera(cam, 2, 0, 0), rast.ws, out, None, None, None)
    assert e.value.status == L.GS_ERR_STATE
    dev = U.device()
    with pytest.raises(L.GSError):
        L.gs_grid_target_resample(torch.zeros((2, 4, 4), device=dev), 10, 10, 3, 3, 0,
                                  torch.empty((2, 4, 4), device=dev))


def _segmentation(H, W, R, seed, block=9):
    """Seeded piecewise-constant region ids (blocks of `block` pixels, about 20 % background)."""
    rng = np.random.default_rng(seed)
    coarse = rng.integers(0, R, size=(-(-H // block), -(-W // block)))
    coarse[rng.uniform(size=coarse.shape) < 0.2] = -1
    return np.repeat(np.repeat(coarse, block, 0), block, 1)[:H, :W].astype(np.int32)


@pytest.mark.parametrize("grid,bf16", [((3, 1, 2), False), ((1, 0, 0), False), ((4, 3, 0), True)])
def test_fused_feature_loss(OG, room, grid, bf16):
    """NEXT-2: the loss and dL/dG_hat produced in the forward's epilogue against the oracle's
    masked L1 + cosine loss (App. D), then the backward driven by that gradient."""
    import torch
    from paper_2603_09632_gb300 import _lib as L
    from paper_2603_09632_gb300.render import Rasterizer, as_camera
    s, ox, oy = grid
    sc, cam = room
    dev = U.device()
    D = sc.n_feat
    R = 25
    seg = _segmentation(cam.H, cam.W, R, seed=5)
    table = np.random.default_rng(6).normal(size=(R, D)).astype(np.float32)
    G, V = OG.target_region(seg, table.astype(np.float64), s, ox, oy)
    Hs, Ws = V.shape
    lam = 0.75
    rast = Rasterizer(dev)
    scene = U.upload(sc, bf16=bf16)
    c = as_camera(cam, s, ox, oy)
    L.gs_project(scene, c, rast.ws)
    L.gs_bin_tiles(rast.ws, sync=True)
    tg = torch.empty((D, Hs, Ws), device=dev)
    mk = torch.empty((Hs, Ws), device=dev)
    L.gs_grid_target_region(torch.from_numpy(seg).to(dev), torch.from_numpy(table).to(dev), s, ox, oy,
                            tg, mk)
    feat = torch.empty((D, Hs, Ws), device=dev)
    gF = torch.empty((D, Hs, Ws), device=dev)
    loss = torch.empty(3, dtype=torch.float64, device=dev)
    L.gs_render_fwd_loss(scene, c, rast.ws, tg, gF, loss, mask=mk, lambda_sem=lam, feat=feat)
    torch.cuda.synchronize()
    got = loss.cpu().numpy()
    # the loss arithmetic itself: the oracle loss of the GPU's own rendered G_hat
    Lr, l1r, lcr, gr = OG.loss(feat.cpu().numpy(), G, V, lam)
    np.testing.assert_allclose(got, [Lr, l1r, lcr], rtol=1e-5)
    np.testing.assert_allclose(gF.cpu().numpy(), gr, rtol=1e-4, atol=1e-4 * np.abs(gr).max())
    # end to end against the oracle's render (bf16 features: the same rounded values)
    feats = U.bf16_round(sc.feats) if bf16 else None
    ref = OG.render(sc, cam, s, ox, oy, "f32", feats=feats)
    L2, l12, lc2, g2 = OG.loss(ref["feat"], G, V, lam)
    np.testing.assert_allclose(got, [L2, l12, lc2], rtol=1e-4)
    assert U.rel_err(gF.cpu().numpy(), g2) <= 1e-3
    # the backward driven by the fused gradient matches the oracle's backward of that loss
    grads = rast.backward(scene, c, None, None, None, gF)
    scb = sc if not bf16 else S.Scene(**{k: getattr(sc, k) for k in
                                         ("means", "scales", "quats", "opacities", "sh")},
                                      feats=feats, sh_degree=sc.sh_degree)
    ref_b = OG.backward(scb, cam, s, ox, oy, {"feat": g2}, "f32")
    for k in GRAD_KEYS:
        if k == "sh":
            continue   # colour gets no gradient from a feature-only loss
        r = U.rel_err(grads[k].cpu().numpy(), ref_b[k])
        assert r <= TOL_BWD, (k, r)
    assert np.abs(grads["sh"].cpu().numpy()).max() == 0.0
    # element by element: both backwards driven by the oracle's loss gradient, zeroed at
    # the samples the oracle flags (the fused gradient itself is checked above; sign(0)
    # flips of the L1 term where G_hat = G* are not a backward difference)
    flags = ref["flags"]
    g3 = np.where(flags[None] != 0, 0.0, g2).astype(np.float32)
    grads3 = rast.backward(scene, c, None, None, None, torch.from_numpy(g3).to(dev))
    ref_3 = OG.backward(scb, cam, s, ox, oy, {"feat": g3}, "f32")
    U.assert_grads_close({k: v.cpu().numpy() for k, v in grads3.items()}, ref_3,
                         [k for k in GRAD_KEYS if k != "sh"],
                         ref_alt=OG.backward(scb, cam, s, ox, oy, {"feat": g3}, "mixed"),
                         label=f"fused-loss gradient, grid s={s} ({int((flags != 0).sum())} flagged)")
