"""GPU (C ABI) vs CPU oracle parity.

Tolerances: tile keys, sorted ids and ranges bit-exact; FP32 rgb/depth/alpha/features
max-abs 1e-4 on pixels the oracle does not flag as within rounding distance of a blend
threshold; BF16-stored features relative 1e-2 against the FP32-feature render; gradients
element by element against the FP32 oracle's analytic backward: every entry within 1e-3 of
its reference value plus 1e-5 of the tensor's largest entry plus the entry's conditioning
term -- the disagreement between the FP32 oracle and the oracle's mixed mode (double
arithmetic with the float projection's visibility, rectangles and list order), two
evaluations of the same gradient that differ only where it is ill-conditioned -- with the
upstream gradient zeroed at the flagged pixels on both sides (which removes exactly their
contribution, so no Gaussian is excluded), and relative (Frobenius) 1e-3 per tensor.
"""
import numpy as np
import pytest

from synth import scenes as S
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

TOL_FWD = 1e-4
GRAD_KEYS = ("means", "scales", "quats", "opacities", "sh", "feats", "pose")


def small_room(n=30_000, W=200, H=136, D=16, deg=3, pose=3):
    sc = S.room_scene(n, n_feat=D, sh_degree=deg, seed=7)
    cams = S.room_trajectory(8, W, H, 0.9 * W)
    return sc, cams[pose]


CASES = {
    "tiny": lambda: (S.config_tiny()[0], S.config_tiny()[1][0]),
    "room_ragged": small_room,
    "room_sh1_d8": lambda: small_room(n=20_000, W=97, H=61, D=8, deg=1, pose=5),
    # 32 and 64 channels: the backward's 8- and 16-Gaussian batch configurations
    "room_d32": lambda: small_room(n=20_000, W=150, H=100, D=32, deg=0, pose=2),
    "room_d64": lambda: small_room(n=20_000, W=150, H=100, D=64, deg=2, pose=6),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request, oracle):
    sc, cam = CASES[request.param]()
    ref = oracle.render(sc, cam, "f32")
    g, nflag = U.mask_flagged(S.upstream_grads(cam.H, cam.W, sc.n_feat), ref["flags"])
    gpu = U.run(sc, cam, g)
    gpu["oracle_fwd"] = ref
    gpu["flagged"] = nflag
    return request.param, sc, cam, g, gpu


def test_projection_bit_exact(oracle, case):
    from paper_2603_09632_gb300 import _lib as L
    name, sc, cam, g, gpu = case
    ref = oracle.project(sc, cam, "f32")
    got = L.gs_get_projection(gpu["rast"].ws, sc.n)
    v = ref["valid"]
    np.testing.assert_array_equal(got["rect"][v], ref["rect"][v])
    assert np.all(got["rect"][~v] == 0)
    for k in ("depth", "mean2d", "conic"):
        np.testing.assert_array_equal(got[k][v].view(np.uint32), ref[k][v].view(np.uint32), err_msg=k)
    np.testing.assert_allclose(got["rgb"][v], ref["rgb"][v], atol=1e-6)


def test_tile_lists_bit_exact(oracle, case):
    from paper_2603_09632_gb300 import _lib as L
    name, sc, cam, g, gpu = case
    TX, TY = oracle.tiles(cam)
    keys, ids, ranges = oracle.tile_lists(sc, cam)
    tiles_g, ids_g, ranges_g = L.gs_get_instances(gpu["rast"].ws, TX * TY)
    assert gpu["instances"] == len(keys)
    depth_g = L.gs_get_projection(gpu["rast"].ws, sc.n)["depth"].view(np.uint32)
    keys_g = (tiles_g.astype(np.uint64) << np.uint64(32)) | depth_g[ids_g].astype(np.uint64)
    np.testing.assert_array_equal(keys_g, keys)
    np.testing.assert_array_equal(ids_g, ids)
    np.testing.assert_array_equal(ranges_g, ranges)


def test_forward_parity(oracle, case):
    from paper_2603_09632_gb300 import _lib as L
    name, sc, cam, g, gpu = case
    ref = gpu["oracle_fwd"]
    flags = ref["flags"]
    assert (flags != 0).mean() < 0.01, "too many near-threshold pixels to be meaningful"
    for k in ("rgb", "depth", "alpha", "feat"):
        err = U.max_abs_unflagged(gpu[k], ref[k], flags)
        assert err <= TOL_FWD, (k, err)
    T, nc = L.gs_get_pixel_state(gpu["rast"].ws, cam.H, cam.W)
    ok = flags == 0
    np.testing.assert_array_equal(nc[ok], ref["n_contrib"][ok])
    assert np.abs(T - ref["T_final"])[ok].max() <= TOL_FWD


def test_backward_parity(oracle, case):
    name, sc, cam, g, gpu = case
    ref = oracle.backward(sc, cam, g, "f32")
    U.assert_grads_close(gpu["grads"], ref, GRAD_KEYS, label=f"{name} ({gpu['flagged']} flagged px)",
                         ref_alt=oracle.backward(sc, cam, g, "mixed"))


def test_bf16_features(oracle):
    sc, cam = small_room(n=30_000, D=64, deg=3)
    gpu = U.run(sc, cam, bf16=True)
    flags = oracle.render(sc, cam, "f32")["flags"]
    # same bf16 values in FP32 arithmetic: FP32 tolerance
    ref_b = oracle.render(sc, cam, "f32", feats=U.bf16_round(sc.feats))
    assert U.max_abs_unflagged(gpu["feat"], ref_b["feat"], flags) <= TOL_FWD
    # against the FP32-feature render: relative 1e-2 per channel map
    ref = oracle.render(sc, cam, "f32")
    ok = flags == 0
    for c in range(sc.n_feat):
        a, b = gpu["feat"][c][ok], ref["feat"][c][ok]
        assert U.rel_err(a, b) <= 1e-2, c
    assert np.abs(gpu["feat"] - ref["feat"])[:, ok].max() / np.abs(ref["feat"]).max() <= 1e-2


def test_bf16_backward(oracle):
    sc, cam = small_room(n=20_000, D=64, deg=0)
    scb = S.Scene(**{k: getattr(sc, k) for k in ("means", "scales", "quats", "opacities", "sh")},
                  feats=U.bf16_round(sc.feats), sh_degree=sc.sh_degree)
    g, nflag = U.mask_flagged(S.upstream_grads(cam.H, cam.W, sc.n_feat),
                              oracle.render(scb, cam, "f32")["flags"])
    gpu = U.run(sc, cam, g, bf16=True)
    ref = oracle.backward(scb, cam, g, "f32")
    U.assert_grads_close(gpu["grads"], ref, GRAD_KEYS, label=f"bf16 d64 ({nflag} flagged px)",
                         ref_alt=oracle.backward(scb, cam, g, "mixed"))


def test_determinism():
    sc, cam = small_room()
    a = U.run(sc, cam)
    b = U.run(sc, cam, rast=a["rast"])
    for k in ("rgb", "depth", "alpha", "feat"):
        np.testing.assert_array_equal(a[k], b[k])


def test_full_size_slam_frame_sampled(oracle):
    """640x480, 200k room Gaussians, 16 f32 features, the bench's launch configuration:
    forward on 3000 sampled pixels, backward of a loss restricted to those pixels."""
    sc, cams = S.config_slam(n_poses=100)
    cam = cams[0]
    rng = np.random.default_rng(12)
    pix = rng.choice(cam.W * cam.H, size=3000, replace=False)
    _sampled_parity(oracle, sc, cam, pix, bf16=False, mode=1)


def _tile_pixels(cam, n_tiles, seed):
    """All pixels of n_tiles random 16x16 tiles (flat indices)."""
    rng = np.random.default_rng(seed)
    TX, TY = (cam.W + 15) // 16, (cam.H + 15) // 16
    out = []
    for t in rng.choice(TX * TY, size=n_tiles, replace=False):
        x0, y0 = (t % TX) * 16, (t // TX) * 16
        ys, xs = np.mgrid[y0:min(y0 + 16, cam.H), x0:min(x0 + 16, cam.W)]
        out.append((ys * cam.W + xs).ravel())
    return np.concatenate(out)


def _sampled_parity(oracle, sc, cam, pix, bf16, mode, max_flagged=0.03):
    """Forward on the pixels ``pix`` and the backward of a loss restricted to them (the
    upstream gradient is zero elsewhere, and at the pixels the oracle flags)."""
    feats = U.bf16_round(sc.feats) if bf16 else None
    scr = sc if feats is None else S.Scene(**{k: getattr(sc, k) for k in
                                               ("means", "scales", "quats", "opacities", "sh")},
                                           feats=feats, sh_degree=sc.sh_degree)
    ref = oracle.render(scr, cam, "f32", pixels=pix, mode=mode)
    flags = ref["flags"]
    assert (flags != 0).mean() < max_flagged   # large Gaussians at 4K cross more thresholds
    keep = pix[flags == 0]
    g = S.upstream_grads(cam.H, cam.W, sc.n_feat)
    mask = np.zeros(cam.W * cam.H, bool)
    mask[keep] = True
    gm = {k: (v.reshape(v.shape[:-2] + (-1,)) * mask).reshape(v.shape) for k, v in g.items()}
    gpu = U.run(sc, cam, gm, bf16=bf16)
    P = cam.W * cam.H
    for k in ("rgb", "depth", "alpha", "feat"):
        v = gpu[k].reshape(gpu[k].shape[:-2] + (P,))[..., pix]
        assert U.max_abs_unflagged(v, ref[k], flags) <= TOL_FWD, k
    gs = {k: v.reshape(v.shape[:-2] + (-1,))[..., keep] for k, v in g.items()}
    rb = oracle.backward(scr, cam, gs, "f32", pixels=keep, mode=mode)
    rm = oracle.backward(scr, cam, gs, "mixed", pixels=keep, mode=mode)
    U.assert_grads_close(gpu["grads"], rb, GRAD_KEYS, ref_alt=rm,
                         label=f"{cam.W}x{cam.H} n={sc.n} D={sc.n_feat} sampled "
                               f"({int((flags != 0).sum())} of {pix.size} px flagged)")
    return gpu


def test_full_size_semantic_frame_sampled(oracle):
    """1200x680, 1M room Gaussians, SH 3, 64 bf16 features: forward on 12 sampled tiles,
    backward of a loss restricted to them (oracle fed the same bf16 feature values)."""
    sc, cams = S.config_semantic(n_poses=100)
    cam = cams[7]
    _sampled_parity(oracle, sc, cam, _tile_pixels(cam, 12, 3), bf16=True, mode=1)


def test_full_size_memory_frame_sampled(oracle):
    """3840x2160, 3M room Gaussians, 32 fp32 features (per-tile recomputation, no stored
    blend lists): 8 sampled tiles, oracle by brute force over all Gaussians per tile."""
    sc, cams = S.config_memory(n_poses=10)
    cam = cams[3]
    gpu = _sampled_parity(oracle, sc, cam, _tile_pixels(cam, 8, 4), bf16=False, mode=0)
    assert gpu["instances"] > 1_000_000


# ---------------------------------------------------------------- edge cases

def test_empty_scene():
    sc = S.cube_scene(0, n_feat=4)
    cam = S.pinhole(40, 30, 40.0, 40.0, np.eye(3), np.array([0, 0, 2.0]))
    g = S.upstream_grads(cam.H, cam.W, 4)
    r = U.run(sc, cam, g)
    assert r["instances"] == 0
    assert np.all(r["rgb"] == 0) and np.all(r["alpha"] == 0) and np.all(r["feat"] == 0)
    np.testing.assert_array_equal(r["grads"]["pose"], np.zeros(6))


def test_all_culled():
    sc = S.cube_scene(500, n_feat=4)
    cam = S.pinhole(64, 48, 50.0, 50.0, np.eye(3), np.array([0, 0, -3.0]))   # scene behind
    g = S.upstream_grads(cam.H, cam.W, 4)
    r = U.run(sc, cam, g)
    assert r["instances"] == 0 and np.all(r["alpha"] == 0)
    for k in GRAD_KEYS:
        assert np.all(r["grads"][k] == 0), k


def test_one_huge_gaussian_and_odd_channels(oracle):
    # one Gaussian covering every tile, D = 3 (padded inside the kernels), SH 2
    sc = S.cube_scene(3, n_feat=3, sh_degree=2, seed=2, log_scale_mu=0.0, log_scale_sd=0.01)
    sc.means[:] = [[0.0, 0.0, 0.0], [0.1, 0.0, 0.3], [-0.2, 0.1, -0.2]]
    cam = S.pinhole(150, 90, 80.0, 80.0, np.eye(3), np.array([0, 0, 2.5]))
    ref = oracle.render(sc, cam, "f32")
    g, nflag = U.mask_flagged(S.upstream_grads(cam.H, cam.W, 3), ref["flags"])
    r = U.run(sc, cam, g)
    for k in ("rgb", "depth", "alpha", "feat"):
        assert U.max_abs_unflagged(r[k], ref[k], ref["flags"]) <= TOL_FWD, k
    rb = oracle.backward(sc, cam, g, "f32")
    U.assert_grads_close(r["grads"], rb, GRAD_KEYS, label=f"one huge Gaussian ({nflag} flagged px)",
                         ref_alt=oracle.backward(sc, cam, g, "mixed"))


def test_no_features():
    sc = S.cube_scene(800, n_feat=0, seed=3)
    cam = S.config_tiny()[1][0]
    g = S.upstream_grads(cam.H, cam.W, 0)
    r = U.run(sc, cam, {k: v for k, v in g.items() if k != "feat"})
    assert r["feat"] is None and r["grads"]["feats"] is None
    assert r["alpha"].max() > 0.5


def test_no_sync_binning_and_overflow():
    from paper_2603_09632_gb300 import _lib as L
    from paper_2603_09632_gb300.render import Rasterizer
    sc, (cam,) = S.config_tiny()
    ref = U.run(sc, cam)
    rast = Rasterizer(U.device())
    rast.reserve(sc.n, ref["instances"], cam.W * cam.H)
    out = U.run(sc, cam, rast=rast, sync=False)
    for k in ("rgb", "alpha", "feat"):
        np.testing.assert_array_equal(out[k], ref[k])
    assert L.gs_workspace_status(rast.ws) == L.GS_OK
    # a workspace reserved too small: the excess is dropped and reported, nothing faults
    small = Rasterizer(U.device())
    small.reserve(sc.n, ref["instances"] // 2, cam.W * cam.H)
    U.run(sc, cam, rast=small, sync=False)
    assert L.gs_workspace_status(small.ws) == L.GS_ERR_DEVICE
    assert L.gs_workspace_status(small.ws) == L.GS_OK      # cleared by the read


def test_l1_grad_matches_sign():
    import torch
    from paper_2603_09632_gb300 import _lib as L
    a = torch.randn(1000, device=U.device())
    b = torch.randn(1000, device=U.device())
    b[:10] = a[:10]
    out = torch.empty_like(a)
    L.gs_l1_grad(a, b, 0.5, out)
    ref = 0.5 * np.sign(a.cpu().numpy() - b.cpu().numpy())
    np.testing.assert_array_equal(out.cpu().numpy(), ref.astype(np.float32))


def test_argument_errors():
    from paper_2603_09632_gb300 import _lib as L
    from paper_2603_09632_gb300.render import Rasterizer
    sc, (cam,) = S.config_tiny()
    scene = U.upload(sc)
    rast = Rasterizer(U.device())
    c = L.make_camera(cam.W, cam.H, cam.fx, cam.fy, cam.cx, cam.cy, cam.R, cam.t)
    with pytest.raises(L.GSError) as e:
        L.gs_render_fwd(scene, c, rast.ws)            # before project/bin
    assert e.value.status == L.GS_ERR_STATE
    bad = L.make_camera(cam.W, cam.H, -1.0, cam.fy, cam.cx, cam.cy, cam.R, cam.t)
    with pytest.raises(L.GSError) as e:
        L.gs_project(scene, bad, rast.ws)
    assert e.value.status == L.GS_ERR_ARG


# ---------------------------------------------------------------- binning edge cases

def _lists_equal(oracle, sc, cam, rast=None):
    from paper_2603_09632_gb300 import _lib as L
    gpu = U.run(sc, cam, rast=rast)
    TX, TY = oracle.tiles(cam)
    keys, ids, ranges = oracle.tile_lists(sc, cam)
    tiles_g, ids_g, ranges_g = L.gs_get_instances(gpu["rast"].ws, TX * TY)
    depth_g = L.gs_get_projection(gpu["rast"].ws, sc.n)["depth"].view(np.uint32)
    keys_g = (tiles_g.astype(np.uint64) << np.uint64(32)) | depth_g[ids_g].astype(np.uint64)
    np.testing.assert_array_equal(ranges_g, ranges)
    np.testing.assert_array_equal(keys_g, keys)
    np.testing.assert_array_equal(ids_g, ids)
    return gpu, ranges


def test_crowded_tiles_longer_than_shared_memory(oracle):
    """Thousands of Gaussians on the same few tiles: their lists exceed the 2048 entries a
    block sorts in shared memory, so they take the chunked global path of the tile sort."""
    rng = np.random.default_rng(21)
    sc = S.cube_scene(7000, n_feat=4, seed=21, log_scale_mu=-5.5, log_scale_sd=0.2)
    sc.means[:] = np.stack([rng.uniform(-0.01, 0.01, 7000), rng.uniform(-0.01, 0.01, 7000),
                            rng.uniform(-0.5, 0.5, 7000)], axis=1)
    cam = S.pinhole(96, 80, 100.0, 100.0, np.eye(3), np.array([0.0, 0.0, 2.0]))
    gpu, ranges = _lists_equal(oracle, sc, cam)
    assert (ranges[:, 1] - ranges[:, 0]).max() > 2048
    ref = oracle.render(sc, cam, "f32")
    for k in ("rgb", "depth", "alpha", "feat"):
        assert U.max_abs_unflagged(gpu[k], ref[k], ref["flags"]) <= TOL_FWD, k


@pytest.mark.parametrize("crowded", [False, True])
def test_equal_depths_are_ordered_by_id(oracle, crowded):
    """A fronto-parallel plane: every Gaussian has the bit-identical camera depth, so each
    tile's order is decided by the id tie-break alone (short and chunked sort paths)."""
    rng = np.random.default_rng(22)
    n = 5000 if crowded else 3000
    sc = S.cube_scene(n, n_feat=4, seed=22, log_scale_mu=-4.0, log_scale_sd=0.3)
    half = 0.01 if crowded else 0.6
    sc.means[:] = np.stack([rng.uniform(-half, half, n), rng.uniform(-half, half, n),
                            np.zeros(n)], axis=1)
    cam = S.pinhole(96, 80, 100.0, 100.0, np.eye(3), np.array([0.0, 0.0, 2.0]))
    proj = oracle.project(sc, cam, "f32")
    assert len(np.unique(proj["depth"][proj["valid"]])) == 1
    gpu, ranges = _lists_equal(oracle, sc, cam)
    if crowded:
        assert (ranges[:, 1] - ranges[:, 0]).max() > 2048


def _large_frame_scene(W, H, n=40_000, seed=31):
    """A room seen at W x H (at least 4096 tiles: the projection counts tile instances as
    per-row differences there) plus a few large Gaussians in front of the camera, whose
    rectangles reach the right and bottom edges of the tile grid (clamped)."""
    sc = S.room_scene(n, n_feat=4, sh_degree=0, seed=seed)
    cam = S.room_trajectory(8, W, H, 0.9 * W)[1]
    R, t = np.asarray(cam.R, np.float64), np.asarray(cam.t, np.float64)
    centre = -R.T @ t
    fwd = R.T @ np.array([0.0, 0.0, 1.0])
    rng = np.random.default_rng(seed)
    for k in range(6):   # overwrite a few Gaussians: 0.3-0.6 m in front, large
        i = k * 997
        right = R.T @ np.array([1.0, 0.0, 0.0])
        down = R.T @ np.array([0.0, 1.0, 0.0])
        sc.means[i] = centre + fwd * rng.uniform(1.0, 2.0) + right * rng.uniform(0.2, 0.8) + down * rng.uniform(0.1, 0.5)
        sc.scales[i] = rng.uniform(0.15, 0.3, 3)
    return sc, cam


@pytest.mark.parametrize("W,H", [(1090, 1030), (1024, 1024)])
def test_tile_lists_bit_exact_row_counted_frames(oracle, W, H):
    """Frames of at least 4096 tiles (ragged and exact tile multiples): the tile counts come
    from per-row differences and the binning's row pass; keys, ids and ranges must equal
    the oracle's, and large Gaussians must reach the last tile column."""
    TX, TY = (W + 15) // 16, (H + 15) // 16
    assert TX * TY >= 4096
    sc, cam = _large_frame_scene(W, H)
    proj = oracle.project(sc, cam, "f32")
    rect = proj["rect"][proj["valid"]]
    assert (rect[:, 2] == TX).any()      # some rectangle is clamped at the right edge
    _lists_equal(oracle, sc, cam)


def test_counting_forms_alternate_on_one_workspace(oracle):
    """Per-row (>= 4096 tiles) and per-tile (< 4096 tiles) counting alternating on one
    rasterizer: each binning must leave the count array clear for the next projection,
    whichever form that projection uses."""
    from paper_2603_09632_gb300.render import Rasterizer
    rast = Rasterizer(U.device())
    big = _large_frame_scene(1090, 1030, n=20_000, seed=33)
    small = small_room(n=20_000, W=200, H=136, D=4, deg=0, pose=2)
    for sc, cam in (big, small, big, small):
        _lists_equal(oracle, sc, cam, rast=rast)
