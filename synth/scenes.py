"""Seeded synthetic scenes, cameras and upstream gradients.

This module only draws random inputs: Gaussian clouds shaped like the indoor
SLAM workloads of X-GS (Sec. 4.1, Table 3: TUM RGB-D / ScanNet rooms), pinhole
cameras on smooth trajectories, and upstream gradients.  It holds none of the
renderer's arithmetic (no projection, no SH basis, no blending) and is shared
by the CPU oracle tests, the GPU parity tests and the benchmark.

Conventions of the drawn data (App. A parameterisation Theta = {mu, Sigma, alpha, c}):
  means     [N,3] f32  world positions
  scales    [N,3] f32  positive (log-normal draw)
  quats     [N,4] f32  (w, x, y, z), unit length unless ``raw_quats``
  opacities [N]   f32  in (0,1) (logit-normal draw)
  sh        [N,K,3] f32, K = (deg+1)^2; the degree-0 coefficient is drawn
            uniform in [-sqrt(pi), sqrt(pi)], which is the coefficient range
            that maps to an RGB colour uniform in [0,1] under the real SH
            basis with the +0.5 offset
  feats     [N,D] f32 N(0,1) (converted to bf16 by the caller where wanted)
Cameras are world->camera (R, t) with OpenCV axes (x right, y down, z forward).
The room has world y pointing down: the floor is the plane y = +1.5.

Seeds: scene = 0, trajectory = 1, upstream grads / targets = 2, serving = 3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_SCENE = 0
SEED_TRAJ = 1
SEED_GRADS = 2
SEED_SERVE = 3

ROOM_LO = np.array([-3.0, -1.5, -2.5])
ROOM_HI = np.array([3.0, 1.5, 2.5])


@dataclass
class Scene:
    means: np.ndarray
    scales: np.ndarray
    quats: np.ndarray
    opacities: np.ndarray
    sh: np.ndarray
    feats: np.ndarray
    sh_degree: int
    log_scales: np.ndarray = field(default=None)
    opacity_logits: np.ndarray = field(default=None)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def n_feat(self) -> int:
        return int(self.feats.shape[1])


@dataclass
class Camera:
    W: int
    H: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray  # [3,3] world->camera rotation
    t: np.ndarray  # [3]
    near: float = 0.2

    def copy_with(self, R=None, t=None) -> "Camera":
        return Camera(self.W, self.H, self.fx, self.fy, self.cx, self.cy,
                      self.R.copy() if R is None else np.asarray(R, np.float64),
                      self.t.copy() if t is None else np.asarray(t, np.float64),
                      self.near)


def _gaussian_attrs(rng, n, log_scale_mu, log_scale_sd, sh_degree, n_feat,
                    sh_hi_sd=0.1, raw_quats=False):
    log_scales = rng.normal(log_scale_mu, log_scale_sd, size=(n, 3))
    q = rng.normal(size=(n, 4))
    if not raw_quats:
        q = q / np.linalg.norm(q, axis=1, keepdims=True)
    logits = rng.normal(size=n)
    K = (sh_degree + 1) ** 2
    sh = np.zeros((n, K, 3))
    sh[:, 0, :] = rng.uniform(-math.sqrt(math.pi), math.sqrt(math.pi), size=(n, 3))
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, sh_hi_sd, size=(n, K - 1, 3))
    feats = rng.normal(size=(n, n_feat))
    return (log_scales, q, logits, sh, feats)


def _finish(means, attrs, sh_degree) -> Scene:
    log_scales, q, logits, sh, feats = attrs
    f32 = np.float32
    return Scene(
        means=np.ascontiguousarray(means, f32),
        scales=np.ascontiguousarray(np.exp(log_scales), f32),
        quats=np.ascontiguousarray(q, f32),
        opacities=np.ascontiguousarray(1.0 / (1.0 + np.exp(-logits)), f32),
        sh=np.ascontiguousarray(sh, f32),
        feats=np.ascontiguousarray(feats, f32),
        sh_degree=sh_degree,
        log_scales=np.ascontiguousarray(log_scales, f32),
        opacity_logits=np.ascontiguousarray(logits, f32),
    )


def cube_scene(n=2000, n_feat=8, sh_degree=0, seed=SEED_SCENE, log_scale_mu=-3.0,
               log_scale_sd=0.5, extent=1.0, raw_quats=False) -> Scene:
    """Configuration 'tiny': means uniform in a cube of side ``extent`` at the origin."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-0.5 * extent, 0.5 * extent, size=(n, 3))
    attrs = _gaussian_attrs(rng, n, log_scale_mu, log_scale_sd, sh_degree, n_feat,
                            raw_quats=raw_quats)
    return _finish(means, attrs, sh_degree)


def _sample_box_faces(rng, lo, hi, m):
    """m points uniform (area-weighted) on the 6 faces of the box [lo, hi]."""
    ext = hi - lo
    areas = np.array([ext[1] * ext[2], ext[1] * ext[2], ext[0] * ext[2],
                      ext[0] * ext[2], ext[0] * ext[1], ext[0] * ext[1]])
    face = rng.choice(6, size=m, p=areas / areas.sum())
    p = lo + rng.uniform(size=(m, 3)) * ext
    axis = face // 2
    side = face % 2
    p[np.arange(m), axis] = np.where(side == 0, lo[axis], hi[axis])
    return p


def room_scene(n=200_000, n_feat=16, sh_degree=0, seed=SEED_SCENE, n_boxes=20,
               wall_frac=0.7, log_scale_mu=-4.0, log_scale_sd=0.5, sh_hi_sd=0.1) -> Scene:
    """Indoor room: ``wall_frac`` of the Gaussians on the walls, floor and ceiling of
    a 6 x 3 x 5 m room, the rest on ``n_boxes`` axis-aligned boxes standing on the floor.
    """
    rng = np.random.default_rng(seed)
    n_wall = int(round(n * wall_frac))
    n_box = n - n_wall
    walls = _sample_box_faces(rng, ROOM_LO, ROOM_HI, n_wall)
    sides = rng.uniform(0.2, 1.0, size=(n_boxes, 3))
    lo = np.empty((n_boxes, 3))
    for a in (0, 2):
        lo[:, a] = rng.uniform(ROOM_LO[a], ROOM_HI[a] - sides[:, a])
    lo[:, 1] = ROOM_HI[1] - sides[:, 1]          # resting on the floor (y down)
    hi = lo + sides
    ext = sides
    box_area = 2 * (ext[:, 0] * ext[:, 1] + ext[:, 1] * ext[:, 2] + ext[:, 0] * ext[:, 2])
    which = rng.choice(n_boxes, size=n_box, p=box_area / box_area.sum())
    boxes = np.empty((n_box, 3))
    for b in range(n_boxes):
        sel = np.nonzero(which == b)[0]
        if sel.size:
            boxes[sel] = _sample_box_faces(rng, lo[b], hi[b], sel.size)
    means = np.concatenate([walls, boxes], axis=0)
    means = means[rng.permutation(n)]
    attrs = _gaussian_attrs(rng, n, log_scale_mu, log_scale_sd, sh_degree, n_feat,
                            sh_hi_sd=sh_hi_sd)
    return _finish(means, attrs, sh_degree)


def look_at(eye, target, up=(0.0, -1.0, 0.0)):
    """World->camera (R, t) for an OpenCV camera at ``eye`` looking at ``target``."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    down = -np.asarray(up, np.float64)
    right = np.cross(down, fwd)
    nr = np.linalg.norm(right)
    if nr < 1e-8:
        right = np.cross(np.array([0.0, 0.0, 1.0]), fwd)
        nr = np.linalg.norm(right)
    right /= nr
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd], axis=0)
    t = -R @ eye
    return R, t


def pinhole(W, H, fx, fy=None, R=None, t=None, near=0.2) -> Camera:
    fy = fx if fy is None else fy
    R = np.eye(3) if R is None else np.asarray(R, np.float64)
    t = np.zeros(3) if t is None else np.asarray(t, np.float64)
    return Camera(W, H, float(fx), float(fy), W / 2.0, H / 2.0, R, t, near)


def _catmull_rom_closed(ctrl, n):
    m = len(ctrl)
    out = []
    for k in range(n):
        s = k * m / n
        i = int(math.floor(s))
        u = s - i
        p0, p1, p2, p3 = (ctrl[(i - 1) % m], ctrl[i % m], ctrl[(i + 1) % m], ctrl[(i + 2) % m])
        out.append(0.5 * ((2 * p1) + (-p0 + p2) * u + (2 * p0 - 5 * p1 + 4 * p2 - p3) * u * u
                          + (-p0 + 3 * p1 - 3 * p2 + p3) * u ** 3))
    return np.array(out)


def room_trajectory(n_poses=100, W=640, H=480, fx=600.0, seed=SEED_TRAJ, n_ctrl=8,
                    margin=0.75):
    """Smooth random camera path inside the room: eyes on a closed Catmull-Rom spline
    through ``n_ctrl`` points of the room shrunk by ``margin``; look-at targets on a
    second spline through random points of the full room; world up is -y."""
    rng = np.random.default_rng(seed)
    lo, hi = ROOM_LO + margin, ROOM_HI - margin
    eyes_c = rng.uniform(lo, hi, size=(n_ctrl, 3))
    tgts_c = rng.uniform(ROOM_LO, ROOM_HI, size=(n_ctrl, 3))
    eyes = _catmull_rom_closed(eyes_c, n_poses)
    tgts = _catmull_rom_closed(tgts_c, n_poses)
    cams = []
    for e, g in zip(eyes, tgts):
        if np.linalg.norm(g - e) < 0.5:
            g = e + np.array([0.0, 0.0, 1.0])
        R, t = look_at(e, g)
        cams.append(pinhole(W, H, fx, fx, R, t))
    return cams


def upstream_grads(H, W, n_feat, seed=SEED_GRADS, scale=1.0):
    """N(0,1) upstream gradients for rgb[3,H,W], depth[H,W], alpha[H,W], feat[D,H,W]."""
    rng = np.random.default_rng(seed)
    f32 = np.float32
    return dict(
        rgb=(scale * rng.normal(size=(3, H, W))).astype(f32),
        depth=(scale * rng.normal(size=(H, W))).astype(f32),
        alpha=(scale * rng.normal(size=(H, W))).astype(f32),
        feat=(scale * rng.normal(size=(n_feat, H, W))).astype(f32),
    )


def region_annotations(H, W, n_feat, n_regions=200, seed=SEED_GRADS, block=8, bg_frac=0.2):
    """Seeded stand-in for precomputed region-indexed semantic annotations (App. D): a
    segmentation [H, W] int32 of piecewise-constant regions on ``block``-pixel cells
    (about ``bg_frac`` background, id -1) and a region-feature table [n_regions, n_feat]
    of N(0, 1) float32 rows."""
    rng = np.random.default_rng(seed + 2000)
    coarse = rng.integers(0, n_regions, size=(-(-H // block), -(-W // block)))
    coarse[rng.uniform(size=coarse.shape) < bg_frac] = -1
    seg = np.repeat(np.repeat(coarse, block, 0), block, 1)[:H, :W].astype(np.int32)
    table = rng.normal(size=(n_regions, n_feat)).astype(np.float32)
    return seg, table


def grid_offsets(n, stride, seed=SEED_GRADS):
    """Per-step grid offsets (o_x, o_y) drawn uniformly from {0..s-1}^2 (App. D)."""
    rng = np.random.default_rng(seed + 3000)
    return [tuple(int(v) for v in rng.integers(0, stride, size=2)) for _ in range(n)]


def feature_target(H, W, n_feat, seed=SEED_GRADS):
    """Seeded N(0,1) target feature map [D,H,W] for the L1 distillation loss."""
    rng = np.random.default_rng(seed + 1000)
    return rng.normal(size=(n_feat, H, W)).astype(np.float32)


# --- the five workload shapes -------------------------------------------------

def config_tiny():
    """2,000 Gaussians in a unit cube, 128x96, fx=fy=100, camera at distance 2."""
    scene = cube_scene(2000, n_feat=8, sh_degree=0)
    cam = pinhole(128, 96, 100.0, 100.0, np.eye(3), np.array([0.0, 0.0, 2.0]))
    return scene, [cam]


def config_slam(n=200_000, n_poses=100):
    """SLAM frame: 200k room Gaussians, SH 0, 16 f32 features, 640x480, fx=fy=600."""
    scene = room_scene(n, n_feat=16, sh_degree=0)
    return scene, room_trajectory(n_poses, 640, 480, 600.0)


def config_semantic(n=1_000_000, n_poses=100):
    """Semantic distillation: 1M room Gaussians, SH 3, 64 bf16 features, 1200x680."""
    scene = room_scene(n, n_feat=64, sh_degree=3)
    return scene, room_trajectory(n_poses, 1200, 680, 600.0)


def config_memory(n=3_000_000, n_poses=10, fx=3600.0):
    """Memory-bound run: 3M room Gaussians, 32 f32 features, 3840x2160."""
    scene = room_scene(n, n_feat=32, sh_degree=0)
    return scene, room_trajectory(n_poses, 3840, 2160, fx)


SERVE_RESOLUTIONS = [(256, 256), (640, 480), (1200, 680), (1920, 1080)]


def serving_scenes(n_scenes=8, seed=SEED_SERVE, n_lo=100_000, n_hi=2_000_000, scale=1.0):
    """Resident scenes for serving: N log-uniform in [n_lo, n_hi] (times ``scale``),
    SH degree = scene id mod 4, D drawn from {16, 32, 64} (stored bf16)."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_scenes):
        n = int(round(scale * math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        d = int(rng.choice([16, 32, 64]))
        out.append(room_scene(max(n, 16), n_feat=d, sh_degree=s % 4, seed=1000 + s))
    return out


def serving_requests(n_req, rate_hz, n_scenes=8, seed=SEED_SERVE, bwd_frac=0.3,
                     resolutions=SERVE_RESOLUTIONS, fx_per_width=600.0 / 640.0):
    """Poisson arrivals: (t_arrive_s, scene_id, camera, want_bwd)."""
    rng = np.random.default_rng(seed + 7)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_req))
    reqs = []
    for k in range(n_req):
        W, H = resolutions[rng.integers(len(resolutions))]
        e = rng.uniform(ROOM_LO + 0.75, ROOM_HI - 0.75)
        g = rng.uniform(ROOM_LO, ROOM_HI)
        if np.linalg.norm(g - e) < 0.5:
            g = e + np.array([0.0, 0.0, 1.0])
        R, tt = look_at(e, g)
        cam = pinhole(W, H, fx_per_width * W, fx_per_width * W, R, tt)
        reqs.append((float(t[k]), int(rng.integers(n_scenes)), cam, bool(rng.uniform() < bwd_frac)))
    return reqs
