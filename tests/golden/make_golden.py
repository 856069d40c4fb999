"""Writes ``tests/golden/hand_scene_40x28.json``: a hand-placed seven-Gaussian scene and the
FP64 oracle's forward values at 60 sampled pixels and every gradient of a seeded upstream
gradient.  Only ``oracle/`` computes the stored values, and the inputs come from this
file and ``synth.scenes.upstream_grads``.

The scene covers the method's cases on a 40 x 28 image (3 x 2 tiles of 16 pixels, ragged on
both axes):
* overlapping Gaussians at different depths (Eq. 1, front-to-back compositing);
* anisotropic, rotated covariances (App. A, Sigma = R S S^T R^T, EWA projection);
* SH degree 1 colour along the view direction (Sec. 3.1 preliminaries);
* one Gaussian across the image edge and one in front of the near plane (culled).

The sampled pixels blend 0 to 6 Gaussians.  Run ``python tests/golden/make_golden.py``
from the repository root to regenerate the fixture; ``tests/test_golden.py`` checks the
oracle (CPU) and the CUDA path (GPU) against it."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from synth import scenes as S   # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hand_scene_40x28.json")
GRAD_SEED = 20260304


def _quat(axis, deg):
    axis = np.asarray(axis, np.float64)
    axis = axis / np.linalg.norm(axis)
    h = np.radians(deg) / 2.0
    return [float(np.cos(h))] + [float(v) for v in np.sin(h) * axis]


def hand_scene():
    """Seven Gaussians (mean, scale, quaternion w x y z, opacity) in front of a camera at the
    origin looking down +z, with degree-1 SH and four feature channels."""
    g = [
        ((0.00, 0.00, 2.0), (0.10, 0.10, 0.10), _quat((0, 0, 1), 0), 0.80),
        ((0.15, -0.05, 2.5), (0.20, 0.05, 0.10), _quat((0, 0, 1), 30), 0.60),
        ((-0.30, 0.10, 3.0), (0.15, 0.15, 0.05), _quat((1, 0, 0), 45), 0.90),
        ((0.35, 0.20, 1.5), (0.03, 0.04, 0.05), _quat((1, 1, 0), 60), 0.95),
        ((-0.10, -0.20, 4.0), (0.40, 0.30, 0.20), _quat((0, 1, 1), 20), 0.50),
        ((0.55, -0.30, 2.2), (0.10, 0.20, 0.10), _quat((1, 0, 1), 75), 0.70),
        ((0.00, 0.00, 0.10), (0.05, 0.05, 0.05), _quat((0, 0, 1), 0), 0.90),   # before the near plane
    ]
    n = len(g)
    sh = np.zeros((n, 4, 3))
    base = np.array([[0.9, 0.1, 0.1], [0.1, 0.8, 0.2], [0.2, 0.3, 0.9], [0.9, 0.9, 0.1],
                     [0.5, 0.5, 0.5], [0.1, 0.9, 0.9], [1.0, 0.0, 1.0]])
    sh[:, 0, :] = (base - 0.5) * 2.0 * np.sqrt(np.pi)   # Y_0 = 1 / (2 sqrt(pi)): colour = base
    for i in range(n):
        sh[i, 1:, :] = 0.2 * np.sin(np.arange(9).reshape(3, 3) + i)
    feats = np.array([[np.cos(0.7 * i + c) for c in range(4)] for i in range(n)])
    f32 = np.float32
    return S.Scene(means=np.array([m for m, _, _, _ in g], f32),
                   scales=np.array([s for _, s, _, _ in g], f32),
                   quats=np.array([q for _, _, q, _ in g], f32),
                   opacities=np.array([o for _, _, _, o in g], f32),
                   sh=sh.astype(f32), feats=feats.astype(f32), sh_degree=1)


def camera():
    return S.pinhole(40, 28, 40.0)


def pixels(cam):
    """Every fifth column and every fourth row, and the four corners."""
    ys, xs = np.mgrid[1:cam.H:4, 2:cam.W:5]
    pix = list((ys * cam.W + xs).ravel())
    pix += [0, cam.W - 1, (cam.H - 1) * cam.W, cam.H * cam.W - 1]
    return np.array(sorted(set(int(p) for p in pix)), np.int64)


def main():
    from oracle import oracle as O
    sc, cam = hand_scene(), camera()
    pix = pixels(cam)
    g = S.upstream_grads(cam.H, cam.W, sc.n_feat, seed=GRAD_SEED)
    fwd = O.render(sc, cam, "f64")
    bwd = O.backward(sc, cam, g, "f64")
    P = cam.W * cam.H
    take = lambda a: np.asarray(a).reshape(np.asarray(a).shape[:-2] + (P,))[..., pix]   # noqa: E731
    doc = {
        "what": "hand-placed 7-Gaussian scene, 40x28 pinhole camera; FP64 oracle forward at "
                "sampled pixels and the gradients of sum(g * outputs) over the whole image",
        "citation": "Eq. 1 (front-to-back alpha compositing; depth and features by "
                    "substitution, App. B, Sec. 3.1); App. A (covariance and EWA projection); "
                    "gradients of the rasterizer (App. B)",
        "written_by": "tests/golden/make_golden.py (oracle/ only)",
        "upstream_grad_seed": GRAD_SEED,
        "pixels": pix.tolist(),
        "forward": {k: take(fwd[k]).tolist() for k in ("rgb", "depth", "alpha", "feat", "T_final")},
        "n_contrib": take(fwd["n_contrib"]).astype(int).tolist(),
        "flags": take(fwd["flags"]).astype(int).tolist(),
        "grads": {k: np.asarray(bwd[k]).tolist()
                  for k in ("means", "scales", "quats", "opacities", "sh", "feats", "pose")},
    }
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=0)
        f.write("\n")
    print(OUT, len(pix), "pixels; n_contrib range",
          int(np.min(doc["n_contrib"])), int(np.max(doc["n_contrib"])))


if __name__ == "__main__":
    main()
