"""Error of the GPU path against the FP64 oracle, per output, on the full semantic-size frame
(1200x680, 1M room Gaussians, SH 3, 64 feature channels): features stored in BF16 and in
FP32, every other quantity (transmittance, conics, pose gradient) in FP32 on the GPU.
Forward outputs on 16 sampled tiles, gradients of a loss restricted to them.

The gates are the parity tests' (FP32 oracle); this test states the FP64 errors and checks
only that they stay in the range the FP32 arithmetic allows.  With GS_PRECISION_REPORT set
to a path it writes the numbers there as JSON."""
import json
import os

import numpy as np
import pytest

from synth import scenes as S
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

GRAD_KEYS = ("means", "scales", "quats", "opacities", "sh", "feats", "pose")
IMG_KEYS = ("rgb", "depth", "alpha", "feat")


def _tile_pixels(cam, n_tiles, seed):
    rng = np.random.default_rng(seed)
    TX, TY = (cam.W + 15) // 16, (cam.H + 15) // 16
    out = []
    for t in rng.choice(TX * TY, size=n_tiles, replace=False):
        x0, y0 = (t % TX) * 16, (t // TX) * 16
        ys, xs = np.mgrid[y0:min(y0 + 16, cam.H), x0:min(x0 + 16, cam.W)]
        out.append((ys * cam.W + xs).ravel())
    return np.concatenate(out)


def _with_feats(sc, feats):
    return S.Scene(**{k: getattr(sc, k) for k in ("means", "scales", "quats", "opacities", "sh")},
                   feats=feats, sh_degree=sc.sh_degree)


def test_errors_against_fp64_per_output(oracle):
    sc, cams = S.config_semantic(n_poses=100)
    cam = cams[11]
    pix = _tile_pixels(cam, 16, 21)
    P = cam.W * cam.H
    g = S.upstream_grads(cam.H, cam.W, sc.n_feat, seed=31)
    mask = np.zeros(P, bool)
    mask[pix] = True
    gm = {k: (v.reshape(v.shape[:-2] + (-1,)) * mask).reshape(v.shape) for k, v in g.items()}
    gs = {k: v.reshape(v.shape[:-2] + (-1,))[..., pix] for k, v in g.items()}

    report = {"frame": "1200x680, 1M Gaussians, SH 3, 64 channels", "pixels": int(pix.size)}
    refs = {}
    for name, feats in (("fp32_features", sc.feats), ("bf16_values", U.bf16_round(sc.feats))):
        scr = _with_feats(sc, feats)
        refs[name] = (oracle.render(scr, cam, "f64", pixels=pix),
                      oracle.backward(scr, cam, gs, "f64", pixels=pix))
    for path, bf16, ref_name in (("fp32 features", False, "fp32_features"),
                                 ("bf16 features", True, "bf16_values"),
                                 ("bf16 features vs fp32-feature reference", True, "fp32_features")):
        gpu = U.run(sc, cam, gm, bf16=bf16)
        ref, rb = refs[ref_name]
        flags = ref["flags"]
        rec = {"unflagged_pixels": int((flags == 0).sum())}
        for k in IMG_KEYS:
            v = gpu[k].reshape(gpu[k].shape[:-2] + (P,))[..., pix]
            rec[k + "_max_abs"] = U.max_abs_unflagged(v, ref[k], flags)
            ok = flags == 0
            rec[k + "_rel"] = U.rel_err(v[..., ok], ref[k][..., ok])
        for k in GRAD_KEYS:
            rec["grad_" + k + "_rel"] = U.rel_err(gpu["grads"][k], rb[k])
        report[path] = rec
    out = os.environ.get("GS_PRECISION_REPORT")
    if out:
        with open(out, "w") as f:
            json.dump(report, f, indent=1)
    # FP32 arithmetic against FP64: well inside the FP32-oracle gates
    for path in ("fp32 features", "bf16 features"):
        r = report[path]
        for k in IMG_KEYS:
            assert r[k + "_max_abs"] <= 1e-4, (path, k, r[k + "_max_abs"])
        for k in GRAD_KEYS:
            assert r["grad_" + k + "_rel"] <= 1e-3, (path, k, r["grad_" + k + "_rel"])
    # BF16 storage of the features: the feature map within relative 1e-2 of the FP32 one
    assert report["bf16 features vs fp32-feature reference"]["feat_rel"] <= 1e-2
