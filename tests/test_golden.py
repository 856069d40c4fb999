"""The stored golden fixture (``tests/golden/hand_scene_40x28.json``, written by
``tests/golden/make_golden.py`` from the FP64 oracle): a hand-placed scene whose sampled
pixels blend 0 to 6 Gaussians, with an anisotropic rotated covariance, SH degree 1, a
Gaussian across the image edge and one in front of the near plane.

On the CPU the oracle must still reproduce the stored values (a change of the oracle's
arithmetic shows here).  On the GPU the CUDA path must match them within the parity
tolerances: forward max-abs 1e-4 and last-contributor counts bit-exact at the sampled
pixels, every gradient entry within 1e-3 of its stored value plus 1e-5 of the tensor's
largest entry (no pixel of the scene is near a blend threshold, so nothing is masked)."""
import json
import os
import sys

import numpy as np
import pytest

from synth import scenes as S

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, HERE)
import make_golden as MG   # noqa: E402

GRAD_KEYS = ("means", "scales", "quats", "opacities", "sh", "feats", "pose")


@pytest.fixture(scope="module")
def golden():
    with open(os.path.join(HERE, "hand_scene_40x28.json")) as f:
        return json.load(f)


def test_fixture_is_what_its_script_describes(golden):
    sc, cam = MG.hand_scene(), MG.camera()
    assert golden["pixels"] == MG.pixels(cam).tolist()
    assert golden["upstream_grad_seed"] == MG.GRAD_SEED
    nc = np.array(golden["n_contrib"])
    assert nc.min() == 0 and nc.max() >= 5          # empty pixels and deep stacks
    assert (np.array(golden["flags"]) == 0).all()   # no pixel near a threshold
    # the Gaussian in front of the near plane gets no gradient, the one across the edge does
    g = {k: np.array(v) for k, v in golden["grads"].items()}
    assert all(np.all(g[k][sc.n - 1] == 0) for k in GRAD_KEYS if k != "pose")
    assert np.abs(g["opacities"][5]) > 0


def test_oracle_reproduces_the_fixture(oracle, golden):
    sc, cam = MG.hand_scene(), MG.camera()
    pix = np.array(golden["pixels"])
    ref = oracle.render(sc, cam, "f64", pixels=pix)
    for k, v in golden["forward"].items():
        np.testing.assert_allclose(ref[k], np.array(v), rtol=1e-12, atol=1e-12, err_msg=k)
    np.testing.assert_array_equal(ref["n_contrib"], golden["n_contrib"])
    g = S.upstream_grads(cam.H, cam.W, sc.n_feat, seed=golden["upstream_grad_seed"])
    rb = oracle.backward(sc, cam, g, "f64")
    for k in GRAD_KEYS:
        np.testing.assert_allclose(rb[k], np.array(golden["grads"][k]), rtol=1e-10, atol=1e-12,
                                   err_msg=k)


@pytest.mark.gpu
def test_cuda_path_matches_the_fixture(golden):
    from paper_2603_09632_gb300 import _lib as L
    from tests import gpu_util as U
    sc, cam = MG.hand_scene(), MG.camera()
    g = S.upstream_grads(cam.H, cam.W, sc.n_feat, seed=golden["upstream_grad_seed"])
    gpu = U.run(sc, cam, g)
    pix = np.array(golden["pixels"])
    P = cam.W * cam.H
    for k, v in golden["forward"].items():
        if k == "T_final":
            continue
        got = gpu[k].reshape(gpu[k].shape[:-2] + (P,))[..., pix]
        assert np.abs(got - np.array(v)).max() <= 1e-4, k
    T, nc = L.gs_get_pixel_state(gpu["rast"].ws, cam.H, cam.W)
    np.testing.assert_array_equal(nc.reshape(-1)[pix], golden["n_contrib"])
    assert np.abs(T.reshape(-1)[pix] - np.array(golden["forward"]["T_final"])).max() <= 1e-4
    U.assert_grads_close(gpu["grads"], {k: np.array(golden["grads"][k]) for k in GRAD_KEYS},
                         GRAD_KEYS, label="golden hand scene 40x28 (FP64 fixture)")
