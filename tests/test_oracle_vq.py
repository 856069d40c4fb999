"""Pins of the VQ oracle (``oracle/vq.py``; Sec. 3.2 Online VQ Module, App. E): softmax
against SciPy, its backward against finite differences, the rendered weight map summing to
the rendered alpha, decode(render(w)) = render(E^T w) (per-pixel and per-Gaussian decodes
agree, App. E), one-hot decodes, and closed-form relevance values."""
import math

import numpy as np
import pytest

from synth import scenes as S


@pytest.fixture(scope="module")
def VQ(oracle):
    from oracle import vq
    return vq


def test_softmax_weights(VQ):
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(1)
    z = rng.normal(scale=3.0, size=(50, 64))
    w = VQ.weights(z)
    np.testing.assert_allclose(w, sp.softmax(z, axis=1), rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(w.sum(1), 1.0, rtol=1e-14)
    np.testing.assert_allclose(VQ.weights(z + 7.5), w, rtol=1e-12)
    assert (w > 0).all()


def test_softmax_backward_finite_differences(VQ):
    rng = np.random.default_rng(2)
    z = rng.normal(size=(6, 16))
    g = rng.normal(size=(6, 16))
    dz = VQ.weights_bwd(z, g)
    h = 1e-6
    for i, l in [(0, 0), (2, 5), (5, 15), (3, 7)]:
        e = np.zeros_like(z)
        e[i, l] = h
        fd = ((VQ.weights(z + e) * g).sum() - (VQ.weights(z - e) * g).sum()) / (2 * h)
        assert abs(fd - dz[i, l]) < 1e-8
    np.testing.assert_allclose(dz.sum(1), 0.0, atol=1e-14)   # softmax is shift invariant


def _scene():
    sc = S.cube_scene(400, n_feat=3, sh_degree=0, seed=4, log_scale_mu=-2.5)
    cam = S.pinhole(48, 40, 40.0, 40.0, np.eye(3), np.array([0.0, 0.0, 2.0]))
    return sc, cam


def test_weight_map_sums_to_alpha(oracle, VQ):
    sc, cam = _scene()
    z = np.random.default_rng(3).normal(size=(sc.n, 32))
    wm = VQ.render_weights(sc, cam, z, "f64")
    alpha = oracle.render(sc, cam, "f64")["alpha"]
    assert alpha.max() > 0.5
    np.testing.assert_allclose(wm.sum(0), alpha, rtol=1e-12, atol=1e-14)


def test_pixel_decode_equals_gaussian_decode(oracle, VQ):
    sc, cam = _scene()
    rng = np.random.default_rng(5)
    L, D = 16, 24
    z = rng.normal(size=(sc.n, L))
    E = rng.normal(size=(L, D))
    F = VQ.decode(VQ.render_weights(sc, cam, z, "f64"), E)
    # App. E decodes per Gaussian (f_i = E^T w_i) and per pixel (F = E^T w(x)); rendering
    # is linear in the features, so both give the same map
    ref = oracle.render(sc, cam, "f64", feats=VQ.weights(z) @ E)["feat"]
    np.testing.assert_allclose(F, ref, rtol=1e-11, atol=1e-13)
    # one-hot weights pick codewords
    onehot = np.zeros((L, 3, 2))
    onehot[4, 1, 0] = 1.0
    onehot[9, 2, 1] = 2.0
    Fo = VQ.decode(onehot, E)
    np.testing.assert_array_equal(Fo[:, 1, 0], E[4])
    np.testing.assert_array_equal(Fo[:, 2, 1], 2.0 * E[9])
    assert np.abs(Fo[:, 0, 0]).max() == 0


def test_relevance_closed_forms(VQ):
    D = 8
    basis = np.eye(D)
    t_pos, t_neg = basis[0], basis[1:5]
    F = np.stack([3.0 * basis[0], basis[2], np.zeros(D), 0.5 * basis[0] + 0.5 * basis[3]], axis=1)
    R = VQ.relevance(F, t_pos, t_neg)
    tau = VQ.TAU
    # along the prompt: every negative is orthogonal -> softmax(tau [1, 0])_1
    assert abs(R[0] - 1.0 / (1.0 + math.exp(-tau))) < 1e-6
    # along a negative: that negative gives softmax(tau [0, 1])_1, the others 0.5 -> max 0.5
    assert abs(R[1] - 0.5) < 1e-12
    # zero feature: all scores 0 -> 0.5
    assert abs(R[2] - 0.5) < 1e-12
    # equal parts prompt and negative 3: s+ = s3- = 1/sqrt(2) -> 0.5 vs the others
    s = 1.0 / math.sqrt(2.0)
    assert abs(R[3] - 1.0 / (1.0 + math.exp(-tau * s))) < 1e-6
    # scale invariance of the normalised feature
    np.testing.assert_allclose(VQ.relevance(7.0 * F[:, :2], t_pos, t_neg), R[:2], rtol=1e-9)
