"""Pins of the oracle's mixed mode: double arithmetic with each Gaussian's visibility, tile
rectangle and list-order depth taken from the float projection.  The readings define the
rectangle and the sort key by separately rounded float operations (App. A's Sigma' feeds a
3-sigma rectangle and the depth-sorted lists of Eq. 1), so the mixed mode is the same
function as the float path evaluated in exact arithmetic; the GPU gradient gates compare
against it."""
import numpy as np

from synth import scenes as S
from tests.test_oracle_backward import fd_camera, fd_scene

KEYS = ("means", "scales", "quats", "opacities", "sh", "feats", "pose")


def _f32_scene(sc):
    return S.Scene(**{k: np.asarray(getattr(sc, k), np.float32).astype(np.float64) for k in
                      ("means", "scales", "quats", "opacities", "sh", "feats")}, sh_degree=sc.sh_degree)


def test_mixed_equals_f64_where_the_decisions_agree(oracle):
    # a scene whose float and double projections agree on every rectangle: the mixed mode
    # must then be the double path bit for bit
    sc = _f32_scene(fd_scene(n=300, deg=2, D=3, seed=5))
    cam = fd_camera(80, 56)
    p32, p64 = oracle.project(sc, cam, "f32"), oracle.project(sc, cam, "f64")
    assert np.array_equal(p32["valid"], p64["valid"])
    assert np.array_equal(p32["rect"][p32["valid"]], p64["rect"][p64["valid"]])
    r64, rmx = oracle.render(sc, cam, "f64"), oracle.render(sc, cam, "mixed")
    for k in ("rgb", "depth", "alpha", "feat", "T_final", "n_contrib"):
        np.testing.assert_array_equal(rmx[k], r64[k], err_msg=k)
    g = {k: v.astype(np.float64) for k, v in S.upstream_grads(cam.H, cam.W, sc.n_feat, seed=4).items()}
    b64, bmx = oracle.backward(sc, cam, g, "f64"), oracle.backward(sc, cam, g, "mixed")
    for k in KEYS:
        np.testing.assert_array_equal(bmx[k], b64[k], err_msg=k)


def test_mixed_takes_the_float_lists(oracle):
    """A room frame with thousands of Gaussians: where the double projection would choose
    another rectangle, the mixed mode keeps the float one, so every pixel's blend list (its
    last-contributor position in the float tile lists) is the float path's, and its values
    differ from the float path only by float rounding."""
    sc = _f32_scene(S.room_scene(30_000, n_feat=8, sh_degree=1, seed=7))
    cam = S.room_trajectory(8, 200, 136, 180.0)[3]
    p32, p64 = oracle.project(sc, cam, "f32"), oracle.project(sc, cam, "f64")
    v = p32["valid"] & p64["valid"]
    differ = int((p32["valid"] != p64["valid"]).sum() + (p32["rect"][v] != p64["rect"][v]).any(1).sum())
    r32, rmx = oracle.render(sc, cam, "f32"), oracle.render(sc, cam, "mixed")
    ok = (r32["flags"] == 0) & (rmx["flags"] == 0)
    np.testing.assert_array_equal(rmx["n_contrib"][ok], r32["n_contrib"][ok])
    for k in ("rgb", "depth", "alpha", "feat"):   # within the forward tolerance of the GPU gates
        assert np.abs(rmx[k] - r32[k])[..., ok].max() <= 1e-4, k
    g = {k: v.astype(np.float64) for k, v in S.upstream_grads(cam.H, cam.W, sc.n_feat, seed=6).items()}
    g = {k: np.where(ok, v, 0.0) for k, v in g.items()}
    b32, bmx = oracle.backward(sc, cam, g, "f32"), oracle.backward(sc, cam, g, "mixed")
    for k in KEYS:
        a, b = bmx[k], b32[k]
        assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(a), (k, differ)


def test_mixed_gradient_is_the_exact_gradient(oracle):
    """Central differences of the mixed forward (step 1e-6 in double, every decision fixed
    by the float projection, no pixel near a threshold) agree with its analytic gradient
    to 1e-6 relative."""
    sc = _f32_scene(fd_scene(n=200, deg=1, D=2, seed=9))
    cam = fd_camera(48, 48)
    g = {k: v.astype(np.float64) for k, v in S.upstream_grads(cam.H, cam.W, sc.n_feat, seed=3).items()}

    def loss(s):
        r = oracle.render(s, cam, "mixed")
        assert (r["flags"] == 0).all()
        return sum(np.sum(g[k] * r[k]) for k in ("rgb", "depth", "alpha", "feat"))

    an = oracle.backward(sc, cam, g, "mixed")
    vis = np.nonzero(oracle.project(sc, cam, "f32")["valid"])[0]
    rng = np.random.default_rng(2)
    for name in ("means", "opacities", "feats", "sh"):
        arr = getattr(sc, name)
        for _ in range(4):
            idx = (int(rng.choice(vis)),) + tuple(int(rng.integers(s)) for s in arr.shape[1:])
            old = arr[idx]
            arr[idx] = old + 1e-6
            lp = loss(sc)
            arr[idx] = old - 1e-6
            lm = loss(sc)
            arr[idx] = old
            fd = (lp - lm) / 2e-6
            assert abs(fd - an[name][idx]) <= 1e-6 * abs(an[name][idx]) + 1e-7 * np.abs(an[name]).max(), \
                (name, idx, fd, an[name][idx])
