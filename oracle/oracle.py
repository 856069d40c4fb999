"""ctypes front-end of the CPU oracle (``gs_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``.  The product library never loads it.

Every function takes numpy arrays from :mod:`synth.scenes` (a ``Scene`` and a
``Camera``) and returns numpy arrays.  ``prec`` is ``"f32"`` (mirrors the GPU's
precision and key-affecting operation order), ``"f64"``, or, for ``render`` and
``backward``, ``"mixed"``: double arithmetic with each Gaussian's visibility, tile
rectangle and list order taken from the float projection (which the readings define in
float), i.e. the same function as the float path evaluated exactly.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

TILE = 16
FLAG_SIGMA, FLAG_LOW, FLAG_CAP, FLAG_STOP = 1, 2, 4, 8


def build(force: bool = False) -> str:
    """Compile the oracle with IEEE float semantics (no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-fopenmp", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            P = C.c_void_p
            i64, i32 = C.c_int64, C.c_int
            for suf in ("f32", "f64"):
                getattr(L, f"or_project_{suf}").argtypes = [i64, P, P, P, P, P, i32, P, i32,
                                                            P, P, P, P, P, P, P]
                getattr(L, f"or_render_{suf}").argtypes = [i64, P, P, P, P, P, i32, P, i32, P,
                                                           i32, i32, P, i64, P, P, P, P, P, P, P]
                getattr(L, f"or_backward_{suf}").argtypes = [i64, P, P, P, P, P, i32, P, i32, P,
                                                             i32, i32, P, i64, P, P, P, P, P, P,
                                                             P, P, P, P, P, P]
            L.or_render_mixed.argtypes = [i64, P, P, P, P, P, i32, P, i32, P, i32, P, i64, P,
                                          P, P, P, P, P, P]
            L.or_backward_mixed.argtypes = [i64, P, P, P, P, P, i32, P, i32, P, i32, P, i64, P,
                                            P, P, P, P, P, P, P, P, P, P, P]
            L.or_tile_lists_f32.argtypes = [i64, P, P, P, P, P, i32, P, i64, P, P, P]
            L.or_tile_lists_f32.restype = i64
            L.or_num_threads.argtypes = [i32]
            L.or_sh_basis_f64.argtypes = [i32, i64, P, P]
            _lib = L
    return _lib


def set_threads(n: int = 0) -> int:
    """Set (n > 0) and return the OpenMP thread count of the oracle."""
    return int(lib().or_num_threads(int(n)))


def cam_array(cam) -> np.ndarray:
    return np.array([cam.W, cam.H, cam.fx, cam.fy, cam.cx, cam.cy, *np.asarray(cam.R).ravel(),
                     *np.asarray(cam.t).ravel(), cam.near], np.float64)


def _dt(prec):
    return np.float32 if prec == "f32" else np.float64   # "f64" and "mixed" are double


def _scene_arrays(scene, prec, feats=None):
    dt = _dt(prec)
    f = scene.feats if feats is None else feats
    arrs = [np.ascontiguousarray(a, dt) for a in
            (scene.means, scene.scales, scene.quats, scene.opacities, scene.sh, f)]
    return arrs


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def tiles(cam):
    return (cam.W + TILE - 1) // TILE, (cam.H + TILE - 1) // TILE


def project(scene, cam, prec="f32", thresholds=True):
    dt = _dt(prec)
    n = scene.n
    means, scales, quats, opac, sh, _ = _scene_arrays(scene, prec)
    out = dict(mean2d=np.zeros((n, 2), dt), conic=np.zeros((n, 3), dt), depth=np.zeros(n, dt),
               rgb=np.zeros((n, 3), dt), rect=np.zeros((n, 4), np.int32),
               radius=np.zeros(n, np.int32), valid=np.zeros(n, np.uint8))
    camv = cam_array(cam)
    getattr(lib(), f"or_project_{prec}")(
        n, _p(means), _p(scales), _p(quats), _p(opac), _p(sh), scene.sh_degree, _p(camv),
        int(thresholds), _p(out["mean2d"]), _p(out["conic"]), _p(out["depth"]), _p(out["rgb"]),
        _p(out["rect"]), _p(out["radius"]), _p(out["valid"]))
    out["valid"] = out["valid"].astype(bool)
    return out


def tile_lists(scene, cam):
    """Stable (tile, depth, id) lists of the float projection: keys u64, ids u32, ranges [T,2]."""
    means, scales, quats, opac, sh, _ = _scene_arrays(scene, "f32")
    camv = cam_array(cam)
    TX, TY = tiles(cam)
    ranges = np.zeros((TX * TY, 2), np.uint32)
    L = lib()
    args = (scene.n, _p(means), _p(scales), _p(quats), _p(opac), _p(sh), scene.sh_degree, _p(camv))
    m = L.or_tile_lists_f32(*args, 0, None, None, _p(ranges))
    keys = np.zeros(m, np.uint64)
    ids = np.zeros(m, np.uint32)
    L.or_tile_lists_f32(*args, m, _p(keys), _p(ids), _p(ranges))
    return keys, ids, ranges


def render(scene, cam, prec="f32", thresholds=True, mode=1, pixels=None, feats=None):
    """Forward render.  ``mode`` 0 = brute force over all Gaussians per pixel, 1 = through
    the sorted tile lists.  Full image outputs are CHW; with ``pixels`` (flat indices
    y*W+x) outputs are [C, len(pixels)]."""
    dt = _dt(prec)
    means, scales, quats, opac, sh, feat = _scene_arrays(scene, prec, feats)
    D = feat.shape[1]
    if pixels is None:
        npix, shp = cam.W * cam.H, (cam.H, cam.W)
        pix = None
    else:
        pix = np.ascontiguousarray(pixels, np.int64)
        npix, shp = pix.size, (pix.size,)
    out = dict(rgb=np.zeros((3, npix), dt), depth=np.zeros(npix, dt), alpha=np.zeros(npix, dt),
               feat=np.zeros((D, npix), dt), T_final=np.zeros(npix, dt),
               n_contrib=np.zeros(npix, np.int32), flags=np.zeros(npix, np.int32))
    camv = cam_array(cam)
    if prec == "mixed":
        assert thresholds, "the mixed mode takes the float decisions of the thresholded path"
        lib().or_render_mixed(
            scene.n, _p(means), _p(scales), _p(quats), _p(opac), _p(sh), scene.sh_degree, _p(feat),
            D, _p(camv), int(mode), _p(pix), npix, _p(out["rgb"]), _p(out["depth"]),
            _p(out["alpha"]), _p(out["feat"]), _p(out["T_final"]), _p(out["n_contrib"]),
            _p(out["flags"]))
    else:
        getattr(lib(), f"or_render_{prec}")(
            scene.n, _p(means), _p(scales), _p(quats), _p(opac), _p(sh), scene.sh_degree, _p(feat),
            D, _p(camv), int(thresholds), int(mode), _p(pix), npix, _p(out["rgb"]), _p(out["depth"]),
            _p(out["alpha"]), _p(out["feat"]), _p(out["T_final"]), _p(out["n_contrib"]),
            _p(out["flags"]))
    out["rgb"] = out["rgb"].reshape((3,) + shp)
    out["feat"] = out["feat"].reshape((D,) + shp)
    for k in ("depth", "alpha", "T_final", "n_contrib", "flags"):
        out[k] = out[k].reshape(shp)
    return out


def backward(scene, cam, grads, prec="f32", thresholds=True, mode=1, pixels=None, feats=None):
    """Analytic gradients of L = sum(g_rgb*rgb) + sum(g_depth*depth) + sum(g_alpha*alpha)
    + sum(g_feat*feat) over the image (or over ``pixels``; grads then [C, len(pixels)]).
    Returns means, scales, quats, opacities, sh, feats, pose (rho, phi) and g2d
    [N,10] = (u, v, A, B, C, o, r, g, b, z)."""
    dt = _dt(prec)
    means, scales, quats, opac, sh, feat = _scene_arrays(scene, prec, feats)
    n, D, K = scene.n, feat.shape[1], (scene.sh_degree + 1) ** 2
    if pixels is None:
        pix, npix = None, cam.W * cam.H
    else:
        pix = np.ascontiguousarray(pixels, np.int64)
        npix = pix.size

    def g(name, shape):
        v = grads.get(name)
        return None if v is None else np.ascontiguousarray(np.asarray(v, dt).reshape(shape))

    gr, gd, ga, gf = g("rgb", (3, npix)), g("depth", (npix,)), g("alpha", (npix,)), g("feat", (D, npix))
    out = dict(means=np.zeros((n, 3), dt), scales=np.zeros((n, 3), dt), quats=np.zeros((n, 4), dt),
               opacities=np.zeros(n, dt), sh=np.zeros((n, K, 3), dt), feats=np.zeros((n, D), dt),
               pose=np.zeros(6, dt), g2d=np.zeros((n, 10), dt))
    camv = cam_array(cam)
    outs = (_p(out["means"]), _p(out["scales"]), _p(out["quats"]), _p(out["opacities"]),
            _p(out["sh"]), _p(out["feats"]), _p(out["pose"]), _p(out["g2d"]))
    if prec == "mixed":
        assert thresholds, "the mixed mode takes the float decisions of the thresholded path"
        lib().or_backward_mixed(
            n, _p(means), _p(scales), _p(quats), _p(opac), _p(sh), scene.sh_degree, _p(feat), D,
            _p(camv), int(mode), _p(pix), npix, _p(gr), _p(gd), _p(ga), _p(gf), *outs)
    else:
        getattr(lib(), f"or_backward_{prec}")(
            n, _p(means), _p(scales), _p(quats), _p(opac), _p(sh), scene.sh_degree, _p(feat), D,
            _p(camv), int(thresholds), int(mode), _p(pix), npix, _p(gr), _p(gd), _p(ga), _p(gf),
            *outs)
    return out


def sh_basis(deg, dirs):
    dirs = np.ascontiguousarray(dirs, np.float64)
    Y = np.zeros((dirs.shape[0], 16))
    lib().or_sh_basis_f64(int(deg), dirs.shape[0], _p(dirs), _p(Y))
    return Y[:, :(deg + 1) ** 2]
