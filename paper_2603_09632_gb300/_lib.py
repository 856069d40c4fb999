"""Thin ctypes binding of libgs (include/gs.h): argument marshalling only.

Every function here has the name of the C entry point it calls and forwards torch
tensors as raw device pointers; all computation happens in the CUDA library.  There is
no fallback: if ``libgs.so`` cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgs.so")

GS_OK, GS_ERR_ARG, GS_ERR_OOM, GS_ERR_CUDA, GS_ERR_DEVICE = 0, 1, 2, 3, 4
GS_ERR_TIMEOUT, GS_ERR_BUSY, GS_ERR_OVER_BUDGET, GS_ERR_STATE, GS_ERR_CANCELLED = 5, 6, 7, 8, 9
GS_F32, GS_BF16 = 0, 1
GS_TIMER_NAMES = ("project", "bin", "fwd", "bwd_raster", "bwd_project")
GS_NUM_TIMERS = len(GS_TIMER_NAMES)


class GSError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


class gs_camera(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("R", C.c_float * 9), ("t", C.c_float * 3),
                ("near_z", C.c_float), ("tile", C.c_int32), ("stride", C.c_int32),
                ("off_x", C.c_int32), ("off_y", C.c_int32)]


class gs_scene(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("n_feat", C.c_int32),
                ("feat_dtype", C.c_int32), ("means", C.c_void_p), ("scales", C.c_void_p),
                ("quats", C.c_void_p), ("opacities", C.c_void_p), ("sh", C.c_void_p),
                ("feats", C.c_void_p)]


class gs_request(C.Structure):
    _fields_ = [("scene_id", C.c_int32), ("cam", gs_camera), ("want_bwd", C.c_int32),
                ("rgb", C.c_void_p), ("depth", C.c_void_p), ("alpha", C.c_void_p), ("feat", C.c_void_p),
                ("g_rgb", C.c_void_p), ("g_depth", C.c_void_p), ("g_alpha", C.c_void_p),
                ("g_feat", C.c_void_p), ("g_means", C.c_void_p), ("g_scales", C.c_void_p),
                ("g_quats", C.c_void_p), ("g_opac", C.c_void_p), ("g_sh", C.c_void_p),
                ("g_feats", C.c_void_p), ("g_pose6", C.c_void_p)]


class gs_result(C.Structure):
    _fields_ = [("status", C.c_int), ("slot", C.c_int32), ("instances", C.c_int64),
                ("queue_us", C.c_double), ("run_us", C.c_double), ("latency_us", C.c_double)]


class gs_serve_stats_t(C.Structure):
    _fields_ = [("scene_bytes", C.c_int64), ("workspace_bytes", C.c_int64), ("arena_bytes", C.c_int64),
                ("arena_peak_bytes", C.c_int64), ("max_pixels", C.c_int64), ("batches", C.c_int64),
                ("lanes", C.c_int32), ("slots_per_lane", C.c_int32), ("peak_batch", C.c_int32),
                ("peak_running", C.c_int32)]


class gs_feat_loss(C.Structure):
    _fields_ = [("target", C.c_void_p), ("mask", C.c_void_p), ("lambda_sem", C.c_float),
                ("g_feat", C.c_void_p), ("loss", C.c_void_p)]


class gs_stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("visible", C.c_int64), ("instances", C.c_int64),
                ("inst_eff", C.c_int64), ("pixels", C.c_int64), ("tiles", C.c_int64),
                ("pairs_eval", C.c_int64), ("pairs_blend", C.c_int64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libgs.so not built ({LIB_PATH}); run __graft_entry__.build() or "
                          "python -m paper_2603_09632_gb300._build")
    L = C.CDLL(LIB_PATH)
    P, i64, i32, st = C.c_void_p, C.c_int64, C.c_int, C.c_int
    sig = {
        "gs_status_string": ([st], C.c_char_p),
        "gs_workspace_create": ([C.POINTER(C.c_void_p), i32], st),
        "gs_workspace_destroy": ([P], None),
        "gs_workspace_reserve": ([P, i64, i64, i64], st),
        "gs_workspace_status": ([P, P], st),
        "gs_workspace_bytes": ([P, C.POINTER(C.c_int64)], st),
        "gs_project": ([P, P, P, P], st),
        "gs_bin_tiles": ([P, P, P], st),
        "gs_render_fwd": ([P, P, P, P, P, P, P, P], st),
        "gs_render_bwd": ([P, P, P] + [P] * 4 + [P] * 7 + [P], st),
        "gs_render_fwd_loss": ([P, P, P, P, P, P, P, P, P], st),
        "gs_l1_grad": ([P, P, i64, C.c_float, P, P], st),
        "gs_get_stats": ([P, P, P], st),
        "gs_get_instances": ([P, P, P, i64, P, P, P], st),
        "gs_get_projection": ([P, P, P, P, P, P, P], st),
        "gs_get_pixel_state": ([P, P, P, P], st),
        "gs_timing_enable": ([P, i32], st),
        "gs_timing_collect": ([P, P, P], st),
        "gs_launch_count": ([], i64),
        "gs_measure_fp32_peak": ([i32, C.POINTER(C.c_double), C.POINTER(C.c_double), P], st),
        "gs_render_fwd_noalloc": ([P, P, P, P, P, P, P], st),
        "gs_serve_create": ([C.POINTER(C.c_void_p), i32, i64, i32], st),
        "gs_serve_destroy": ([P], None),
        "gs_serve_add_scene": ([P, P, C.POINTER(C.c_int)], st),
        "gs_serve_submit": ([P, P, C.POINTER(C.c_uint64)], st),
        "gs_serve_poll": ([P, C.c_uint64, i64, P], st),
        "gs_serve_cancel": ([P, C.c_uint64], st),
        "gs_serve_info": ([P, P, P, P, P], st),
        "gs_serve_stats": ([P, P], st),
        "gs_grid_target_region": ([P, i32, i32, P, i32, i32, i32, i32, i32, P, P, P], st),
        "gs_vq_weights": ([P, i64, i32, i32, P, P], st),
        "gs_vq_weights_bwd": ([P, P, i64, i32, P, P], st),
        "gs_vq_decode": ([P, i64, i32, P, i32, P, P, i32, C.c_float, P, P, P], st),
        "gs_grid_target_resample": ([P, i32, i32, i32, i32, i32, i32, i32, i32, P, P, P], st),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


lib = _load()


def status_string(s: int) -> str:
    return lib.gs_status_string(int(s)).decode()


def _check(s, where):
    if s != GS_OK:
        raise GSError(s, where)


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------- value types

def make_camera(W, H, fx, fy, cx, cy, R, t, near=0.2, stride=1, off_x=0, off_y=0) -> gs_camera:
    c = gs_camera()
    c.W, c.H, c.fx, c.fy, c.cx, c.cy = int(W), int(H), float(fx), float(fy), float(cx), float(cy)
    R = np.asarray(R, np.float64).reshape(9)
    t = np.asarray(t, np.float64).reshape(3)
    for k in range(9):
        c.R[k] = float(R[k])
    for k in range(3):
        c.t[k] = float(t[k])
    c.near_z, c.tile, c.stride, c.off_x, c.off_y = float(near), 16, int(stride), int(off_x), int(off_y)
    return c


class Scene:
    """Device tensors of one scene plus the C struct pointing at them (post-activation)."""

    def __init__(self, means, scales, quats, opacities, sh, feats=None):
        dev = means.device
        self.means = means.contiguous().float()
        self.scales = scales.contiguous().float()
        self.quats = quats.contiguous().float()
        self.opacities = opacities.contiguous().float()
        self.sh = sh.contiguous().float()
        n = self.means.shape[0]
        K = self.sh.shape[1] if self.sh.dim() == 3 else 1
        deg = int(round(math.sqrt(K))) - 1
        if (deg + 1) ** 2 != K:
            raise ValueError("sh must be [n, (deg+1)^2, 3]")
        if feats is None:
            feats = torch.zeros((n, 0), device=dev, dtype=torch.float32)
        self.feats = feats.contiguous()
        if self.feats.dtype not in (torch.float32, torch.bfloat16):
            raise ValueError("features must be float32 or bfloat16")
        s = gs_scene()
        s.n, s.sh_degree, s.n_feat = n, deg, int(self.feats.shape[1])
        s.feat_dtype = GS_BF16 if self.feats.dtype == torch.bfloat16 else GS_F32
        s.means, s.scales, s.quats = self.means.data_ptr(), self.scales.data_ptr(), self.quats.data_ptr()
        s.opacities, s.sh = self.opacities.data_ptr(), self.sh.data_ptr()
        s.feats = self.feats.data_ptr() if s.n_feat > 0 else None
        self.c = s

    @property
    def n(self):
        return int(self.c.n)

    @property
    def n_feat(self):
        return int(self.c.n_feat)

    @property
    def sh_degree(self):
        return int(self.c.sh_degree)


class Workspace:
    """Library-owned workspace (gs_workspace_create / gs_workspace_destroy)."""

    def __init__(self, device=None):
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(torch.device("cuda", device).index if isinstance(device, int) else
                          torch.device(device).index or 0)
        h = C.c_void_p()
        _check(lib.gs_workspace_create(C.byref(h), self.device), "gs_workspace_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib.gs_workspace_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- entry points

def gs_workspace_reserve(ws, n_gauss, n_instances, n_pixels):
    _check(lib.gs_workspace_reserve(ws.h, int(n_gauss), int(n_instances), int(n_pixels)),
           "gs_workspace_reserve")


def gs_workspace_status(ws, stream=None):
    return lib.gs_workspace_status(ws.h, _stream(stream))


def gs_workspace_bytes(ws) -> int:
    """Device memory held by the workspace (its high-water mark), in bytes."""
    b = C.c_int64()
    _check(lib.gs_workspace_bytes(ws.h, C.byref(b)), "gs_workspace_bytes")
    return int(b.value)


def gs_project(scene, cam, ws, stream=None):
    _check(lib.gs_project(C.byref(scene.c), C.byref(cam), ws.h, _stream(stream)), "gs_project")


def gs_bin_tiles(ws, sync=True, stream=None):
    """Returns the instance count when ``sync`` (one stream synchronisation), else None."""
    if sync:
        n = C.c_int64()
        _check(lib.gs_bin_tiles(ws.h, C.byref(n), _stream(stream)), "gs_bin_tiles")
        return int(n.value)
    _check(lib.gs_bin_tiles(ws.h, None, _stream(stream)), "gs_bin_tiles")
    return None


def gs_render_fwd(scene, cam, ws, rgb=None, depth=None, alpha=None, feat=None, stream=None):
    _check(lib.gs_render_fwd(C.byref(scene.c), C.byref(cam), ws.h, _ptr(rgb), _ptr(depth),
                             _ptr(alpha), _ptr(feat), _stream(stream)), "gs_render_fwd")


def gs_render_fwd_loss(scene, cam, ws, target, g_feat, loss, mask=None, lambda_sem=1.0, rgb=None,
                       depth=None, alpha=None, feat=None, stream=None):
    """Forward render with the masked L1 + cosine feature loss fused in: writes dL/dG_hat
    into ``g_feat`` [D,rows,cols] and (L, L_1, L_cos) into ``loss`` (float64 device [3])."""
    fl = gs_feat_loss()
    fl.target, fl.mask, fl.lambda_sem = _ptr(target), _ptr(mask), float(lambda_sem)
    fl.g_feat, fl.loss = _ptr(g_feat), _ptr(loss)
    _check(lib.gs_render_fwd_loss(C.byref(scene.c), C.byref(cam), ws.h, _ptr(rgb), _ptr(depth),
                                  _ptr(alpha), _ptr(feat), C.byref(fl), _stream(stream)),
           "gs_render_fwd_loss")


def gs_render_bwd(scene, cam, ws, g_rgb=None, g_depth=None, g_alpha=None, g_feat=None,
                  g_means=None, g_scales=None, g_quats=None, g_opac=None, g_sh=None,
                  g_feats=None, g_pose6=None, stream=None):
    _check(lib.gs_render_bwd(C.byref(scene.c), C.byref(cam), ws.h, _ptr(g_rgb), _ptr(g_depth),
                             _ptr(g_alpha), _ptr(g_feat), _ptr(g_means), _ptr(g_scales),
                             _ptr(g_quats), _ptr(g_opac), _ptr(g_sh), _ptr(g_feats),
                             _ptr(g_pose6), _stream(stream)), "gs_render_bwd")


def gs_l1_grad(pred, target, scale, grad, stream=None):
    _check(lib.gs_l1_grad(_ptr(pred), _ptr(target), int(pred.numel()), float(scale), _ptr(grad),
                          _stream(stream)), "gs_l1_grad")


def gs_get_stats(ws, stream=None) -> dict:
    s = gs_stats()
    _check(lib.gs_get_stats(ws.h, C.byref(s), _stream(stream)), "gs_get_stats")
    return {k: int(getattr(s, k)) for k, _ in gs_stats._fields_}


def gs_get_instances(ws, n_tiles, stream=None):
    n = C.c_int64()
    _check(lib.gs_get_instances(ws.h, None, None, 0, C.byref(n), None, _stream(stream)),
           "gs_get_instances")
    m = int(n.value)
    tiles = np.zeros(m, np.uint32)
    ids = np.zeros(m, np.uint32)
    ranges = np.zeros((n_tiles, 2), np.uint32)
    P = C.c_void_p
    _check(lib.gs_get_instances(ws.h, P(tiles.ctypes.data), P(ids.ctypes.data), m, C.byref(n),
                                P(ranges.ctypes.data), _stream(stream)), "gs_get_instances")
    return tiles, ids, ranges


def gs_get_projection(ws, n, stream=None):
    out = dict(mean2d=np.zeros((n, 2), np.float32), conic=np.zeros((n, 3), np.float32),
               depth=np.zeros(n, np.float32), rgb=np.zeros((n, 3), np.float32),
               rect=np.zeros((n, 4), np.int32))
    P = C.c_void_p
    _check(lib.gs_get_projection(ws.h, *(P(out[k].ctypes.data) for k in
                                         ("mean2d", "conic", "depth", "rgb", "rect")),
                                 _stream(stream)), "gs_get_projection")
    return out


def gs_get_pixel_state(ws, H, W, stream=None):
    T = np.zeros((H, W), np.float32)
    nc = np.zeros((H, W), np.uint32)
    P = C.c_void_p
    _check(lib.gs_get_pixel_state(ws.h, P(T.ctypes.data), P(nc.ctypes.data), _stream(stream)),
           "gs_get_pixel_state")
    return T, nc


class Server:
    """Serving loop (gs_serve_*): resident scenes, continuous admission by an HBM budget."""

    def __init__(self, hbm_budget_bytes, max_slots, device=None):
        dev = torch.cuda.current_device() if device is None else int(device)
        h = C.c_void_p()
        _check(lib.gs_serve_create(C.byref(h), dev, int(hbm_budget_bytes), int(max_slots)),
               "gs_serve_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib.gs_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gs_serve_add_scene(server, scene):
    sid = C.c_int()
    _check(lib.gs_serve_add_scene(server.h, C.byref(scene.c), C.byref(sid)), "gs_serve_add_scene")
    return int(sid.value)


def make_request(scene_id, cam, outputs, grads_in=None, grads_out=None):
    """gs_request from dicts of device tensors (outputs: rgb/depth/alpha/feat; grads_in:
    rgb/depth/alpha/feat upstream; grads_out: means/scales/quats/opacities/sh/feats/pose)."""
    r = gs_request()
    r.scene_id, r.cam, r.want_bwd = int(scene_id), cam, int(grads_in is not None)
    for k in ("rgb", "depth", "alpha", "feat"):
        setattr(r, k, outputs[k].data_ptr() if outputs.get(k) is not None else None)
    if grads_in is not None:
        for k in ("rgb", "depth", "alpha", "feat"):
            v = grads_in.get(k)
            setattr(r, "g_" + k, v.data_ptr() if v is not None else None)
        names = dict(means="g_means", scales="g_scales", quats="g_quats", opacities="g_opac",
                     sh="g_sh", feats="g_feats", pose="g_pose6")
        for k, f in names.items():
            v = grads_out.get(k)
            setattr(r, f, v.data_ptr() if v is not None else None)
    return r


def gs_serve_submit(server, req):
    """Returns (status, ticket); the status is not raised so callers can see refusals."""
    t = C.c_uint64()
    s = lib.gs_serve_submit(server.h, C.byref(req), C.byref(t))
    return int(s), int(t.value)


def gs_serve_poll(server, ticket, timeout_us=-1):
    """Returns (status, result dict or None); GS_ERR_BUSY when not finished in time."""
    r = gs_result()
    s = lib.gs_serve_poll(server.h, C.c_uint64(ticket), int(timeout_us), C.byref(r))
    if s != GS_OK:
        return int(s), None
    return GS_OK, {k: getattr(r, k) for k, _ in gs_result._fields_}


def gs_serve_cancel(server, ticket):
    return int(lib.gs_serve_cancel(server.h, C.c_uint64(ticket)))


def gs_serve_info(server):
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    d = C.c_int32()
    _check(lib.gs_serve_info(server.h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)), "gs_serve_info")
    return dict(scene_bytes=a.value, in_flight_bytes=b.value, peak_in_flight_bytes=c.value,
                peak_running=d.value)


def gs_serve_stats(server):
    """How the server divided its budget (scenes, workspaces, arena) and how it batched."""
    r = gs_serve_stats_t()
    _check(lib.gs_serve_stats(server.h, C.byref(r)), "gs_serve_stats")
    return {k: getattr(r, k) for k, _ in gs_serve_stats_t._fields_}


def gs_render_fwd_noalloc(scene, cam, rgb=None, depth=None, alpha=None, feat=None, stream=None):
    """Forward render with no allocation (library-held fixed scratch; small scenes only).
    Returns the status code instead of raising, so callers can test GS_ERR_OVER_BUDGET."""
    return lib.gs_render_fwd_noalloc(C.byref(scene.c), C.byref(cam), _ptr(rgb), _ptr(depth),
                                     _ptr(alpha), _ptr(feat), _stream(stream))


def gs_grid_target_region(seg, table, stride, off_x, off_y, target, mask=None, stream=None):
    """Region-indexed grid targets: seg [H,W] int32 (device), table [R,D] float32 -> target
    [D,Hs,Ws], mask [Hs,Ws] (caller-allocated device tensors)."""
    H, W = seg.shape
    R, D = table.shape
    _check(lib.gs_grid_target_region(_ptr(seg), H, W, _ptr(table), R, D, int(stride), int(off_x),
                                     int(off_y), _ptr(target), _ptr(mask), _stream(stream)),
           "gs_grid_target_region")


def gs_grid_target_resample(fmap, H, W, stride, off_x, off_y, target, mask=None, stream=None):
    """Continuous-map grid targets: fmap [D,Hf,Wf] float32 (device) for an H x W image."""
    D, Hf, Wf = fmap.shape
    _check(lib.gs_grid_target_resample(_ptr(fmap), D, Hf, Wf, int(H), int(W), int(stride),
                                       int(off_x), int(off_y), _ptr(target), _ptr(mask),
                                       _stream(stream)), "gs_grid_target_resample")


def gs_vq_weights(logits, out, stream=None):
    """Softmax mixture weights: logits [n, L] float32 -> out [n, L] (float32 or bfloat16)."""
    n, L = logits.shape
    dt = GS_BF16 if out.dtype == torch.bfloat16 else GS_F32
    _check(lib.gs_vq_weights(_ptr(logits), n, L, dt, _ptr(out), _stream(stream)), "gs_vq_weights")


def gs_vq_weights_bwd(logits, g_w, g_logits, stream=None):
    n, L = logits.shape
    _check(lib.gs_vq_weights_bwd(_ptr(logits), _ptr(g_w), n, L, _ptr(g_logits), _stream(stream)),
           "gs_vq_weights_bwd")


def gs_vq_decode(wmap, codebook, F_out=None, text=None, tau=10.0, relevance=None, err=None,
                 stream=None):
    """F = E^T w(x) and/or prompt relevance from a weight map [L, ...] (channel-major)."""
    L = wmap.shape[0]
    P = wmap.numel() // L
    Lc, D = codebook.shape
    if Lc != L:
        raise ValueError("codebook rows must equal the weight channels")
    n_text = 0 if text is None else text.shape[0]
    _check(lib.gs_vq_decode(_ptr(wmap), P, L, _ptr(codebook), D, _ptr(F_out), _ptr(text), n_text,
                            float(tau), _ptr(relevance), _ptr(err), _stream(stream)), "gs_vq_decode")


def gs_launch_count() -> int:
    return int(lib.gs_launch_count())


def gs_measure_fp32_peak(iters=65536, stream=None):
    """(TFLOP/s, ms) of the FP32 FMA microbenchmark on the current device."""
    tf, ms = C.c_double(), C.c_double()
    _check(lib.gs_measure_fp32_peak(int(iters), C.byref(tf), C.byref(ms), _stream(stream)),
           "gs_measure_fp32_peak")
    return tf.value, ms.value


def gs_timing_enable(ws, enable=True):
    _check(lib.gs_timing_enable(ws.h, int(bool(enable))), "gs_timing_enable")


def gs_timing_collect(ws) -> dict:
    ms = (C.c_double * GS_NUM_TIMERS)()
    cnt = (C.c_int64 * GS_NUM_TIMERS)()
    _check(lib.gs_timing_collect(ws.h, ms, cnt), "gs_timing_collect")
    return {name: (float(ms[k]), int(cnt[k])) for k, name in enumerate(GS_TIMER_NAMES)}
