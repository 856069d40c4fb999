"""Helpers for the GPU parity tests: upload a numpy scene, run the C-ABI path, compare."""
from __future__ import annotations

import numpy as np
import torch

from synth import scenes as S


def device():
    return torch.device("cuda:0")


def upload(sc: S.Scene, bf16=False, feats=None):
    from paper_2603_09632_gb300 import _lib as L
    dev = device()
    f = sc.feats if feats is None else feats
    ft = torch.from_numpy(np.ascontiguousarray(f, np.float32)).to(dev)
    if bf16:
        ft = ft.to(torch.bfloat16)
    t = [torch.from_numpy(np.ascontiguousarray(getattr(sc, k), np.float32)).to(dev)
         for k in ("means", "scales", "quats", "opacities", "sh")]
    return L.Scene(*t, ft)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest even) and back, exactly as torch does."""
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(torch.bfloat16).float().numpy()


def run(sc, cam, grads=None, bf16=False, rast=None, sync=True):
    from paper_2603_09632_gb300.render import Rasterizer
    scene = upload(sc, bf16)
    rast = rast or Rasterizer(device())
    out = rast.forward(scene, cam, sync=sync)
    res = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in out.items()}
    if grads is not None:
        gt = {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).to(device())
              for k, v in grads.items()}
        g = rast.backward(scene, cam, gt.get("rgb"), gt.get("depth"), gt.get("alpha"), gt.get("feat"))
        res["grads"] = {k: (v.cpu().numpy() if v is not None else None) for k, v in g.items()}
    torch.cuda.synchronize()
    res["rast"] = rast
    res["scene"] = scene
    return res


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def max_abs_unflagged(gpu, ref, flags):
    ok = flags == 0
    d = np.abs(np.asarray(gpu, np.float64) - np.asarray(ref, np.float64))
    d = d[..., ok] if d.ndim == flags.ndim + 1 else d[ok]
    return float(d.max()) if d.size else 0.0


# ---------------------------------------------------------------- element-wise gradient gates
#
# A pixel the oracle flags (one of its blend decisions -- sigma < 0, alpha against 1/255 or
# 0.99, T(1 - alpha) against 1e-4 -- lies within rounding distance of its threshold) may take
# the other branch on the GPU.  Its contribution to every gradient is linear in its upstream
# gradient, so zeroing the upstream gradient at the flagged pixels, on both sides, removes it
# exactly from every Gaussian's gradient and from the pose's.  Nothing else is excluded: every
# entry of every gradient tensor is then compared one by one.

GRAD_RTOL = 1e-3      # per entry, relative to the reference entry
GRAD_FLOOR = 1e-5     # per entry, absolute floor as a fraction of the tensor's largest entry


def mask_flagged(grads, flags):
    """Upstream gradients (name -> [C, H, W] or [H, W] image) with the pixels the oracle
    flags ([H, W]) zeroed.  Returns (masked copies, number of flagged pixels)."""
    bad = np.asarray(flags) != 0
    out = {}
    for k, v in grads.items():
        a = np.array(v, copy=True)
        a[..., bad] = 0
        out[k] = a
    return out, int(bad.sum())


def grad_violations(got, ref, rtol=GRAD_RTOL, floor=GRAD_FLOOR, ref_alt=None):
    """Entries with |got - ref| > rtol |ref| + floor max|ref| (+ |ref - ref_alt|): (count,
    worst ratio of the error to its bound, number of entries compared)."""
    g = np.asarray(got, np.float64).reshape(-1)
    r = np.asarray(ref, np.float64).reshape(-1)
    if r.size == 0:
        return 0, 0.0, 0
    bound = rtol * np.abs(r) + floor * max(np.abs(r).max(), 1e-30)
    if ref_alt is not None:
        bound = bound + np.abs(r - np.asarray(ref_alt, np.float64).reshape(-1))
    err = np.abs(g - r)
    ratio = err / bound
    return int((err > bound).sum()), float(ratio.max()), int(r.size)


def assert_grads_close(got, ref, keys, rtol=GRAD_RTOL, floor=GRAD_FLOOR, norm_tol=1e-3, label="",
                       ref_alt=None):
    """Every entry of every gradient within its bound, and the relative Frobenius error of
    each tensor within ``norm_tol``.  ``ref_alt``: a second evaluation of the same gradients
    (the oracle's mixed mode next to its float mode); each entry's bound then grows by the
    two evaluations' disagreement, which is ~0 where the gradient is well conditioned and
    the float oracle's own error where it is not.  Returns {key: (violations, worst ratio,
    entries)}."""
    stats, bad = {}, []
    for k in keys:
        g, r = got[k], ref[k]
        if g is None and r is None:
            continue
        alt = None if ref_alt is None else ref_alt[k]
        n, worst, m = grad_violations(g, r, rtol, floor, alt)
        rel = rel_err(g, r)
        stats[k] = (n, worst, m)
        if alt is not None:   # how much the conditioning term contributed, for the report
            stats[k] = (n, worst, m, grad_violations(g, r, rtol, floor)[1])
        if n or rel > norm_tol:
            bad.append((k, f"{n}/{m} entries over the bound (worst {worst:.3g}x)", f"rel {rel:.3g}"))
    _report(label, stats)
    assert not bad, (label, bad)
    return stats


def _report(label, stats):
    """Append the per-tensor comparison to $GS_PARITY_REPORT (JSON lines) when set."""
    import json
    import os
    path = os.environ.get("GS_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"case": label, "grads": {
                k: dict({"violations": v[0], "worst": v[1], "entries": v[2]},
                        **({"worst_without_conditioning": v[3]} if len(v) > 3 else {}))
                for k, v in stats.items()}}) + "\n")
