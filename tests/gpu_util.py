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
