"""CPU oracle of grid-sampled semantic supervision (X-GS, Sec. 3.2 "Grid-Sampled Semantic
Supervision" and App. D).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and the benchmark's CPU leg; the product
library never loads it.  It shares no code with the CUDA library.

What it computes, each function following one passage of App. D:
  * sample_coords    -- the sampled locations (u, v) = (o_h + m s, o_w + n s)
  * render/backward  -- the compact prediction G_hat[:, m, n] = the rendered feature at
                        (u, v): the full-resolution oracle (``oracle.render`` /
                        ``oracle.backward``) evaluated at exactly those pixels
  * target_region    -- region-indexed targets and mask (segmentation S, table Phi)
  * target_resample  -- continuous-map targets by rounded coordinate alignment
  * loss             -- lambda_sem [L_cos(V.G_hat, V.G*) + L_1(V.G_hat, V.G*)] and its
                        gradient with respect to G_hat
Readings of what App. D leaves open (all listed in the design notes):
  * the compact shape is H_s = ceil(H / s), W_s = ceil(W / s) for every offset; samples
    that fall outside the image (large offsets) render nothing (alpha 0, T = 1) and have
    mask 0;
  * ``round`` in the continuous alignment is round-half-away-from-zero, evaluated exactly
    on the rational u (H_f - 1) / max(H - 1, 1);
  * region ids outside [0, R) other than -1 are treated like background (mask 0);
  * L_1 is the mean absolute difference over all D H_s W_s entries and L_cos the mean over
    the H_s W_s pixels of 1 - cos, with cos(a, b) = a.b / (max(|a|, eps) max(|b|, eps)),
    eps = 1e-8 (masked-out pixels therefore add a constant 1 and no gradient).
"""
from __future__ import annotations

import numpy as np

from . import oracle as O

COS_EPS = 1e-8


def grid_shape(H, W, stride):
    """Compact resolution (H_s, W_s) of a stride-s grid over an H x W image."""
    return -(-H // stride), -(-W // stride)


def sample_coords(H, W, stride, off_x, off_y):
    """Row coordinates u[m] = o_h + m s, column coordinates v[n] = o_w + n s, and the
    in-image mask [H_s, W_s] (App. D, sampled locations)."""
    if stride < 1 or not (0 <= off_x < stride) or not (0 <= off_y < stride):
        raise ValueError("need stride >= 1 and 0 <= offset < stride")
    Hs, Ws = grid_shape(H, W, stride)
    u = off_y + stride * np.arange(Hs, dtype=np.int64)
    v = off_x + stride * np.arange(Ws, dtype=np.int64)
    inb = (u[:, None] < H) & (v[None, :] < W)
    return u, v, inb


def _pixels(cam, stride, off_x, off_y):
    u, v, inb = sample_coords(cam.H, cam.W, stride, off_x, off_y)
    flat = u[:, None] * cam.W + v[None, :]
    return flat[inb], inb


def render(scene, cam, stride, off_x, off_y, prec="f32", feats=None, thresholds=True):
    """Compact rgb [3,H_s,W_s], depth, alpha, feat [D,H_s,W_s], T_final, n_contrib, flags:
    the full-resolution render at the sampled pixels, zero (T = 1) outside the image."""
    pix, inb = _pixels(cam, stride, off_x, off_y)
    Hs, Ws = inb.shape
    r = O.render(scene, cam, prec, thresholds=thresholds, pixels=pix, feats=feats)
    dt = r["rgb"].dtype
    D = r["feat"].shape[0]
    out = dict(rgb=np.zeros((3, Hs, Ws), dt), depth=np.zeros((Hs, Ws), dt),
               alpha=np.zeros((Hs, Ws), dt), feat=np.zeros((D, Hs, Ws), dt),
               T_final=np.ones((Hs, Ws), dt), n_contrib=np.zeros((Hs, Ws), np.int32),
               flags=np.zeros((Hs, Ws), np.int32))
    out["rgb"][:, inb] = r["rgb"]
    out["feat"][:, inb] = r["feat"]
    for k in ("depth", "alpha", "T_final", "n_contrib", "flags"):
        out[k][inb] = r[k]
    return out


def backward(scene, cam, stride, off_x, off_y, grads, prec="f32", feats=None, thresholds=True):
    """Gradients of sum(g . compact outputs); ``grads`` holds compact maps (rgb [3,H_s,W_s],
    depth, alpha [H_s,W_s], feat [D,H_s,W_s]).  Entries outside the image carry no
    gradient (nothing is rendered there)."""
    pix, inb = _pixels(cam, stride, off_x, off_y)
    sub = {}
    for k, g in grads.items():
        if g is None:
            continue
        g = np.asarray(g)
        sub[k] = g[:, inb] if g.ndim == 3 else g[inb]
    return O.backward(scene, cam, sub, prec, thresholds=thresholds, pixels=pix, feats=feats)


def target_region(seg, table, stride, off_x, off_y):
    """Region-indexed targets (App. D): V = [S(u,v) != -1], G* = Phi[S(u,v)] where valid,
    0 elsewhere.  ``seg`` [H,W] int, ``table`` [R,D].  Returns G* [D,H_s,W_s], V [H_s,W_s]."""
    H, W = seg.shape
    R, D = table.shape
    u, v, inb = sample_coords(H, W, stride, off_x, off_y)
    Hs, Ws = inb.shape
    G = np.zeros((D, Hs, Ws), np.float64)
    V = np.zeros((Hs, Ws), np.float64)
    for m in range(Hs):
        for n in range(Ws):
            if not inb[m, n]:
                continue
            sid = int(seg[u[m], v[n]])
            if 0 <= sid < R:
                V[m, n] = 1.0
                G[:, m, n] = table[sid]
    return G, V


def round_half_away(num, den):
    """round(num / den) for integers num >= 0, den > 0, halves away from zero."""
    return (2 * num + den) // (2 * den)


def target_resample(P, H, W, stride, off_x, off_y):
    """Continuous-map targets (App. D): u~ = round(u (H_f - 1) / max(H - 1, 1)),
    v~ = round(v (W_f - 1) / max(W - 1, 1)), G* = P[:, u~, v~], V = 1 inside the image
    (0 at samples outside it).  ``P`` [D,H_f,W_f].  Returns G*, V."""
    D, Hf, Wf = P.shape
    u, v, inb = sample_coords(H, W, stride, off_x, off_y)
    Hs, Ws = inb.shape
    G = np.zeros((D, Hs, Ws), np.float64)
    V = np.zeros((Hs, Ws), np.float64)
    for m in range(Hs):
        uu = round_half_away(int(u[m]) * (Hf - 1), max(H - 1, 1))
        for n in range(Ws):
            if not inb[m, n]:
                continue
            vv = round_half_away(int(v[n]) * (Wf - 1), max(W - 1, 1))
            V[m, n] = 1.0
            G[:, m, n] = P[:, uu, vv]
    return G, V


def loss(G_hat, G_star, V, lam=1.0):
    """Masked L1 + cosine loss (App. D) in FP64.  Returns (L, L_1, L_cos, dL/dG_hat)."""
    Gh = np.asarray(G_hat, np.float64)
    Gs = np.asarray(G_star, np.float64)
    Vm = np.asarray(V, np.float64)
    D, Hs, Ws = Gh.shape
    a = Vm[None] * Gh
    b = Vm[None] * Gs
    # L_1: mean over all entries
    diff = a - b
    l1 = np.abs(diff).sum() / (D * Hs * Ws)
    # L_cos: mean over pixels of 1 - cos, norms clamped at eps separately
    la = np.sqrt((a * a).sum(0))
    lb = np.sqrt((b * b).sum(0))
    na = np.maximum(la, COS_EPS)
    nb = np.maximum(lb, COS_EPS)
    dot = (a * b).sum(0)
    cos = dot / (na * nb)
    lcos = (1.0 - cos).sum() / (Hs * Ws)
    L = lam * (lcos + l1)
    # gradient with respect to a, then through a = V G_hat
    g_l1 = np.sign(diff) / (D * Hs * Ws)
    dcos = b / (na * nb)[None]
    big = la > COS_EPS
    dcos = dcos - np.where(big, cos / np.where(big, la * la, 1.0), 0.0)[None] * a
    g_cos = -dcos / (Hs * Ws)
    grad = lam * Vm[None] * (g_l1 + g_cos)
    return L, l1, lcos, grad
