"""CPU oracle of the VQ semantic parameterisation and its per-pixel decode (X-GS Sec. 3.2
"Online VQ Module" and App. E "3D Visual Grounding Details").

TEST INFRASTRUCTURE ONLY: imported by ``tests/``; the product library never loads it.  It
shares no code with the CUDA library.  Everything is FP64.

What it computes:
  * weights        -- w_i = softmax(z_i) of each Gaussian's logit vector (Sec. 3.2)
  * weights_bwd    -- dL/dz_i from dL/dw_i through the softmax
  * render_weights -- the weight map w(x): the rasterizer's feature substitution f_i -> w_i
                      (App. E: the renderer splats the mixture weights), via the
                      rasterizer oracle
  * decode         -- F(x) = E^T w(x) per pixel (App. E)
  * relevance      -- F~ = F / (|F| + eps) and R(x | p) = max_n softmax(tau [F~.t+, F~.t_n-])_1
                      with tau = 10 (App. E)
Readings (also in the design notes): the CLIP embedding width D is a free parameter (the
workloads use 512); eps = 1e-8; text embeddings are unit vectors given by the caller.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O

TAU = 10.0
EPS = 1e-8


def weights(z):
    """Row-wise softmax of the logits z [N, L] (Sec. 3.2)."""
    z = np.asarray(z, np.float64)
    e = np.exp(z - z.max(axis=1, keepdims=True))
    return e / e.sum(axis=1, keepdims=True)


def weights_bwd(z, g_w):
    """dL/dz from dL/dw through w = softmax(z): w * (g - sum_l g_l w_l)."""
    w = weights(z)
    g = np.asarray(g_w, np.float64)
    return w * (g - (g * w).sum(axis=1, keepdims=True))


def render_weights(scene, cam, z, prec="f32", pixels=None):
    """Weight map w(x) [L, H, W] (or [L, len(pixels)]): the rasterizer oracle with the
    per-Gaussian features replaced by the softmax weights."""
    return O.render(scene, cam, prec, pixels=pixels, feats=weights(z))["feat"]


def decode(wmap, E):
    """F(x) = E^T w(x) for every pixel: wmap [L, ...], codebook E [L, D] -> F [D, ...]."""
    w = np.asarray(wmap, np.float64)
    L = w.shape[0]
    E = np.asarray(E, np.float64)
    return (E.T @ w.reshape(L, -1)).reshape((E.shape[1],) + w.shape[1:])


def relevance(F, t_pos, t_neg, tau=TAU, eps=EPS):
    """R(x | p) (App. E) for F [D, ...], the prompt embedding t_pos [D] and the generic
    negatives t_neg [N_neg, D]."""
    F = np.asarray(F, np.float64)
    D = F.shape[0]
    Fm = F.reshape(D, -1)
    Ft = Fm / (np.sqrt((Fm * Fm).sum(axis=0)) + eps)
    sp = np.asarray(t_pos, np.float64) @ Ft
    best = np.zeros_like(sp)
    for t in np.asarray(t_neg, np.float64):
        sn = t @ Ft
        # first entry of softmax(tau [s+, s-])
        m = np.maximum(sp, sn)
        ep, en = np.exp(tau * (sp - m)), np.exp(tau * (sn - m))
        best = np.maximum(best, ep / (ep + en))
    return best.reshape(F.shape[1:])
