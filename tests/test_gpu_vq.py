"""NEXT-4 on the GPU against the VQ oracle (``oracle/vq.py``; Sec. 3.2, App. E): softmax
weights and their backward, the tensor-core decode F = E^T w(x) of a rendered weight map,
structured one-hot maps that expose any operand-layout error, and the prompt relevance map.

The decode's products are 3xTF32 (each operand split into two tf32 parts: the split leaves
at most 2^-22 of each operand, the dropped lo x lo term at most 2^-22 of the product) and
its sums FP32 over L <= 64 terms (at most 64 x 2^-24 of sum_l |w_l E_l|), so every entry
must lie within BOUND_REL = 2e-5 of sum_l |w_l E_l| of the FP64 decode: about four times
the sum of those terms, for the tensor core's own accumulation order and rounding."""
import numpy as np
import pytest

from synth import scenes as S
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

BOUND_REL = 2e-5


def assert_decode_within_bound(VQ, got, w, E):
    """|F - E^T w| <= BOUND_REL sum_l |w_l E_l| entry by entry (FP64 reference)."""
    ref = VQ.decode(w, E)
    bound = VQ.decode(np.abs(np.asarray(w, np.float64)), np.abs(np.asarray(E, np.float64)))
    err = np.abs(np.asarray(got, np.float64) - ref)
    worst = float((err / np.maximum(bound, 1e-30)).max())
    assert (err <= BOUND_REL * bound + 1e-30).all(), f"worst |err| / sum|w E| = {worst:.3e}"
    return worst


@pytest.fixture(scope="module")
def VQ(oracle):
    from oracle import vq
    return vq


def _t(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(U.device())
    return t if dtype is None else t.to(dtype)


def test_weights_and_backward(VQ):
    import torch
    from paper_2603_09632_gb300 import _lib as L
    rng = np.random.default_rng(1)
    for n, Lw in [(1000, 64), (333, 16), (17, 40), (5, 1)]:
        z = rng.normal(scale=2.0, size=(n, Lw)).astype(np.float32)
        w32 = torch.empty((n, Lw), device=U.device())
        wbf = torch.empty((n, Lw), device=U.device(), dtype=torch.bfloat16)
        L.gs_vq_weights(_t(z), w32)
        L.gs_vq_weights(_t(z), wbf)
        ref = VQ.weights(z)
        np.testing.assert_allclose(w32.cpu().numpy(), ref, rtol=2e-5, atol=1e-7)
        np.testing.assert_allclose(wbf.float().cpu().numpy(), ref, rtol=8e-3, atol=1e-6)
        g = rng.normal(size=(n, Lw)).astype(np.float32)
        gz = torch.empty((n, Lw), device=U.device())
        L.gs_vq_weights_bwd(_t(z), _t(g), gz)
        ref_gz = VQ.weights_bwd(z, g)
        assert U.rel_err(gz.cpu().numpy(), ref_gz) <= 1e-5
        # element by element: gz_l = w_l (g_l - d), d = sum_k w_k g_k.  With each weight within
        # 2e-5 w + 1e-7 of the FP64 value (checked above) and d summed in FP32 over L terms,
        # |error of gz_l| <= 2e-5 |gz_l| + 1e-7 |g_l - d| + w_l (4e-5 sum_k |w_k g_k| + 1e-7 sum_k |g_k|)
        wr = VQ.weights(z)
        gd = np.asarray(g, np.float64)
        d = (wr * gd).sum(axis=1, keepdims=True)
        bound = (2e-5 * np.abs(ref_gz) + 1e-7 * np.abs(gd - d)
                 + wr * (4e-5 * np.abs(wr * gd).sum(axis=1, keepdims=True)
                         + 1e-7 * np.abs(gd).sum(axis=1, keepdims=True)) + 1e-9)
        over = np.abs(gz.cpu().numpy() - ref_gz) > bound
        assert not over.any(), (n, Lw, int(over.sum()))


@pytest.mark.parametrize("Lw,D,P", [(64, 512, 27_200), (16, 48, 1000), (8, 16, 129), (32, 272, 128)])
def test_decode_one_hot_maps(VQ, Lw, D, P):
    """Pixel p carries weight 1 on codeword p mod L (and 0.5 on codeword (p // L) mod L):
    every pixel must reproduce its codewords, so a transposed or shifted operand shows."""
    import torch
    from paper_2603_09632_gb300 import _lib as L
    rng = np.random.default_rng(2)
    E = rng.normal(size=(Lw, D)).astype(np.float32)
    w = np.zeros((Lw, P), np.float32)
    p = np.arange(P)
    w[p % Lw, p] = 1.0
    w[(p // Lw) % Lw, p] += 0.5
    F = torch.empty((D, P), device=U.device())
    err = torch.zeros(1, dtype=torch.int32, device=U.device())
    L.gs_vq_decode(_t(w), _t(E), F_out=F, err=err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    assert_decode_within_bound(VQ, F.cpu().numpy(), w, E)


def test_decode_of_rendered_weights_and_relevance(oracle, VQ):
    """Render the softmax weights of a room scene as 64 bf16 channels, decode on the tensor
    cores with the relevance epilogue, and compare with the oracle's decode and relevance of
    the same weight map."""
    import torch
    from paper_2603_09632_gb300 import _lib as L
    from paper_2603_09632_gb300.render import Rasterizer
    rng = np.random.default_rng(3)
    Lw, D = 64, 512
    sc = S.room_scene(30_000, n_feat=Lw, sh_degree=0, seed=9)
    cam = S.room_trajectory(8, 203, 139, 180.0)[2]
    z = rng.normal(scale=2.0, size=(sc.n, Lw)).astype(np.float32)
    wbf = torch.empty((sc.n, Lw), device=U.device(), dtype=torch.bfloat16)
    L.gs_vq_weights(_t(z), wbf)
    scene = U.upload(sc, bf16=True)
    scene = L.Scene(scene.means, scene.scales, scene.quats, scene.opacities, scene.sh, wbf)
    out = Rasterizer(U.device()).forward(scene, cam)
    wmap = out["feat"]                                   # [64, H, W]
    # the weight map sums to alpha (softmax weights sum to 1 per Gaussian, up to bf16)
    assert torch.allclose(wmap.sum(0), out["alpha"], atol=2e-2)
    E = rng.normal(size=(Lw, D)).astype(np.float32) / 8.0
    text = rng.normal(size=(5, D))
    text = (text / np.linalg.norm(text, axis=1, keepdims=True)).astype(np.float32)
    F = torch.empty((D, cam.H, cam.W), device=U.device())
    R = torch.empty((cam.H, cam.W), device=U.device())
    err = torch.zeros(1, dtype=torch.int32, device=U.device())
    L.gs_vq_decode(wmap, _t(E), F_out=F, text=_t(text), tau=10.0, relevance=R, err=err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    wm = wmap.double().cpu().numpy()
    Fr = VQ.decode(wm, E)
    assert_decode_within_bound(VQ, F.cpu().numpy(), wm, E)
    Rr = VQ.relevance(Fr, text[0], text[1:])
    got = R.cpu().numpy()
    assert np.abs(got - Rr).max() <= 1e-3
    assert 0.0 <= got.min() and got.max() <= 1.0 and got.std() > 1e-3
    # relevance alone (no F written) is the same map
    R2 = torch.empty_like(R)
    L.gs_vq_decode(wmap, _t(E), text=_t(text), tau=10.0, relevance=R2)
    torch.cuda.synchronize()
    assert torch.equal(R, R2)


@pytest.mark.parametrize("Lw,D,P", [(64, 512, 5_000), (64, 272, 3_333), (16, 128, 2_049), (40, 256, 257)])
def test_decode_random_maps_and_relevance(VQ, Lw, D, P):
    """Softmax-like weight maps (non-negative, summing to at most 1) of ragged pixel counts:
    every entry of F within the 3xTF32 bound, and the relevance against the oracle's
    relevance of the oracle's F, for one CTA per tile (D <= 256) and for two CTAs that
    split the columns and exchange their half norms (D > 256, uneven halves at 272)."""
    import torch
    from paper_2603_09632_gb300 import _lib as L
    rng = np.random.default_rng(5 + D)
    z = rng.normal(scale=2.0, size=(P, Lw))
    w = np.exp(z - z.max(1, keepdims=True))
    w = (w / w.sum(1, keepdims=True) * rng.uniform(0.2, 1.0, size=(P, 1))).T.astype(np.float32)
    E = (rng.normal(size=(Lw, D)) / 8.0).astype(np.float32)
    text = rng.normal(size=(6, D))
    text = (text / np.linalg.norm(text, axis=1, keepdims=True)).astype(np.float32)
    F = torch.empty((D, P), device=U.device())
    R = torch.empty((P,), device=U.device())
    err = torch.zeros(1, dtype=torch.int32, device=U.device())
    L.gs_vq_decode(_t(w), _t(E), F_out=F, text=_t(text), tau=10.0, relevance=R, err=err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    worst = assert_decode_within_bound(VQ, F.cpu().numpy(), w, E)
    Rr = VQ.relevance(VQ.decode(w, E), text[0], text[1:])
    rel_err = float(np.abs(R.cpu().numpy() - Rr).max())
    print(f"L={Lw} D={D} P={P}: worst |err| / sum|w E| = {worst:.3e}, relevance max abs err = {rel_err:.3e}")
    assert rel_err <= 1e-4


def test_decode_full_size_sampled(VQ):
    """The bench's decode launch at full size: 1200x680 pixels, L = 64 -> D = 512 with the
    relevance epilogue (6375 tiles over clusters of two CTAs), softmax-like weight maps
    drawn on the device; 4096 sampled pixels against the FP64 oracle, F entry by entry
    within the 3xTF32 bound and the relevance within 1e-4."""
    import torch
    from paper_2603_09632_gb300 import _lib as L
    dev = U.device()
    H, W, Lw, D = 680, 1200, 64, 512
    P = H * W
    g = torch.Generator(device=dev).manual_seed(21)
    z = torch.randn((P, Lw), generator=g, device=dev) * 2.0
    alpha = torch.rand((P, 1), generator=g, device=dev) * 0.8 + 0.2
    w = (torch.softmax(z, dim=1) * alpha).t().contiguous()            # [L, P]
    del z
    rng = np.random.default_rng(22)
    E = (rng.normal(size=(Lw, D)) / 8.0).astype(np.float32)
    text = rng.normal(size=(5, D))
    text = (text / np.linalg.norm(text, axis=1, keepdims=True)).astype(np.float32)
    F = torch.empty((D, P), device=dev)
    R = torch.empty((P,), device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    L.gs_vq_decode(w, _t(E), F_out=F, text=_t(text), tau=10.0, relevance=R, err=err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    idx = np.sort(rng.choice(P, size=4096, replace=False))
    ti = torch.from_numpy(idx).to(dev)
    ws = w[:, ti].double().cpu().numpy()
    worst = assert_decode_within_bound(VQ, F[:, ti].cpu().numpy(), ws, E)
    Rr = VQ.relevance(VQ.decode(ws, E), text[0], text[1:])
    rel_err = float(np.abs(R[ti].cpu().numpy() - Rr).max())
    print(f"full-size decode: worst |err| / sum|w E| = {worst:.3e}, relevance max abs err = {rel_err:.3e}")
    assert rel_err <= 1e-4


def test_decode_argument_errors():
    import torch
    from paper_2603_09632_gb300 import _lib as L
    dev = U.device()
    w = torch.zeros((12, 10), device=dev)
    with pytest.raises(L.GSError):
        L.gs_vq_decode(w, torch.zeros((12, 16), device=dev), F_out=torch.empty((16, 10), device=dev))
    w = torch.zeros((16, 10), device=dev)
    with pytest.raises(L.GSError):
        L.gs_vq_decode(w, torch.zeros((16, 520), device=dev), F_out=torch.empty((520, 10), device=dev))
    with pytest.raises(L.GSError):   # relevance needs a prompt and at least one negative
        L.gs_vq_decode(w, torch.zeros((16, 16), device=dev), text=torch.zeros((1, 16), device=dev),
                       relevance=torch.empty(10, device=dev))
