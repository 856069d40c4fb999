"""Serving loop on the GPU: several resident scenes, a mix of forward and forward+backward
requests at mixed resolutions submitted together; requests run concurrently on the slots
and each result equals the same request rendered alone (forward bit for bit, gradients
within the backward tolerance, since atomic additions may land in another order)."""
import numpy as np
import pytest

from synth import scenes as S
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

RES = [(256, 256), (320, 240), (640, 480)]


def _outputs(torch, dev, cam, D):
    return dict(rgb=torch.empty((3, cam.H, cam.W), device=dev), depth=torch.empty((cam.H, cam.W), device=dev),
                alpha=torch.empty((cam.H, cam.W), device=dev),
                feat=torch.empty((D, cam.H, cam.W), device=dev) if D else None)


def _grad_outputs(torch, dev, n, K, D):
    return dict(means=torch.empty((n, 3), device=dev), scales=torch.empty((n, 3), device=dev),
                quats=torch.empty((n, 4), device=dev), opacities=torch.empty(n, device=dev),
                sh=torch.empty((n, K, 3), device=dev), feats=torch.empty((n, D), device=dev) if D else None,
                pose=torch.empty(6, device=dev))


def test_mix_equals_alone():
    import torch
    from paper_2603_09632_gb300 import _lib as L
    from paper_2603_09632_gb300.render import Rasterizer, as_camera
    dev = U.device()
    specs = [(30_000, 0, 16, False), (60_000, 1, 32, True), (90_000, 3, 8, False)]
    scenes, tensors = [], []
    for k, (n, deg, D, bf) in enumerate(specs):
        sc = S.room_scene(n, n_feat=D, sh_degree=deg, seed=50 + k)
        scenes.append(sc)
        tensors.append(U.upload(sc, bf16=bf))
    server = L.Server(8 << 30, 16, dev.index)   # four lanes of up to four requests
    ids = [L.gs_serve_add_scene(server, t) for t in tensors]
    rng = np.random.default_rng(8)
    reqs = []
    for i in range(9):
        s = i % 3
        W, H = RES[rng.integers(len(RES))]
        if i == 4:   # a frame of >= 4096 tiles: its projection counts tiles by row differences
            W, H = 1088, 1024
        cam = S.room_trajectory(12, W, H, 0.9 * W, seed=100 + i)[int(rng.integers(12))]
        D = scenes[s].n_feat
        out = _outputs(torch, dev, cam, D)
        want_bwd = i % 3 == 1
        gin = gout = None
        if want_bwd:
            g = S.upstream_grads(H, W, D, seed=7 + i)
            gin = {k: torch.from_numpy(v).to(dev) for k, v in g.items()}
            K = (scenes[s].sh_degree + 1) ** 2
            gout = _grad_outputs(torch, dev, scenes[s].n, K, D)
        req = L.make_request(ids[s], as_camera(cam), out, gin, gout)
        reqs.append((s, cam, out, gin, gout, req))
    tickets = []
    for r in reqs:
        st, t = L.gs_serve_submit(server, r[-1])
        assert st == L.GS_OK
        tickets.append(t)
    results = []
    for t in tickets:
        st, res = L.gs_serve_poll(server, t, 60_000_000)
        assert st == L.GS_OK and res["status"] == L.GS_OK, (st, res)
        results.append(res)
    torch.cuda.synchronize()
    info = L.gs_serve_info(server)
    stats = L.gs_serve_stats(server)
    assert info["peak_running"] >= 2            # requests did run concurrently
    assert len({r["slot"] for r in results}) >= 2
    assert stats["peak_batch"] >= 2             # and shared raster launches
    assert stats["batches"] < len(reqs)
    assert info["peak_in_flight_bytes"] <= stats["arena_bytes"]
    # admission used the real instance counts: every request's granted range is its count
    assert all(r["instances"] > 0 for r in results)

    rast = Rasterizer(dev)
    for (s, cam, out, gin, gout, _), res in zip(reqs, results):
        alone = rast.forward(tensors[s], cam)
        for k in ("rgb", "depth", "alpha", "feat"):
            if out[k] is not None:
                assert torch.equal(out[k], alone[k]), k
        assert res["instances"] == alone["instances"]
        if gin is not None:
            ga = rast.backward(tensors[s], cam, gin["rgb"], gin["depth"], gin["alpha"], gin["feat"])
            keys = [k for k in ("means", "scales", "quats", "opacities", "sh", "feats", "pose")
                    if gout[k] is not None]
            # same kernels, another atomic order: every entry within the gradient bound
            U.assert_grads_close({k: gout[k].cpu().numpy() for k in keys},
                                 {k: ga[k].cpu().numpy() for k in keys}, keys,
                                 label="served in the mix vs alone")
    server.close()


def test_budget_refusals_and_cancel():
    import torch
    from paper_2603_09632_gb300 import _lib as L
    from paper_2603_09632_gb300.render import as_camera
    dev = U.device()
    sc = S.room_scene(20_000, n_feat=4, sh_degree=0, seed=3)
    t = U.upload(sc)
    tiny = L.Server(1 << 20, 2, dev.index)                 # 1 MiB: the scene cannot fit
    with pytest.raises(L.GSError) as e:
        L.gs_serve_add_scene(tiny, t)
    assert e.value.status == L.GS_ERR_OVER_BUDGET
    tiny.close()
    server = L.Server(64 << 20, 1, dev.index)               # fits the scene, not a 4K request
    sid = L.gs_serve_add_scene(server, t)
    # large Gaussians seen from close by: far more tile instances than the arena holds
    crowd = S.cube_scene(20_000, n_feat=4, seed=4, log_scale_mu=-1.5, log_scale_sd=0.1)
    cid = L.gs_serve_add_scene(server, U.upload(crowd))
    big = S.pinhole(3840, 2160, 3600.0, 3600.0, np.eye(3), np.array([0.0, 0.0, 3.0]))
    out = _outputs(torch, dev, S.pinhole(64, 64, 60.0), 4)
    st, _ = L.gs_serve_submit(server, L.make_request(sid, as_camera(big), out))
    assert st == L.GS_ERR_OVER_BUDGET
    st, _ = L.gs_serve_submit(server, L.make_request(sid + 5, as_camera(big), out))
    assert st == L.GS_ERR_ARG
    # the budget is divided at the first submit: no more scenes
    with pytest.raises(L.GSError) as e:
        L.gs_serve_add_scene(server, t)
    assert e.value.status == L.GS_ERR_STATE
    stats = L.gs_serve_stats(server)
    assert stats["scene_bytes"] + stats["workspace_bytes"] + stats["arena_bytes"] <= 64 << 20
    assert stats["max_pixels"] < 3840 * 2160
    # admission by the real instance count: a request that needs more than the whole arena
    # is refused after its projection, and nothing is written
    close = S.pinhole(1280, 1024, 1000.0, 1000.0, np.eye(3), np.array([0.0, 0.0, 2.0]))
    o2 = _outputs(torch, dev, close, 4)
    o2["alpha"].fill_(-7.0)
    st, tb = L.gs_serve_submit(server, L.make_request(cid, as_camera(close), o2))
    assert st == L.GS_OK
    st, res = L.gs_serve_poll(server, tb, 10_000_000)
    assert st == L.GS_OK and res["status"] == L.GS_ERR_OVER_BUDGET and res["slot"] == -1
    assert res["instances"] == 0
    torch.cuda.synchronize()
    assert (o2["alpha"] == -7.0).all()
    # cancel queued requests behind running ones (one request per lane)
    cams = S.room_trajectory(4, 64, 64, 60.0)
    tk = []
    for c in cams:
        st, ticket = L.gs_serve_submit(server, L.make_request(sid, as_camera(c), _outputs(torch, dev, c, 4)))
        assert st == L.GS_OK
        tk.append(ticket)
    cancelled = [L.gs_serve_cancel(server, x) for x in tk[1:]]
    for x, c in zip(tk[1:], cancelled):
        st, res = L.gs_serve_poll(server, x, 10_000_000)
        assert st == L.GS_OK
        assert res["status"] == (L.GS_ERR_CANCELLED if c == L.GS_OK else L.GS_OK)
    st, res = L.gs_serve_poll(server, tk[0], 10_000_000)
    assert st == L.GS_OK and res["status"] == L.GS_OK
    server.close()
