"""Benchmark: Mpix/s of forward + backward (RGB + depth + alpha + features) on one GB300.

One step = one camera pose of the workload through the whole path: gs_project ->
gs_bin_tiles -> gs_render_fwd -> gs_render_bwd (gradients to every Gaussian parameter and
the 6-DoF pose), inputs resident in HBM.  The default workload is the largest
single-GPU configuration, the memory form: 3M room Gaussians, SH 0, 32 fp32 feature
channels, 3840x2160, fx = fy = 3600, per-tile recomputation in the backward (no stored
blend lists), cycling over a 10-pose trajectory.  The SLAM frame (200k, 640x480, 16
channels) and the semantic frame (1M, SH 3, 64 bf16 channels, 1200x680) are selected with
--workload.  L2 is flushed (a 256 MiB write) between timed steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle instead (the
reference arm: there is no runnable reference implementation of this path).
Multi-GPU (torchrun, N > 1): poses are independent, so each rank renders its own poses
with no data-path collective (weak scaling); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import scenes as S  # noqa: E402

WORKLOADS = {
    "slam_640x480_200k": dict(make=lambda: S.config_slam(n_poses=100), bf16=False, l1=False,
                              desc="room 200k Gaussians, SH0, 16 fp32 feats, 640x480, fx=600"),
    "semantic_1200x680_1m": dict(make=lambda: S.config_semantic(n_poses=100), bf16=True, l1=True,
                                 desc="room 1M Gaussians, SH3, 64 bf16 feats, 1200x680, fx=600, L1 loss"),
    "tiny_128x96_2k": dict(make=S.config_tiny, bf16=False, l1=False,
                           desc="cube 2k Gaussians, SH0, 8 fp32 feats, 128x96, fx=100"),
    "memory_3840x2160_3m": dict(make=lambda: S.config_memory(n_poses=10), bf16=False, l1=False,
                                desc="room 3M Gaussians, SH0, 32 fp32 feats, 3840x2160, fx=3600, "
                                     "per-tile recomputation (no stored blend lists)",
                                cpu_mode=0, cpu_tiles=64),
    # the memory form's kernels (32 fp32 channels, every gradient) at a size a full ncu
    # capture can take (about 2 GB on the device); profiling size, not a headline
    "memory_1920x1080_1m": dict(make=lambda: (S.room_scene(1_000_000, n_feat=32, sh_degree=0),
                                              S.room_trajectory(10, 1920, 1080, 1800.0)),
                                bf16=False, l1=False, cpu_mode=0, cpu_tiles=64,
                                desc="room 1M Gaussians, SH0, 32 fp32 feats, 1920x1080, fx=1800 "
                                     "(profiling size of the memory form)"),
}
# Semantic distillation phase (Sec. 3.2, App. D): grid-sampled rendering with random offsets,
# region-indexed targets, the masked L1 + cosine loss fused into the forward, and the
# features-only backward (geometry frozen).  Stride 1 is the same phase at full resolution.
# VQ pixel decode (Sec. 3.2, App. E): softmax weights of 64 logits per Gaussian rendered as
# 64 bf16 channels, then F = E^T w(x) (512-d) and the prompt relevance on the tensor cores.
WORKLOADS["vq_decode_640x480_200k"] = dict(
    make=lambda: S.config_slam(n_poses=100), bf16=True, l1=False, vq=(64, 512),
    desc="room 200k Gaussians, 64 VQ logits -> bf16 weights rendered at 640x480, "
         "decode F = E^T w(x) to 512-d fp32 + prompt relevance (tcgen05 tf32); profiling size")
WORKLOADS["vq_decode_1200x680_1m"] = dict(
    make=lambda: S.config_semantic(n_poses=100), bf16=True, l1=False, vq=(64, 512),
    desc="room 1M Gaussians, 64 VQ logits -> bf16 weights rendered at 1200x680, "
         "decode F = E^T w(x) to 512-d fp32 + prompt relevance (tcgen05 tf32)")
for _s in (1, 2, 4):
    WORKLOADS[f"semantic_grid_s{_s}_1200x680_1m"] = dict(
        make=lambda: S.config_semantic(n_poses=100), bf16=True, l1=False, grid=_s,
        desc=f"room 1M Gaussians, SH3, 64 bf16 feats, 1200x680, grid stride {_s} (random offsets), "
             "region targets, fused masked L1+cos loss, features-only backward")
DEFAULT_WORKLOAD = "memory_3840x2160_3m"
METRIC = "Mpix/s fwd+bwd (RGB+D+feat) at 1 GB300"
L2_FLUSH_BYTES = 256 << 20


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def rank_poses(rank, n_poses, count):
    """Pose indices a rank renders: a walk over the trajectory offset by 37 poses per rank,
    so the ranks of a weak-scaling run render different poses and exchange no data."""
    return [(rank * 37 + k) % n_poses for k in range(count)]


def max_over_ranks(ms, dist, device):
    """Time of the whole job: the slowest rank's time (all_reduce MAX); ms itself at N = 1."""
    if not dist:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, steps, units_per_step, ms):
    """Whole-job throughput in millions of units per second: every rank processed
    steps x units_per_step in at most ms milliseconds."""
    return world * steps * units_per_step / (ms * 1e-3) / 1e6


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------- algorithmic model

def stage_bytes(st, D, bf, K):
    """Algorithmic bytes per launch of each stage (the byte model of the design notes)."""
    N, V, I, Ie, P = st["n"], st["visible"], st["instances"], st["inst_eff"], st["pixels"]
    pix_io = P * (20 + 4 * D + 8)
    return {
        "project": N * 44 + V * (12 * K + 48),
        "bin": I * 24 + N * 8 + V * 20,
        "fwd": Ie * (44 + D * bf) + pix_io,
        "bwd_raster": pix_io + Ie * (44 + D * bf) + V * (40 + 4 * D),
        "bwd_project": V * (40 + 44 + 12 * K) + V * (44 + 12 * K) + 24,
    }


def stage_bytes_semantic(st, D, bf):
    """Byte model of the semantic-phase step: the forward reads the target and mask and
    writes dL/dG_hat instead of images; the features-only backward reads that gradient and
    adds into the feature gradients."""
    V, I, Ie, P = st["visible"], st["instances"], st["inst_eff"], st["pixels"]
    return {
        "project": st["n"] * 44 + V * (12 * 16 + 48),
        "bin": I * 24 + st["n"] * 8 + V * 20,
        "fwd": Ie * (44 + D * bf) + P * (4 * D + 4 + 4 * D + 8),
        "bwd_raster": P * (4 * D + 8) + Ie * (44 + D * bf) + V * 4 * D,
        "bwd_project": 0,
    }


def stage_flops_semantic(st, D):
    """FLOP model of the semantic-phase step: per evaluated pair ~12 FLOPs (sigma, alpha,
    transmittance), per blended pair 2D (feature blend, or the W^T g_F contraction), and
    ~10D per sample for the fused loss."""
    V, E, Eb, P = st["visible"], st["pairs_eval"], st["pairs_blend"], st["pixels"]
    return {
        "project": V * (150 + 6 * 16),
        "bin": 0,
        "fwd": 12 * E + 2 * D * Eb + 10 * D * P,
        "bwd_raster": 12 * E + 2 * D * Eb,
        "bwd_project": 0,
    }


def stage_flops(st, D, K):
    """Algorithmic FP32 FLOPs per launch (FMA = 2, exp = 1) from the exact pair counts:
    E = pairs up to each pixel's last contributor, Eb = pairs blended."""
    V, E, Eb = st["visible"], st["pairs_eval"], st["pairs_blend"]
    return {
        "project": V * (150 + 6 * K),
        "bin": 0,
        "fwd": 12 * E + 2 * (4 + D) * Eb,
        "bwd_raster": 30 * E + 6 * (4 + D) * Eb,
        "bwd_project": V * (400 + 12 * K),
    }


def fp32_peak_tflops(peaks):
    """FP32 FMA peak derived from the unit counts: 152 SMs x 128 lanes x 2 FLOP x max clock
    (used only when no measurement is available)."""
    return 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12


def measure_fp32_peak(L, dev, index, iters=65536, reps=3):
    """FP32 FMA rate of this GPU from the library's microbenchmark (independent FMA chains
    at full occupancy, CUDA events), with the SM clock sampled while it runs.  Untimed:
    taken before the timed region.  Returns the best of ``reps`` runs."""
    clocks = make_clock_sampler(dev, index)
    clocks.start()
    runs = [L.gs_measure_fp32_peak(iters) for _ in range(reps)]
    clk = clocks.stop()
    tf, ms = max(runs)
    return {"tflops": round(tf, 2), "ms": round(ms, 3), "runs_tflops": [round(r[0], 2) for r in runs],
            "sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"),
            "reasons": clk.get("reasons"),
            "how": "gs_measure_fp32_peak: 8 independent FMA chains per thread (scalar fmaf and "
                   "packed f32x2 pairs, the larger rate), every SM at its occupancy limit, CUDA "
                   "events; best of %d, SM clock sampled meanwhile" % reps}


KERNEL_SOURCES = {
    "bwd_raster": ["gs_raster_bwd.cu", "gs_blend.cuh", "gs_internal.cuh"],
    "fwd": ["gs_raster_fwd.cu", "gs_blend.cuh", "gs_internal.cuh"],
    "bin": ["gs_sort.cu", "gs_internal.cuh"],
    "project": ["gs_project_fwd.cu", "gs_internal.cuh"],
    "bwd_project": ["gs_project_bwd.cu", "gs_internal.cuh"],
    "vq_decode": ["gs_vq.cu", "gs_internal.cuh"],
}


# the grid-sampled workloads run the grid kernels for their fwd / bwd_raster stages
GRID_KERNEL_SOURCES = {"fwd": ["gs_raster_grid.cu", "gs_blend.cuh", "gs_internal.cuh"],
                       "bwd_raster": ["gs_raster_grid.cu", "gs_blend.cuh", "gs_internal.cuh"]}


def source_hash(stage, workload=""):
    import hashlib
    h = hashlib.sha256()
    files = KERNEL_SOURCES[stage]
    if "grid" in workload and stage in GRID_KERNEL_SOURCES:
        files = GRID_KERNEL_SOURCES[stage]
    for f in files:
        with open(os.path.join(ROOT, "paper_2603_09632_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(stage, workload):
    """DRAM bytes per launch from the committed ncu capture, if the kernel source is unchanged."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(workload, {}).get(stage)
    if e and e.get("source_sha") == source_hash(stage, workload):
        return e["dram_bytes_per_launch"]
    return None


# ---------------------------------------------------------------- clocks

class NvmlClockSampler:
    """SM clock and clock-event reasons every ~1 ms through NVML (libnvidia-ml)
    (read-only queries), for timed regions far shorter than nvidia-smi's sampling period."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, torch_device):
        import ctypes
        self.C = ctypes
        self.nv = ctypes.CDLL("libnvidia-ml.so.1")
        if self.nv.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        import torch
        pr = torch.cuda.get_device_properties(torch_device)
        bus = f"{getattr(pr, 'pci_domain_id', 0):08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0"
        self.h = ctypes.c_void_p()
        if self.nv.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(self.h)) != 0:
            raise OSError("no NVML handle for " + bus)
        self.getr = getattr(self.nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.nv.nvmlDeviceGetCurrentClocksThrottleReasons
        self.samples, self.reasons, self.run = [], 0, False
        mx = ctypes.c_uint()
        self.nv.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx))
        self.max_mhz = float(mx.value)

    def _loop(self):
        C = self.C
        v, r = C.c_uint(), C.c_ulonglong()
        while self.run:
            if self.nv.nvmlDeviceGetClockInfo(self.h, 1, C.byref(v)) == 0:
                self.samples.append(float(v.value))
            if self.getr(self.h, C.byref(r)) == 0:
                self.reasons |= int(r.value)
            time.sleep(0.001)

    def start(self):
        self.run = True
        self.t = threading.Thread(target=self._loop, daemon=True)
        self.t.start()

    def stop(self):
        self.run = False
        self.t.join(timeout=2)
        return {"sm_mhz": statistics.median(self.samples) if self.samples else None,
                "sm_max_mhz": self.max_mhz,
                "reasons": sorted(n for b, n in self.REASONS.items() if self.reasons & b),
                "samples": len(self.samples), "source": "nvml"}


def make_clock_sampler(dev, index):
    try:
        return NvmlClockSampler(dev)
    except (OSError, AttributeError):
        return ClockSampler(index)


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- GPU arm

def build_roofline(stage, sb_tot, sf_tot, pairs, steps, workload, fp32=None, sm_mhz=None):
    """Roofline of the dominant stage: algorithmic bytes and FLOPs per launch (summed over
    the timed poses in sb_tot / sf_tot) against the measured stage time; the binding
    bound is whichever of the HBM and FP32 times is larger.  ``fp32`` is the measured FP32
    peak (measure_fp32_peak; the unit-count derivation only without it) and ``sm_mhz`` the
    median SM clock of the timed region, which gives the FP32 fraction at the clock the
    kernel ran at as well."""
    stage_ms = {name: stage[name][0] / max(stage[name][1], 1) for name in stage}
    dom = max(stage_ms, key=stage_ms.get)
    peaks, src = load_peaks()
    alg_b = sb_tot[dom] / steps
    alg_f = sf_tot[dom] / steps
    if fp32 and fp32.get("tflops"):
        p_alu = float(fp32["tflops"])
        alu_src = ("measured: FMA microbenchmark (gs_measure_fp32_peak) on this GPU in this run, "
                   f"at {fp32.get('sm_mhz')} MHz median SM clock")
    else:
        p_alu = fp32_peak_tflops(peaks)
        alu_src = "derived: 152 SMs x 128 FP32 lanes x 2 FLOP x max SM clock"
    t_hbm = alg_b / (peaks["hbm_gbs"] * 1e9)
    t_alu = alg_f / (p_alu * 1e12)
    t_meas = stage_ms[dom] * 1e-3
    traffic = captured_traffic(dom, workload)
    if t_alu > t_hbm:
        achieved = alg_f / t_meas / 1e12
        roofline = {"bound": "alu", "kernel": dom, "achieved": round(achieved, 3), "peak": round(p_alu, 1),
                    "unit": "TFLOP/s", "frac": round(achieved / p_alu, 4), "peak_source": alu_src}
    else:
        achieved = alg_b / t_meas / 1e9
        roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
                    "peak_source": src}
    roofline.update({
        "traffic": traffic, "alg_bytes": int(alg_b), "alg_flops": int(alg_f),
        "hbm_frac": round(alg_b / t_meas / 1e9 / peaks["hbm_gbs"], 4),
        "alu_frac": round(alg_f / t_meas / 1e12 / p_alu, 4),
        "alu_peak_tflops": round(p_alu, 2),
        "pairs_eval_per_step": int(pairs[0] / steps), "pairs_blend_per_step": int(pairs[1] / steps),
        "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()},
        "stage_alg_mb": {k: round(v / steps / 1e6, 3) for k, v in sb_tot.items()},
        "stage_alg_gflop": {k: round(v / steps / 1e9, 3) for k, v in sf_tot.items()}})
    if sm_mhz:
        # the dominant stage in cycles (ms x MHz = thousands of cycles), comparable across
        # clocks, and its FP32 fraction against the peak scaled to the clock it ran at
        roofline["stage_kcycles"] = round(stage_ms[dom] * sm_mhz, 1)
        if fp32 and fp32.get("tflops") and fp32.get("sm_mhz"):
            p_clk = p_alu * sm_mhz / fp32["sm_mhz"]
            roofline["alu_frac_at_kernel_clock"] = round(alg_f / t_meas / 1e12 / p_clk, 4)
    return roofline


def run_gpu(args):
    import torch
    from paper_2603_09632_gb300 import _lib as L
    from paper_2603_09632_gb300.render import as_camera

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    wl = WORKLOADS[args.workload]
    scene_np, cams = wl["make"]()
    D, K = scene_np.n_feat, (scene_np.sh_degree + 1) ** 2
    bf = 2 if wl["bf16"] else 4
    H, W = cams[0].H, cams[0].W
    P = H * W

    def dev_t(a, dtype=torch.float32):
        return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev).to(dtype)

    fdt = torch.bfloat16 if wl["bf16"] else torch.float32
    scene = L.Scene(dev_t(scene_np.means), dev_t(scene_np.scales), dev_t(scene_np.quats),
                    dev_t(scene_np.opacities), dev_t(scene_np.sh), dev_t(scene_np.feats, fdt))
    g = S.upstream_grads(H, W, D)
    gr, gd, ga, gf = (dev_t(g[k]) for k in ("rgb", "depth", "alpha", "feat"))
    target = dev_t(S.feature_target(H, W, D)) if wl["l1"] else None
    out = dict(rgb=torch.empty((3, H, W), device=dev), depth=torch.empty((H, W), device=dev),
               alpha=torch.empty((H, W), device=dev), feat=torch.empty((D, H, W), device=dev))
    grads = dict(means=torch.empty((scene.n, 3), device=dev), scales=torch.empty((scene.n, 3), device=dev),
                 quats=torch.empty((scene.n, 4), device=dev), opac=torch.empty(scene.n, device=dev),
                 sh=torch.empty((scene.n, K, 3), device=dev), feats=torch.empty((scene.n, D), device=dev),
                 pose=torch.empty(6, device=dev))
    gcams = [as_camera(c) for c in cams]
    ws = L.Workspace(local)
    stream = torch.cuda.current_stream()

    # size the workspace once (max instance count over the trajectory, +25 %), so that the
    # timed steps never synchronise or allocate
    max_inst = 0
    for c in gcams:
        L.gs_project(scene, c, ws)
        max_inst = max(max_inst, L.gs_bin_tiles(ws, sync=True))
    L.gs_workspace_reserve(ws, scene.n, int(max_inst * 1.25) + 1024, P)

    def step(c, gfeat):
        L.gs_project(scene, c, ws, stream)
        L.gs_bin_tiles(ws, sync=False, stream=stream)
        L.gs_render_fwd(scene, c, ws, out["rgb"], out["depth"], out["alpha"], out["feat"], stream)
        if target is not None:
            L.gs_l1_grad(out["feat"], target, 1.0 / out["feat"].numel(), gf, stream)
        L.gs_render_bwd(scene, c, ws, gr, gd, ga, gfeat, grads["means"], grads["scales"],
                        grads["quats"], grads["opac"], grads["sh"], grads["feats"], grads["pose"],
                        stream)

    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)
    poses = rank_poses(rank, len(gcams), args.warmup + args.steps)
    for k in range(args.warmup):
        step(gcams[poses[k]], gf)
        flush.fill_(float(k))
    torch.cuda.synchronize()
    if L.gs_workspace_status(ws) != L.GS_OK:
        raise RuntimeError("instance capacity overflow during warm-up")

    fp32 = measure_fp32_peak(L, dev, local)          # untimed, before the timed region
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    clocks = make_clock_sampler(dev, local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    n0 = L.gs_launch_count()
    torch.cuda.nvtx.range_push("timed")   # lets a profiler capture exactly these steps
    for k in range(args.steps):
        evs[k][0].record(stream)
        step(gcams[poses[args.warmup + k]], gf)
        evs[k][1].record(stream)
        flush.fill_(float(k))
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = L.gs_launch_count() - n0
    clk = clocks.stop()
    status = L.gs_workspace_status(ws)
    ms = sum(a.elapsed_time(b) for a, b in evs)
    ms = max_over_ranks(ms, dist, dev)
    value = job_throughput(world, args.steps, P, ms)

    # per-stage times: a separate, untimed pass over the same poses with the library's
    # stage events enabled (they add event records, so they stay out of the timed steps)
    L.gs_timing_enable(ws, True)
    L.gs_timing_collect(ws)
    for k in range(args.steps):
        step(gcams[poses[args.warmup + k]], gf)
        flush.fill_(float(k))
    stage = L.gs_timing_collect(ws)
    L.gs_timing_enable(ws, False)

    # algorithmic bytes per stage, averaged over the timed poses (untimed recount)
    sb_tot, sf_tot, pairs = {}, {}, [0, 0]
    for k in range(args.steps):
        c = gcams[poses[args.warmup + k]]
        L.gs_project(scene, c, ws)
        L.gs_bin_tiles(ws, sync=True)
        L.gs_render_fwd(scene, c, ws, out["rgb"], out["depth"], out["alpha"], out["feat"])
        st = L.gs_get_stats(ws)
        pairs[0] += st["pairs_eval"]
        pairs[1] += st["pairs_blend"]
        for name, b in stage_bytes(st, D, bf, K).items():
            sb_tot[name] = sb_tot.get(name, 0.0) + b
        for name, f in stage_flops(st, D, K).items():
            sf_tot[name] = sf_tot.get(name, 0.0) + f
    roofline = build_roofline(stage, sb_tot, sf_tot, pairs, args.steps, args.workload, fp32,
                              clk.get("sm_mhz"))
    # device memory of the step: the scene, images and gradients (torch; the L2 flush buffer
    # excluded) and the library workspace's high-water mark
    torch_peak = int(torch.cuda.max_memory_allocated(dev)) - flush.numel() * flush.element_size()
    ws_bytes = L.gs_workspace_bytes(ws)
    memory = {"torch_peak_bytes": torch_peak, "workspace_bytes": ws_bytes,
              "total_bytes": torch_peak + ws_bytes,
              "what": "peak device memory of the timed steps: torch allocations (scene, images, "
                      "gradients; not the L2 flush buffer) + the library workspace"}

    # end to end through the public API with host buffers
    e2e = run_e2e(args, L, scene, gcams, poses, dev, stream, ws, K, D, H, W)

    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "Mpix/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl["desc"], "gaussians": scene.n,
                   "pixels_per_step": P, "poses": len(gcams), "l2": "flushed (256 MiB write) between steps",
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "e2e": e2e, "gpu_launches": int(launches), "clocks": clk, "roofline": roofline,
        "fp32_peak": fp32, "memory": memory, "device_status": L.status_string(status),
    }
    if rank == 0 and not args.no_serve:
        # p50/p99 serve latency next to the throughput: the serving mix at saturation (2x
        # the plain arm's capacity), both arms on the same arrivals
        line["serve"] = serve_summary(serve_measure(args, dev, local, (SERVE_SAT,)))
    if rank == 0 and not args.no_cpu and world == 1:
        line["cpu_baseline"] = cpu_baseline(args, scene_np, cams, target_budget_s=args.cpu_budget,
                                            mode=wl.get("cpu_mode", 1))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_e2e(args, L, scene, gcams, poses, dev, stream, ws, K, D, H, W):
    """Same metric through the C ABI with host data: the map (the Gaussians) stays resident
    on the device as it does in SLAM; every step copies its per-frame input -- the upstream
    gradient images rgb/depth/alpha/features standing in for the observed frame -- from
    pinned host memory, runs project -> bin -> fwd -> bwd and reads the step's result (the
    6-DoF pose gradient) back into pinned host memory.  Inputs are double-buffered: a copy
    stream uploads step k+1 while step k computes."""
    import torch
    n = scene.n
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory()
    h_g = []
    for v in range(2):
        g = S.upstream_grads(H, W, D, seed=20 + v)
        h_g.append([pin(g[k]) for k in ("rgb", "depth", "alpha", "feat")])
    d_g = [[torch.empty_like(t, device=dev) for t in h_g[0]] for _ in range(2)]
    outs = [torch.empty((3, H, W), device=dev), torch.empty((H, W), device=dev),
            torch.empty((H, W), device=dev), torch.empty((D, H, W), device=dev)]
    grads = [torch.empty((n, 3), device=dev), torch.empty((n, 3), device=dev),
             torch.empty((n, 4), device=dev), torch.empty(n, device=dev),
             torch.empty((n, K, 3), device=dev), torch.empty((n, D), device=dev),
             torch.empty(6, device=dev)]
    h_pose = [torch.empty(6).pin_memory() for _ in range(2)]
    bi = sum(t.numel() * t.element_size() for t in h_g[0])
    bo = h_pose[0].numel() * h_pose[0].element_size()
    copy_stream = torch.cuda.Stream(device=dev)
    total = min(3, args.warmup) + args.steps
    ev_in = [torch.cuda.Event() for _ in range(total)]
    ev_used = [torch.cuda.Event() for _ in range(total)]

    def step(k, c):
        buf = d_g[k % 2]
        with torch.cuda.stream(copy_stream):
            if k >= 2:
                copy_stream.wait_event(ev_used[k - 2])   # buffer free again
            for d, h in zip(buf, h_g[k % 2]):
                d.copy_(h, non_blocking=True)
            ev_in[k].record(copy_stream)
        stream.wait_event(ev_in[k])
        L.gs_project(scene, c, ws, stream)
        L.gs_bin_tiles(ws, sync=False, stream=stream)
        L.gs_render_fwd(scene, c, ws, *outs, stream)
        L.gs_render_bwd(scene, c, ws, *buf, *grads, stream)
        ev_used[k].record(stream)
        h_pose[k % 2].copy_(grads[-1], non_blocking=True)

    nw = min(3, args.warmup)
    for k in range(nw):
        step(k, gcams[poses[k]])
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    copy_stream.wait_event(a)
    for k in range(args.steps):
        step(nw + k, gcams[poses[args.warmup + k]])
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    return {"value": round(args.steps * H * W / (ms * 1e-3) / 1e6, 2), "unit": "Mpix/s",
            "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(bo),
            "ms_per_step": round(ms / args.steps, 4),
            "what": "per step: upstream gradient images host->device (double-buffered on a copy "
                    "stream), pose gradient device->host (a tracking loop's result); the Gaussians "
                    "stay resident; no rendered image and no Gaussian gradient is read back"}


def run_grid(args):
    """Semantic distillation phase on the sample grid: per step project -> bin (no sync) ->
    region targets on the grid -> forward with the fused masked L1 + cosine loss ->
    features-only backward.  Offsets are drawn per step from {0..s-1}^2 (seeded)."""
    import torch
    from paper_2603_09632_gb300 import _lib as L
    from paper_2603_09632_gb300.render import as_camera, grid_shape

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    wl = WORKLOADS[args.workload]
    stride = wl["grid"]
    scene_np, cams = wl["make"]()
    D = scene_np.n_feat
    bf = 2 if wl["bf16"] else 4
    H, W = cams[0].H, cams[0].W
    fdt = torch.bfloat16 if wl["bf16"] else torch.float32

    def dev_t(a, dtype=torch.float32):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev).to(dtype)

    scene = L.Scene(dev_t(scene_np.means), dev_t(scene_np.scales), dev_t(scene_np.quats),
                    dev_t(scene_np.opacities), dev_t(scene_np.sh), dev_t(scene_np.feats, fdt))
    seg_np, table_np = S.region_annotations(H, W, D)
    seg, table = dev_t(seg_np, torch.int32), dev_t(table_np)
    nsteps = args.warmup + args.steps
    offs = S.grid_offsets(nsteps, stride, seed=2 + rank)
    poses = rank_poses(rank, len(cams), nsteps)
    gcams = [as_camera(cams[poses[k]], stride, *offs[k]) for k in range(nsteps)]
    Hs, Ws = grid_shape(gcams[0])
    P = Hs * Ws
    tgt = torch.empty((D, Hs, Ws), device=dev)
    mask = torch.empty((Hs, Ws), device=dev)
    gF = torch.empty((D, Hs, Ws), device=dev)
    loss = torch.zeros(3, dtype=torch.float64, device=dev)
    g_feats = torch.empty((scene.n, D), device=dev)
    ws = L.Workspace(local)
    stream = torch.cuda.current_stream()
    max_inst = 0
    for c in gcams:
        L.gs_project(scene, c, ws)
        max_inst = max(max_inst, L.gs_bin_tiles(ws, sync=True))
    L.gs_workspace_reserve(ws, scene.n, int(max_inst * 1.25) + 1024, P)

    def step(c):
        L.gs_project(scene, c, ws, stream)
        L.gs_bin_tiles(ws, sync=False, stream=stream)
        L.gs_grid_target_region(seg, table, c.stride, c.off_x, c.off_y, tgt, mask, stream)
        L.gs_render_fwd_loss(scene, c, ws, tgt, gF, loss, mask=mask, lambda_sem=1.0, stream=stream)
        L.gs_render_bwd(scene, c, ws, g_feat=gF, g_feats=g_feats, stream=stream)

    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)
    for k in range(args.warmup):
        step(gcams[k])
        flush.fill_(float(k))
    torch.cuda.synchronize()
    if L.gs_workspace_status(ws) != L.GS_OK:
        raise RuntimeError("instance capacity overflow during warm-up")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    L.gs_timing_enable(ws, True)
    L.gs_timing_collect(ws)
    clocks = make_clock_sampler(dev, local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    n0 = L.gs_launch_count()
    torch.cuda.nvtx.range_push("timed")
    for k in range(args.steps):
        evs[k][0].record(stream)
        step(gcams[args.warmup + k])
        evs[k][1].record(stream)
        flush.fill_(float(k))
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = L.gs_launch_count() - n0
    clk = clocks.stop()
    stage = L.gs_timing_collect(ws)
    L.gs_timing_enable(ws, False)
    status = L.gs_workspace_status(ws)
    ms = sum(a.elapsed_time(b) for a, b in evs)
    ms = max_over_ranks(ms, dist, dev)
    value = job_throughput(world, args.steps, P, ms)
    sb_tot, sf_tot, pairs = {}, {}, [0, 0]
    for k in range(args.steps):
        c = gcams[args.warmup + k]
        L.gs_project(scene, c, ws)
        L.gs_bin_tiles(ws, sync=True)
        L.gs_render_fwd(scene, c, ws, None, None, None, gF)
        st = L.gs_get_stats(ws)
        pairs[0] += st["pairs_eval"]
        pairs[1] += st["pairs_blend"]
        for name, b in stage_bytes_semantic(st, D, bf).items():
            sb_tot[name] = sb_tot.get(name, 0.0) + b
        for name, f in stage_flops_semantic(st, D).items():
            sf_tot[name] = sf_tot.get(name, 0.0) + f
    roofline = build_roofline(stage, sb_tot, sf_tot, pairs, args.steps, args.workload)

    # end to end with host data: the Gaussians stay resident; every step uploads its frame's
    # annotations (segmentation and region table; double-buffered on a copy stream) and
    # reads the loss back
    pin = lambda t: t.cpu().pin_memory()
    h_in = [[pin(seg), pin(table)], [pin(torch.flip(seg, dims=(1,))), pin(table.flip(0))]]
    d_in = [[torch.empty_like(t, device=dev) for t in h_in[0]] for _ in range(2)]
    h_loss = [torch.empty(3, dtype=torch.float64).pin_memory() for _ in range(2)]
    copy_stream = torch.cuda.Stream(device=dev)
    nw = min(3, args.warmup)
    ev_in = [torch.cuda.Event() for _ in range(nw + args.steps)]
    ev_used = [torch.cuda.Event() for _ in range(nw + args.steps)]

    def e2e_step(k, c):
        buf = d_in[k % 2]
        with torch.cuda.stream(copy_stream):
            if k >= 2:
                copy_stream.wait_event(ev_used[k - 2])
            for d, h in zip(buf, h_in[k % 2]):
                d.copy_(h, non_blocking=True)
            ev_in[k].record(copy_stream)
        stream.wait_event(ev_in[k])
        L.gs_project(scene, c, ws, stream)
        L.gs_bin_tiles(ws, sync=False, stream=stream)
        L.gs_grid_target_region(buf[0], buf[1], c.stride, c.off_x, c.off_y, tgt, mask, stream)
        ev_used[k].record(stream)
        L.gs_render_fwd_loss(scene, c, ws, tgt, gF, loss, mask=mask, lambda_sem=1.0, stream=stream)
        L.gs_render_bwd(scene, c, ws, g_feat=gF, g_feats=g_feats, stream=stream)
        h_loss[k % 2].copy_(loss, non_blocking=True)

    for k in range(nw):
        e2e_step(k, gcams[k])
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    copy_stream.wait_event(a)
    for k in range(args.steps):
        e2e_step(nw + k, gcams[args.warmup + k])
    b.record(stream)
    torch.cuda.synchronize()
    ems = a.elapsed_time(b)
    e2e = {"value": round(args.steps * P / (ems * 1e-3) / 1e6, 2), "unit": "Mpix/s",
           "h2d_bytes_per_step": int(sum(t.numel() * t.element_size() for t in h_in[0])),
           "d2h_bytes_per_step": int(h_loss[0].numel() * h_loss[0].element_size()),
           "ms_per_step": round(ems / args.steps, 4),
           "what": "per step: frame annotations host->device (double-buffered on a copy stream), "
                   "loss device->host; the Gaussians stay resident"}
    line = {
        "metric": "Mpix/s supervised samples, semantic phase fwd+bwd (grid, fused loss, features-only)",
        "value": round(value, 2), "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (bf16 features)", "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl["desc"], "gaussians": scene.n,
                   "stride": stride, "samples_per_step": P, "image": [W, H], "poses": len(cams),
                   "l2": "flushed (256 MiB write) between steps",
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "e2e": e2e, "gpu_launches": int(launches), "clocks": clk, "roofline": roofline,
        "device_status": L.status_string(status),
    }
    if rank == 0 and not args.no_cpu and world == 1:
        line["cpu_baseline"] = cpu_baseline(args, scene_np, [cams[p] for p in poses],
                                            target_budget_s=args.cpu_budget, stride=stride)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_vq(args):
    """VQ decode step: softmax weights (N x L) -> project -> bin (no sync) -> render the
    weights as L bf16 channels -> tensor-core decode writing F [D, H, W] and the relevance
    map.  The roofline is the decode kernel's, timed alone with CUDA events."""
    import torch
    from paper_2603_09632_gb300 import _lib as L
    from paper_2603_09632_gb300.render import as_camera

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    wl = WORKLOADS[args.workload]
    Lw, Dc = wl["vq"]
    scene_np, cams = wl["make"]()
    H, W = cams[0].H, cams[0].W
    P = H * W
    rng = np.random.default_rng(11)

    def dev_t(a, dtype=torch.float32):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev).to(dtype)

    n = scene_np.n
    logits = dev_t(rng.normal(scale=2.0, size=(n, Lw)).astype(np.float32))
    wts = torch.empty((n, Lw), device=dev, dtype=torch.bfloat16)
    scene = L.Scene(dev_t(scene_np.means), dev_t(scene_np.scales), dev_t(scene_np.quats),
                    dev_t(scene_np.opacities), dev_t(scene_np.sh), wts)
    E = dev_t((rng.normal(size=(Lw, Dc)) / 8.0).astype(np.float32))
    text = rng.normal(size=(5, Dc))
    text = dev_t((text / np.linalg.norm(text, axis=1, keepdims=True)).astype(np.float32))
    wmap = torch.empty((Lw, H, W), device=dev)
    F = torch.empty((Dc, H, W), device=dev)
    R = torch.empty((H, W), device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    gcams = [as_camera(c) for c in cams]
    ws = L.Workspace(local)
    stream = torch.cuda.current_stream()
    L.gs_vq_weights(logits, wts)
    max_inst = 0
    for c in gcams:
        L.gs_project(scene, c, ws)
        max_inst = max(max_inst, L.gs_bin_tiles(ws, sync=True))
    L.gs_workspace_reserve(ws, n, int(max_inst * 1.25) + 1024, P)
    dec = []

    def step(c, k):
        L.gs_vq_weights(logits, wts, stream)
        L.gs_project(scene, c, ws, stream)
        L.gs_bin_tiles(ws, sync=False, stream=stream)
        L.gs_render_fwd(scene, c, ws, None, None, None, wmap, stream)
        a, b = dec[k]
        a.record(stream)
        L.gs_vq_decode(wmap, E, F_out=F, text=text, tau=10.0, relevance=R, err=err, stream=stream)
        b.record(stream)

    nsteps = args.warmup + args.steps
    dec = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(nsteps)]
    poses = rank_poses(rank, len(gcams), nsteps)
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)
    for k in range(args.warmup):
        step(gcams[poses[k]], k)
        flush.fill_(float(k))
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    clocks = make_clock_sampler(dev, local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    n0 = L.gs_launch_count()
    for k in range(args.steps):
        evs[k][0].record(stream)
        step(gcams[poses[args.warmup + k]], args.warmup + k)
        evs[k][1].record(stream)
        flush.fill_(float(k))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = L.gs_launch_count() - n0
    clk = clocks.stop()
    if int(err.item()) != 0:
        raise RuntimeError("tensor-core decode reported a timed-out wait")
    ms = sum(a.elapsed_time(b) for a, b in evs)
    ms = max_over_ranks(ms, dist, dev)
    dec_ms = sum(dec[args.warmup + k][0].elapsed_time(dec[args.warmup + k][1])
                 for k in range(args.steps)) / args.steps
    value = job_throughput(world, args.steps, P, ms)
    peaks, src = load_peaks()
    alg_bytes = P * (Lw * 4 + Dc * 4 + 4)
    alg_flops = 2.0 * P * Lw * Dc + P * Dc * 2 * 6
    tf32_peak = peaks.get("bf16_tflops", 1900.0) * (1.1 / 2.25)
    achieved_b = alg_bytes / (dec_ms * 1e-3) / 1e9
    achieved_f = alg_flops / (dec_ms * 1e-3) / 1e12
    t_hbm = alg_bytes / (peaks["hbm_gbs"] * 1e9)
    t_tc = alg_flops / (tf32_peak * 1e12)
    if t_hbm >= t_tc:
        roofline = {"bound": "hbm", "kernel": "k_vq_decode", "achieved": round(achieved_b, 1),
                    "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": round(achieved_b / peaks["hbm_gbs"], 4), "peak_source": src}
    else:
        roofline = {"bound": "tensor", "kernel": "k_vq_decode", "achieved": round(achieved_f, 2),
                    "peak": round(tf32_peak, 1), "unit": "TFLOP/s",
                    "frac": round(achieved_f / tf32_peak, 4),
                    "peak_source": "measured bf16 burst x nominal tf32/bf16 ratio 1.1/2.25"}
    roofline.update({"traffic": captured_traffic("vq_decode", args.workload),
                     "alg_bytes": int(alg_bytes), "alg_flops": int(alg_flops),
                     "decode_ms": round(dec_ms, 4),
                     "tensor_frac": round(achieved_f / tf32_peak, 4),
                     "hbm_frac": round(achieved_b / peaks["hbm_gbs"], 4)})
    line = {
        "metric": "Mpix/s VQ weights + render + tensor-core decode (F 512-d + relevance)",
        "value": round(value, 2), "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "tf32 decode, f32 accumulate", "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl["desc"], "gaussians": n, "L": Lw, "D": Dc,
                   "pixels_per_step": P, "l2": "flushed (256 MiB write) between steps"},
        "gpu_launches": int(launches), "clocks": clk, "roofline": roofline,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------- CPU oracle

def sample_grads(n_feat, n_pix, seed):
    """Seeded N(0,1) upstream gradients at the sampled pixels only ([C, n_pix])."""
    rng = np.random.default_rng(seed)
    return {k: rng.standard_normal((c, n_pix)).astype(np.float32)
            for k, c in (("rgb", 3), ("depth", 1), ("alpha", 1), ("feat", n_feat))}


def oracle_step(O, scene_np, cam, pixels, gs, mode=1):
    """One bounded sample of the workload through the CPU oracle (FP32): forward and
    backward of a loss restricted to ``pixels`` (flat indices) with upstream gradients
    ``gs`` at those pixels.  ``mode`` 1 builds the sorted tile lists of the whole frame, 0
    takes each sampled tile's candidates by brute force over all Gaussians (at 4K the
    frame's lists hold ~10^8 instances, which a sample does not need)."""
    O.render(scene_np, cam, "f32", pixels=pixels, mode=mode)
    O.backward(scene_np, cam, gs, "f32", pixels=pixels, mode=mode)


def sample_pixels(cam, n_tiles, rng, stride=1):
    """Image pixels of n_tiles random 16x16 tiles of the rendered grid (the image, or the
    stride-s sample grid with a random offset)."""
    ox, oy = (int(v) for v in rng.integers(0, stride, size=2))
    Ws, Hs = -(-cam.W // stride), -(-cam.H // stride)
    TX, TY = (Ws + 15) // 16, (Hs + 15) // 16
    tiles = rng.choice(TX * TY, size=min(n_tiles, TX * TY), replace=False)
    pix = []
    for t in tiles:
        x0, y0 = (t % TX) * 16, (t // TX) * 16
        ms, ns = np.mgrid[y0:min(y0 + 16, Hs), x0:min(x0 + 16, Ws)]
        ys, xs = oy + stride * ms, ox + stride * ns
        ok = (ys < cam.H) & (xs < cam.W)
        pix.append((ys * cam.W + xs)[ok].ravel())
    return np.concatenate(pix)


def cpu_tiles(args, wl):
    return args.cpu_tiles if args.cpu_tiles else wl.get("cpu_tiles", 300)


def cpu_baseline(args, scene_np, cams, target_budget_s=15.0, stride=1, mode=1):
    from oracle import oracle as O
    O.build()
    cores = O.set_threads(os.cpu_count() or 1)
    rng = np.random.default_rng(5)
    n_tiles = cpu_tiles(args, WORKLOADS[args.workload])
    t_tot, px_tot, k = 0.0, 0, 0
    while t_tot < target_budget_s and k < len(cams):
        cam = cams[k]
        pix = sample_pixels(cam, n_tiles, rng, stride)
        gs = sample_grads(scene_np.n_feat, pix.size, 100 + k)
        t0 = time.perf_counter()
        oracle_step(O, scene_np, cam, pix, gs, mode)
        t_tot += time.perf_counter() - t0
        px_tot += pix.size
        k += 1
    lists = ("tile lists of the full frame" if mode == 1 else
             "brute-force candidates of each sampled tile")
    return {"value": round(px_tot / t_tot / 1e6, 5), "unit": "Mpix/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{k} poses x {n_tiles} random 16x16 tiles"
                      + (f" of the stride-{stride} sample grid" if stride > 1 else "")
                      + f", FP32 oracle forward + backward (projection of the full scene and {lists} "
                      f"each pose), {t_tot:.1f} s"}


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    cores = O.set_threads(os.cpu_count() or 1)
    wl = WORKLOADS[args.workload]
    scene_np, cams = wl["make"]()
    rng = np.random.default_rng(5)
    times, px = [], 0
    n_tiles = cpu_tiles(args, wl)
    for k in range(args.warmup + args.steps):
        cam = cams[k % len(cams)]
        pix = sample_pixels(cam, n_tiles, rng, wl.get("grid", 1))
        gs = sample_grads(scene_np.n_feat, pix.size, 100 + k)
        t0 = time.perf_counter()
        oracle_step(O, scene_np, cam, pix, gs, wl.get("cpu_mode", 1))
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            px += pix.size
    tot = sum(times)
    value = px / tot / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "Mpix/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * tot / args.steps, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"], "gaussians": scene_np.n,
                       "pixels_per_step": int(px / args.steps), "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": round(value, 5), "unit": "Mpix/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"{n_tiles} random 16x16 tiles per step, FP32 oracle "
                                       "forward + backward on the host cores"},
            "e2e": {"value": round(value, 5), "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


SERVE_RATES = (0.25, 0.5, 1.0, 1.5, 2.0)
SERVE_SAT = 2.0   # the rate of the serving summary in the main line (x plain capacity)


def wait_until(t):
    """Sleep until perf_counter() reaches t (spinning only for the last 0.2 ms, so that
    other Python threads keep running)."""
    while True:
        d = t - time.perf_counter()
        if d <= 0:
            return
        time.sleep(d - 2e-4) if d > 4e-4 else time.sleep(0)


def _pct(xs, q):
    return float(np.percentile(np.asarray(xs, np.float64), q)) if len(xs) else float("nan")


def serve_measure(args, dev, local, rates):
    """Serving mix: 8 resident scenes (100k-2M Gaussians, SH = id mod 4, 16/32/64 bf16
    feature channels), Poisson arrivals of single-pose requests at resolutions drawn from
    {256x256, 640x480, 1200x680, 1920x1080}, 30 % with backward.  Two arms on the same
    request sequence and arrival times:
      plain: one request at a time through gs_project -> gs_bin_tiles -> gs_render_fwd
             (-> gs_render_bwd) on one stream, synchronised per request;
      serve: the serving loop (gs_serve_submit / gs_serve_poll) with --serve-slots slots:
             batches of requests projected together, admitted by their real tile-instance
             counts and rendered by shared persistent raster launches.
    The rate is given as multiples of the plain arm's closed-loop capacity.  Latency runs
    from the scheduled arrival to poll-visible completion (so time a request waits for a
    client buffer counts); throughput is served pixels over first arrival -> last
    completion.  Returns the measurement as a dict."""
    import torch
    from paper_2603_09632_gb300 import _lib as L
    from paper_2603_09632_gb300.render import as_camera

    scenes_np = S.serving_scenes(scale=args.serve_scale)
    scenes = []
    for sc in scenes_np:
        t = [torch.from_numpy(np.ascontiguousarray(getattr(sc, k), np.float32)).to(dev)
             for k in ("means", "scales", "quats", "opacities", "sh")]
        ft = torch.from_numpy(np.ascontiguousarray(sc.feats, np.float32)).to(dev).to(torch.bfloat16)
        scenes.append(L.Scene(*t, ft))
    reqs = S.serving_requests(args.serve_requests, 1.0)     # arrival times at 1 request/s
    max_pix = max(c.W * c.H for _, _, c, _ in reqs)
    max_d = max(sc.n_feat for sc in scenes_np)
    max_n = max(sc.n for sc in scenes_np)

    def align(x):
        return (x + 63) // 64 * 64

    out_floats = align(5 * max_pix) + align(max_d * max_pix)
    g_floats = align(max_n * 3) * 2 + align(max_n * 4) + align(max_n) + align(max_n * 48) \
        + align(max_n * max_d) + 64
    n_sets = 4 * args.serve_slots
    pool = [(torch.empty(out_floats, device=dev), torch.empty(g_floats, device=dev))
            for _ in range(n_sets)]
    # upstream gradients per resolution (read-only, shared by every request)
    ups = {}
    for _, _, c, _ in reqs:
        if (c.W, c.H) not in ups:
            g = S.upstream_grads(c.H, c.W, max_d)
            ups[(c.W, c.H)] = {k: torch.from_numpy(v).to(dev) for k, v in g.items()}

    def views(k, sid, cam, want_bwd):
        ob, gb = pool[k]
        P, D, n = cam.W * cam.H, scenes_np[sid].n_feat, scenes_np[sid].n
        Kc = (scenes_np[sid].sh_degree + 1) ** 2
        out = dict(rgb=ob[:3 * P].view(3, cam.H, cam.W), depth=ob[3 * P:4 * P].view(cam.H, cam.W),
                   alpha=ob[4 * P:5 * P].view(cam.H, cam.W),
                   feat=ob[align(5 * P):align(5 * P) + D * P].view(D, cam.H, cam.W))
        if not want_bwd:
            return out, None, None
        u = ups[(cam.W, cam.H)]
        gin = dict(rgb=u["rgb"], depth=u["depth"], alpha=u["alpha"], feat=u["feat"][:D])
        o, gout = 0, {}
        for name, m in (("means", 3), ("scales", 3), ("quats", 4), ("opacities", 1), ("sh", Kc * 3),
                        ("feats", D), ("pose", 0)):
            sz = 6 if name == "pose" else n * m
            gout[name] = gb[o:o + sz]
            o += align(sz)
        return out, gin, gout

    cams = [as_camera(c) for _, _, c, _ in reqs]
    pixels = [c.W * c.H for _, _, c, _ in reqs]
    ws = L.Workspace(local)
    L.gs_workspace_reserve(ws, max_n, 0, max_pix)
    stream = torch.cuda.current_stream()

    def plain_one(i):
        _, sid, cam, bwd = reqs[i]
        out, gin, gout = views(i % n_sets, sid, cam, bwd)
        sc = scenes[sid]
        L.gs_project(sc, cams[i], ws, stream)
        L.gs_bin_tiles(ws, sync=True, stream=stream)
        L.gs_render_fwd(sc, cams[i], ws, out["rgb"], out["depth"], out["alpha"], out["feat"], stream)
        if bwd:
            L.gs_render_bwd(sc, cams[i], ws, gin["rgb"], gin["depth"], gin["alpha"], gin["feat"],
                            gout["means"], gout["scales"], gout["quats"], gout["opacities"],
                            gout["sh"], gout["feats"], gout["pose"], stream)
        stream.synchronize()

    # warm-up and plain closed-loop capacity
    for i in range(min(len(reqs), 3 * args.warmup)):
        plain_one(i)
    m = min(len(reqs), args.serve_capacity_requests)
    t0 = time.perf_counter()
    for i in range(m):
        plain_one(i)
    t_cap = time.perf_counter() - t0
    cap_rps = m / t_cap
    cap_mpix = sum(pixels[:m]) / t_cap / 1e6

    def plain_open(rate):
        lat, t0 = [], time.perf_counter()
        last = t0
        for i, (ta, _, _, _) in enumerate(reqs):
            arrive = t0 + ta / rate
            wait_until(arrive)
            plain_one(i)
            last = time.perf_counter()
            lat.append(last - arrive)
        return lat, last - (t0 + reqs[0][0] / rate)

    server = L.Server(int(args.serve_budget_gb * (1 << 30)), args.serve_slots, local)
    ids = [L.gs_serve_add_scene(server, sc) for sc in scenes]

    def serve_open(rate, n_req=None):
        n_req = len(reqs) if n_req is None else n_req
        free = list(range(n_sets))
        cv = threading.Condition()
        outstanding = {}      # ticket -> (i, set, t_submit, arrive)
        lat = [None] * n_req
        fail = []
        done_flag = [False]

        def poller():
            while True:
                with cv:
                    items = list(outstanding.items())
                    if not items and done_flag[0]:
                        return
                got = False
                for t, (i, k, ts, ta) in items:
                    st, res = L.gs_serve_poll(server, t, 0)
                    if st == L.GS_OK:
                        got = True
                        if res["status"] != L.GS_OK:
                            fail.append((i, res["status"]))
                        lat[i] = (ts - ta) + res["latency_us"] * 1e-6
                        with cv:
                            del outstanding[t]
                            free.append(k)
                            cv.notify_all()
                if not got:
                    time.sleep(50e-6)

        th = threading.Thread(target=poller, daemon=True)
        th.start()
        t0 = time.perf_counter()
        for i in range(n_req):
            ta, sid, cam, bwd = reqs[i]
            arrive = t0 + ta / rate
            wait_until(arrive)
            with cv:
                while not free:
                    cv.wait()
                k = free.pop()
            out, gin, gout = views(k, sid, cam, bwd)
            ts = time.perf_counter()
            st, t = L.gs_serve_submit(server, L.make_request(ids[sid], cams[i], out, gin, gout))
            if st != L.GS_OK:
                raise RuntimeError(f"gs_serve_submit: {L.status_string(st)}")
            with cv:
                outstanding[t] = (i, k, ts, arrive)
        with cv:
            done_flag[0] = True
        th.join()
        if fail:
            raise RuntimeError(f"served requests failed: {fail[:4]}")
        first = t0 + reqs[0][0] / rate
        last = max(t0 + reqs[i][0] / rate + lat[i] for i in range(n_req))
        return lat, last - first

    serve_open(cap_rps, min(len(reqs), 4 * args.serve_slots))     # warm the slots
    rows = []
    for x in rates:
        rate = x * cap_rps
        lp, tp = plain_open(rate)
        ls, tsv = serve_open(rate)
        px = sum(pixels)
        rows.append({"x_capacity": x, "rate_rps": round(rate, 2),
                     "plain": {"mpix_s": round(px / tp / 1e6, 2), "p50_ms": round(1e3 * _pct(lp, 50), 3),
                               "p99_ms": round(1e3 * _pct(lp, 99), 3)},
                     "serve": {"mpix_s": round(px / tsv / 1e6, 2), "p50_ms": round(1e3 * _pct(ls, 50), 3),
                               "p99_ms": round(1e3 * _pct(ls, 99), 3)}})
    info = L.gs_serve_info(server)
    stats = L.gs_serve_stats(server)
    server.close()
    return {"plain_capacity": {"rps": round(cap_rps, 2), "mpix_s": round(cap_mpix, 2), "requests": m},
            "sweep": rows, "server": dict(info, **stats),
            "config": {"workload": "serve_mix_8_scenes", "scenes": [
                {"n": sc.n, "sh": sc.sh_degree, "feat": sc.n_feat} for sc in scenes_np],
                "requests": len(reqs), "slots": args.serve_slots,
                "budget_gb": args.serve_budget_gb, "client_buffer_sets": n_sets,
                "resolutions": sorted({(c.W, c.H) for _, _, c, _ in reqs}),
                "bwd_fraction": round(sum(r[3] for r in reqs) / len(reqs), 3)}}


def serve_summary(res):
    """Serving figures at the highest swept rate: both arms' Mpix/s and p50/p99 latency."""
    top = res["sweep"][-1]
    return {"rate_x_plain_capacity": top["x_capacity"], "rate_rps": top["rate_rps"],
            "serve_mpix_s": top["serve"]["mpix_s"], "serve_p50_ms": top["serve"]["p50_ms"],
            "serve_p99_ms": top["serve"]["p99_ms"], "plain_mpix_s": top["plain"]["mpix_s"],
            "plain_p50_ms": top["plain"]["p50_ms"], "plain_p99_ms": top["plain"]["p99_ms"],
            "throughput_x_plain": round(top["serve"]["mpix_s"] / max(top["plain"]["mpix_s"], 1e-9), 3),
            "batches": res["server"]["batches"], "peak_batch": res["server"]["peak_batch"],
            "workload": res["config"]["workload"], "requests": res["config"]["requests"]}


def run_serve(args):
    """The serving sweep (serve_measure) from 0.25x to 2x the plain capacity, one JSON line."""
    import torch
    rank, world, local = env_rank()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    res = serve_measure(args, dev, local, SERVE_RATES)
    top = res["sweep"][-1]
    line = {"metric": "serving Mpix/s with p50/p99 latency, mixed scenes/resolutions, 30% fwd+bwd",
            "value": top["serve"]["mpix_s"], "unit": "Mpix/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32 (bf16 features)", "data": "synthetic",
            "plain_capacity": res["plain_capacity"], "sweep": res["sweep"],
            "config": res["config"], "server": res["server"], "summary": serve_summary(res)}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--cpu-tiles", type=int, default=0,
                    help="16x16 tiles per oracle sample (0: the workload's default, 300 or 64 at 4K)")
    ap.add_argument("--serve", action="store_true", help="serving-loop benchmark instead")
    ap.add_argument("--no-serve", action="store_true",
                    help="leave the serving summary (p50/p99 at saturation) out of the main line")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-capacity-requests", type=int, default=100)
    ap.add_argument("--serve-budget-gb", type=float, default=16.0)
    ap.add_argument("--serve-scale", type=float, default=1.0, help="scale of the scene sizes")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.serve:
        run_serve(args)
    elif "grid" in WORKLOADS[args.workload]:
        run_grid(args)
    elif "vq" in WORKLOADS[args.workload]:
        run_vq(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
