// Serving: resident scenes, continuous batching, two-phase admission by an HBM budget.
//
// A server owns copies of the scenes it serves and, once the first request arrives, every
// buffer it will use: up to four lanes, each a CUDA stream with its own request workspaces
// (reserved for the largest resident scene and a per-request pixel limit), and one arena of
// tile-instance buffers that takes the rest of the budget.  Nothing is allocated or freed
// while requests run.
//
// The scheduler (serve_core.hpp) forms a batch from the oldest pending requests for a free
// lane.  Phase A projects each of them on the lane's stream and reads back their tile
// instance counts (one synchronisation per batch): that count, not an estimate, is what a
// request needs from the arena.  Admission grants arena ranges in arrival order.  Phase B
// bins each admitted request into its range, then renders all of them in ONE persistent
// forward raster launch whose queue holds every (request, tile) item of the batch (one
// launch per feature layout), and likewise one backward raster launch for the requests
// that want gradients, followed by their projection backward.  Lanes are independent
// workers, so while one lane's batch is on the device the others project, admit and launch
// theirs: requests that arrive meanwhile start as soon as a lane and memory free up, and
// their work overlaps on the device.
// Results are bit-identical to the same request rendered alone (forward) and equal within
// atomic reordering (backward).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "gs_internal.cuh"
#include "gs_serve_ws.hpp"
#include "serve_core.hpp"

namespace {

using gs::RasterJob;

constexpr int kMaxLanes = 4;
constexpr double kAgingS = 0.05;          // a request that waited 50 ms is not overtaken
constexpr int64_t kInstBytes = 16;        // per instance: (key, id) pair, scratch key, sorted id
constexpr int64_t kGaussBytes = 112;      // per Gaussian in a request workspace (planning)
constexpr int64_t kPixBytes = 8;          // per pixel: final transmittance, last contributor
constexpr int64_t kMaxPixPerRequest = 3840LL * 2160LL;
constexpr int64_t kMinPixPerRequest = 256LL * 256LL;

struct SceneStore {
  gs_scene view;                   // points at the buffers below
  std::vector<void*> buffers;
  size_t bytes = 0;
};

struct Lane {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  uint32_t* h_inst = nullptr;          // pinned, one count per workspace
  uint32_t* queue = nullptr;           // device: forward queue [0, 1], backward [2, 3]
  std::vector<gs_workspace*> ws;
};

size_t feat_elem_bytes(const gs_scene& s) { return s.feat_dtype == GS_BF16 ? 2 : 4; }

int64_t tiles_of(int64_t W, int64_t H) { return ((W + 15) / 16) * ((H + 15) / 16); }

}  // namespace

struct gs_server {
  int device = 0;
  int64_t budget = 0;
  int n_lanes = 1, slots_per_lane = 1;
  std::mutex mu;                   // scenes and start-up
  std::vector<SceneStore> scenes;
  int64_t scene_bytes = 0;
  int64_t max_n = 0;               // largest resident scene
  bool started = false;
  int64_t pix_cap = 0, tile_cap = 0;   // per-request limits of the reserved workspaces
  int64_t fixed_bytes = 0;             // workspaces, queues
  Lane lanes[kMaxLanes];
  void* arena = nullptr;
  int64_t arena_inst = 0;              // instance slots in the arena
  uint2* kv = nullptr;                 // (key, id) pairs [arena_inst]
  uint32_t* arr[2] = {};               // scratch keys, sorted ids: [arena_inst] each
  std::unique_ptr<gs_serve::Scheduler<gs_request>> sched;
};

namespace {

struct Grouping {
  int dp;
  int dtype;
  bool operator<(const Grouping& o) const { return dp != o.dp ? dp < o.dp : dtype < o.dtype; }
};

gs_scene scene_of(gs_server* sv, int id) {
  std::lock_guard<std::mutex> lk(sv->mu);
  return sv->scenes[(size_t)id].view;
}

// Phase A: project every request of the batch and read back its tile-instance count.
void measure(gs_server* sv, int lane, std::vector<gs_serve::Item<gs_request>>& items) {
  cudaSetDevice(sv->device);
  Lane& ln = sv->lanes[lane];
  for (auto& it : items) {
    gs_workspace* ws = ln.ws[(size_t)it.slot];
    const gs_scene sc = scene_of(sv, it.req.scene_id);
    gs_status s = gs_project(&sc, &it.req.cam, ws, ln.stream);
    if (s == GS_OK) s = gs::ws_instances_async(ws, ln.h_inst + it.slot, ln.stream);
    it.status = s;
  }
  if (cudaStreamSynchronize(ln.stream) != cudaSuccess)
    for (auto& it : items) it.status = it.status ? it.status : GS_ERR_CUDA;
  for (auto& it : items)
    if (it.status == GS_OK) it.cost = (int64_t)ln.h_inst[it.slot];
}

// Phase B: bin each admitted request into its arena range, then one forward raster launch
// (and one backward raster launch) per feature layout for the whole batch.
void launch(gs_server* sv, int lane, std::vector<gs_serve::Item<gs_request>>& items) {
  cudaSetDevice(sv->device);
  Lane& ln = sv->lanes[lane];
  std::map<Grouping, std::vector<std::pair<size_t, RasterJob>>> fwd, bwd;
  for (size_t k = 0; k < items.size(); ++k) {
    auto& it = items[k];
    gs_workspace* ws = ln.ws[(size_t)it.slot];
    const gs_scene sc = scene_of(sv, it.req.scene_id);
    const int64_t o = it.offset;
    gs::ws_lend_instances(ws, sv->kv + o, sv->arr[0] + o, sv->arr[1] + o, it.cost);
    gs_status s = gs_bin_tiles(ws, nullptr, ln.stream);
    RasterJob j;
    if (s == GS_OK) s = gs::ws_job(ws, sc, &j);
    if (s != GS_OK) {
      it.status = s;
      continue;
    }
    const gs_request& r = it.req;
    const int D = sc.n_feat;
    j.rgb = r.rgb;
    j.depth = r.depth;
    j.alpha = r.alpha;
    j.feat = D > 0 ? r.feat : nullptr;
    fwd[Grouping{j.feat ? gs::padded_feat(D) : 0, sc.feat_dtype}].push_back({k, j});
    if (r.want_bwd) {
      if ((s = gs::ws_bwd_clear(ws, D, D > 0 ? r.g_feats : nullptr, ln.stream)) != GS_OK) {
        it.status = s;
        continue;
      }
      j.g_rgb = r.g_rgb;
      j.g_depth = r.g_depth;
      j.g_alpha = r.g_alpha;
      j.g_feat = D > 0 ? r.g_feat : nullptr;
      j.g_feats = D > 0 ? r.g_feats : nullptr;
      bwd[Grouping{j.g_feat ? gs::padded_feat(D) : 0, sc.feat_dtype}].push_back({k, j});
    }
  }
  const gs::TileQueue fq{ln.queue, ln.queue + 1, nullptr, 0};
  for (auto& g : fwd) {
    std::vector<RasterJob> jobs;
    int end = 0;
    for (auto& e : g.second) {
      if (items[e.first].status != GS_OK) continue;
      end += gs::kFwdItemsPerTile * e.second.cam.TX * e.second.cam.TY;
      e.second.item_end = end;
      jobs.push_back(e.second);
    }
    gs::launch_raster_fwd_jobs(jobs.data(), (int)jobs.size(), g.first.dtype, g.first.dp > 0, fq,
                               ln.stream);
  }
  const gs::TileQueue bq{ln.queue + 2, ln.queue + 3, nullptr, 0};
  for (auto& g : bwd) {
    std::vector<RasterJob> jobs;
    int end = 0;
    for (auto& e : g.second) {
      if (items[e.first].status != GS_OK) continue;
      end += e.second.cam.TX * e.second.cam.TY;
      e.second.item_end = end;
      jobs.push_back(e.second);
    }
    if (jobs.empty()) continue;
    // the backward kernels leave their queue to the host: zeroed before each launch
    cudaMemsetAsync(ln.queue + 2, 0, 8, ln.stream);
    gs::launch_raster_bwd_jobs(jobs.data(), (int)jobs.size(), g.first.dtype, g.first.dp > 0, bq,
                               ln.stream);
  }
  for (auto& it : items) {
    const gs_request& r = it.req;
    if (!r.want_bwd || it.status != GS_OK) continue;
    const gs_scene sc = scene_of(sv, r.scene_id);
    it.status = gs::ws_project_bwd(ln.ws[(size_t)it.slot], sc, r.g_means, r.g_scales, r.g_quats,
                                   r.g_opac, r.g_sh, r.g_pose6, ln.stream);
  }
  if (cudaGetLastError() != cudaSuccess)
    for (auto& it : items) it.status = it.status ? it.status : GS_ERR_CUDA;
  cudaEventRecord(ln.done, ln.stream);
}

void finish(gs_server* sv, int lane, std::vector<gs_serve::Item<gs_request>>& items) {
  cudaSetDevice(sv->device);
  Lane& ln = sv->lanes[lane];
  const bool ok = cudaEventSynchronize(ln.done) == cudaSuccess;
  for (auto& it : items) {
    it.instances = it.cost;
    if (it.status != GS_OK) continue;
    if (!ok) {
      it.status = GS_ERR_CUDA;
      continue;
    }
    it.status = gs_workspace_status(ln.ws[(size_t)it.slot], ln.stream);
  }
}

void free_lanes(gs_server* sv) {
  for (Lane& ln : sv->lanes) {
    for (gs_workspace* w : ln.ws) gs_workspace_destroy(w);
    ln.ws.clear();
    if (ln.queue) cudaFree(ln.queue);
    if (ln.h_inst) cudaFreeHost(ln.h_inst);
    if (ln.done) cudaEventDestroy(ln.done);
    if (ln.stream) cudaStreamDestroy(ln.stream);
    ln = Lane{};
  }
}

// Start-up at the first request (under sv->mu): reserve the request workspaces (half of
// the budget left after the scenes at most) and give the rest to the instance arena.
gs_status start_locked(gs_server* sv) {
  if (sv->started) return GS_OK;
  if (sv->scenes.empty()) return GS_ERR_STATE;
  cudaSetDevice(sv->device);
  const int nws = sv->n_lanes * sv->slots_per_lane;
  const int64_t left = sv->budget - sv->scene_bytes;
  const int64_t per_ws = left / 2 / nws - sv->max_n * kGaussBytes;
  int64_t pix = std::min<int64_t>(kMaxPixPerRequest, per_ws / (kPixBytes + 1));
  if (pix < kMinPixPerRequest) return GS_ERR_OVER_BUDGET;
  const int64_t tiles = pix / 256 + 4096;
  int64_t fixed = 0;
  for (int l = 0; l < sv->n_lanes; ++l) {
    Lane& ln = sv->lanes[l];
    if (cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ln.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&ln.h_inst, sizeof(uint32_t) * gs::kMaxJobs) != cudaSuccess ||
        cudaMalloc(&ln.queue, 4 * sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(ln.queue, 0, 4 * sizeof(uint32_t)) != cudaSuccess) {
      free_lanes(sv);
      return GS_ERR_OOM;
    }
    fixed += 16;
    for (int k = 0; k < sv->slots_per_lane; ++k) {
      gs_workspace* w = nullptr;
      gs_status s = gs_workspace_create(&w, sv->device);
      if (s == GS_OK) {
        ln.ws.push_back(w);
        s = gs::ws_reserve_fixed(w, sv->max_n, pix, tiles);
      }
      int64_t b = 0;
      if (s == GS_OK) s = gs_workspace_bytes(w, &b);
      if (s != GS_OK) {
        free_lanes(sv);
        return s == GS_ERR_OOM ? GS_ERR_OVER_BUDGET : s;
      }
      fixed += b;
    }
  }
  const int64_t arena_bytes = left - fixed;
  int64_t inst = std::min<int64_t>(arena_bytes / kInstBytes, (int64_t(1) << 31) - 1);
  inst = inst / 64 * 64;
  if (inst < 1024) {
    free_lanes(sv);
    return GS_ERR_OVER_BUDGET;
  }
  if (cudaMalloc(&sv->arena, (size_t)inst * kInstBytes) != cudaSuccess) {
    free_lanes(sv);
    return GS_ERR_OOM;
  }
  sv->kv = static_cast<uint2*>(sv->arena);
  for (int k = 0; k < 2; ++k) sv->arr[k] = reinterpret_cast<uint32_t*>(sv->kv + inst) + (size_t)k * inst;
  if (cudaDeviceSynchronize() != cudaSuccess) return GS_ERR_CUDA;
  sv->pix_cap = pix;
  sv->tile_cap = tiles;
  sv->fixed_bytes = fixed;
  sv->arena_inst = inst;
  gs_serve::Executor<gs_request> ex;
  ex.measure = [sv](int l, std::vector<gs_serve::Item<gs_request>>& b) { measure(sv, l, b); };
  ex.launch = [sv](int l, std::vector<gs_serve::Item<gs_request>>& b) { launch(sv, l, b); };
  ex.finish = [sv](int l, std::vector<gs_serve::Item<gs_request>>& b) { finish(sv, l, b); };
  sv->sched.reset(new gs_serve::Scheduler<gs_request>(sv->n_lanes, sv->slots_per_lane, inst, kAgingS, ex));
  sv->started = true;
  return GS_OK;
}

}  // namespace

extern "C" {

gs_status gs_serve_create(gs_server** out, int device, int64_t hbm_budget_bytes, int max_slots) {
  if (!out || hbm_budget_bytes <= 0 || max_slots <= 0 || max_slots > 64) return GS_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return GS_ERR_CUDA;
  gs_server* sv = new (std::nothrow) gs_server();
  if (!sv) return GS_ERR_OOM;
  sv->device = device;
  sv->budget = hbm_budget_bytes;
  // up to four lanes (independent pipelines on the device), the rest as batch width
  sv->n_lanes = std::min(kMaxLanes, max_slots);
  sv->slots_per_lane = std::max(1, std::min(gs::kMaxJobs, (max_slots + sv->n_lanes - 1) / sv->n_lanes));
  *out = sv;
  return GS_OK;
}

void gs_serve_destroy(gs_server* sv) {
  if (!sv) return;
  sv->sched.reset();   // joins the dispatcher and lanes; pending requests are cancelled
  cudaSetDevice(sv->device);
  free_lanes(sv);
  if (sv->arena) cudaFree(sv->arena);
  for (SceneStore& s : sv->scenes)
    for (void* p : s.buffers) cudaFree(p);
  delete sv;
}

gs_status gs_serve_add_scene(gs_server* sv, const gs_scene* scene, int* scene_id) {
  if (!sv || !scene || !scene_id || scene->n <= 0 || scene->sh_degree < 0 || scene->sh_degree > 3 ||
      scene->n_feat < 0 || scene->n_feat > gs::kMaxFeat ||
      (scene->feat_dtype != GS_F32 && scene->feat_dtype != GS_BF16))
    return GS_ERR_ARG;
  const int64_t n = scene->n;
  const int K = (scene->sh_degree + 1) * (scene->sh_degree + 1);
  const size_t sizes[6] = {(size_t)n * 12, (size_t)n * 12, (size_t)n * 16, (size_t)n * 4,
                           (size_t)n * K * 12, (size_t)n * scene->n_feat * feat_elem_bytes(*scene)};
  const void* src[6] = {scene->means, scene->scales, scene->quats, scene->opacities, scene->sh,
                        scene->feats};
  size_t total = 0;
  for (size_t b : sizes) total += b;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->started) return GS_ERR_STATE;   // the budget was divided at the first request
  if (sv->scene_bytes + (int64_t)total > sv->budget) return GS_ERR_OVER_BUDGET;
  cudaSetDevice(sv->device);
  SceneStore st;
  void* dst[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  for (int k = 0; k < 6; ++k) {
    if (sizes[k] == 0) continue;
    if (!src[k] || cudaMalloc(&dst[k], sizes[k]) != cudaSuccess ||
        cudaMemcpy(dst[k], src[k], sizes[k], cudaMemcpyDeviceToDevice) != cudaSuccess) {
      for (void* p : dst)
        if (p) cudaFree(p);
      return src[k] ? GS_ERR_OOM : GS_ERR_ARG;
    }
    st.buffers.push_back(dst[k]);
  }
  st.view = *scene;
  st.view.means = static_cast<const float*>(dst[0]);
  st.view.scales = static_cast<const float*>(dst[1]);
  st.view.quats = static_cast<const float*>(dst[2]);
  st.view.opacities = static_cast<const float*>(dst[3]);
  st.view.sh = static_cast<const float*>(dst[4]);
  st.view.feats = dst[5];
  st.bytes = total;
  sv->scene_bytes += (int64_t)total;
  sv->max_n = std::max<int64_t>(sv->max_n, n);
  sv->scenes.push_back(st);
  *scene_id = (int)sv->scenes.size() - 1;
  return GS_OK;
}

gs_status gs_serve_submit(gs_server* sv, const gs_request* req, uint64_t* ticket) {
  if (!sv || !req || !ticket) return GS_ERR_ARG;
  gs_serve::Scheduler<gs_request>* sched = nullptr;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (req->scene_id < 0 || req->scene_id >= (int)sv->scenes.size()) return GS_ERR_ARG;
    const gs_camera& c = req->cam;
    if (c.W <= 0 || c.H <= 0 || c.tile != gs::kTile || !(c.fx > 0.f) || !(c.fy > 0.f) ||
        !(c.near_z > 0.f) || c.stride != 1 || c.off_x != 0 || c.off_y != 0)
      return GS_ERR_ARG;
    if (req->want_bwd && (!req->g_rgb && !req->g_depth && !req->g_alpha && !req->g_feat))
      return GS_ERR_ARG;
    gs_status s = start_locked(sv);
    if (s != GS_OK) return s;
    if ((int64_t)c.W * c.H > sv->pix_cap || tiles_of(c.W, c.H) > sv->tile_cap)
      return GS_ERR_OVER_BUDGET;
    sched = sv->sched.get();
  }
  return (gs_status)sched->submit(*req, 0, ticket);
}

gs_status gs_serve_poll(gs_server* sv, uint64_t ticket, int64_t timeout_us, gs_result* out) {
  if (!sv) return GS_ERR_ARG;
  if (!sv->sched) return GS_ERR_ARG;   // no request was ever submitted
  gs_serve::Result r;
  const int s = sv->sched->poll(ticket, timeout_us, &r);
  if (s != 0) return (gs_status)s;
  if (out) {
    out->status = (gs_status)r.status;
    out->slot = r.slot;
    out->instances = r.instances;
    out->queue_us = r.queue_us;
    out->run_us = r.run_us;
    out->latency_us = r.latency_us;
  }
  return GS_OK;
}

gs_status gs_serve_cancel(gs_server* sv, uint64_t ticket) {
  if (!sv || !sv->sched) return GS_ERR_ARG;
  return (gs_status)sv->sched->cancel(ticket);
}

gs_status gs_serve_info(gs_server* sv, int64_t* scene_bytes, int64_t* in_flight_bytes,
                        int64_t* peak_in_flight_bytes, int32_t* peak_running) {
  if (!sv) return GS_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (scene_bytes) *scene_bytes = sv->scene_bytes;
  }
  gs_serve::Scheduler<gs_request>* s = sv->sched.get();
  if (in_flight_bytes) *in_flight_bytes = s ? s->arena_used() * kInstBytes : 0;
  if (peak_in_flight_bytes) *peak_in_flight_bytes = s ? s->arena_peak() * kInstBytes : 0;
  if (peak_running) *peak_running = s ? s->peak_running() : 0;
  return GS_OK;
}

gs_status gs_serve_stats(gs_server* sv, gs_serve_stats_t* out) {
  if (!sv || !out) return GS_ERR_ARG;
  std::memset(out, 0, sizeof(*out));
  std::lock_guard<std::mutex> lk(sv->mu);
  out->scene_bytes = sv->scene_bytes;
  out->workspace_bytes = sv->fixed_bytes;
  out->arena_bytes = sv->arena_inst * kInstBytes;
  out->max_pixels = sv->pix_cap;
  out->lanes = sv->started ? sv->n_lanes : 0;
  out->slots_per_lane = sv->slots_per_lane;
  if (gs_serve::Scheduler<gs_request>* s = sv->sched.get()) {
    out->arena_peak_bytes = s->arena_peak() * kInstBytes;
    out->batches = s->batches();
    out->peak_batch = s->peak_batch();
    out->peak_running = s->peak_running();
  }
  return GS_OK;
}

}  // extern "C"
