// Serving: resident scenes, continuous admission by an HBM budget, overlapping execution.
//
// A server owns copies of the scenes it serves (device memory counted against its
// budget) and a pool of slots.  Each slot is a worker thread with its own CUDA stream and
// workspace; a worker takes the oldest pending request whose memory estimate fits what is
// left of the budget and runs project -> bin -> render (-> backward) on its stream, so
// requests that arrive while others are on the GPU are admitted as soon as a slot and the
// memory free up and their kernels overlap with the running ones.  Results are
// bit-identical to the same request rendered alone (forward) and equal within atomic
// reordering (backward).
#include <algorithm>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "gs_internal.cuh"
#include "serve_core.hpp"

namespace {

struct SceneStore {
  gs_scene view;                   // points at the buffers below
  std::vector<void*> buffers;
  size_t bytes = 0;
};

struct Slot {
  gs_workspace* ws = nullptr;
  cudaStream_t stream = nullptr;
  int64_t res_n = 0, res_pix = 0;   // what the workspace was last reserved for (worker-owned)
};

size_t feat_elem_bytes(const gs_scene& s) { return s.feat_dtype == GS_BF16 ? 2 : 4; }

}  // namespace

struct gs_server {
  int device = 0;
  int64_t budget = 0;
  std::mutex mu;                   // scenes
  std::vector<SceneStore> scenes;
  int64_t scene_bytes = 0;
  int64_t max_n = 0;               // largest resident scene
  std::vector<Slot> slots;
  std::unique_ptr<gs_serve::Scheduler<gs_request>> sched;
};

namespace {

// Admission estimate of the device memory a request's intermediates need: per Gaussian
// ~112 bytes (record, keys, sort buffers, gradient accumulators), per pixel 12 bytes,
// per tile instance 16 bytes with an assumed 8 instances per Gaussian.
int64_t request_cost(const gs_scene& s, const gs_camera& c) {
  return s.n * 112 + (int64_t)c.W * c.H * 12 + s.n * 8 * 16 + (1 << 20);
}

int run_request(gs_server* sv, int slot, const gs_request& r, int64_t* instances) {
  cudaSetDevice(sv->device);
  Slot& sl = sv->slots[slot];
  gs_scene sc;
  int64_t max_n;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (r.scene_id < 0 || r.scene_id >= (int)sv->scenes.size()) return GS_ERR_ARG;
    sc = sv->scenes[r.scene_id].view;
    max_n = sv->max_n;
  }
  // Grow this slot's workspace to the largest resident scene at once (and to the pixel
  // count with headroom), so that the device-wide synchronisation of a reallocation
  // happens rarely rather than whenever a slot meets a larger scene or frame.
  const int64_t pix = (int64_t)r.cam.W * r.cam.H;
  if (max_n > sl.res_n || pix > sl.res_pix) {
    const int64_t want_pix = std::max<int64_t>(sl.res_pix, pix + pix / 4);
    gs_status s = gs_workspace_reserve(sl.ws, max_n, 0, want_pix);
    if (s != GS_OK) return s;
    sl.res_n = max_n;
    sl.res_pix = want_pix;
  }
  gs_status s = gs_project(&sc, &r.cam, sl.ws, sl.stream);
  if (s != GS_OK) return s;
  if ((s = gs_bin_tiles(sl.ws, instances, sl.stream)) != GS_OK) return s;
  if ((s = gs_render_fwd(&sc, &r.cam, sl.ws, r.rgb, r.depth, r.alpha, r.feat, sl.stream)) != GS_OK)
    return s;
  if (r.want_bwd &&
      (s = gs_render_bwd(&sc, &r.cam, sl.ws, r.g_rgb, r.g_depth, r.g_alpha, r.g_feat, r.g_means,
                         r.g_scales, r.g_quats, r.g_opac, r.g_sh, r.g_feats, r.g_pose6,
                         sl.stream)) != GS_OK)
    return s;
  if (cudaStreamSynchronize(sl.stream) != cudaSuccess) return GS_ERR_CUDA;
  return gs_workspace_status(sl.ws, sl.stream);
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
  cudaSetDevice(device);
  for (int i = 0; i < max_slots; ++i) {
    Slot sl;
    if (gs_workspace_create(&sl.ws, device) != GS_OK ||
        cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
      if (sl.ws) gs_workspace_destroy(sl.ws);
      for (Slot& o : sv->slots) {
        gs_workspace_destroy(o.ws);
        cudaStreamDestroy(o.stream);
      }
      delete sv;
      return GS_ERR_CUDA;
    }
    sv->slots.push_back(sl);
  }
  sv->sched.reset(new gs_serve::Scheduler<gs_request>(
      max_slots, hbm_budget_bytes,
      [sv](int slot, const gs_request& r, int64_t* inst) { return run_request(sv, slot, r, inst); }));
  *out = sv;
  return GS_OK;
}

void gs_serve_destroy(gs_server* sv) {
  if (!sv) return;
  sv->sched.reset();   // joins the workers; pending requests are cancelled
  cudaSetDevice(sv->device);
  for (Slot& o : sv->slots) {
    gs_workspace_destroy(o.ws);
    cudaStreamDestroy(o.stream);
  }
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
  sv->sched->set_budget(sv->budget - sv->scene_bytes);
  return GS_OK;
}

gs_status gs_serve_submit(gs_server* sv, const gs_request* req, uint64_t* ticket) {
  if (!sv || !req || !ticket) return GS_ERR_ARG;
  gs_scene sc;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (req->scene_id < 0 || req->scene_id >= (int)sv->scenes.size()) return GS_ERR_ARG;
    sc = sv->scenes[req->scene_id].view;
  }
  const gs_camera& c = req->cam;
  if (c.W <= 0 || c.H <= 0 || c.tile != gs::kTile || !(c.fx > 0.f) || !(c.fy > 0.f)) return GS_ERR_ARG;
  if (req->want_bwd && (!req->g_rgb && !req->g_depth && !req->g_alpha && !req->g_feat)) return GS_ERR_ARG;
  const int64_t room = sv->budget - sv->scene_bytes;
  const int64_t cost = request_cost(sc, c);
  if (cost > room) return GS_ERR_OVER_BUDGET;
  const int s = sv->sched->submit(*req, cost, ticket);
  return (gs_status)s;
}

gs_status gs_serve_poll(gs_server* sv, uint64_t ticket, int64_t timeout_us, gs_result* out) {
  if (!sv) return GS_ERR_ARG;
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
  if (!sv) return GS_ERR_ARG;
  return (gs_status)sv->sched->cancel(ticket);
}

gs_status gs_serve_info(gs_server* sv, int64_t* scene_bytes, int64_t* in_flight_bytes,
                        int64_t* peak_in_flight_bytes, int32_t* peak_running) {
  if (!sv) return GS_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (scene_bytes) *scene_bytes = sv->scene_bytes;
  }
  if (in_flight_bytes) *in_flight_bytes = sv->sched->in_flight_bytes();
  if (peak_in_flight_bytes) *peak_in_flight_bytes = sv->sched->peak_in_flight_bytes();
  if (peak_running) *peak_running = sv->sched->peak_running();
  return GS_OK;
}

}  // extern "C"
