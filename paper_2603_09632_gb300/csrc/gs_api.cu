// C ABI of libgs: workspace management and the entry points declared in include/gs.h.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "gs_internal.cuh"
#include "gs_serve_ws.hpp"

using namespace gs;

namespace gs {
static std::atomic<int64_t> g_launches{0};
void note_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int resident_ctas(const void* kern, int threads, size_t smem) {
  struct Entry {
    const void* kern;
    int threads;
    size_t smem;
    int dev;
    int ctas;
  };
  static std::mutex mu;   // the serving threads launch concurrently
  static std::vector<Entry> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(mu);
    for (const Entry& e : cache)
      if (e.kern == kern && e.threads == threads && e.smem == smem && e.dev == dev) return e.ctas;
  }
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (smem > 0) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  const int ctas = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  std::lock_guard<std::mutex> lk(mu);
  cache.push_back(Entry{kern, threads, smem, dev, ctas});
  return ctas;
}
}  // namespace gs

namespace {

template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t cap = 0;      // elements
  bool owned = true;   // false: memory lent by the caller (a serving arena range)
  cudaError_t ensure(size_t n) {
    if (n <= cap) return cudaSuccess;
    // a buffer that has to grow grows by at least a quarter, so that sizes drifting upwards
    // (instance counts over a trajectory) do not reallocate (and synchronise) every call
    const size_t m = std::max<size_t>(std::max<size_t>(n, 16), cap + cap / 4);
    if (p && owned) cudaFree(p);
    p = nullptr;
    cap = 0;
    owned = true;
    cudaError_t e = cudaMalloc(&p, m * sizeof(T));
    if (e == cudaSuccess) cap = m;
    return e;
  }
  void lend(T* q, size_t n) {
    release();
    p = q;
    cap = n;
    owned = false;
  }
  // as ensure(), and a (re)allocated buffer is filled with zeros
  cudaError_t ensure_zeroed(size_t n) {
    if (n <= cap) return cudaSuccess;
    cudaError_t e = ensure(n);
    return e == cudaSuccess ? cudaMemset(p, 0, cap * sizeof(T)) : e;
  }
  void release() {
    if (p && owned) cudaFree(p);
    p = nullptr;
    cap = 0;
    owned = true;
  }
};

constexpr int kTimerRing = 256;

}  // namespace

struct gs_workspace {
  int device = 0;
  // per Gaussian
  DevBuf<GaussRec> rec;
  DevBuf<uint32_t> depth_key, ntiles;
  DevBuf<uint2> rect;
  DevBuf<uint32_t> item_max;   // per grid work item, statistics only
  bool tile_counts_dirty = false;   // tile_count holds a projection's counts not yet scanned
  DevBuf<float> g2d;
  DevBuf<float> pose_partials;
  // per instance: sorted depth keys and ids, their ping-pong space, the slot's tile
  DevBuf<uint32_t> inst_key, inst_id;   // sort scratch keys, sorted ids
  DevBuf<uint2> inst_kv;                 // scattered (key, id) pairs
  // per tile / pixel
  DevBuf<uint2> ranges;
  DevBuf<uint32_t> tile_order, queue;   // heavy-first tile order; persistent-kernel queues
                                        // (head, leave count): fwd [0, 1], bwd [2, 3], sort [4, 5]
  DevBuf<uint32_t> tile_count, tile_cursor;   // binning scratch
  bool ordered = false;
  DevBuf<float> T_final;
  DevBuf<uint32_t> n_contrib;
  // scratch
  DevBuf<uint32_t> counters;
  DevBuf<unsigned long long> stats64;     // pair counts (statistics only)
  CamDev cam{};                           // camera of the last gs_project
  uint32_t* h_counters = nullptr;   // pinned mirror
  // state
  int64_t n = 0;
  int W = 0, H = 0, TX = 0, TY = 0;
  int stage = 0;             // 1 projected, 2 binned, 3 rendered
  int64_t inst_bound = 0;    // host bound on I used for grids
  const uint32_t* id_sorted = nullptr;    // Gaussian id of every instance slot
  // timing
  bool timing = false;
  cudaEvent_t ev[GS_NUM_TIMERS][kTimerRing][2];
  int ev_count[GS_NUM_TIMERS] = {0};
  bool ev_created = false;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

gs_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return GS_OK;
  if (e == cudaErrorMemoryAllocation) return GS_ERR_OOM;
  return GS_ERR_CUDA;
}

#define GS_TRY(expr)                              \
  do {                                            \
    cudaError_t _e = (expr);                      \
    if (_e != cudaSuccess) return cuda_status(_e); \
  } while (0)

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

gs_status check_scene(const gs_scene* sc) {
  if (!sc) return GS_ERR_ARG;
  if (sc->n < 0 || sc->n >= (int64_t(1) << 31)) return GS_ERR_ARG;
  if (sc->sh_degree < 0 || sc->sh_degree > 3) return GS_ERR_ARG;
  if (sc->n_feat < 0 || sc->n_feat > kMaxFeat) return GS_ERR_ARG;
  if (sc->feat_dtype != GS_F32 && sc->feat_dtype != GS_BF16) return GS_ERR_ARG;
  if (sc->n > 0) {
    if (!sc->means || !sc->scales || !sc->quats || !sc->opacities || !sc->sh) return GS_ERR_ARG;
    if (sc->n_feat > 0 && !sc->feats) return GS_ERR_ARG;
    if (!aligned16(sc->means) || !aligned16(sc->scales) || !aligned16(sc->quats) ||
        !aligned16(sc->sh) || (sc->feats && !aligned16(sc->feats)))
      return GS_ERR_ARG;
  }
  return GS_OK;
}

gs_status make_cam(const gs_camera* c, CamDev* out) {
  if (!c) return GS_ERR_ARG;
  if (c->W <= 0 || c->H <= 0 || c->W > 65535 * kTile || c->H > 65535 * kTile) return GS_ERR_ARG;
  if (c->tile != kTile) return GS_ERR_ARG;
  if ((int64_t)((c->W + kTile - 1) / kTile) * ((c->H + kTile - 1) / kTile) > (int64_t(1) << 24))
    return GS_ERR_ARG;
  if (!(c->fx > 0.f) || !(c->fy > 0.f) || !(c->near_z > 0.f)) return GS_ERR_ARG;
  // rendered pixels: the image (stride 1) or the stride-s sample grid with offsets in
  // [0, s) (App. D), of fixed size ceil(H / s) x ceil(W / s)
  if (c->stride < 1 || c->stride > kMaxStride || c->off_x < 0 || c->off_x >= c->stride ||
      c->off_y < 0 || c->off_y >= c->stride)
    return GS_ERR_ARG;
  out->W = c->W;
  out->H = c->H;
  out->TX = (c->W + kTile - 1) / kTile;
  out->TY = (c->H + kTile - 1) / kTile;
  out->stride = c->stride;
  out->ox = c->off_x;
  out->oy = c->off_y;
  out->GW = (c->W + c->stride - 1) / c->stride;
  out->GH = (c->H + c->stride - 1) / c->stride;
  out->fx = c->fx;
  out->fy = c->fy;
  out->cx = c->cx;
  out->cy = c->cy;
  std::memcpy(out->R, c->R, sizeof(out->R));
  std::memcpy(out->t, c->t, sizeof(out->t));
  out->near_z = c->near_z;
  return GS_OK;
}

// Same image and the same rendered grid (a render must use the projection's grid).
bool same_grid(const CamDev& a, const CamDev& b) {
  return a.W == b.W && a.H == b.H && a.stride == b.stride && a.ox == b.ox && a.oy == b.oy;
}

struct StageTimer {
  gs_workspace* ws;
  int which;
  cudaStream_t st;
  int slot = -1;
  StageTimer(gs_workspace* w, int k, cudaStream_t s) : ws(w), which(k), st(s) {
    if (ws->timing && ws->ev_count[k] < kTimerRing) {
      slot = ws->ev_count[k]++;
      cudaEventRecord(ws->ev[k][slot][0], st);
    }
  }
  ~StageTimer() {
    if (slot >= 0) cudaEventRecord(ws->ev[which][slot][1], st);
  }
};

cudaError_t ensure_gauss(gs_workspace* ws, int64_t n) {
  const size_t m = (size_t)std::max<int64_t>(n, 1);
  cudaError_t e;
  if ((e = ws->rec.ensure(m)) || (e = ws->depth_key.ensure(m)) || (e = ws->ntiles.ensure(m)) ||
      (e = ws->rect.ensure(m)) || (e = ws->g2d.ensure(m * kG2D)) ||
      (e = ws->pose_partials.ensure((size_t)project_bwd_blocks(n) * 8)))
    return e;
  return cudaSuccess;
}

cudaError_t ensure_inst(gs_workspace* ws, int64_t cap) {
  const size_t m = (size_t)std::max<int64_t>(cap, 1);
  cudaError_t e;
  if ((e = ws->inst_key.ensure(m)) || (e = ws->inst_id.ensure(m)) || (e = ws->inst_kv.ensure(m)))
    return e;
  return cudaSuccess;
}

cudaError_t ensure_pix(gs_workspace* ws, int64_t npix, int64_t ntiles) {
  cudaError_t e;
  if ((e = ws->T_final.ensure((size_t)std::max<int64_t>(npix, 1))) ||
      (e = ws->n_contrib.ensure((size_t)std::max<int64_t>(npix, 1))))
    return e;
  const size_t t = (size_t)std::max<int64_t>(ntiles, 1);
  // the tile counts are kept as per-row differences: TY (TX + 1) <= 2 TX TY words
  if ((e = ws->tile_order.ensure(t)) || (e = ws->tile_count.ensure_zeroed(2 * t)) ||
      (e = ws->tile_cursor.ensure(t)))
    return e;
  return ws->ranges.ensure(t);
}

}  // namespace

extern "C" {

const char* gs_status_string(gs_status s) {
  switch (s) {
    case GS_OK: return "ok";
    case GS_ERR_ARG: return "invalid argument";
    case GS_ERR_OOM: return "out of device memory";
    case GS_ERR_CUDA: return "CUDA runtime error";
    case GS_ERR_DEVICE: return "device-side error";
    case GS_ERR_TIMEOUT: return "timeout";
    case GS_ERR_BUSY: return "busy";
    case GS_ERR_OVER_BUDGET: return "over memory budget";
    case GS_ERR_STATE: return "calls out of order";
    case GS_ERR_CANCELLED: return "cancelled";
  }
  return "unknown status";
}

gs_status gs_workspace_create(gs_workspace** out, int device) {
  if (!out) return GS_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return GS_ERR_CUDA;
  gs_workspace* ws = new (std::nothrow) gs_workspace();
  if (!ws) return GS_ERR_OOM;
  ws->device = device;
  DeviceGuard g(device);
  if (ws->counters.ensure(kCntNum) != cudaSuccess || ws->queue.ensure(8) != cudaSuccess ||
      cudaMemset(ws->counters.p, 0, kCntNum * sizeof(uint32_t)) != cudaSuccess ||
      cudaMemset(ws->queue.p, 0, 8 * sizeof(uint32_t)) != cudaSuccess ||
      cudaMallocHost(&ws->h_counters, kCntNum * sizeof(uint32_t)) != cudaSuccess) {
    gs_workspace_destroy(ws);
    return GS_ERR_OOM;
  }
  *out = ws;
  return GS_OK;
}

void gs_workspace_destroy(gs_workspace* ws) {
  if (!ws) return;
  {
    DeviceGuard g(ws->device);
    cudaDeviceSynchronize();
    ws->rec.release(); ws->depth_key.release(); ws->ntiles.release();
    ws->rect.release(); ws->item_max.release(); ws->g2d.release(); ws->pose_partials.release();
    ws->inst_key.release(); ws->inst_id.release(); ws->inst_kv.release();
    ws->ranges.release(); ws->T_final.release(); ws->n_contrib.release();
    ws->tile_order.release(); ws->queue.release(); ws->tile_count.release(); ws->tile_cursor.release();
    ws->counters.release(); ws->stats64.release();
    if (ws->h_counters) cudaFreeHost(ws->h_counters);
    if (ws->ev_created)
      for (int k = 0; k < GS_NUM_TIMERS; ++k)
        for (int s = 0; s < kTimerRing; ++s) {
          cudaEventDestroy(ws->ev[k][s][0]);
          cudaEventDestroy(ws->ev[k][s][1]);
        }
  }
  delete ws;
}

gs_status gs_workspace_reserve(gs_workspace* ws, int64_t n_gauss, int64_t n_instances,
                               int64_t n_pixels) {
  if (!ws || n_gauss < 0 || n_instances < 0 || n_pixels < 0) return GS_ERR_ARG;
  DeviceGuard g(ws->device);
  GS_TRY(ensure_gauss(ws, n_gauss));
  GS_TRY(ensure_inst(ws, n_instances));
  GS_TRY(ensure_pix(ws, n_pixels, gs::ceil_div(n_pixels, 256) + 4096));
  GS_TRY(cudaDeviceSynchronize());
  return GS_OK;
}

gs_status gs_workspace_status(gs_workspace* ws, void* stream) {
  if (!ws) return GS_ERR_ARG;
  DeviceGuard g(ws->device);
  cudaStream_t st = (cudaStream_t)stream;
  GS_TRY(cudaMemcpyAsync(ws->h_counters, ws->counters.p, kCntNum * sizeof(uint32_t),
                         cudaMemcpyDeviceToHost, st));
  GS_TRY(cudaStreamSynchronize(st));
  const uint32_t s = ws->h_counters[kCntStatus];
  if (s) {
    GS_TRY(cudaMemsetAsync(ws->counters.p + kCntStatus, 0, 4, st));
    GS_TRY(cudaStreamSynchronize(st));
    return GS_ERR_DEVICE;
  }
  return GS_OK;
}

gs_status gs_workspace_bytes(gs_workspace* ws, int64_t* bytes) {
  if (!ws || !bytes) return GS_ERR_ARG;
  size_t b = 0;
  auto add = [&b](const auto& buf) { b += buf.cap * sizeof(*buf.p); };
  add(ws->rec); add(ws->depth_key); add(ws->ntiles); add(ws->rect); add(ws->item_max);
  add(ws->g2d); add(ws->pose_partials);
  add(ws->inst_key); add(ws->inst_id); add(ws->inst_kv);
  add(ws->ranges); add(ws->tile_order); add(ws->queue); add(ws->tile_count); add(ws->tile_cursor);
  add(ws->T_final); add(ws->n_contrib); add(ws->counters); add(ws->stats64);
  *bytes = (int64_t)b;
  return GS_OK;
}

gs_status gs_project(const gs_scene* scene, const gs_camera* cam, gs_workspace* ws, void* stream) {
  if (!ws) return GS_ERR_ARG;
  gs_status s = check_scene(scene);
  if (s != GS_OK) return s;
  CamDev cd;
  if ((s = make_cam(cam, &cd)) != GS_OK) return s;
  cd.n_gauss = (int)scene->n;
  DeviceGuard g(ws->device);
  cudaStream_t st = (cudaStream_t)stream;
  GS_TRY(ensure_gauss(ws, scene->n));
  GS_TRY(ensure_pix(ws, (int64_t)cd.GW * cd.GH, (int64_t)cd.TX * cd.TY));
  StageTimer tm(ws, GS_TIMER_PROJECT, st);
  GS_TRY(cudaMemsetAsync(ws->counters.p + kCntVisible, 0, 2 * sizeof(uint32_t), st));
  // the tile counts are zero unless a projection was not followed by a binning (whose scan
  // clears them after reading)
  if (ws->tile_counts_dirty)
    GS_TRY(cudaMemsetAsync(ws->tile_count.p, 0, sizeof(uint32_t) * ws->tile_count.cap, st));
  launch_project(*scene, cd, ws->rec.p, ws->depth_key.p, ws->ntiles.p, ws->rect.p, ws->counters.p,
                 ws->tile_count.p, st);
  ws->tile_counts_dirty = true;
  GS_TRY(cudaGetLastError());
  ws->n = scene->n;
  ws->cam = cd;
  // W, H: the rendered pixels (the compact grid at stride > 1); TX, TY: the image tiles in
  // which Gaussians are binned
  ws->W = cd.GW;
  ws->H = cd.GH;
  ws->TX = cd.TX;
  ws->TY = cd.TY;
  ws->stage = 1;
  return GS_OK;
}

gs_status gs_bin_tiles(gs_workspace* ws, int64_t* n_instances_out, void* stream) {
  if (!ws) return GS_ERR_ARG;
  if (ws->stage < 1) return GS_ERR_STATE;
  DeviceGuard g(ws->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (ws->stage >= 2 && !ws->tile_counts_dirty) {
    // this projection is binned already (its scan consumed the tile counts): nothing to redo
    if (n_instances_out) {
      GS_TRY(cudaMemcpyAsync(ws->h_counters, ws->counters.p, kCntNum * sizeof(uint32_t),
                             cudaMemcpyDeviceToHost, st));
      GS_TRY(cudaStreamSynchronize(st));
      *n_instances_out = (int64_t)ws->h_counters[kCntInst];
    }
    return GS_OK;
  }
  const int64_t n = ws->n;
  const int ntl = ws->TX * ws->TY;
  StageTimer tm(ws, GS_TIMER_BIN, st);
  uint32_t* cnt = ws->counters.p;
  int64_t bound;
  if (n_instances_out) {
    // I was counted by the projection: one synchronisation, then size the instance buffers
    GS_TRY(cudaMemcpyAsync(ws->h_counters, cnt, kCntNum * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    GS_TRY(cudaStreamSynchronize(st));
    bound = (int64_t)ws->h_counters[kCntInst];
    GS_TRY(ensure_inst(ws, bound));
    *n_instances_out = bound;
  } else {
    bound = (int64_t)ws->inst_id.cap;
  }
  const int64_t cap = (int64_t)ws->inst_id.cap;
  // count -> scan (ranges, heavy-first order) -> scatter -> per-tile radix sort
  BinArgs b;
  b.n = n;
  b.ntiles = ws->ntiles.p;
  b.rect = ws->rect.p;
  b.depth_key = ws->depth_key.p;
  b.TX = ws->TX;
  b.n_tiles = ntl;
  b.cap = cap;
  b.tile_count = ws->tile_count.p;
  b.cursor = ws->tile_cursor.p;
  b.ranges = ws->ranges.p;
  b.order = ws->tile_order.p;
  b.queue = ws->queue.p + 4;
  b.kv = ws->inst_kv.p;
  b.key0 = ws->inst_key.p;
  b.id0 = ws->inst_id.p;
  b.counters = cnt;
  ws->ordered = launch_bin(b, st);
  ws->tile_counts_dirty = false;   // the scan cleared them
  ws->id_sorted = ws->inst_id.p;
  GS_TRY(cudaGetLastError());
  ws->inst_bound = std::min(bound, cap);
  ws->stage = 2;
  return GS_OK;
}

namespace {

gs_status render_fwd(const gs_scene* scene, const gs_camera* cam, gs_workspace* ws, float* rgb,
                     float* depth, float* alpha, float* feat, const gs_feat_loss* loss,
                     void* stream) {
  if (!ws) return GS_ERR_ARG;
  gs_status s = check_scene(scene);
  if (s != GS_OK) return s;
  CamDev cd;
  if ((s = make_cam(cam, &cd)) != GS_OK) return s;
  cd.n_gauss = (int)scene->n;
  if (ws->stage < 2 || scene->n != ws->n || !same_grid(cd, ws->cam)) return GS_ERR_STATE;
  if (feat && scene->n_feat > 0 && !aligned16(feat)) return GS_ERR_ARG;
  FeatLoss fl{};
  if (loss) {
    if (scene->n_feat <= 0 || !loss->target || !loss->g_feat || !loss->loss ||
        !(loss->lambda_sem >= 0.f))
      return GS_ERR_ARG;
    const double P = (double)cd.GW * cd.GH, D = (double)scene->n_feat;
    fl.target = loss->target;
    fl.mask = loss->mask;
    fl.g_feat = loss->g_feat;
    fl.loss = loss->loss;
    fl.lambda = loss->lambda_sem;
    fl.s_l1 = 1.0 / (D * P);
    fl.s_cos = 1.0 / P;
    fl.w_l1 = (float)(fl.lambda * fl.s_l1);
    fl.w_cos = (float)(fl.lambda * fl.s_cos);
  }
  DeviceGuard g(ws->device);
  cudaStream_t st = (cudaStream_t)stream;
  StageTimer tm(ws, GS_TIMER_FWD, st);
  if (loss) GS_TRY(cudaMemsetAsync(loss->loss, 0, 3 * sizeof(double), st));
  const TileQueue tq{ws->queue.p, ws->queue.p + 1, ws->ordered ? ws->tile_order.p : nullptr,
                     cd.TX * cd.TY};
  if (cd.stride > 1)
    launch_grid_fwd(cd, tq, ws->rec.p, scene->feats, scene->feat_dtype, scene->n_feat, ws->ranges.p,
                    ws->id_sorted, rgb, depth, alpha, scene->n_feat > 0 ? feat : nullptr,
                    ws->T_final.p, ws->n_contrib.p, loss ? &fl : nullptr, st);
  else
    launch_raster_fwd(cd, tq, ws->rec.p, scene->feats, scene->feat_dtype, scene->n_feat,
                      ws->ranges.p, ws->id_sorted, rgb, depth, alpha,
                      scene->n_feat > 0 ? feat : nullptr, ws->T_final.p, ws->n_contrib.p,
                      loss ? &fl : nullptr, st);
  GS_TRY(cudaGetLastError());
  ws->stage = 3;
  return GS_OK;
}

}  // namespace

gs_status gs_render_fwd(const gs_scene* scene, const gs_camera* cam, gs_workspace* ws, float* rgb,
                        float* depth, float* alpha, float* feat, void* stream) {
  return render_fwd(scene, cam, ws, rgb, depth, alpha, feat, nullptr, stream);
}

gs_status gs_render_fwd_loss(const gs_scene* scene, const gs_camera* cam, gs_workspace* ws,
                             float* rgb, float* depth, float* alpha, float* feat,
                             const gs_feat_loss* loss, void* stream) {
  if (!loss) return GS_ERR_ARG;
  return render_fwd(scene, cam, ws, rgb, depth, alpha, feat, loss, stream);
}

gs_status gs_render_bwd(const gs_scene* scene, const gs_camera* cam, gs_workspace* ws,
                        const float* g_rgb, const float* g_depth, const float* g_alpha,
                        const float* g_feat, float* g_means, float* g_scales, float* g_quats,
                        float* g_opac, float* g_sh, float* g_feats, float* g_pose6, void* stream) {
  if (!ws) return GS_ERR_ARG;
  gs_status s = check_scene(scene);
  if (s != GS_OK) return s;
  CamDev cd;
  if ((s = make_cam(cam, &cd)) != GS_OK) return s;
  cd.n_gauss = (int)scene->n;
  if (ws->stage < 3 || scene->n != ws->n || !same_grid(cd, ws->cam)) return GS_ERR_STATE;
  if (g_feats && !aligned16(g_feats)) return GS_ERR_ARG;
  if (g_quats && !aligned16(g_quats)) return GS_ERR_ARG;
  DeviceGuard g(ws->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = scene->n;
  const int D = scene->n_feat;
  // Features-only backward (geometry and colour frozen, Sec. 3.2): only g_feats is asked
  // for, so the rasterizer skips every geometry term and the projection backward is not run.
  const bool features_only = D > 0 && g_feat && g_feats && !g_means && !g_scales && !g_quats &&
                             !g_opac && !g_sh && !g_pose6;
  {
    StageTimer tm(ws, GS_TIMER_BWD_RASTER, st);
    if (n > 0 && !features_only)
      GS_TRY(cudaMemsetAsync(ws->g2d.p, 0, sizeof(float) * kG2D * (size_t)n, st));
    if (g_feats && n > 0 && D > 0)
      GS_TRY(cudaMemsetAsync(g_feats, 0, sizeof(float) * (size_t)n * D, st));
    // the backward kernels leave their queue to the host: zeroed before each launch (a
    // self-resetting queue measured slower in these kernels)
    GS_TRY(cudaMemsetAsync(ws->queue.p + 2, 0, 8, st));
    const TileQueue tq{ws->queue.p + 2, ws->queue.p + 3, ws->ordered ? ws->tile_order.p : nullptr,
                       cd.TX * cd.TY};
    const float* gf = D > 0 ? g_feat : nullptr;
    float* gfe = D > 0 ? g_feats : nullptr;
    if (cd.stride > 1)
      launch_grid_bwd(cd, tq, ws->rec.p, scene->feats, scene->feat_dtype, D, ws->ranges.p,
                      ws->id_sorted, ws->T_final.p, ws->n_contrib.p, g_rgb, g_depth, g_alpha, gf,
                      ws->g2d.p, gfe, features_only, st);
    else
      launch_raster_bwd(cd, tq, ws->rec.p, scene->feats, scene->feat_dtype, D, ws->ranges.p,
                        ws->id_sorted, ws->T_final.p, ws->n_contrib.p, g_rgb, g_depth, g_alpha, gf,
                        ws->g2d.p, gfe, features_only, st);
    GS_TRY(cudaGetLastError());
  }
  if (!features_only) {
    StageTimer tm(ws, GS_TIMER_BWD_PROJECT, st);
    launch_project_bwd(*scene, cd, ws->rec.p, ws->ntiles.p, ws->g2d.p, g_means, g_scales, g_quats,
                       g_opac, g_sh, ws->pose_partials.p, g_pose6, st);
    GS_TRY(cudaGetLastError());
  }
  return GS_OK;
}

gs_status gs_l1_grad(const float* pred, const float* target, int64_t n, float scale, float* grad,
                     void* stream) {
  if (n < 0 || (n > 0 && (!pred || !target || !grad))) return GS_ERR_ARG;
  launch_l1_grad(pred, target, n, scale, grad, (cudaStream_t)stream);
  GS_TRY(cudaGetLastError());
  return GS_OK;
}

gs_status gs_get_stats(gs_workspace* ws, gs_stats* out, void* stream) {
  if (!ws || !out) return GS_ERR_ARG;
  DeviceGuard g(ws->device);
  cudaStream_t st = (cudaStream_t)stream;
  const bool grid = ws->cam.stride > 1;
  if (ws->stage >= 3 && !grid)
    launch_inst_eff(ws->n_contrib.p, ws->TX, ws->TY, ws->W, ws->H, ws->counters.p, st);
  unsigned long long pairs[2] = {0ull, 0ull};
  if (ws->stage >= 3) {
    GS_TRY(ws->stats64.ensure(2));
    if (grid) {
      // I_eff and pair counts of the grid's work items (one pass per sample)
      GS_TRY(ws->item_max.ensure((size_t)ws->TX * ws->TY * grid_chunks_per_tile(ws->cam.stride)));
      launch_grid_stats(ws->cam, ws->rec.p, ws->ranges.p, ws->id_sorted, ws->n_contrib.p,
                        ws->item_max.p, ws->counters.p, ws->stats64.p, st);
    } else {
      launch_pair_stats(ws->cam, ws->rec.p, ws->ranges.p, ws->id_sorted, ws->n_contrib.p,
                        ws->stats64.p, st);
    }
    GS_TRY(cudaMemcpyAsync(pairs, ws->stats64.p, sizeof(pairs), cudaMemcpyDeviceToHost, st));
  }
  GS_TRY(cudaMemcpyAsync(ws->h_counters, ws->counters.p, kCntNum * sizeof(uint32_t),
                         cudaMemcpyDeviceToHost, st));
  GS_TRY(cudaStreamSynchronize(st));
  out->n = ws->n;
  out->visible = ws->stage >= 2 ? ws->h_counters[kCntVisible] : 0;
  out->instances = ws->stage >= 2 ? ws->h_counters[kCntInst] : 0;
  out->inst_eff = ws->stage >= 3 ? ws->h_counters[kCntInstEff] : 0;
  out->pixels = (int64_t)ws->W * ws->H;
  out->tiles = (int64_t)ws->TX * ws->TY;
  out->pairs_eval = (int64_t)pairs[0];
  out->pairs_blend = (int64_t)pairs[1];
  return GS_OK;
}

gs_status gs_get_instances(gs_workspace* ws, uint32_t* tiles_out, uint32_t* ids_out, int64_t cap,
                           int64_t* n_out, uint32_t* ranges_out, void* stream) {
  if (!ws || cap < 0) return GS_ERR_ARG;
  if (ws->stage < 2) return GS_ERR_STATE;
  DeviceGuard g(ws->device);
  cudaStream_t st = (cudaStream_t)stream;
  GS_TRY(cudaMemcpyAsync(ws->h_counters, ws->counters.p, kCntNum * sizeof(uint32_t),
                         cudaMemcpyDeviceToHost, st));
  GS_TRY(cudaStreamSynchronize(st));
  const int64_t I = std::min<int64_t>(ws->h_counters[kCntInst], ws->inst_bound);
  if (n_out) *n_out = ws->h_counters[kCntInst];
  const int64_t m = std::min(I, cap);
  const int ntl = ws->TX * ws->TY;
  std::vector<uint2> rg((size_t)ntl);
  if (m > 0 && ids_out)
    GS_TRY(cudaMemcpyAsync(ids_out, ws->id_sorted, m * 4, cudaMemcpyDeviceToHost, st));
  if (ntl > 0)
    GS_TRY(cudaMemcpyAsync(rg.data(), ws->ranges.p, sizeof(uint2) * (size_t)ntl,
                           cudaMemcpyDeviceToHost, st));
  GS_TRY(cudaStreamSynchronize(st));
  if (ranges_out && ntl > 0) std::memcpy(ranges_out, rg.data(), sizeof(uint2) * (size_t)ntl);
  if (tiles_out) {   // the tile of every slot, from the tile ranges
    for (int t = 0; t < ntl; ++t)
      for (int64_t j = rg[(size_t)t].x; j < (int64_t)rg[(size_t)t].y && j < m; ++j)
        tiles_out[j] = (uint32_t)t;
  }
  return GS_OK;
}

gs_status gs_get_projection(gs_workspace* ws, float* mean2d, float* conic, float* depth, float* rgb,
                            int32_t* rect, void* stream) {
  if (!ws) return GS_ERR_ARG;
  if (ws->stage < 1) return GS_ERR_STATE;
  DeviceGuard g(ws->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = ws->n;
  std::vector<GaussRec> rec((size_t)n);
  std::vector<uint2> rc((size_t)n);
  if (n > 0) {
    GS_TRY(cudaMemcpyAsync(rec.data(), ws->rec.p, sizeof(GaussRec) * n, cudaMemcpyDeviceToHost, st));
    GS_TRY(cudaMemcpyAsync(rc.data(), ws->rect.p, sizeof(uint2) * n, cudaMemcpyDeviceToHost, st));
  }
  GS_TRY(cudaStreamSynchronize(st));
  for (int64_t i = 0; i < n; ++i) {
    if (rc[i].x == 0u && rc[i].y == 0u) rec[i] = GaussRec{};   // culled: no record was written
    const GaussRec& r = rec[i];
    if (mean2d) { mean2d[2 * i] = r.r0.x; mean2d[2 * i + 1] = r.r0.y; }
    if (conic) { conic[3 * i] = r.r0.z; conic[3 * i + 1] = r.r0.w; conic[3 * i + 2] = r.r1.x; }
    if (depth) depth[i] = r.r1.z;
    if (rgb) { rgb[3 * i] = r.r2.x; rgb[3 * i + 1] = r.r2.y; rgb[3 * i + 2] = r.r2.z; }
    if (rect) {
      rect[4 * i] = (int32_t)(rc[i].x & 0xFFFF);
      rect[4 * i + 1] = (int32_t)(rc[i].x >> 16);
      rect[4 * i + 2] = (int32_t)(rc[i].y & 0xFFFF);
      rect[4 * i + 3] = (int32_t)(rc[i].y >> 16);
    }
  }
  return GS_OK;
}

gs_status gs_get_pixel_state(gs_workspace* ws, float* T_final, uint32_t* n_contrib, void* stream) {
  if (!ws) return GS_ERR_ARG;
  if (ws->stage < 3) return GS_ERR_STATE;
  DeviceGuard g(ws->device);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t P = (size_t)ws->W * ws->H;
  if (T_final) GS_TRY(cudaMemcpyAsync(T_final, ws->T_final.p, P * 4, cudaMemcpyDeviceToHost, st));
  if (n_contrib) GS_TRY(cudaMemcpyAsync(n_contrib, ws->n_contrib.p, P * 4, cudaMemcpyDeviceToHost, st));
  GS_TRY(cudaStreamSynchronize(st));
  return GS_OK;
}

int64_t gs_launch_count(void) { return gs::g_launches.load(std::memory_order_relaxed); }

gs_status gs_timing_enable(gs_workspace* ws, int enable) {
  if (!ws) return GS_ERR_ARG;
  DeviceGuard g(ws->device);
  if (enable && !ws->ev_created) {
    for (int k = 0; k < GS_NUM_TIMERS; ++k)
      for (int s = 0; s < kTimerRing; ++s) {
        GS_TRY(cudaEventCreate(&ws->ev[k][s][0]));
        GS_TRY(cudaEventCreate(&ws->ev[k][s][1]));
      }
    ws->ev_created = true;
  }
  ws->timing = enable != 0;
  return GS_OK;
}

gs_status gs_timing_collect(gs_workspace* ws, double* ms_out, int64_t* count_out) {
  if (!ws || !ms_out) return GS_ERR_ARG;
  DeviceGuard g(ws->device);
  for (int k = 0; k < GS_NUM_TIMERS; ++k) {
    double tot = 0.0;
    for (int s = 0; s < ws->ev_count[k]; ++s) {
      GS_TRY(cudaEventSynchronize(ws->ev[k][s][1]));
      float ms = 0.f;
      GS_TRY(cudaEventElapsedTime(&ms, ws->ev[k][s][0], ws->ev[k][s][1]));
      tot += ms;
    }
    ms_out[k] = tot;
    if (count_out) count_out[k] = ws->ev_count[k];
    ws->ev_count[k] = 0;
  }
  return GS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- serving helpers
// Internal (C++) interface of the serving executor (gs_serve.cu): a request's workspace is
// reserved once, its instance buffers are ranges of the server's arena, and its raster
// work joins a multi-request launch.
namespace gs {

gs_status ws_reserve_fixed(gs_workspace* ws, int64_t n_gauss, int64_t n_pixels, int64_t n_tiles) {
  if (!ws || n_gauss < 0 || n_pixels < 0 || n_tiles < 0) return GS_ERR_ARG;
  DeviceGuard g(ws->device);
  GS_TRY(ensure_gauss(ws, n_gauss));
  GS_TRY(ensure_pix(ws, n_pixels, n_tiles));
  return GS_OK;
}

void ws_lend_instances(gs_workspace* ws, uint2* kv, uint32_t* key0, uint32_t* id0, int64_t cap) {
  const size_t m = (size_t)std::max<int64_t>(cap, 0);
  ws->inst_kv.lend(kv, m);
  ws->inst_key.lend(key0, m);
  ws->inst_id.lend(id0, m);
}

bool ws_fits(const gs_workspace* ws, int64_t n_gauss, int64_t n_pixels, int64_t n_tiles) {
  return (int64_t)ws->rec.cap >= n_gauss && (int64_t)ws->T_final.cap >= n_pixels &&
         (int64_t)ws->ranges.cap >= n_tiles;
}

gs_status ws_instances_async(gs_workspace* ws, uint32_t* host, cudaStream_t st) {
  if (ws->stage < 1) return GS_ERR_STATE;
  GS_TRY(cudaMemcpyAsync(host, ws->counters.p + kCntInst, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  return GS_OK;
}

gs_status ws_job(gs_workspace* ws, const gs_scene& sc, RasterJob* j) {
  if (ws->stage < 2 || sc.n != ws->n) return GS_ERR_STATE;
  *j = RasterJob{};
  j->cam = ws->cam;
  j->rec = ws->rec.p;
  j->feats = sc.feats;
  j->D = sc.n_feat;
  j->ranges = ws->ranges.p;
  j->inst_id = ws->id_sorted;
  j->order = ws->ordered ? ws->tile_order.p : nullptr;
  j->T_final = ws->T_final.p;
  j->n_contrib = ws->n_contrib.p;
  j->g2d = ws->g2d.p;
  return GS_OK;
}

int ws_tiles(const gs_workspace* ws) { return ws->TX * ws->TY; }

gs_status ws_bwd_clear(gs_workspace* ws, int D, float* g_feats, cudaStream_t st) {
  const int64_t n = ws->n;
  if (n > 0) GS_TRY(cudaMemsetAsync(ws->g2d.p, 0, sizeof(float) * kG2D * (size_t)n, st));
  if (g_feats && n > 0 && D > 0) GS_TRY(cudaMemsetAsync(g_feats, 0, sizeof(float) * (size_t)n * D, st));
  return GS_OK;
}

gs_status ws_project_bwd(gs_workspace* ws, const gs_scene& sc, float* g_means, float* g_scales,
                         float* g_quats, float* g_opac, float* g_sh, float* g_pose6, cudaStream_t st) {
  launch_project_bwd(sc, ws->cam, ws->rec.p, ws->ntiles.p, ws->g2d.p, g_means, g_scales, g_quats,
                     g_opac, g_sh, ws->pose_partials.p, g_pose6, st);
  GS_TRY(cudaGetLastError());
  return GS_OK;
}

}  // namespace gs

