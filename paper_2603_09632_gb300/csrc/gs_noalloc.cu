// gs_render_fwd_noalloc: a forward render that allocates no memory.
//
// For callers that cannot allocate device memory when they render -- a plugin that
// runs inside a host application owning every allocation, code running under a fixed
// device-memory budget, or a renderer called from a context where a cudaMalloc would
// stall or fail -- this entry point renders small scenes with every intermediate buffer
// (projection records, sort buffers, tile lists, per-pixel state) carved out of one
// file-scope device array of fixed size that the library holds for as long as it is
// loaded.  The caller passes only the scene, the camera and the output images.
//
// It runs the same kernels as gs_project -> gs_bin_tiles -> gs_render_fwd, so its images
// are the same.  Limits: at most kNaMaxGauss Gaussians, kNaMaxInst tile instances,
// kNaMaxPix pixels and kNaMaxTiles tiles; larger requests return GS_ERR_OVER_BUDGET.
#include <mutex>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int64_t kNaMaxGauss = 16384;
constexpr int64_t kNaMaxInst = 131072;
constexpr int64_t kNaMaxPix = 65536;
constexpr int64_t kNaMaxTiles = 1024;
constexpr int kNaMaxDevices = 64;

constexpr size_t al(size_t x) { return (x + 255) & ~size_t(255); }
// byte offsets of the sub-buffers inside the scratch array
constexpr size_t oRec = 0;
constexpr size_t oKey = al(oRec + kNaMaxGauss * sizeof(GaussRec));
constexpr size_t oNt = al(oKey + kNaMaxGauss * 4);
constexpr size_t oRect = al(oNt + kNaMaxGauss * 4);
constexpr size_t oKV = al(oRect + kNaMaxGauss * 8);        // instance (key, id) pairs
constexpr size_t oK0 = al(oKV + kNaMaxInst * 8);          // sort scratch keys
constexpr size_t oI0 = al(oK0 + kNaMaxInst * 4);          // sorted ids
constexpr size_t oTf = al(oI0 + kNaMaxInst * 4);
constexpr size_t oNc = al(oTf + kNaMaxPix * 4);
constexpr size_t oRanges = al(oNc + kNaMaxPix * 4);
constexpr size_t oOrder = al(oRanges + kNaMaxTiles * 8);
constexpr size_t oTCount = al(oOrder + kNaMaxTiles * 4);    // binning scratch
constexpr size_t oTCursor = al(oTCount + kNaMaxTiles * 8);   // (per-row differences: <= 2 words a tile)
constexpr size_t oCnt = al(oTCursor + kNaMaxTiles * 4);     // counters
constexpr size_t oQueue = al(oCnt + kCntNum * 4);           // persistent-kernel queues
constexpr size_t kNaBytes = al(oQueue + 8 * 4);

}  // namespace
}  // namespace gs

// The scratch: one array per device, shared by every call (about 4 MB).
static __device__ __align__(256) unsigned char g_noalloc_scratch[gs::kNaBytes];

namespace gs {
namespace {

std::mutex g_na_mu;
unsigned char* g_na_ptr[kNaMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
gs_status na_scratch(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kNaMaxDevices) return GS_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GS_ERR_CUDA;
    g_na_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_na_ptr[dev];
  return GS_OK;
}

bool na_aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_render_fwd_noalloc(const gs_scene* scene, const gs_camera* c, float* rgb,
                                           float* depth, float* alpha, float* feat, void* stream) {
  if (!scene || !c) return GS_ERR_ARG;
  if (scene->n < 0 || scene->sh_degree < 0 || scene->sh_degree > 3 || scene->n_feat < 0 ||
      scene->n_feat > kMaxFeat || (scene->feat_dtype != GS_F32 && scene->feat_dtype != GS_BF16))
    return GS_ERR_ARG;
  if (scene->n > 0 && (!scene->means || !scene->scales || !scene->quats || !scene->opacities ||
                       !scene->sh || (scene->n_feat > 0 && !scene->feats)))
    return GS_ERR_ARG;
  if (!na_aligned16(scene->means) || !na_aligned16(scene->scales) || !na_aligned16(scene->quats) ||
      !na_aligned16(scene->sh) || (scene->feats && !na_aligned16(scene->feats)) ||
      (feat && !na_aligned16(feat)))
    return GS_ERR_ARG;
  if (c->W <= 0 || c->H <= 0 || c->tile != kTile || !(c->fx > 0.f) || !(c->fy > 0.f) ||
      !(c->near_z > 0.f) || c->stride != 1 || c->off_x != 0 || c->off_y != 0)
    return GS_ERR_ARG;
  // size limits first, so that the tile counts below cannot overflow an int
  if (scene->n > kNaMaxGauss || c->W > kNaMaxPix || c->H > kNaMaxPix ||
      (int64_t)c->W * c->H > kNaMaxPix)
    return GS_ERR_OVER_BUDGET;
  CamDev cd;
  cd.W = c->W;
  cd.H = c->H;
  cd.TX = (c->W + kTile - 1) / kTile;
  cd.TY = (c->H + kTile - 1) / kTile;
  cd.n_gauss = (int)scene->n;
  cd.fx = c->fx;
  cd.fy = c->fy;
  cd.cx = c->cx;
  cd.cy = c->cy;
  for (int k = 0; k < 9; ++k) cd.R[k] = c->R[k];
  for (int k = 0; k < 3; ++k) cd.t[k] = c->t[k];
  cd.near_z = c->near_z;
  cd.stride = 1;
  cd.ox = cd.oy = 0;
  cd.GW = cd.W;
  cd.GH = cd.H;
  const int64_t ntl = (int64_t)cd.TX * cd.TY;
  if (ntl > kNaMaxTiles) return GS_ERR_OVER_BUDGET;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GS_ERR_CUDA;
  unsigned char* base = nullptr;
  gs_status s = na_scratch(dev, &base);
  if (s != GS_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  GaussRec* rec = reinterpret_cast<GaussRec*>(base + oRec);
  uint32_t* key = reinterpret_cast<uint32_t*>(base + oKey);
  uint32_t* nt = reinterpret_cast<uint32_t*>(base + oNt);
  uint2* rect = reinterpret_cast<uint2*>(base + oRect);
  uint2* kv = reinterpret_cast<uint2*>(base + oKV);
  uint32_t *k0 = reinterpret_cast<uint32_t*>(base + oK0), *i0 = reinterpret_cast<uint32_t*>(base + oI0);
  float* Tf = reinterpret_cast<float*>(base + oTf);
  uint32_t* nc = reinterpret_cast<uint32_t*>(base + oNc);
  uint2* ranges = reinterpret_cast<uint2*>(base + oRanges);
  uint32_t* order = reinterpret_cast<uint32_t*>(base + oOrder);
  uint32_t* tcount = reinterpret_cast<uint32_t*>(base + oTCount);
  uint32_t* tcursor = reinterpret_cast<uint32_t*>(base + oTCursor);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(base + oCnt);
  uint32_t* queue = reinterpret_cast<uint32_t*>(base + oQueue);

  // the array keeps the previous call's contents: clear what must start at zero (counters,
  // the tile counts the projection adds to, and the queues, which reset themselves but are
  // cleared here as well since nothing else initialises this array)
  if (cudaMemsetAsync(cnt, 0, kCntNum * 4, st) != cudaSuccess ||
      cudaMemsetAsync(queue, 0, 8 * 4, st) != cudaSuccess ||
      cudaMemsetAsync(tcount, 0, (size_t)cd.TY * (cd.TX + 1) * 4, st) != cudaSuccess)
    return GS_ERR_CUDA;
  launch_project(*scene, cd, rec, key, nt, rect, cnt, tcount, st);
  // the instance count decides whether the request fits: one synchronisation
  uint32_t h_cnt[kCntNum];
  if (cudaMemcpyAsync(h_cnt, cnt, sizeof(h_cnt), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return GS_ERR_CUDA;
  const int64_t I = h_cnt[kCntInst];
  // too many tile instances: nothing is written; the tile counts the projection added are
  // cleared by the next call, like every other value that must start at zero
  if (I > kNaMaxInst) return GS_ERR_OVER_BUDGET;
  BinArgs b;
  b.n = scene->n;
  b.ntiles = nt;
  b.rect = rect;
  b.depth_key = key;
  b.TX = cd.TX;
  b.n_tiles = (int)ntl;
  b.cap = kNaMaxInst;
  b.tile_count = tcount;
  b.cursor = tcursor;
  b.ranges = ranges;
  b.order = order;
  b.queue = queue + 2;
  b.kv = kv;
  b.key0 = k0;
  b.id0 = i0;
  b.counters = cnt;
  const bool ordered = launch_bin(b, st);
  const TileQueue tq{queue, queue + 1, ordered ? order : nullptr, (int)ntl};
  launch_raster_fwd(cd, tq, rec, scene->feats, scene->feat_dtype, scene->n_feat, ranges, i0, rgb,
                    depth, alpha, scene->n_feat > 0 ? feat : nullptr, Tf, nc, nullptr, st);
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
