// CPU oracle for the differentiable Gaussian-splatting rasterizer of X-GS.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
// load this file; only the tests, the package's smoke check and the
// benchmark's CPU-baseline leg use it.  It shares no code with the CUDA
// library: it is a plain, slow, per-pixel restatement of the method.
//
// What it computes (X-GS, App. A and App. B, Sec. 3.1):
//   * Sigma = R S S^T R^T                          (App. A, covariance parameterisation)
//   * Sigma' = J W Sigma W^T J^T                    (App. A, EWA projection)
//   * G(x) = exp(-1/2 (x-mu)^T Sigma^-1 (x-mu))     (App. A, evaluated in 2D with Sigma')
//   * C(x) = sum_i c_i a'_i prod_{j<i} (1 - a'_j)   (Eq. 1 / discrete rendering, App. B)
//   * depth by substituting c_i -> d_i              (App. B)
//   * features by substituting c_i -> f_i           (Sec. 3.1, Preliminaries)
//   * gradients w.r.t. every Gaussian parameter and the camera pose
//     ("the rasterizer is natively differentiable", App. B; tracking Eq. 2,
//      mapping Eq. 3).
// The readings of what the paper leaves open (camera model, near plane,
// guard band, low-pass dilation, 3-sigma tile rectangle, blend thresholds,
// SH basis, pose twist) are listed in the repository's design notes.
//
// Everything is templated on the scalar type: float mirrors the GPU's
// precision (and, for the key-affecting projection, its exact operation
// order), double is the FP64 reference.  Build with -ffp-contract=off so
// that float results are the IEEE results of the written expressions.
// A third mode evaluates everything in double but takes each Gaussian's
// discrete projection decisions -- visibility, 3-sigma tile rectangle and
// the depth that orders the tile lists -- from the float projection: the
// readings define those with separately rounded float operations, so this
// is the same function in exact arithmetic (the "mixed" entry points).
//
// Parity pins: see tests/test_oracle_*.py (closed forms, invariants, brute
// force, finite differences, SH orthonormality, Monte-Carlo/FD projection).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int TILE = 16;

// ---------------------------------------------------------------- camera
template <class S>
struct Cam {
  int W, H, TX, TY;
  S fx, fy, cx, cy, R[9], t[3], near_z;
  bool thresholds;
};

// cam layout (doubles): W, H, fx, fy, cx, cy, R[9] (row-major, world->camera), t[3], near
template <class S>
Cam<S> make_cam(const double* c, int thresholds) {
  Cam<S> k;
  k.W = (int)c[0];
  k.H = (int)c[1];
  k.TX = (k.W + TILE - 1) / TILE;
  k.TY = (k.H + TILE - 1) / TILE;
  k.fx = (S)c[2]; k.fy = (S)c[3]; k.cx = (S)c[4]; k.cy = (S)c[5];
  for (int i = 0; i < 9; ++i) k.R[i] = (S)c[6 + i];
  for (int i = 0; i < 3; ++i) k.t[i] = (S)c[15 + i];
  k.near_z = (S)c[18];
  k.thresholds = thresholds != 0;
  return k;
}

// ---------------------------------------------------------------- real SH basis
// Real spherical harmonics up to degree 3 on the unit sphere, ordered (l, m=-l..l),
// orthonormal, written as harmonic polynomials of the unit direction (x, y, z),
// without the Condon-Shortley phase.  Y[k] and its gradient dY[k][3] w.r.t. (x,y,z).
template <class S>
void sh_basis(int deg, S x, S y, S z, S* Y, S (*dY)[3]) {
  const double PI = 3.14159265358979323846;
  const S c0 = (S)(0.5 / std::sqrt(PI));
  const S c1 = (S)std::sqrt(3.0 / (4.0 * PI));
  const S c2a = (S)(0.5 * std::sqrt(15.0 / PI));
  const S c2b = (S)(0.25 * std::sqrt(5.0 / PI));
  const S c2c = (S)(0.25 * std::sqrt(15.0 / PI));
  const S c3a = (S)(0.25 * std::sqrt(35.0 / (2.0 * PI)));
  const S c3b = (S)(0.5 * std::sqrt(105.0 / PI));
  const S c3c = (S)(0.25 * std::sqrt(21.0 / (2.0 * PI)));
  const S c3d = (S)(0.25 * std::sqrt(7.0 / PI));
  const S c3e = (S)(0.25 * std::sqrt(105.0 / PI));
  auto set = [&](int k, S v, S gx, S gy, S gz) {
    Y[k] = v;
    if (dY) { dY[k][0] = gx; dY[k][1] = gy; dY[k][2] = gz; }
  };
  set(0, c0, 0, 0, 0);
  if (deg < 1) return;
  set(1, c1 * y, 0, c1, 0);
  set(2, c1 * z, 0, 0, c1);
  set(3, c1 * x, c1, 0, 0);
  if (deg < 2) return;
  set(4, c2a * x * y, c2a * y, c2a * x, 0);
  set(5, c2a * y * z, 0, c2a * z, c2a * y);
  set(6, c2b * (2 * z * z - x * x - y * y), -2 * c2b * x, -2 * c2b * y, 4 * c2b * z);
  set(7, c2a * x * z, c2a * z, 0, c2a * x);
  set(8, c2c * (x * x - y * y), 2 * c2c * x, -2 * c2c * y, 0);
  if (deg < 3) return;
  set(9, c3a * y * (3 * x * x - y * y), 6 * c3a * x * y, c3a * (3 * x * x - 3 * y * y), 0);
  set(10, c3b * x * y * z, c3b * y * z, c3b * x * z, c3b * x * y);
  set(11, c3c * y * (4 * z * z - x * x - y * y), -2 * c3c * x * y,
      c3c * (4 * z * z - x * x - 3 * y * y), 8 * c3c * y * z);
  set(12, c3d * z * (2 * z * z - 3 * x * x - 3 * y * y), -6 * c3d * x * z, -6 * c3d * y * z,
      c3d * (6 * z * z - 3 * x * x - 3 * y * y));
  set(13, c3c * x * (4 * z * z - x * x - y * y), c3c * (4 * z * z - 3 * x * x - y * y),
      -2 * c3c * x * y, 8 * c3c * x * z);
  set(14, c3e * z * (x * x - y * y), 2 * c3e * x * z, -2 * c3e * y * z, c3e * (x * x - y * y));
  set(15, c3a * x * (x * x - 3 * y * y), c3a * (3 * x * x - 3 * y * y), -6 * c3a * x * y, 0);
}

// ---------------------------------------------------------------- projection
template <class S>
struct Proj {
  bool valid = false;
  S p[3];                 // camera-space mean
  S qn[4], qlen;          // normalised quaternion (w,x,y,z), original length
  S Rq[9];                // rotation of the quaternion
  S M[9];                 // Rq * diag(s)
  S Sig[9];               // world covariance (symmetric)
  S Sc[9];                // camera covariance W Sigma W^T (symmetric)
  S tx, ty, txc, tyc;     // x/z, y/z and their guard-band clamps
  bool clx, cly;          // clamp active
  S J[4];                 // j00, j02, j11, j12
  S cov[3];               // Sigma' + dilation: a, b, c
  S det;
  S conic[3];             // A, B, C of Sigma'^{-1}
  S u, v, depth;
  S key;                  // depth that orders the tile lists (the float depth in mixed mode)
  int radius;
  int rect[4];            // x0, y0, x1, y1 in tiles, [x0,x1) x [y0,y1)
  S dir[3], dlen;         // unit view direction and the length it came from
  S rgb[3];
  bool rgb_pos[3];        // colour not clamped at 0
};

// Sigma = R S S^T R^T, Sigma' = J W Sigma W^T J^T (App. A) with the readings:
// guard band 1.3 x half-FOV on J, +0.3 px^2 low-pass on the diagonal, 3-sigma radius.
// The operation order below is the key-affecting convention (see design notes).
// d32 (mixed mode): the float projection of the same Gaussian, whose visibility, tile
// rectangle and depth key are taken as they are.
template <class S>
Proj<S> project_one(const Cam<S>& k, const S* mu, const S* s, const S* q, const S* sh,
                    int deg, const Proj<float>* d32 = nullptr) {
  Proj<S> P;
  if (d32 && !d32->valid) return P;
  const S* R = k.R;
  P.p[0] = ((R[0] * mu[0] + R[1] * mu[1]) + R[2] * mu[2]) + k.t[0];
  P.p[1] = ((R[3] * mu[0] + R[4] * mu[1]) + R[5] * mu[2]) + k.t[1];
  P.p[2] = ((R[6] * mu[0] + R[7] * mu[1]) + R[8] * mu[2]) + k.t[2];
  const S x = P.p[0], y = P.p[1], z = P.p[2];
  if (!d32 && !(z > k.near_z)) return P;

  S qq = ((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3];
  P.qlen = std::sqrt(qq);
  const S w = q[0] / P.qlen, qx = q[1] / P.qlen, qy = q[2] / P.qlen, qz = q[3] / P.qlen;
  P.qn[0] = w; P.qn[1] = qx; P.qn[2] = qy; P.qn[3] = qz;
  S* Rq = P.Rq;
  Rq[0] = (S)1 - (S)2 * (qy * qy + qz * qz);
  Rq[1] = (S)2 * (qx * qy - w * qz);
  Rq[2] = (S)2 * (qx * qz + w * qy);
  Rq[3] = (S)2 * (qx * qy + w * qz);
  Rq[4] = (S)1 - (S)2 * (qx * qx + qz * qz);
  Rq[5] = (S)2 * (qy * qz - w * qx);
  Rq[6] = (S)2 * (qx * qz - w * qy);
  Rq[7] = (S)2 * (qy * qz + w * qx);
  Rq[8] = (S)1 - (S)2 * (qx * qx + qy * qy);
  for (int i = 0; i < 3; ++i)
    for (int c = 0; c < 3; ++c) P.M[i * 3 + c] = Rq[i * 3 + c] * s[c];
  // Sigma = M M^T (upper triangle computed, mirrored)
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      S v = (P.M[i * 3 + 0] * P.M[j * 3 + 0] + P.M[i * 3 + 1] * P.M[j * 3 + 1]) +
            P.M[i * 3 + 2] * P.M[j * 3 + 2];
      P.Sig[i * 3 + j] = v;
      P.Sig[j * 3 + i] = v;
    }
  // Sc = W Sigma W^T with W = R (upper triangle, mirrored)
  S A[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      A[i * 3 + j] = (R[i * 3 + 0] * P.Sig[0 * 3 + j] + R[i * 3 + 1] * P.Sig[1 * 3 + j]) +
                     R[i * 3 + 2] * P.Sig[2 * 3 + j];
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      S v = (A[i * 3 + 0] * R[j * 3 + 0] + A[i * 3 + 1] * R[j * 3 + 1]) +
            A[i * 3 + 2] * R[j * 3 + 2];
      P.Sc[i * 3 + j] = v;
      P.Sc[j * 3 + i] = v;
    }
  // J of the pinhole map (u,v) = (fx x/z + cx, fy y/z + cy), guard-banded.
  const S tanx = ((S)0.5 * (S)k.W) / k.fx, tany = ((S)0.5 * (S)k.H) / k.fy;
  const S limx = (S)1.3 * tanx, limy = (S)1.3 * tany;
  P.tx = x / z;
  P.ty = y / z;
  P.txc = std::min(limx, std::max(-limx, P.tx));
  P.tyc = std::min(limy, std::max(-limy, P.ty));
  P.clx = !(P.tx > -limx && P.tx < limx);
  P.cly = !(P.ty > -limy && P.ty < limy);
  const S j00 = k.fx / z, j02 = -((k.fx * P.txc) / z);
  const S j11 = k.fy / z, j12 = -((k.fy * P.tyc) / z);
  P.J[0] = j00; P.J[1] = j02; P.J[2] = j11; P.J[3] = j12;
  const S* Sc = P.Sc;
  const S T00 = j00 * Sc[0] + j02 * Sc[2];
  const S T01 = j00 * Sc[1] + j02 * Sc[5];
  const S T02 = j00 * Sc[2] + j02 * Sc[8];
  const S T11 = j11 * Sc[4] + j12 * Sc[5];
  const S T12 = j11 * Sc[5] + j12 * Sc[8];
  const S a = (T00 * j00 + T02 * j02) + (S)0.3;
  const S b = T01 * j11 + T02 * j12;
  const S c = (T11 * j11 + T12 * j12) + (S)0.3;
  P.cov[0] = a; P.cov[1] = b; P.cov[2] = c;
  P.det = a * c - b * b;
  if (!d32 && !(P.det > 0)) return P;
  const S mid = (S)0.5 * (a + c);
  const S lam = mid + std::sqrt(std::max((S)0.1, mid * mid - P.det));
  const S r = std::ceil((S)3 * std::sqrt(lam));
  P.u = k.fx * P.tx + k.cx;
  P.v = k.fy * P.ty + k.cy;
  auto clampi = [](S f, int hi) -> int {
    f = std::min(std::max(f, (S)0), (S)hi);
    return (int)f;
  };
  P.rect[0] = clampi(std::floor((P.u - r) / (S)TILE), k.TX);
  P.rect[2] = clampi(std::floor((P.u + r) / (S)TILE) + (S)1, k.TX);
  P.rect[1] = clampi(std::floor((P.v - r) / (S)TILE), k.TY);
  P.rect[3] = clampi(std::floor((P.v + r) / (S)TILE) + (S)1, k.TY);
  P.radius = (int)std::min(r, (S)2147483647.0);
  if (d32) {
    for (int i = 0; i < 4; ++i) P.rect[i] = d32->rect[i];
    P.radius = d32->radius;
  } else if (k.thresholds && (P.rect[2] <= P.rect[0] || P.rect[3] <= P.rect[1])) {
    return P;
  }
  P.depth = z;
  P.key = d32 ? (S)d32->depth : z;
  P.conic[0] = c / P.det;
  P.conic[1] = -b / P.det;
  P.conic[2] = a / P.det;
  // colour from SH along the view direction mu - camera centre
  S cp[3];
  for (int i = 0; i < 3; ++i)
    cp[i] = -((R[0 * 3 + i] * k.t[0] + R[1 * 3 + i] * k.t[1]) + R[2 * 3 + i] * k.t[2]);
  S d[3] = {mu[0] - cp[0], mu[1] - cp[1], mu[2] - cp[2]};
  P.dlen = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  for (int i = 0; i < 3; ++i) P.dir[i] = d[i] / P.dlen;
  S Y[16];
  sh_basis<S>(deg, P.dir[0], P.dir[1], P.dir[2], Y, nullptr);
  const int K = (deg + 1) * (deg + 1);
  for (int ch = 0; ch < 3; ++ch) {
    S acc = 0;
    for (int kk = 0; kk < K; ++kk) acc += sh[kk * 3 + ch] * Y[kk];
    acc += (S)0.5;
    P.rgb_pos[ch] = acc > 0;
    P.rgb[ch] = acc > 0 ? acc : (S)0;
  }
  P.valid = true;
  return P;
}

template <class S>
struct Inputs {
  int64_t n;
  const S *means, *scales, *quats, *opac, *sh, *feat;
  int deg, D;
};

template <class S>
std::vector<Proj<S>> project_all(const Cam<S>& k, const Inputs<S>& in,
                                 const std::vector<Proj<float>>* d32 = nullptr) {
  const int K = (in.deg + 1) * (in.deg + 1);
  std::vector<Proj<S>> P((size_t)in.n);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < in.n; ++i)
    P[i] = project_one<S>(k, in.means + 3 * i, in.scales + 3 * i, in.quats + 4 * i,
                          in.sh + (size_t)K * 3 * i, in.deg, d32 ? &(*d32)[(size_t)i] : nullptr);
  return P;
}

// ---------------------------------------------------------------- candidate lists
template <class S>
bool covers(const Proj<S>& P, const Cam<S>& k, int tx, int ty) {
  if (!P.valid) return false;
  if (!k.thresholds) return true;
  return tx >= P.rect[0] && tx < P.rect[2] && ty >= P.rect[1] && ty < P.rect[3];
}

template <class S>
bool depth_less(const std::vector<Proj<S>>& P, int64_t a, int64_t b) {
  if (P[a].key != P[b].key) return P[a].key < P[b].key;
  return a < b;
}

// Brute force: every Gaussian whose rectangle covers the pixel's tile, by (depth, id).
template <class S>
std::vector<int64_t> brute_candidates(const std::vector<Proj<S>>& P, const Cam<S>& k, int tx,
                                      int ty) {
  std::vector<int64_t> c;
  for (int64_t i = 0; i < (int64_t)P.size(); ++i)
    if (covers(P[i], k, tx, ty)) c.push_back(i);
  std::sort(c.begin(), c.end(), [&](int64_t a, int64_t b) { return depth_less(P, a, b); });
  return c;
}

uint32_t float_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}

// Tile lists: emit (tile, depth) keys per Gaussian in id order, tiles row-major,
// then a stable sort by the 64-bit key (tile << 32 | depth bits).
template <class S>
void tile_lists(const std::vector<Proj<S>>& P, const Cam<S>& k, std::vector<uint64_t>& keys,
                std::vector<uint32_t>& ids, std::vector<uint32_t>& ranges) {
  keys.clear();
  ids.clear();
  for (int64_t i = 0; i < (int64_t)P.size(); ++i) {
    if (!P[i].valid) continue;
    const uint32_t db = float_bits((float)P[i].key);
    for (int ty = P[i].rect[1]; ty < P[i].rect[3]; ++ty)
      for (int tx = P[i].rect[0]; tx < P[i].rect[2]; ++tx) {
        keys.push_back(((uint64_t)(ty * k.TX + tx) << 32) | db);
        ids.push_back((uint32_t)i);
      }
  }
  std::vector<size_t> order(keys.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](size_t a, size_t b) { return keys[a] < keys[b]; });
  std::vector<uint64_t> k2(keys.size());
  std::vector<uint32_t> i2(keys.size());
  for (size_t j = 0; j < order.size(); ++j) {
    k2[j] = keys[order[j]];
    i2[j] = ids[order[j]];
  }
  keys.swap(k2);
  ids.swap(i2);
  const int T = k.TX * k.TY;
  ranges.assign((size_t)2 * T, 0);
  for (size_t j = 0; j < keys.size(); ++j) {
    const uint32_t t = (uint32_t)(keys[j] >> 32);
    if (j == 0 || (uint32_t)(keys[j - 1] >> 32) != t) ranges[2 * t] = (uint32_t)j;
    if (j + 1 == keys.size() || (uint32_t)(keys[j + 1] >> 32) != t) ranges[2 * t + 1] = (uint32_t)(j + 1);
  }
}

// ---------------------------------------------------------------- per-pixel blending
template <class S>
struct Contrib {
  int64_t id;
  S alpha, G, T, dx, dy;
  bool clamped;  // alpha hit the 0.99 cap
};

enum : int32_t {
  FLAG_SIGMA = 1,   // sigma < 0 met
  FLAG_LOW = 2,     // alpha within margin of 1/255
  FLAG_CAP = 4,     // o*G within margin of 0.99
  FLAG_STOP = 8,    // T(1-alpha) within margin of 1e-4
};

template <class S>
struct PixelOut {
  S rgb[3], depth, T;
  std::vector<S> feat;
  int32_t n_contrib;
  int32_t flags;
  std::vector<Contrib<S>> list;
};

// Eq. 1 (front-to-back alpha blending) with rgb, depth (App. B) and features (Sec. 3.1),
// thresholds: skip sigma<0 or alpha<1/255, alpha capped at 0.99, stop before a
// Gaussian that would take T below 1e-4.
template <class S>
PixelOut<S> blend_pixel(const std::vector<Proj<S>>& P, const Cam<S>& k, const Inputs<S>& in,
                        const std::vector<int64_t>& cand, int px, int py, bool keep_list) {
  PixelOut<S> o;
  o.rgb[0] = o.rgb[1] = o.rgb[2] = 0;
  o.depth = 0;
  o.feat.assign((size_t)in.D, (S)0);
  o.n_contrib = 0;
  o.flags = 0;
  S T = 1;
  const S cxp = (S)px + (S)0.5, cyp = (S)py + (S)0.5;
  const S lo = (S)1 / (S)255;
  const double mrel = 2e-5, mT = 1e-3;
  for (size_t j = 0; j < cand.size(); ++j) {
    const Proj<S>& g = P[cand[j]];
    const S dx = cxp - g.u, dy = cyp - g.v;
    const S sigma = (S)0.5 * (g.conic[0] * dx * dx + g.conic[2] * dy * dy) + g.conic[1] * dx * dy;
    const S op = in.opac[cand[j]];
    if (k.thresholds && sigma < 0) {
      o.flags |= FLAG_SIGMA;
      continue;
    }
    const S G = std::exp(-sigma);
    const S oG = op * G;
    S alpha = oG;
    bool clamped = false;
    if (k.thresholds) {
      if (std::fabs((double)oG - 0.99) <= mrel * 0.99) o.flags |= FLAG_CAP;
      if (oG > (S)0.99) { alpha = (S)0.99; clamped = true; }
      if (std::fabs((double)alpha - (double)lo) <= mrel * (double)lo) o.flags |= FLAG_LOW;
      if (alpha < lo) continue;
    }
    const S Tn = T * ((S)1 - alpha);
    if (k.thresholds) {
      if (std::fabs((double)Tn - 1e-4) <= mT * 1e-4) o.flags |= FLAG_STOP;
      if (Tn < (S)0.0001) break;
    }
    const S w = alpha * T;
    for (int ch = 0; ch < 3; ++ch) o.rgb[ch] += g.rgb[ch] * w;
    o.depth += g.depth * w;
    const S* f = in.feat + (size_t)in.D * cand[j];
    for (int c = 0; c < in.D; ++c) o.feat[c] += f[c] * w;
    if (keep_list) o.list.push_back(Contrib<S>{cand[j], alpha, G, T, dx, dy, clamped});
    T = Tn;
    o.n_contrib = (int32_t)(j + 1);
  }
  o.T = T;
  return o;
}

// Per-pixel candidate list: by brute force (mode 0) or through the sorted tile lists (mode 1).
template <class S>
struct CandidateSource {
  const std::vector<Proj<S>>& P;
  const Cam<S>& k;
  int mode;
  std::vector<uint64_t> keys;
  std::vector<uint32_t> ids, ranges;
  CandidateSource(const std::vector<Proj<S>>& P_, const Cam<S>& k_, int mode_)
      : P(P_), k(k_), mode(mode_) {
    if (mode == 1 && k.thresholds) tile_lists<S>(P, k, keys, ids, ranges);
  }
  std::vector<int64_t> get(int tx, int ty) const {
    if (mode == 1 && k.thresholds) {
      const int t = ty * k.TX + tx;
      std::vector<int64_t> c;
      for (uint32_t j = ranges[2 * t]; j < ranges[2 * t + 1]; ++j) c.push_back(ids[j]);
      return c;
    }
    return brute_candidates<S>(P, k, tx, ty);
  }
};

template <class S>
std::vector<int64_t> pixel_set(const Cam<S>& k, const int64_t* pix, int64_t npix) {
  std::vector<int64_t> v;
  if (pix) {
    v.assign(pix, pix + npix);
  } else {
    v.resize((size_t)k.W * k.H);
    std::iota(v.begin(), v.end(), 0);
  }
  return v;
}

// Candidate lists per tile, built once and shared by the pixels of that tile.
template <class S>
std::vector<std::vector<int64_t>> tile_candidates(const CandidateSource<S>& src, const Cam<S>& k,
                                                  const std::vector<int64_t>& pixels) {
  std::vector<std::vector<int64_t>> per_tile((size_t)k.TX * k.TY);
  std::vector<char> need((size_t)k.TX * k.TY, 0);
  for (int64_t p : pixels) need[(p % k.W) / TILE + (p / k.W) / TILE * k.TX] = 1;
#pragma omp parallel for schedule(dynamic)
  for (int64_t t = 0; t < (int64_t)need.size(); ++t)
    if (need[t]) per_tile[t] = src.get((int)(t % k.TX), (int)(t / k.TX));
  return per_tile;
}

template <class S>
int render(const Inputs<S>& in, const Cam<S>& k, int mode, const int64_t* pix, int64_t npix,
           S* rgb, S* depth, S* alpha, S* feat, S* T_final, int32_t* n_contrib, int32_t* flags,
           const std::vector<Proj<float>>* d32 = nullptr) {
  auto P = project_all<S>(k, in, d32);
  CandidateSource<S> src(P, k, mode);
  auto pixels = pixel_set<S>(k, pix, npix);
  auto per_tile = tile_candidates<S>(src, k, pixels);
  const int64_t np = (int64_t)pixels.size();
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t q = 0; q < np; ++q) {
    const int64_t p = pixels[q];
    const int px = (int)(p % k.W), py = (int)(p / k.W);
    const auto& cand = per_tile[px / TILE + py / TILE * k.TX];
    PixelOut<S> o = blend_pixel<S>(P, k, in, cand, px, py, false);
    if (rgb) for (int ch = 0; ch < 3; ++ch) rgb[ch * np + q] = o.rgb[ch];
    if (depth) depth[q] = o.depth;
    if (alpha) alpha[q] = (S)1 - o.T;
    if (feat) for (int c = 0; c < in.D; ++c) feat[(int64_t)c * np + q] = o.feat[c];
    if (T_final) T_final[q] = o.T;
    if (n_contrib) n_contrib[q] = o.n_contrib;
    if (flags) flags[q] = o.flags;
  }
  return 0;
}

// ---------------------------------------------------------------- backward
// Per-Gaussian gradient w.r.t. the 2D quantities of the blend.
template <class S>
struct Grad2D {
  S u = 0, v = 0, A = 0, B = 0, C = 0, o = 0, rgb[3] = {0, 0, 0}, z = 0;
};

// Reverse-mode derivative of blend_pixel for one pixel.  With w_i = alpha_i T_i and
// T_i = prod_{j<i}(1 - alpha_j):
//   dC/dalpha_i = T_i (c_i - S_i),  S_i = sum_{k>i} c_k alpha_k prod_{i<j<k}(1-alpha_j)
//   d(1 - T_final)/dalpha_i = T_final / (1 - alpha_i)
template <class S>
void pixel_backward(const std::vector<Proj<S>>& P, const Inputs<S>& in, const PixelOut<S>& o,
                    const S* gC, S gD, S gA, const S* gF, std::vector<Grad2D<S>>& g2,
                    std::vector<S>& gfeat) {
  const int D = in.D;
  S sC[3] = {0, 0, 0}, sD = 0;
  std::vector<S> sF((size_t)D, (S)0);
  const S Tf = o.T;
  for (int j = (int)o.list.size() - 1; j >= 0; --j) {
    const Contrib<S>& c = o.list[j];
    const Proj<S>& g = P[c.id];
    const S* f = in.feat + (size_t)D * c.id;
    const S w = c.alpha * c.T;
    S dalpha = 0;
    for (int ch = 0; ch < 3; ++ch) dalpha += gC[ch] * (g.rgb[ch] - sC[ch]);
    dalpha += gD * (g.depth - sD);
    for (int d = 0; d < D; ++d) dalpha += gF[d] * (f[d] - sF[d]);
    dalpha *= c.T;
    dalpha += gA * Tf / ((S)1 - c.alpha);
    for (int ch = 0; ch < 3; ++ch) sC[ch] = c.alpha * g.rgb[ch] + ((S)1 - c.alpha) * sC[ch];
    sD = c.alpha * g.depth + ((S)1 - c.alpha) * sD;
    for (int d = 0; d < D; ++d) sF[d] = c.alpha * f[d] + ((S)1 - c.alpha) * sF[d];

    Grad2D<S>& G2 = g2[c.id];
    for (int ch = 0; ch < 3; ++ch) G2.rgb[ch] += w * gC[ch];
    G2.z += w * gD;
    for (int d = 0; d < D; ++d) gfeat[(size_t)D * c.id + d] += w * gF[d];
    if (c.clamped) continue;
    const S op = in.opac[c.id];
    G2.o += dalpha * c.G;
    const S dsigma = -dalpha * op * c.G;  // alpha = o exp(-sigma)
    G2.A += dsigma * (S)0.5 * c.dx * c.dx;
    G2.B += dsigma * c.dx * c.dy;
    G2.C += dsigma * (S)0.5 * c.dy * c.dy;
    // dx = px - u: dsigma/du = -(A dx + B dy), dsigma/dv = -(C dy + B dx)
    G2.u += -dsigma * (g.conic[0] * c.dx + g.conic[1] * c.dy);
    G2.v += -dsigma * (g.conic[2] * c.dy + g.conic[1] * c.dx);
  }
}

// Chain rule from the 2D quantities back to (mu, s, q, o, sh) and the pose twist
// xi = (rho, phi) of a left perturbation T <- Exp(xi) T.
template <class S>
void project_backward(const Cam<S>& k, const Inputs<S>& in, const std::vector<Proj<S>>& P,
                      const std::vector<Grad2D<S>>& g2, S* g_means, S* g_scales, S* g_quats,
                      S* g_opac, S* g_sh, S* g_pose) {
  const int K = (in.deg + 1) * (in.deg + 1);
  S pose[6] = {0, 0, 0, 0, 0, 0};
  const S* R = k.R;
  for (int64_t i = 0; i < in.n; ++i) {
    S* gm = g_means + 3 * i;
    S* gs = g_scales + 3 * i;
    S* gq = g_quats + 4 * i;
    S* gsh = g_sh + (size_t)K * 3 * i;
    for (int c = 0; c < 3; ++c) gm[c] = gs[c] = 0;
    for (int c = 0; c < 4; ++c) gq[c] = 0;
    for (int c = 0; c < K * 3; ++c) gsh[c] = 0;
    g_opac[i] = 0;
    const Proj<S>& g = P[i];
    if (!g.valid) continue;
    const Grad2D<S>& d2 = g2[i];
    g_opac[i] = d2.o;
    const S x = g.p[0], y = g.p[1], z = g.p[2];
    S gp[3] = {0, 0, 0};  // dL/d p_cam
    // mean2d: u = fx x/z + cx, v = fy y/z + cy
    gp[0] += d2.u * k.fx / z;
    gp[1] += d2.v * k.fy / z;
    gp[2] += -d2.u * k.fx * x / (z * z) - d2.v * k.fy * y / (z * z);
    // depth = z
    gp[2] += d2.z;
    // conic Q = cov^{-1}: dL/dcov = -Q Gq Q with Gq the symmetric gradient of Q
    const S Qa = g.conic[0], Qb = g.conic[1], Qc = g.conic[2];
    const S Ga = d2.A, Gb = (S)0.5 * d2.B, Gc = d2.C;
    // X = Q Gq
    const S X00 = Qa * Ga + Qb * Gb, X01 = Qa * Gb + Qb * Gc;
    const S X10 = Qb * Ga + Qc * Gb, X11 = Qb * Gb + Qc * Gc;
    // Y = X Q, Gcov = -Y (symmetric)
    const S C00 = -(X00 * Qa + X01 * Qb);
    const S C01 = -(X00 * Qb + X01 * Qc);
    const S C11 = -(X10 * Qb + X11 * Qc);
    // cov = J Sc J^T + 0.3 I: dL/dSc = J^T Gcov J, dL/dJ = 2 Gcov J Sc
    S Jm[6] = {g.J[0], 0, g.J[1], 0, g.J[2], g.J[3]};  // 2x3
    S Gcov[4] = {C00, C01, C01, C11};
    S GSc[9];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        S acc = 0;
        for (int r = 0; r < 2; ++r)
          for (int s = 0; s < 2; ++s) acc += Jm[r * 3 + a] * Gcov[r * 2 + s] * Jm[s * 3 + b];
        GSc[a * 3 + b] = acc;
      }
    S GJ[6];
    for (int r = 0; r < 2; ++r)
      for (int b = 0; b < 3; ++b) {
        S acc = 0;
        for (int s = 0; s < 2; ++s)
          for (int c = 0; c < 3; ++c) acc += Gcov[r * 2 + s] * Jm[s * 3 + c] * g.Sc[c * 3 + b];
        GJ[r * 3 + b] = (S)2 * acc;
      }
    // J = [[fx/z, 0, -fx txc/z], [0, fy/z, -fy tyc/z]]
    gp[2] += -GJ[0] * k.fx / (z * z) - GJ[4] * k.fy / (z * z);
    gp[2] += GJ[2] * k.fx * g.txc / (z * z) + GJ[5] * k.fy * g.tyc / (z * z);
    if (!g.clx) {
      const S gt = -GJ[2] * k.fx / z;  // d/d txc
      gp[0] += gt / z;
      gp[2] += -gt * x / (z * z);
    }
    if (!g.cly) {
      const S gt = -GJ[5] * k.fy / z;
      gp[1] += gt / z;
      gp[2] += -gt * y / (z * z);
    }
    // Sc = W Sigma W^T: dL/dSigma = W^T GSc W
    S GSig[9];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        S acc = 0;
        for (int r = 0; r < 3; ++r)
          for (int s = 0; s < 3; ++s) acc += R[r * 3 + a] * GSc[r * 3 + s] * R[s * 3 + b];
        GSig[a * 3 + b] = acc;
      }
    // Sigma = M M^T: dL/dM = 2 GSig M
    S GM[9];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        S acc = 0;
        for (int r = 0; r < 3; ++r) acc += GSig[a * 3 + r] * g.M[r * 3 + b];
        GM[a * 3 + b] = (S)2 * acc;
      }
    // M = Rq diag(s)
    S GR[9];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) GR[a * 3 + b] = GM[a * 3 + b] * in.scales[3 * i + b];
    for (int b = 0; b < 3; ++b) {
      S acc = 0;
      for (int a = 0; a < 3; ++a) acc += GM[a * 3 + b] * g.Rq[a * 3 + b];
      gs[b] = acc;
    }
    // Rq(w,x,y,z) of the unit quaternion
    const S w = g.qn[0], qx = g.qn[1], qy = g.qn[2], qz = g.qn[3];
    S gn[4];
    gn[0] = (S)2 * (-qz * GR[1] + qy * GR[2] + qz * GR[3] - qx * GR[5] - qy * GR[6] + qx * GR[7]);
    gn[1] = (S)2 * (qy * GR[1] + qz * GR[2] + qy * GR[3] - (S)2 * qx * GR[4] - w * GR[5] +
                    qz * GR[6] + w * GR[7] - (S)2 * qx * GR[8]);
    gn[2] = (S)2 * (-(S)2 * qy * GR[0] + qx * GR[1] + w * GR[2] + qx * GR[3] + qz * GR[5] -
                    w * GR[6] + qz * GR[7] - (S)2 * qy * GR[8]);
    gn[3] = (S)2 * (-(S)2 * qz * GR[0] - w * GR[1] + qx * GR[2] + w * GR[3] - (S)2 * qz * GR[4] +
                    qy * GR[5] + qx * GR[6] + qy * GR[7]);
    // q_hat = q / |q|
    const S dotn = gn[0] * g.qn[0] + gn[1] * g.qn[1] + gn[2] * g.qn[2] + gn[3] * g.qn[3];
    for (int c = 0; c < 4; ++c) gq[c] = (gn[c] - g.qn[c] * dotn) / g.qlen;
    // SH colour: rgb_ch = max(0, sum_k sh[k,ch] Y_k(dir) + 0.5), dir = (mu - cam)/|mu - cam|
    S Y[16], dY[16][3];
    sh_basis<S>(in.deg, g.dir[0], g.dir[1], g.dir[2], Y, dY);
    S gdir[3] = {0, 0, 0};
    const S* sh = in.sh + (size_t)K * 3 * i;
    for (int ch = 0; ch < 3; ++ch) {
      if (!g.rgb_pos[ch]) continue;
      const S gc = d2.rgb[ch];
      for (int kk = 0; kk < K; ++kk) {
        gsh[kk * 3 + ch] = gc * Y[kk];
        for (int e = 0; e < 3; ++e) gdir[e] += gc * sh[kk * 3 + ch] * dY[kk][e];
      }
    }
    const S dd = gdir[0] * g.dir[0] + gdir[1] * g.dir[1] + gdir[2] * g.dir[2];
    S gdv[3];
    for (int e = 0; e < 3; ++e) gdv[e] = (gdir[e] - g.dir[e] * dd) / g.dlen;
    // p_cam = W mu + t
    for (int c = 0; c < 3; ++c)
      gm[c] = (R[0 * 3 + c] * gp[0] + R[1 * 3 + c] * gp[1] + R[2 * 3 + c] * gp[2]) + gdv[c];
    // pose twist: d p_cam = rho + phi x p_cam ; d Sc = [phi]x Sc - Sc [phi]x ;
    // d campos = -W^T rho (campos enters through -gdv)
    S Am[9];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        S acc = 0;
        for (int r = 0; r < 3; ++r) acc += g.Sc[a * 3 + r] * GSc[r * 3 + b] - GSc[a * 3 + r] * g.Sc[r * 3 + b];
        Am[a * 3 + b] = acc;
      }
    for (int c = 0; c < 3; ++c)
      pose[c] += gp[c] + (R[c * 3 + 0] * gdv[0] + R[c * 3 + 1] * gdv[1] + R[c * 3 + 2] * gdv[2]);
    pose[3] += (y * gp[2] - z * gp[1]) + (Am[5] - Am[7]);
    pose[4] += (z * gp[0] - x * gp[2]) + (Am[6] - Am[2]);
    pose[5] += (x * gp[1] - y * gp[0]) + (Am[1] - Am[3]);
  }
  if (g_pose)
    for (int c = 0; c < 6; ++c) g_pose[c] = pose[c];
}

template <class S>
int backward(const Inputs<S>& in, const Cam<S>& k, int mode, const int64_t* pix, int64_t npix,
             const S* g_rgb, const S* g_depth, const S* g_alpha, const S* g_feat, S* g_means,
             S* g_scales, S* g_quats, S* g_opac, S* g_sh, S* g_featp, S* g_pose, S* g2d_out,
             const std::vector<Proj<float>>* d32 = nullptr) {
  auto P = project_all<S>(k, in, d32);
  CandidateSource<S> src(P, k, mode);
  auto pixels = pixel_set<S>(k, pix, npix);
  auto per_tile = tile_candidates<S>(src, k, pixels);
  const int64_t np = (int64_t)pixels.size();
  const int D = in.D;
  std::vector<PixelOut<S>> outs((size_t)np);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t q = 0; q < np; ++q) {
    const int64_t p = pixels[q];
    const int px = (int)(p % k.W), py = (int)(p / k.W);
    outs[q] = blend_pixel<S>(P, k, in, per_tile[px / TILE + py / TILE * k.TX], px, py, true);
  }
  std::vector<Grad2D<S>> g2((size_t)in.n);
  std::vector<S> gfeat((size_t)in.n * D, (S)0);
  std::vector<S> gF((size_t)D);
  for (int64_t q = 0; q < np; ++q) {  // fixed order: deterministic sums
    S gC[3];
    for (int ch = 0; ch < 3; ++ch) gC[ch] = g_rgb ? g_rgb[ch * np + q] : (S)0;
    for (int d = 0; d < D; ++d) gF[d] = g_feat ? g_feat[(int64_t)d * np + q] : (S)0;
    pixel_backward<S>(P, in, outs[q], gC, g_depth ? g_depth[q] : (S)0,
                      g_alpha ? g_alpha[q] : (S)0, gF.data(), g2, gfeat);
    outs[q].list.clear();
    outs[q].list.shrink_to_fit();
  }
  if (g_featp) std::copy(gfeat.begin(), gfeat.end(), g_featp);
  if (g2d_out)
    for (int64_t i = 0; i < in.n; ++i) {
      const Grad2D<S>& d = g2[i];
      S v[10] = {d.u, d.v, d.A, d.B, d.C, d.o, d.rgb[0], d.rgb[1], d.rgb[2], d.z};
      std::copy(v, v + 10, g2d_out + 10 * i);
    }
  project_backward<S>(k, in, P, g2, g_means, g_scales, g_quats, g_opac, g_sh, g_pose);
  return 0;
}

template <class S>
Inputs<S> make_inputs(int64_t n, const S* means, const S* scales, const S* quats, const S* opac,
                      const S* sh, int deg, const S* feat, int D) {
  Inputs<S> in;
  in.n = n; in.means = means; in.scales = scales; in.quats = quats; in.opac = opac;
  in.sh = sh; in.deg = deg; in.feat = feat; in.D = D;
  return in;
}

template <class S>
int project_out(int64_t n, const S* means, const S* scales, const S* quats, const S* opac,
                const S* sh, int deg, const double* cam, int thresholds, S* mean2d, S* conic,
                S* depth, S* rgb, int32_t* rect, int32_t* radius, uint8_t* valid) {
  const Cam<S> k = make_cam<S>(cam, thresholds);
  auto in = make_inputs<S>(n, means, scales, quats, opac, sh, deg, nullptr, 0);
  auto P = project_all<S>(k, in);
  for (int64_t i = 0; i < n; ++i) {
    const Proj<S>& g = P[i];
    valid[i] = g.valid ? 1 : 0;
    mean2d[2 * i] = g.valid ? g.u : (S)0;
    mean2d[2 * i + 1] = g.valid ? g.v : (S)0;
    for (int c = 0; c < 3; ++c) conic[3 * i + c] = g.valid ? g.conic[c] : (S)0;
    depth[i] = g.valid ? g.depth : (S)0;
    for (int c = 0; c < 3; ++c) rgb[3 * i + c] = g.valid ? g.rgb[c] : (S)0;
    for (int c = 0; c < 4; ++c) rect[4 * i + c] = g.valid ? g.rect[c] : 0;
    radius[i] = g.valid ? g.radius : 0;
  }
  return 0;
}

}  // namespace

// ---------------------------------------------------------------- C entry points
extern "C" {

int or_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

#define OR_PROJECT(S, SUF)                                                                      \
  int or_project_##SUF(int64_t n, const S* means, const S* scales, const S* quats,             \
                       const S* opac, const S* sh, int deg, const double* cam, int thresholds, \
                       S* mean2d, S* conic, S* depth, S* rgb, int32_t* rect, int32_t* radius,  \
                       uint8_t* valid) {                                                        \
    return project_out<S>(n, means, scales, quats, opac, sh, deg, cam, thresholds, mean2d,     \
                          conic, depth, rgb, rect, radius, valid);                              \
  }
OR_PROJECT(float, f32)
OR_PROJECT(double, f64)

// Sorted tile lists of the float projection.  Returns the instance count; copies at
// most `cap` keys/ids.  ranges has 2*TX*TY entries.
int64_t or_tile_lists_f32(int64_t n, const float* means, const float* scales, const float* quats,
                          const float* opac, const float* sh, int deg, const double* cam,
                          int64_t cap, uint64_t* keys, uint32_t* ids, uint32_t* ranges) {
  const Cam<float> k = make_cam<float>(cam, 1);
  auto in = make_inputs<float>(n, means, scales, quats, opac, sh, deg, nullptr, 0);
  auto P = project_all<float>(k, in);
  std::vector<uint64_t> kk;
  std::vector<uint32_t> ii, rr;
  tile_lists<float>(P, k, kk, ii, rr);
  const int64_t m = std::min<int64_t>(cap, (int64_t)kk.size());
  if (keys) std::copy(kk.begin(), kk.begin() + m, keys);
  if (ids) std::copy(ii.begin(), ii.begin() + m, ids);
  if (ranges) std::copy(rr.begin(), rr.end(), ranges);
  return (int64_t)kk.size();
}

#define OR_RENDER(S, SUF)                                                                       \
  int or_render_##SUF(int64_t n, const S* means, const S* scales, const S* quats, const S* opac, \
                      const S* sh, int deg, const S* feat, int D, const double* cam,            \
                      int thresholds, int mode, const int64_t* pix, int64_t npix, S* rgb,       \
                      S* depth, S* alpha, S* featout, S* T_final, int32_t* n_contrib,           \
                      int32_t* flags) {                                                         \
    const Cam<S> k = make_cam<S>(cam, thresholds);                                              \
    auto in = make_inputs<S>(n, means, scales, quats, opac, sh, deg, feat, D);                  \
    return render<S>(in, k, mode, pix, npix, rgb, depth, alpha, featout, T_final, n_contrib,    \
                     flags);                                                                    \
  }
OR_RENDER(float, f32)
OR_RENDER(double, f64)

#define OR_BACKWARD(S, SUF)                                                                      \
  int or_backward_##SUF(int64_t n, const S* means, const S* scales, const S* quats,             \
                        const S* opac, const S* sh, int deg, const S* feat, int D,              \
                        const double* cam, int thresholds, int mode, const int64_t* pix,        \
                        int64_t npix, const S* g_rgb, const S* g_depth, const S* g_alpha,       \
                        const S* g_feat, S* g_means, S* g_scales, S* g_quats, S* g_opac,        \
                        S* g_sh, S* g_featp, S* g_pose, S* g2d) {                               \
    const Cam<S> k = make_cam<S>(cam, thresholds);                                               \
    auto in = make_inputs<S>(n, means, scales, quats, opac, sh, deg, feat, D);                   \
    return backward<S>(in, k, mode, pix, npix, g_rgb, g_depth, g_alpha, g_feat, g_means,        \
                       g_scales, g_quats, g_opac, g_sh, g_featp, g_pose, g2d);                  \
  }
OR_BACKWARD(float, f32)
OR_BACKWARD(double, f64)

// Mixed mode: double arithmetic with the float projection's visibility, tile rectangles and
// list order (the same function as the float path in exact arithmetic; see the header).
struct FloatCopy {
  std::vector<float> means, scales, quats, opac, sh;
};
static std::vector<Proj<float>> float_decisions(int64_t n, const double* means,
                                                const double* scales, const double* quats,
                                                const double* opac, const double* sh, int deg,
                                                const double* cam) {
  const int K = (deg + 1) * (deg + 1);
  FloatCopy f;
  f.means.assign(means, means + 3 * n);
  f.scales.assign(scales, scales + 3 * n);
  f.quats.assign(quats, quats + 4 * n);
  f.opac.assign(opac, opac + n);
  f.sh.assign(sh, sh + (size_t)K * 3 * n);
  const Cam<float> k = make_cam<float>(cam, 1);
  auto in = make_inputs<float>(n, f.means.data(), f.scales.data(), f.quats.data(), f.opac.data(),
                               f.sh.data(), deg, nullptr, 0);
  return project_all<float>(k, in);
}

int or_render_mixed(int64_t n, const double* means, const double* scales, const double* quats,
                    const double* opac, const double* sh, int deg, const double* feat, int D,
                    const double* cam, int mode, const int64_t* pix, int64_t npix, double* rgb,
                    double* depth, double* alpha, double* featout, double* T_final,
                    int32_t* n_contrib, int32_t* flags) {
  const auto d32 = float_decisions(n, means, scales, quats, opac, sh, deg, cam);
  const Cam<double> k = make_cam<double>(cam, 1);
  auto in = make_inputs<double>(n, means, scales, quats, opac, sh, deg, feat, D);
  return render<double>(in, k, mode, pix, npix, rgb, depth, alpha, featout, T_final, n_contrib,
                        flags, &d32);
}

int or_backward_mixed(int64_t n, const double* means, const double* scales, const double* quats,
                      const double* opac, const double* sh, int deg, const double* feat, int D,
                      const double* cam, int mode, const int64_t* pix, int64_t npix,
                      const double* g_rgb, const double* g_depth, const double* g_alpha,
                      const double* g_feat, double* g_means, double* g_scales, double* g_quats,
                      double* g_opac, double* g_sh, double* g_featp, double* g_pose, double* g2d) {
  const auto d32 = float_decisions(n, means, scales, quats, opac, sh, deg, cam);
  const Cam<double> k = make_cam<double>(cam, 1);
  auto in = make_inputs<double>(n, means, scales, quats, opac, sh, deg, feat, D);
  return backward<double>(in, k, mode, pix, npix, g_rgb, g_depth, g_alpha, g_feat, g_means,
                          g_scales, g_quats, g_opac, g_sh, g_featp, g_pose, g2d, &d32);
}

// Real SH basis values [npts, 16] for testing orthonormality.
void or_sh_basis_f64(int deg, int64_t npts, const double* dirs, double* Y) {
  for (int64_t i = 0; i < npts; ++i) {
    double y[16] = {0};
    sh_basis<double>(deg, dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], y, nullptr);
    std::copy(y, y + 16, Y + 16 * i);
  }
}

}  // extern "C"
