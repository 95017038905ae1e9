// Confidence-filtered fusion of submap points into one global point buffer.
//
// The paper takes "the global coordinates of all points in the current
// submap" from the estimated submap transforms (Sec. III-C, Point
// Correction); every pixel of a submap carries a confidence (Sec. III-C,
// Feed-Forward Inference).  Kept points (confidence > threshold) are written
// in ascending flat index, so the compaction is unique and its indices are
// exact:
//
//   k_fuse_count    one CTA per tile of 8192 points of one submap: keep count
//                   and the tile's 1-bit keep mask
//   k_fuse_scan     one CTA: exclusive scan of the tile counts from *cursor,
//                   advances *cursor by the total
//   k_fuse_scatter  one CTA per tile: ordered block-wide compaction in rounds
//                   of 1024 points (the keep bits from the mask), Sim(3)
//                   transform in FP32 (FMA), writes the point and its int64
//                   global index
//
// Bytes per input point: 4 + 1/8 (count) + 12 + 1/8 (scatter read) + 20 per
// kept point.
#include <cfloat>

#include "common.cuh"

namespace ec3r {
namespace fuse {

constexpr int TILE = 8192;
constexpr int THREADS = 256;
constexpr int ROUND = 4 * THREADS;  // points per compaction round

__device__ __forceinline__ bool keep(float c, float thr) { return c > thr; }  // NaN -> false

constexpr int MASK_WORDS = TILE / 32;  // keep-mask words per tile

// Kept points per tile and the tile's keep mask: bit i % 32 of word
// t * MASK_WORDS + i / 32 is point i of tile t (bits past the tile's end are
// 0).  A round covers 1024 points, 4 per thread, so 8 consecutive lanes fill
// one word.
template <bool VEC>
__global__ void __launch_bounds__(THREADS) k_fuse_count(const float* __restrict__ conf,
                                                        int64_t n, int tps, float thr,
                                                        int32_t* __restrict__ tile_count,
                                                        uint32_t* __restrict__ mask) {
  const int64_t t = blockIdx.x;
  const int64_t m = t / tps;
  const int c = (int)(t - m * tps);
  const int64_t base = m * n + (int64_t)c * TILE;
  const int64_t rem = n - (int64_t)c * TILE;
  const int npx = rem < TILE ? (int)rem : TILE;
  const int lane = threadIdx.x & 31;
  int cnt = 0;
  for (int r0 = 0; r0 < npx; r0 += 4 * THREADS) {  // every lane takes every round
    const int i0 = r0 + 4 * threadIdx.x;
    unsigned nib = 0;
    if (VEC && i0 + 4 <= npx) {
      const float4 v = __ldcs(reinterpret_cast<const float4*>(conf + base + i0));
      nib = (unsigned)keep(v.x, thr) | (unsigned)keep(v.y, thr) << 1 |
            (unsigned)keep(v.z, thr) << 2 | (unsigned)keep(v.w, thr) << 3;
    } else {
      for (int j = 0; j < 4; ++j)
        if (i0 + j < npx && keep(conf[base + i0 + j], thr)) nib |= 1u << j;
    }
    cnt += __popc(nib);
    unsigned w = nib << (4 * (lane & 7));
    w |= __shfl_xor_sync(0xffffffffu, w, 1);
    w |= __shfl_xor_sync(0xffffffffu, w, 2);
    w |= __shfl_xor_sync(0xffffffffu, w, 4);
    if ((lane & 7) == 0) mask[t * MASK_WORDS + (r0 >> 5) + (threadIdx.x >> 3)] = w;
  }
  // words past the last round of a short tile
  for (int w = ((npx + 4 * THREADS - 1) / (4 * THREADS)) * (4 * THREADS / 32) + threadIdx.x;
       w < MASK_WORDS; w += THREADS)
    mask[t * MASK_WORDS + w] = 0u;
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  __shared__ int red[THREADS / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < THREADS / 32; ++w) s += red[w];
    tile_count[t] = s;
  }
}

// Single-CTA exclusive scan of the tile counts.  tile_off[t] = *cursor + sum
// of counts before t; *cursor += total.
__global__ void __launch_bounds__(1024) k_fuse_scan(const int32_t* __restrict__ tile_count,
                                                    int64_t n_tiles,
                                                    int64_t* __restrict__ tile_off,
                                                    int64_t* cursor) {
  __shared__ int64_t wsum[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = *cursor;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t b = 0; b < n_tiles; b += 1024) {
    const int64_t i = b + threadIdx.x;
    const int64_t v = i < n_tiles ? tile_count[i] : 0;
    int64_t x = v;  // inclusive warp scan
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int64_t ws = wsum[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws += y;
      }
      wsum[lane] = ws;  // inclusive over warps
    }
    __syncthreads();
    const int64_t before = (warp > 0 ? wsum[warp - 1] : 0) + x - v;
    if (i < n_tiles) tile_off[i] = carry + before;
    __syncthreads();
    if (threadIdx.x == 0) carry += wsum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) *cursor = carry;
}

// One compaction round of a scatter CTA: this thread's kept points (mask km
// over its 4 points i0..i0+3 of the tile) get consecutive slots in point order
// (warp scan, then across warps), `point(j, dst)` writes point j's three
// global coordinates into shared memory, and the round's kept points are
// written with coalesced stores at [pos, pos + total) (nothing at or past
// `capacity`); pos advances by the round's total.
template <class Point>
__device__ __forceinline__ void emit_round(unsigned km, int i0, int64_t gbase, int64_t& pos,
                                           int64_t capacity, bool& overflow,
                                           float* __restrict__ out_xyz,
                                           int64_t* __restrict__ out_idx, int* wcnt, float* sx,
                                           int64_t* sidx, Point&& point) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cnt = __popc(km);
  int x = cnt;  // inclusive warp scan of counts (thread order = point order)
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wcnt[warp] = x;
  __syncthreads();
  int wbefore = 0, total = 0;
  for (int w = 0; w < THREADS / 32; ++w) {
    const int v = wcnt[w];
    wbefore += w < warp ? v : 0;
    total += v;
  }
  int q = wbefore + (x - cnt);  // slot of this thread's first kept point in the round
  for (int j = 0; j < 4; ++j) {
    if (!(km & (1u << j))) continue;
    point(j, sx + 3 * q);
    sidx[q] = gbase + i0 + j;
    ++q;
  }
  __syncthreads();
  int64_t lim = pos < 0 ? 0 : capacity - pos;  // points that still fit (none past a bad cursor)
  if (lim < 0) lim = 0;
  const int nw = (int)(total < lim ? total : lim);
  if (nw < total) overflow = true;
  float* ox = out_xyz + 3 * pos;
  for (int i = threadIdx.x; i < 3 * nw; i += THREADS) ox[i] = sx[i];
  for (int i = threadIdx.x; i < nw; i += THREADS) out_idx[pos + i] = sidx[i];
  pos += total;
  __syncthreads();
}

// One CTA per tile, rounds of 1024 points (4 per thread).  The keep decision
// comes from the count pass's mask (1 bit per point instead of a 4-byte
// confidence); the next round's loads are in flight while the current one is
// compacted, and each round's kept points are staged in shared memory and
// written with coalesced stores.
template <bool VEC>
__global__ void __launch_bounds__(THREADS) k_fuse_scatter(
    const float* __restrict__ xyz, const uint32_t* __restrict__ mask, int64_t n, int tps,
    const ec3r_sim3* __restrict__ poses, int64_t index_base,
    const int64_t* __restrict__ tile_off, float* __restrict__ out_xyz,
    int64_t* __restrict__ out_idx, int64_t capacity, unsigned* flags) {
  const int64_t t = blockIdx.x;
  const int64_t m = t / tps;
  const int c = (int)(t - m * tps);
  const int64_t tile0 = (int64_t)c * TILE;
  const int64_t base = m * n + tile0;
  const int64_t rem = n - tile0;
  const int npx = rem < TILE ? (int)rem : TILE;
  __shared__ float A[12];
  __shared__ int wcnt[THREADS / 32];
  __shared__ float sx[3 * ROUND];
  __shared__ int64_t sidx[ROUND];
  if (threadIdx.x < 12) {
    const ec3r_sim3& P = poses[m];
    const int r = threadIdx.x / 4, col = threadIdx.x % 4;
    A[threadIdx.x] = col < 3 ? (float)(P.s * P.R[3 * r + col]) : (float)P.t[r];
  }
  __syncthreads();
  const float a00 = A[0], a01 = A[1], a02 = A[2], a03 = A[3];
  const float a10 = A[4], a11 = A[5], a12 = A[6], a13 = A[7];
  const float a20 = A[8], a21 = A[9], a22 = A[10], a23 = A[11];
  int64_t pos = tile_off[t];
  bool overflow = false;

  const uint32_t* tmask = mask + t * MASK_WORDS;
  unsigned nb;
  float p[12];
  auto load = [&](int r0) {
    const int i0 = r0 + 4 * threadIdx.x;
    nb = (tmask[(r0 >> 5) + (threadIdx.x >> 3)] >> (4 * (threadIdx.x & 7))) & 0xFu;
    if (VEC && i0 + 4 <= npx) {
      const float4* X = reinterpret_cast<const float4*>(xyz + 3 * (base + i0));
      const float4 u = __ldcs(X), w = __ldcs(X + 1), z = __ldcs(X + 2);
      p[0] = u.x; p[1] = u.y; p[2] = u.z; p[3] = u.w; p[4] = w.x; p[5] = w.y;
      p[6] = w.z; p[7] = w.w; p[8] = z.x; p[9] = z.y; p[10] = z.z; p[11] = z.w;
    } else {
      for (int j = 0; j < 4; ++j) {
        const bool in = i0 + j < npx;
        for (int d = 0; d < 3; ++d) p[3 * j + d] = in ? xyz[3 * (base + i0 + j) + d] : 0.f;
      }
    }
  };
  if (npx > 0) load(0);
  for (int r0 = 0; r0 < npx; r0 += ROUND) {
    const int i0 = r0 + 4 * threadIdx.x;
    float cp[12];
    const unsigned cnb = nb;
    for (int j = 0; j < 12; ++j) cp[j] = p[j];
    if (r0 + ROUND < npx) load(r0 + ROUND);  // next round in flight
    unsigned km = 0;
    for (int j = 0; j < 4; ++j) km |= (i0 + j < npx && ((cnb >> j) & 1u)) ? (1u << j) : 0u;
    emit_round(km, i0, index_base + base, pos, capacity, overflow, out_xyz, out_idx, wcnt, sx,
               sidx, [&](int j, float* dst) {
                 const float x0 = cp[3 * j], x1 = cp[3 * j + 1], x2 = cp[3 * j + 2];
                 dst[0] = fmaf(a00, x0, fmaf(a01, x1, fmaf(a02, x2, a03)));
                 dst[1] = fmaf(a10, x0, fmaf(a11, x1, fmaf(a12, x2, a13)));
                 dst[2] = fmaf(a20, x0, fmaf(a21, x1, fmaf(a22, x2, a23)));
               });
  }
  if (overflow && threadIdx.x == 0) atomicOr(flags, FLAG_CAPACITY);
}

// --------------------------------------------------------------------------
// fusion straight from depth maps and cameras
// --------------------------------------------------------------------------
// A point exists where the frame's camera is usable (finite, fx, fy != 0) and
// the depth is finite and > 0; it is kept when, in addition, its confidence is
// strictly above the threshold.  Tiles are 8192 pixels of one frame, so the
// flat index of every point is g = frame * H * W + pixel, the same as the
// pointmap fusion's (submap-major, then frame, row, column).
__device__ __forceinline__ bool cam_usable(const ec3r_camera& c) {
  bool ok = c.fx != 0.f && c.fy != 0.f;
  const float* f = &c.fx;
  for (int i = 0; i < 16; ++i) ok &= fabsf(f[i]) <= FLT_MAX;
  return ok;
}

__device__ __forceinline__ bool keepz(float d, float c, float thr) {
  return d > 0.f && d <= FLT_MAX && c > thr;
}

// Kept points per tile and the tile's keep mask, in k_fuse_count's layout
// (an unusable camera keeps nothing).
template <bool VEC>
__global__ void __launch_bounds__(THREADS) k_fusez_count(const float* __restrict__ depth,
                                                         const float* __restrict__ conf,
                                                         const ec3r_camera* __restrict__ cams,
                                                         int64_t hw, int tpf, float thr,
                                                         int32_t* __restrict__ tile_count,
                                                         uint32_t* __restrict__ mask) {
  const int64_t t = blockIdx.x;
  const int64_t fr = t / tpf;
  const int c = (int)(t - fr * tpf);
  const int64_t base = fr * hw + (int64_t)c * TILE;
  const int64_t rem = hw - (int64_t)c * TILE;
  const int npx = rem < TILE ? (int)rem : TILE;
  const bool usable = cam_usable(cams[fr]);
  const int lane = threadIdx.x & 31;
  int cnt = 0;
  for (int r0 = 0; r0 < npx; r0 += 4 * THREADS) {  // every lane takes every round
    const int i0 = r0 + 4 * threadIdx.x;
    unsigned nib = 0;
    if (usable) {
      if (VEC && i0 + 4 <= npx) {
        const float4 d = __ldcs(reinterpret_cast<const float4*>(depth + base + i0));
        const float4 v = __ldcs(reinterpret_cast<const float4*>(conf + base + i0));
        nib = (unsigned)keepz(d.x, v.x, thr) | (unsigned)keepz(d.y, v.y, thr) << 1 |
              (unsigned)keepz(d.z, v.z, thr) << 2 | (unsigned)keepz(d.w, v.w, thr) << 3;
      } else {
        for (int j = 0; j < 4; ++j)
          if (i0 + j < npx && keepz(depth[base + i0 + j], conf[base + i0 + j], thr))
            nib |= 1u << j;
      }
    }
    cnt += __popc(nib);
    unsigned w = nib << (4 * (lane & 7));
    w |= __shfl_xor_sync(0xffffffffu, w, 1);
    w |= __shfl_xor_sync(0xffffffffu, w, 2);
    w |= __shfl_xor_sync(0xffffffffu, w, 4);
    if ((lane & 7) == 0) mask[t * MASK_WORDS + (r0 >> 5) + (threadIdx.x >> 3)] = w;
  }
  // words past the last round of a short tile
  for (int w = ((npx + 4 * THREADS - 1) / (4 * THREADS)) * (4 * THREADS / 32) + threadIdx.x;
       w < MASK_WORDS; w += THREADS)
    mask[t * MASK_WORDS + w] = 0u;
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  __shared__ int red[THREADS / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < THREADS / 32; ++w) s += red[w];
    tile_count[t] = s;
  }
}

// As k_fuse_scatter, the point of a kept pixel (row v, column u) being
// A (d (u - cx)/fx, d (v - cy)/fy, d) + a with (A, a) = the submap pose composed
// with the camera pose, formed in FP64 and rounded to FP32 once per CTA.
template <bool VEC>
__global__ void __launch_bounds__(THREADS) k_fusez_scatter(
    const float* __restrict__ depth, const uint32_t* __restrict__ mask,
    const ec3r_camera* __restrict__ cams, int W, int64_t hw, int tpf, int frames,
    const ec3r_sim3* __restrict__ poses, int64_t index_base,
    const int64_t* __restrict__ tile_off, float* __restrict__ out_xyz,
    int64_t* __restrict__ out_idx, int64_t capacity, unsigned* flags) {
  const int64_t t = blockIdx.x;
  const int64_t fr = t / tpf;
  const int c = (int)(t - fr * tpf);
  const int64_t tile0 = (int64_t)c * TILE;
  const int64_t base = fr * hw + tile0;
  const int64_t rem = hw - tile0;
  const int npx = rem < TILE ? (int)rem : TILE;
  __shared__ float A[16];
  __shared__ int wcnt[THREADS / 32];
  __shared__ float sx[3 * ROUND];
  __shared__ int64_t sidx[ROUND];
  const ec3r_camera& cam = cams[fr];
  if (threadIdx.x < 12) {
    const ec3r_sim3& P = poses[fr / frames];
    const int r = threadIdx.x / 4, col = threadIdx.x % 4;
    double v = 0.0;  // (s R_m [R_f | t_f]) + [0 | t_m], row r, column col
    for (int k = 0; k < 3; ++k)
      v += P.s * P.R[3 * r + k] * (col < 3 ? (double)cam.R[3 * k + col] : (double)cam.t[k]);
    A[threadIdx.x] = (float)(col < 3 ? v : v + P.t[r]);
  } else if (threadIdx.x == 12) {
    A[12] = 1.f / cam.fx;
    A[13] = 1.f / cam.fy;
    A[14] = cam.cx;
    A[15] = cam.cy;
  }
  __syncthreads();
  const float a00 = A[0], a01 = A[1], a02 = A[2], a03 = A[3];
  const float a10 = A[4], a11 = A[5], a12 = A[6], a13 = A[7];
  const float a20 = A[8], a21 = A[9], a22 = A[10], a23 = A[11];
  const float ifx = A[12], ify = A[13], cx = A[14], cy = A[15];
  int64_t pos = tile_off[t];
  bool overflow = false;

  // the keep decision from the count pass's mask (1 bit per point instead of
  // a 4-byte confidence); the depth is read for the kept points' coordinates
  const uint32_t* tmask = mask + t * MASK_WORDS;
  unsigned nb;
  float dd[4];
  auto load = [&](int r0) {
    const int i0 = r0 + 4 * threadIdx.x;
    nb = (tmask[(r0 >> 5) + (threadIdx.x >> 3)] >> (4 * (threadIdx.x & 7))) & 0xFu;
    if (VEC && i0 + 4 <= npx) {
      const float4 d = __ldcs(reinterpret_cast<const float4*>(depth + base + i0));
      dd[0] = d.x; dd[1] = d.y; dd[2] = d.z; dd[3] = d.w;
    } else {
      for (int j = 0; j < 4; ++j) dd[j] = i0 + j < npx ? depth[base + i0 + j] : 0.f;
    }
  };
  if (npx > 0) load(0);
  for (int r0 = 0; r0 < npx; r0 += ROUND) {
    const int i0 = r0 + 4 * threadIdx.x;
    float cd[4];
    const unsigned cnb = nb;
    for (int j = 0; j < 4; ++j) cd[j] = dd[j];
    if (r0 + ROUND < npx) load(r0 + ROUND);  // next round in flight
    unsigned km = 0;
    for (int j = 0; j < 4; ++j) km |= (i0 + j < npx && ((cnb >> j) & 1u)) ? (1u << j) : 0u;
    const unsigned pix0 = (unsigned)(tile0 + i0);  // < 2^31
    const unsigned v0 = pix0 / (unsigned)W;
    const unsigned u0 = pix0 - v0 * (unsigned)W;
    emit_round(km, i0, index_base + base, pos, capacity, overflow, out_xyz, out_idx, wcnt, sx,
               sidx, [&](int j, float* dst) {
                 unsigned u = u0 + j, v = v0;
                 while (u >= (unsigned)W) { u -= (unsigned)W; ++v; }  // at most 3 steps
                 const float d = cd[j];
                 const float x0 = d * (((float)u - cx) * ifx), x1 = d * (((float)v - cy) * ify);
                 dst[0] = fmaf(a00, x0, fmaf(a01, x1, fmaf(a02, d, a03)));
                 dst[1] = fmaf(a10, x0, fmaf(a11, x1, fmaf(a12, d, a13)));
                 dst[2] = fmaf(a20, x0, fmaf(a21, x1, fmaf(a22, d, a23)));
               });
  }
  if (overflow && threadIdx.x == 0) atomicOr(flags, FLAG_CAPACITY);
}

}  // namespace fuse
}  // namespace ec3r

using namespace ec3r;
using namespace ec3r::fuse;

// Argument checks shared by the pointmap fusion entries; *tps and *n_tiles
// receive the tiling.  EC3R_OK with n_tiles = 0 means nothing to do.
static ec3r_status fuse_args(ec3r_ctx* ctx, int n_submaps, int64_t pts_per_submap,
                             float conf_threshold, int64_t* tps, int64_t* n_tiles) {
  *tps = *n_tiles = 0;
  if (n_submaps < 0 || pts_per_submap < 0)
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "negative size");
  if (n_submaps == 0 || pts_per_submap == 0) return EC3R_OK;
  if (conf_threshold != conf_threshold)
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "conf_threshold is NaN");
  *tps = (pts_per_submap + TILE - 1) / TILE;
  *n_tiles = *tps * n_submaps;
  if (*n_tiles >= ((int64_t)1 << 31) || *tps >= ((int64_t)1 << 30))
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "problem too large for one call");
  return EC3R_OK;
}

static void launch_count(ec3r_ctx* ctx, cudaStream_t s, const float* d_conf,
                         int64_t pts_per_submap, int64_t tps, int64_t n_tiles,
                         float conf_threshold, int32_t* cnt, uint32_t* mask) {
  const bool vec = (pts_per_submap % 4 == 0) && ((uintptr_t)d_conf % 16 == 0);
  traced(ctx, s, "fuse_count", [&] {
    if (vec)
      k_fuse_count<true><<<(unsigned)n_tiles, THREADS, 0, s>>>(d_conf, pts_per_submap, (int)tps,
                                                               conf_threshold, cnt, mask);
    else
      k_fuse_count<false><<<(unsigned)n_tiles, THREADS, 0, s>>>(
          d_conf, pts_per_submap, (int)tps, conf_threshold, cnt, mask);
  });
}

// Scan of the tile counts (after the running cursor) and the ordered scatter.
static ec3r_status scan_scatter(ec3r_ctx* ctx, cudaStream_t s, int64_t pts_per_submap,
                                int64_t tps, int64_t n_tiles, const float* d_xyz,
                                const int32_t* cnt, const uint32_t* mask,
                                const ec3r_sim3* d_poses, int64_t index_base, float* d_out_xyz,
                                int64_t* d_out_idx, int64_t capacity, int64_t* d_cursor) {
  void* p_off;
  ec3r_status st;
  if ((st = ensure_buf(ctx, "fuse.off", sizeof(int64_t) * (size_t)n_tiles, s, &p_off))) return st;
  int64_t* off = (int64_t*)p_off;
  const bool vec = (pts_per_submap % 4 == 0) && ((uintptr_t)d_xyz % 16 == 0);
  const dim3 grid((unsigned)n_tiles);
  traced(ctx, s, "fuse_scan", [&] { k_fuse_scan<<<1, 1024, 0, s>>>(cnt, n_tiles, off, d_cursor); });
  traced(ctx, s, "fuse_scatter", [&] {
    if (vec)
      k_fuse_scatter<true><<<grid, THREADS, 0, s>>>(d_xyz, mask, pts_per_submap, (int)tps,
                                                    d_poses, index_base, off, d_out_xyz,
                                                    d_out_idx, capacity, ctx->d_flags);
    else
      k_fuse_scatter<false><<<grid, THREADS, 0, s>>>(d_xyz, mask, pts_per_submap, (int)tps,
                                                     d_poses, index_base, off, d_out_xyz,
                                                     d_out_idx, capacity, ctx->d_flags);
  });
  EC3R_CUDA_TRY(ctx, cudaGetLastError());
  return EC3R_OK;
}

extern "C" ec3r_status ec3r_fuse_points(ec3r_ctx* ctx, int n_submaps, int64_t pts_per_submap,
                                        const float* d_xyz, const float* d_conf,
                                        const ec3r_sim3* d_poses, float conf_threshold,
                                        int64_t index_base, float* d_out_xyz,
                                        int64_t* d_out_idx, int64_t capacity,
                                        int64_t* d_cursor, void* stream) {
  if (!ctx) return EC3R_ERR_INVALID_ARG;
  if (capacity < 0 || index_base < 0)
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "negative size");
  int64_t tps, n_tiles;
  ec3r_status st = fuse_args(ctx, n_submaps, pts_per_submap, conf_threshold, &tps, &n_tiles);
  if (st != EC3R_OK || n_tiles == 0) return st;
  if (!d_xyz || !d_conf || !d_poses || !d_cursor || (capacity > 0 && (!d_out_xyz || !d_out_idx)))
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "a required pointer is NULL");
  EC3R_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  void *p_cnt, *p_mask;
  if ((st = ensure_buf(ctx, "fuse.count", sizeof(int32_t) * (size_t)n_tiles, s, &p_cnt)))
    return st;
  if ((st = ensure_buf(ctx, "fuse.mask", sizeof(uint32_t) * MASK_WORDS * (size_t)n_tiles, s,
                       &p_mask)))
    return st;
  int32_t* cnt = (int32_t*)p_cnt;
  uint32_t* mask = (uint32_t*)p_mask;
  launch_count(ctx, s, d_conf, pts_per_submap, tps, n_tiles, conf_threshold, cnt, mask);
  return scan_scatter(ctx, s, pts_per_submap, tps, n_tiles, d_xyz, cnt, mask, d_poses,
                      index_base, d_out_xyz, d_out_idx, capacity, d_cursor);
}

extern "C" ec3r_status ec3r_fuse_count(ec3r_ctx* ctx, int n_submaps, int64_t pts_per_submap,
                                       const float* d_conf, float conf_threshold,
                                       int32_t* d_tile_counts, uint32_t* d_keep_mask,
                                       void* stream) {
  if (!ctx) return EC3R_ERR_INVALID_ARG;
  int64_t tps, n_tiles;
  ec3r_status st = fuse_args(ctx, n_submaps, pts_per_submap, conf_threshold, &tps, &n_tiles);
  if (st != EC3R_OK || n_tiles == 0) return st;
  if (!d_conf || !d_tile_counts || !d_keep_mask)
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "a required pointer is NULL");
  EC3R_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  launch_count(ctx, (cudaStream_t)stream, d_conf, pts_per_submap, tps, n_tiles, conf_threshold,
               d_tile_counts, d_keep_mask);
  EC3R_CUDA_TRY(ctx, cudaGetLastError());
  return EC3R_OK;
}

extern "C" ec3r_status ec3r_fuse_points_counted(
    ec3r_ctx* ctx, int n_submaps, int64_t pts_per_submap, const float* d_xyz,
    const int32_t* d_tile_counts, const uint32_t* d_keep_mask, const ec3r_sim3* d_poses,
    int64_t index_base, float* d_out_xyz, int64_t* d_out_idx, int64_t capacity,
    int64_t* d_cursor, void* stream) {
  if (!ctx) return EC3R_ERR_INVALID_ARG;
  if (capacity < 0 || index_base < 0)
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "negative size");
  int64_t tps, n_tiles;
  ec3r_status st = fuse_args(ctx, n_submaps, pts_per_submap, 0.f, &tps, &n_tiles);
  if (st != EC3R_OK || n_tiles == 0) return st;
  if (!d_xyz || !d_tile_counts || !d_keep_mask || !d_poses || !d_cursor ||
      (capacity > 0 && (!d_out_xyz || !d_out_idx)))
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "a required pointer is NULL");
  EC3R_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  return scan_scatter(ctx, (cudaStream_t)stream, pts_per_submap, tps, n_tiles, d_xyz,
                      d_tile_counts, d_keep_mask, d_poses, index_base, d_out_xyz, d_out_idx,
                      capacity, d_cursor);
}

extern "C" ec3r_status ec3r_fuse_points_depth(ec3r_ctx* ctx, int n_submaps, int frames, int H,
                                              int W, const float* d_depth, const float* d_conf,
                                              const ec3r_camera* d_cams,
                                              const ec3r_sim3* d_poses, float conf_threshold,
                                              int64_t index_base, float* d_out_xyz,
                                              int64_t* d_out_idx, int64_t capacity,
                                              int64_t* d_cursor, void* stream) {
  if (!ctx) return EC3R_ERR_INVALID_ARG;
  if (n_submaps < 0 || frames < 0 || H < 0 || W < 0 || capacity < 0 || index_base < 0)
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "negative size");
  if (n_submaps == 0 || frames == 0 || H == 0 || W == 0) return EC3R_OK;
  if (!d_depth || !d_conf || !d_cams || !d_poses || !d_cursor ||
      (capacity > 0 && (!d_out_xyz || !d_out_idx)))
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "a required pointer is NULL");
  if (conf_threshold != conf_threshold)
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "conf_threshold is NaN");
  const int64_t hw = (int64_t)H * W;
  const int64_t tpf = (hw + TILE - 1) / TILE;
  const int64_t n_frames = (int64_t)n_submaps * frames;
  const int64_t n_tiles = tpf * n_frames;
  if (hw >= ((int64_t)1 << 31) || n_tiles >= ((int64_t)1 << 31))
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "problem too large for one call");
  EC3R_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  void *p_cnt, *p_off, *p_mask;
  ec3r_status st;
  if ((st = ensure_buf(ctx, "fuse.count", sizeof(int32_t) * (size_t)n_tiles, s, &p_cnt))) return st;
  if ((st = ensure_buf(ctx, "fuse.off", sizeof(int64_t) * (size_t)n_tiles, s, &p_off))) return st;
  if ((st = ensure_buf(ctx, "fuse.mask", sizeof(uint32_t) * MASK_WORDS * (size_t)n_tiles, s,
                       &p_mask)))
    return st;
  // (buffers that grew dropped the graphs holding older ones; re-read them all)
  int32_t* cnt = (int32_t*)ctx->bufs["fuse.count"].ptr;
  int64_t* off = (int64_t*)ctx->bufs["fuse.off"].ptr;
  uint32_t* mask = (uint32_t*)ctx->bufs["fuse.mask"].ptr;
  const bool vec = (hw % 4 == 0) && ((uintptr_t)d_depth % 16 == 0) &&
                   ((uintptr_t)d_conf % 16 == 0);
  const dim3 grid((unsigned)n_tiles);
  traced(ctx, s, "fusez_count", [&] {
    if (vec)
      k_fusez_count<true><<<grid, THREADS, 0, s>>>(d_depth, d_conf, d_cams, hw, (int)tpf,
                                                   conf_threshold, cnt, mask);
    else
      k_fusez_count<false><<<grid, THREADS, 0, s>>>(d_depth, d_conf, d_cams, hw, (int)tpf,
                                                    conf_threshold, cnt, mask);
  });
  traced(ctx, s, "fuse_scan", [&] { k_fuse_scan<<<1, 1024, 0, s>>>(cnt, n_tiles, off, d_cursor); });
  traced(ctx, s, "fusez_scatter", [&] {
    if (vec)
      k_fusez_scatter<true><<<grid, THREADS, 0, s>>>(
          d_depth, mask, d_cams, W, hw, (int)tpf, frames, d_poses, index_base, off, d_out_xyz,
          d_out_idx, capacity, ctx->d_flags);
    else
      k_fusez_scatter<false><<<grid, THREADS, 0, s>>>(
          d_depth, mask, d_cams, W, hw, (int)tpf, frames, d_poses, index_base, off, d_out_xyz,
          d_out_idx, capacity, ctx->d_flags);
  });
  EC3R_CUDA_TRY(ctx, cudaGetLastError());
  return EC3R_OK;
}
