// Batched Sim(3) registration straight from depth maps and cameras (Sec. III-C:
// a submap is the inverse projection of the predicted depths D through the
// predicted cameras g; every pixel of a keyframe is one point).
//
// The result is the registration of the unprojected pointmaps
//   X(v, u) = R_f (d(v, u) K_f^-1 [u, v, 1]^T) + t_f     (pixel row v, column u)
// but the sweeps never form X in submap coordinates.  A link (src frame f_p,
// tgt frame f_q) is swept in its two cameras' frames: x = d_p ray_p(u, v),
// y = d_q ray_q(u, v), read as 4-byte depths instead of 12-byte points (16 B
// per correspondence with the confidences, against 32 B).  With p = R_p x +
// t_p and q = R_q y + t_q the residual of a pair estimate (A, b) is
// |A (p - P) + b - (q - Q)| = |A_l (x - X_l) + b_l - (y - Y_l)| with
// A_l = R_q^T A R_p, b_l = R_q^T b, X_l = R_p^T (P - t_p), Y_l = R_q^T (Q - t_q),
// so the per-pixel arithmetic is that of the pointmap sweep with per-link
// constants.  The per-link moments are rotated back to the pair's frame in
// FP64 before the solve: Sp = R_p Sx, Sq = R_q Sy, Sqp = R_q Syx R_p^T, while
// W, Spp, the cost and the count are invariant.
//
//   k_setup_depth   one CTA per pair: link checks, pivots P, Q (mean of 1024
//                   sampled valid correspondences, unprojected to submap
//                   coordinates), per-link pivots and rays, identity estimate
//   k_sweep_depth   one CTA per tile of 8192 pixels of one link
//   k_solve_depth   one warp per pair: per-link FP64 tile sums, rotation to the
//                   pair frame, weighted Umeyama, per-link constants of the new
//                   estimate
#include <cfloat>

#include "align_impl.cuh"

namespace ec3r {
namespace align {

// Per-link constants of the depth sweep (FP32, camera frames).
struct LinkState {
  float A[9], b[3];    // current estimate seen from the link's cameras
  float Ap[9], bp[3];  // previous estimate
  float px[3], py[3];  // pivots X_l, Y_l
  float kp[4], kq[4];  // (1/fx, 1/fy, cx, cy) of the src and tgt cameras
  int ok;              // both cameras finite with nonzero focal lengths
};

// A camera is usable when all its entries are finite and fx, fy != 0 (else
// every point of its frame is invalid, as the unprojection gives no point).
__device__ __forceinline__ bool camera_ok(const ec3r_camera& c) {
  bool ok = c.fx != 0.f && c.fy != 0.f;
  const float* f = &c.fx;
  for (int i = 0; i < 16; ++i) ok &= finitef(f[i]);
  return ok;
}

__device__ __forceinline__ bool depth_ok(float d) { return d > 0.f && d <= FLT_MAX; }

// Camera-frame point of depth d at pixel (v, u); k = (1/fx, 1/fy, cx, cy).
// A non-positive or non-finite depth gives NaN (an invalid point).
__device__ __forceinline__ void cam_point(float d, float u, float v, const float* k, float& x0,
                                          float& x1, float& x2) {
  const float dd = depth_ok(d) ? d : __int_as_float(0x7fc00000);
  x0 = dd * ((u - k[2]) * k[0]);
  x1 = dd * ((v - k[3]) * k[1]);
  x2 = dd;
}

__global__ void __launch_bounds__(THREADS) k_setup_depth(
    const float* __restrict__ depth, const float* __restrict__ conf,
    const ec3r_camera* __restrict__ cams, int64_t n_frames, int W, int64_t hw, int n_pairs,
    int64_t n_links, const int32_t* __restrict__ link_off, const int32_t* __restrict__ src,
    const int32_t* __restrict__ tgt, const float* __restrict__ pair_cmin, float cmin_default,
    int32_t* __restrict__ link_pair, const int32_t* __restrict__ malformed,
    PairState* __restrict__ st, LinkState* __restrict__ ls, unsigned* flags) {
  const int k = blockIdx.x;
  __shared__ int bad;
  __shared__ float red[THREADS / 32][7];
  __shared__ float piv[6];
  // a malformed offset array (k_check_offsets) marks every pair of the batch
  const int64_t l0 = *malformed ? 0 : link_off[k], l1 = *malformed ? 0 : link_off[k + 1];
  if (threadIdx.x == 0) bad = *malformed;
  __syncthreads();
  if (!bad) {
    for (int64_t l = l0 + threadIdx.x; l < l1; l += THREADS) {
      const int a = src[l], b = tgt[l];
      if (a < 0 || a >= n_frames || b < 0 || b >= n_frames) bad = 1;
    }
  }
  __syncthreads();
  const float cmin = pair_cmin ? pair_cmin[k] : cmin_default;
  if (!bad) {
    for (int64_t l = l0 + threadIdx.x; l < l1; l += THREADS) link_pair[l] = k;
  }
  // pivots: mean of up to 1024 valid correspondences sampled evenly, in
  // submap coordinates
  float acc[7] = {0, 0, 0, 0, 0, 0, 0};
  if (!bad && l1 > l0) {
    const int64_t npix = (l1 - l0) * hw;
    for (int j = threadIdx.x; j < 1024; j += THREADS) {
      int64_t f = (int64_t)((double)j * (double)npix / 1024.0);
      if (f >= npix) f = npix - 1;
      const int64_t l = l0 + f / hw, px = f % hw;
      const float u = (float)(px % W), v = (float)(px / W);
      const ec3r_camera& cp_ = cams[src[l]];
      const ec3r_camera& cq_ = cams[tgt[l]];
      const float dp = depth[(int64_t)src[l] * hw + px], dq = depth[(int64_t)tgt[l] * hw + px];
      const float cp = conf[(int64_t)src[l] * hw + px], cq = conf[(int64_t)tgt[l] * hw + px];
      const float kp[4] = {1.f / cp_.fx, 1.f / cp_.fy, cp_.cx, cp_.cy};
      const float kq[4] = {1.f / cq_.fx, 1.f / cq_.fy, cq_.cx, cq_.cy};
      float x[3], y[3];
      cam_point(dp, u, v, kp, x[0], x[1], x[2]);
      cam_point(dq, u, v, kq, y[0], y[1], y[2]);
      float p[3], q[3];
      for (int i = 0; i < 3; ++i) {
        p[i] = cp_.R[3 * i] * x[0] + cp_.R[3 * i + 1] * x[1] + cp_.R[3 * i + 2] * x[2] + cp_.t[i];
        q[i] = cq_.R[3 * i] * y[0] + cq_.R[3 * i + 1] * y[1] + cq_.R[3 * i + 2] * y[2] + cq_.t[i];
      }
      const bool ok = finitef(p[0]) && finitef(p[1]) && finitef(p[2]) && finitef(q[0]) &&
                      finitef(q[1]) && finitef(q[2]) && finitef(cp) && finitef(cq) &&
                      cp > cmin && cq > cmin;
      if (ok) {
        acc[0] += p[0]; acc[1] += p[1]; acc[2] += p[2];
        acc[3] += q[0]; acc[4] += q[1]; acc[5] += q[2];
        acc[6] += 1.f;
      }
    }
  }
  for (int m = 0; m < 7; ++m)
    for (int o = 16; o > 0; o >>= 1) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], o);
  if ((threadIdx.x & 31) == 0)
    for (int m = 0; m < 7; ++m) red[threadIdx.x >> 5][m] = acc[m];
  __syncthreads();
  if (threadIdx.x == 0) {
    float s[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int w = 0; w < THREADS / 32; ++w)
      for (int m = 0; m < 7; ++m) s[m] += red[w][m];
    PairState& S = st[k];
    const float inv = s[6] > 0.f ? 1.f / s[6] : 0.f;
    for (int i = 0; i < 3; ++i) {
      S.piv_p[i] = s[i] * inv;
      S.piv_q[i] = s[3 + i] * inv;
      piv[i] = S.piv_p[i];
      piv[3 + i] = S.piv_q[i];
    }
    for (int i = 0; i < 9; ++i) {
      S.A[i] = S.Ap[i] = (i % 4 == 0) ? 1.f : 0.f;
      S.Ad[i] = S.Adp[i] = (i % 4 == 0) ? 1.0 : 0.0;
    }
    for (int i = 0; i < 3; ++i) {
      S.b[i] = S.bp[i] = 0.f;
      S.bd[i] = S.bdp[i] = 0.0;
    }
    S.cmin = cmin;
    S.active = bad ? 0 : 1;
    S.status = bad ? (int)EC3R_PAIR_BAD_INPUT : 0;
    if (bad) atomicOr(flags, FLAG_BAD_INDEX);
  }
  __syncthreads();
  if (bad) return;
  // per-link constants: pivots in the cameras' frames, rays, and the identity
  // pair estimate seen from the cameras (A_l = R_q^T R_p, b_l = 0)
  for (int64_t l = l0 + threadIdx.x; l < l1; l += THREADS) {
    const ec3r_camera& a = cams[src[l]];
    const ec3r_camera& c = cams[tgt[l]];
    LinkState& L = ls[l];
    L.ok = camera_ok(a) && camera_ok(c);
    if (!L.ok) {  // no valid pixel; finite zero constants keep the sums finite
      for (int i = 0; i < 9; ++i) L.A[i] = L.Ap[i] = 0.f;
      for (int i = 0; i < 3; ++i) L.b[i] = L.bp[i] = L.px[i] = L.py[i] = 0.f;
      for (int i = 0; i < 4; ++i) L.kp[i] = L.kq[i] = 0.f;
      continue;
    }
    for (int i = 0; i < 3; ++i) {
      L.px[i] = a.R[i] * (piv[0] - a.t[0]) + a.R[3 + i] * (piv[1] - a.t[1]) +
                a.R[6 + i] * (piv[2] - a.t[2]);
      L.py[i] = c.R[i] * (piv[3] - c.t[0]) + c.R[3 + i] * (piv[4] - c.t[1]) +
                c.R[6 + i] * (piv[5] - c.t[2]);
    }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const float v = c.R[i] * a.R[j] + c.R[3 + i] * a.R[3 + j] + c.R[6 + i] * a.R[6 + j];
        L.A[3 * i + j] = L.Ap[3 * i + j] = v;
      }
    for (int i = 0; i < 3; ++i) L.b[i] = L.bp[i] = 0.f;
    L.kp[0] = 1.f / a.fx; L.kp[1] = 1.f / a.fy; L.kp[2] = a.cx; L.kp[3] = a.cy;
    L.kq[0] = 1.f / c.fx; L.kq[1] = 1.f / c.fy; L.kq[2] = c.cx; L.kq[3] = c.cy;
  }
}

// Per-tile partial moments of one link in its cameras' frames (FP32 per point,
// FP64 across warps): the pointmap sweep's point operation on unprojected
// depths.  An invalid pixel's depth is replaced by 0 before the unprojection,
// so its (finite) point carries zero weight and no per-coordinate masking is
// needed; one finiteness test of the coordinates' sum covers overflow.
template <int KIND>
struct DepthOp {
  float A[9], b[3], Ap[9], bp[3];  // residual constants (Ap, bp: the cost's weights)
  float px[3], py[3];              // the link's pivots
  float kp[4], kq[4];              // (1/fx, 1/fy, cx, cy) per side
  float delta, cmin;
  int rule;
  bool link_ok;

  // From both confidences; returns the pixel's weight as the later sweeps
  // read it (NaN: invalid).  A pixel whose unprojection overflows is invalid
  // and its coordinates are zeroed, so that its zero weight keeps the sums
  // finite.
  __device__ __forceinline__ float operator()(float dp, float dq, float cp, float cq, float u,
                                              float v, float* acc) const {
    const bool ok = link_ok && dp > 0.f && dq > 0.f && dp <= FLT_MAX && dq <= FLT_MAX &&
                    cp > cmin && cq > cmin && cp <= FLT_MAX && cq <= FLT_MAX;
    const float zp = ok ? dp : 0.f, zq = ok ? dq : 0.f;
    float x0 = zp * ((u - kp[2]) * kp[0]) - px[0];
    float x1 = zp * ((v - kp[3]) * kp[1]) - px[1];
    float x2 = zp - px[2];
    float y0 = zq * ((u - kq[2]) * kq[0]) - py[0];
    float y1 = zq * ((v - kq[3]) * kq[1]) - py[1];
    float y2 = zq - py[2];
    const bool valid = ok && finitef(((x0 + x1) + (x2 + y0)) + (y1 + y2));
    if (!valid) x0 = x1 = x2 = y0 = y1 = y2 = 0.f;
    const float w = rule == 0 ? cp * cq : cp;
    point(x0, x1, x2, y0, y1, y2, valid, valid ? w : 0.f, acc);
    return valid ? w : __int_as_float(0x7fc00000);
  }

  // From the weight the first sweep stored: no validity tests per pixel, and
  // 12 bytes read instead of 16
  __device__ __forceinline__ void operator()(float dp, float dq, float wv, float u, float v,
                                             float* acc) const {
    const bool valid = wv == wv;
    const float zp = valid ? dp : 0.f, zq = valid ? dq : 0.f;
    const float x0 = zp * ((u - kp[2]) * kp[0]) - px[0];
    const float x1 = zp * ((v - kp[3]) * kp[1]) - px[1];
    const float x2 = zp - px[2];
    const float y0 = zq * ((u - kq[2]) * kq[0]) - py[0];
    const float y1 = zq * ((v - kq[3]) * kq[1]) - py[1];
    const float y2 = zq - py[2];
    point(x0, x1, x2, y0, y1, y2, valid, valid ? wv : 0.f, acc);
  }

  __device__ __forceinline__ void point(float x0, float x1, float x2, float y0, float y1,
                                        float y2, bool valid, float w, float* acc) const {
    float h = 1.f, r2 = 0.f;
    if (KIND != FIRST) {
      const float* a = (KIND == COST) ? Ap : A;
      const float* c = (KIND == COST) ? bp : b;
      const float e0 = a[0] * x0 + a[1] * x1 + a[2] * x2 + c[0] - y0;
      const float e1 = a[3] * x0 + a[4] * x1 + a[5] * x2 + c[1] - y1;
      const float e2 = a[6] * x0 + a[7] * x1 + a[8] * x2 + c[2] - y2;
      const float rr = e0 * e0 + e1 * e1 + e2 * e2;
      h = fminf(1.f, delta * rsqrtf(rr));
      if (KIND == COST) {
        const float f0 = A[0] * x0 + A[1] * x1 + A[2] * x2 + b[0] - y0;
        const float f1 = A[3] * x0 + A[4] * x1 + A[5] * x2 + b[1] - y1;
        const float f2 = A[6] * x0 + A[7] * x1 + A[8] * x2 + b[2] - y2;
        r2 = f0 * f0 + f1 * f1 + f2 * f2;
      } else {
        r2 = rr;
      }
    }
    const float om = w * h;
    acc[M_W] += om;
    acc[M_COST] += om * r2;
    acc[M_CNT] += valid ? 1.f : 0.f;
    if (KIND == COST) return;
    const float wx0 = om * x0, wx1 = om * x1, wx2 = om * x2;
    const float wy0 = om * y0, wy1 = om * y1, wy2 = om * y2;
    acc[M_SP + 0] += wx0; acc[M_SP + 1] += wx1; acc[M_SP + 2] += wx2;
    acc[M_SQ + 0] += wy0; acc[M_SQ + 1] += wy1; acc[M_SQ + 2] += wy2;
    acc[M_PP] += wx0 * x0 + wx1 * x1 + wx2 * x2;
    acc[M_QP + 0] += wy0 * x0; acc[M_QP + 1] += wy0 * x1; acc[M_QP + 2] += wy0 * x2;
    acc[M_QP + 3] += wy1 * x0; acc[M_QP + 4] += wy1 * x1; acc[M_QP + 5] += wy1 * x2;
    acc[M_QP + 6] += wy2 * x0; acc[M_QP + 7] += wy2 * x1; acc[M_QP + 8] += wy2 * x2;
  }
};

// `wbuf` [n_links][hw]: the first sweep stores every link pixel's weight
// there (NaN: invalid); with WGT a later sweep reads it instead of both
// confidences and the validity tests.
template <int KIND, bool VEC, bool WGT>
__global__ void __launch_bounds__(THREADS, 4) k_sweep_depth(
    const float* __restrict__ depth, const float* __restrict__ conf, int W, int64_t hw, int tpl,
    const int32_t* __restrict__ src, const int32_t* __restrict__ tgt,
    const int32_t* __restrict__ link_pair, const PairState* __restrict__ st,
    const LinkState* __restrict__ ls, float delta, int rule, double* __restrict__ partials,
    float* __restrict__ wbuf) {
  const int64_t t = blockIdx.x;
  const int64_t l = t / tpl;
  const int c = (int)(t - l * tpl);
  const int k = link_pair[l];
  if (k < 0) return;
  if (!st[k].active) return;
  const LinkState& L = ls[l];
  DepthOp<KIND> op;
  for (int i = 0; i < 9; ++i) { op.A[i] = L.A[i]; op.Ap[i] = L.Ap[i]; }
  for (int i = 0; i < 3; ++i) {
    op.b[i] = L.b[i]; op.bp[i] = L.bp[i];
    op.px[i] = L.px[i]; op.py[i] = L.py[i];
  }
  for (int i = 0; i < 4; ++i) { op.kp[i] = L.kp[i]; op.kq[i] = L.kq[i]; }
  op.delta = delta;
  op.cmin = st[k].cmin;
  op.rule = rule;
  op.link_ok = L.ok != 0;

  const int64_t fs = src[l], ft = tgt[l];
  const int64_t px0 = (int64_t)c * TILE;
  const float* DP = depth + fs * hw + px0;
  const float* DQ = depth + ft * hw + px0;
  const float* CP = conf + fs * hw + px0;
  const float* CQ = conf + ft * hw + px0;
  float* WB = wbuf ? wbuf + l * hw + px0 : nullptr;  // FIRST: written; WGT: read
  const int64_t rem = hw - px0;
  const int npx = rem < TILE ? (int)rem : TILE;
  const float fW = (float)W;

  float acc[NMOM];
#pragma unroll
  for (int m = 0; m < NMOM; ++m) acc[m] = 0.f;

#pragma unroll 2
  for (int g = threadIdx.x; g < TILE / 4; g += THREADS) {
    const int i0 = 4 * g;
    if (i0 >= npx) break;
    const unsigned pix = (unsigned)(px0 + i0);  // pixel index within the frame (< 2^31)
    const unsigned v0 = pix / (unsigned)W;
    float v = (float)v0, u = (float)(pix - v0 * (unsigned)W);
    if (VEC && i0 + 4 <= npx) {
      const float4 dp = __ldcs(reinterpret_cast<const float4*>(DP + i0));
      const float4 dq = __ldcs(reinterpret_cast<const float4*>(DQ + i0));
      const float dpa[4] = {dp.x, dp.y, dp.z, dp.w}, dqa[4] = {dq.x, dq.y, dq.z, dq.w};
      if constexpr (WGT) {
        const float4 w = __ldcs(reinterpret_cast<const float4*>(WB + i0));
        const float wa[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          op(dpa[j], dqa[j], wa[j], u, v, acc);
          u += 1.f;  // exact: pixel coordinates are integers < 2^24
          if (u == fW) { u = 0.f; v += 1.f; }
        }
      } else {
        const float4 cp = __ldcs(reinterpret_cast<const float4*>(CP + i0));
        const float4 cq = __ldcs(reinterpret_cast<const float4*>(CQ + i0));
        const float cpa[4] = {cp.x, cp.y, cp.z, cp.w}, cqa[4] = {cq.x, cq.y, cq.z, cq.w};
        float wo[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          wo[j] = op(dpa[j], dqa[j], cpa[j], cqa[j], u, v, acc);
          u += 1.f;
          if (u == fW) { u = 0.f; v += 1.f; }
        }
        if (KIND == FIRST && WB)
          __stcs(reinterpret_cast<float4*>(WB + i0), make_float4(wo[0], wo[1], wo[2], wo[3]));
      }
    } else {
      const int n = min(4, npx - i0);
      for (int j = 0; j < n; ++j) {
        if constexpr (WGT) {
          op(DP[i0 + j], DQ[i0 + j], __ldcs(WB + i0 + j), u, v, acc);
        } else {
          const float wo = op(DP[i0 + j], DQ[i0 + j], CP[i0 + j], CQ[i0 + j], u, v, acc);
          if (KIND == FIRST && WB) __stcs(WB + i0 + j, wo);
        }
        u += 1.f;
        if (u == fW) { u = 0.f; v += 1.f; }
      }
    }
  }
#pragma unroll
  for (int m = 0; m < NMOM; ++m)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], o);
  __shared__ double red[THREADS / 32][NMOM];
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int m = 0; m < NMOM; ++m) red[warp][m] = (double)acc[m];
  __syncthreads();
  if (threadIdx.x < NMOM) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < THREADS / 32; ++w) s += red[w][threadIdx.x];
    partials[t * NMOM + threadIdx.x] = s;
  }
}

// One warp per pair: per link, FP64 sums of its tiles (lane m owns moment m),
// rotation of the link's moments to the pair frame (summed over links in link
// order), weighted Umeyama on lane 0, then the per-link constants of the new
// estimate (lanes over links).
__global__ void __launch_bounds__(256) k_solve_depth(
    int n_pairs, const int32_t* __restrict__ link_off, int tpl, const double* __restrict__ partials,
    const int32_t* __restrict__ src, const int32_t* __restrict__ tgt,
    const ec3r_camera* __restrict__ cams, PairState* __restrict__ st, LinkState* __restrict__ ls,
    ec3r_sim3* __restrict__ out, int32_t* __restrict__ status_out, int last) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  __shared__ double lm[8][NMOM];   // one link's moments, camera frames
  __shared__ double rot[8][18];    // R_p, R_q of that link
  __shared__ double mom[8][NMOM];  // the pair's moments
  __shared__ double est[8][12];    // new A = s R (9) and b (3)
  __shared__ int ok[8];
  if (warp >= n_pairs) return;
  PairState& S = st[warp];
  if (!S.active) {
    if (last && lane == 0) {
      write_identity(&out[warp]);
      status_out[warp] = S.status;
    }
    return;
  }
  const int l0 = link_off[warp], l1 = link_off[warp + 1];
  double acc = 0.0;  // lane m < NMOM: pair moment m
  for (int l = l0; l < l1; ++l) {
    if (!ls[l].ok) continue;  // no valid pixel (and possibly a non-finite camera)
    if (lane < NMOM)
      lm[wib][lane] = tile_sum<NMOM>(partials, (int64_t)l * tpl, (int64_t)(l + 1) * tpl, lane);
    if (lane < 9) {
      rot[wib][lane] = (double)cams[src[l]].R[lane];
      rot[wib][9 + lane] = (double)cams[tgt[l]].R[lane];
    }
    __syncwarp();
    const double* m = lm[wib];
    const double* Rp = rot[wib];
    const double* Rq = rot[wib] + 9;
    if (lane == M_W || lane == M_PP || lane == M_COST || lane == M_CNT) {
      acc += m[lane];
    } else if (lane >= M_SP && lane < M_SP + 3) {
      const int i = lane - M_SP;
      acc += Rp[3 * i] * m[M_SP] + Rp[3 * i + 1] * m[M_SP + 1] + Rp[3 * i + 2] * m[M_SP + 2];
    } else if (lane >= M_SQ && lane < M_SQ + 3) {
      const int i = lane - M_SQ;
      acc += Rq[3 * i] * m[M_SQ] + Rq[3 * i + 1] * m[M_SQ + 1] + Rq[3 * i + 2] * m[M_SQ + 2];
    } else if (lane >= M_QP && lane < M_QP + 9) {
      // (R_q Syx R_p^T)_ij = sum_ab Rq_ia Syx_ab Rp_jb
      const int i = (lane - M_QP) / 3, j = (lane - M_QP) % 3;
      double v = 0.0;
      for (int a = 0; a < 3; ++a) {
        const double r = Rp[3 * j] * m[M_QP + 3 * a] + Rp[3 * j + 1] * m[M_QP + 3 * a + 1] +
                         Rp[3 * j + 2] * m[M_QP + 3 * a + 2];
        v += Rq[3 * i + a] * r;
      }
      acc += v;
    }
    __syncwarp();
  }
  if (lane < NMOM) mom[wib][lane] = acc;
  __syncwarp();
  if (lane == 0) {
    double R[9], s = 1.0, b[3];
    const unsigned status = umeyama_from_moments(mom[wib], R, s, b);
    commit_estimate(S, status, R, s, b, last != 0, out[warp], status_out[warp]);
    ok[wib] = status == 0;
    for (int i = 0; i < 9; ++i) est[wib][i] = s * R[i];
    for (int i = 0; i < 3; ++i) est[wib][9 + i] = b[i];
  }
  __syncwarp();
  if (!ok[wib]) return;
  // the new estimate seen from each link's cameras: A_l = R_q^T A R_p, b_l = R_q^T b
  const double* A = est[wib];
  const double* b = est[wib] + 9;
  for (int l = l0 + lane; l < l1; l += 32) {
    const ec3r_camera& a = cams[src[l]];
    const ec3r_camera& c = cams[tgt[l]];
    LinkState& L = ls[l];
    if (!L.ok) continue;
    double T[9];  // A R_p
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        T[3 * i + j] = A[3 * i] * a.R[j] + A[3 * i + 1] * a.R[3 + j] + A[3 * i + 2] * a.R[6 + j];
    for (int i = 0; i < 9; ++i) L.Ap[i] = L.A[i];
    for (int i = 0; i < 3; ++i) L.bp[i] = L.b[i];
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j)
        L.A[3 * i + j] =
            (float)(c.R[i] * T[j] + c.R[3 + i] * T[3 + j] + c.R[6 + i] * T[6 + j]);
      L.b[i] = (float)(c.R[i] * b[0] + c.R[3 + i] * b[1] + c.R[6 + i] * b[2]);
    }
  }
}

// The first sweep stores the link pixels' weights in `wbuf`; the later ones
// read them.
template <bool VEC>
static void launch_sweep_depth(int kind, int64_t n_tiles, cudaStream_t s, const float* depth,
                               const float* conf, int W, int64_t hw, int tpl, const int32_t* src,
                               const int32_t* tgt, const int32_t* link_pair, const PairState* st,
                               const LinkState* ls, float delta, int rule, double* partials,
                               float* wbuf) {
  const dim3 grid((unsigned)n_tiles);
  if (kind == FIRST)
    k_sweep_depth<FIRST, VEC, false><<<grid, THREADS, 0, s>>>(
        depth, conf, W, hw, tpl, src, tgt, link_pair, st, ls, delta, rule, partials, wbuf);
  else if (kind == IRLS)
    k_sweep_depth<IRLS, VEC, true><<<grid, THREADS, 0, s>>>(
        depth, conf, W, hw, tpl, src, tgt, link_pair, st, ls, delta, rule, partials, wbuf);
  else
    k_sweep_depth<COST, VEC, true><<<grid, THREADS, 0, s>>>(
        depth, conf, W, hw, tpl, src, tgt, link_pair, st, ls, delta, rule, partials, wbuf);
}

}  // namespace align
}  // namespace ec3r

using namespace ec3r;
using namespace ec3r::align;

extern "C" ec3r_status ec3r_align_submaps_depth(
    ec3r_ctx* ctx, const float* d_depth, const float* d_conf, const ec3r_camera* d_cams,
    int64_t n_frames, int H, int W, int n_pairs, int64_t n_links, const int32_t* d_link_off,
    const int32_t* d_src, const int32_t* d_tgt, const float* d_pair_conf_min,
    const ec3r_align_opts* opts, ec3r_sim3* d_out, int32_t* d_pair_status, double* d_pair_cost,
    void* stream) {
  if (!ctx) return EC3R_ERR_INVALID_ARG;
  if (!opts) return set_error(ctx, EC3R_ERR_INVALID_ARG, "opts is NULL");
  if (n_pairs < 0 || n_links < 0 || H <= 0 || W <= 0 || n_frames <= 0)
    return set_error(ctx, EC3R_ERR_INVALID_ARG,
                     "bad sizes (n_pairs %d, n_links %lld, H %d, W %d, n_frames %lld)", n_pairs,
                     (long long)n_links, H, W, (long long)n_frames);
  if (n_pairs == 0) return EC3R_OK;
  if (!d_depth || !d_conf || !d_cams || !d_link_off || !d_out || !d_pair_status ||
      (n_links > 0 && (!d_src || !d_tgt)))
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "a required pointer is NULL");
  if (!(opts->huber_delta > 0.f) || !(opts->huber_delta <= FLT_MAX) || opts->iters < 1 ||
      opts->iters > 64 || (opts->weight_rule != 0 && opts->weight_rule != 1) ||
      opts->precision != EC3R_PREC_FP32C || opts->conf_min != opts->conf_min)
    return set_error(ctx, EC3R_ERR_INVALID_ARG,
                     "bad ec3r_align_opts (the depth path computes FP32 moments only)");
  if (opts->want_cost && !d_pair_cost)
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "want_cost set but d_pair_cost is NULL");
  const int64_t hw = (int64_t)H * W;
  const int64_t tpl = (hw + TILE - 1) / TILE;
  const int64_t n_tiles = n_links * tpl;
  if (n_tiles >= ((int64_t)1 << 31) || n_frames > ((int64_t)1 << 40) / hw ||
      n_links >= ((int64_t)1 << 31) || hw >= ((int64_t)1 << 31))
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "problem too large for one call");
  EC3R_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  void *p_state, *p_part, *p_lp, *p_ls, *p_w;
  ec3r_status st;
  if ((st = ensure_buf(ctx, "depth.state", sizeof(PairState) * (size_t)n_pairs, s, &p_state)))
    return st;
  if ((st = ensure_buf(ctx, "depth.partials", sizeof(double) * NMOM * (size_t)(n_tiles + 1), s,
                       &p_part)))
    return st;
  // link -> pair map, then one word for the result of k_check_offsets
  if ((st = ensure_buf(ctx, "depth.link_pair", sizeof(int32_t) * (size_t)(n_links + 2), s,
                       &p_lp)))
    return st;
  if ((st = ensure_buf(ctx, "depth.links", sizeof(LinkState) * (size_t)(n_links + 1), s,
                       &p_ls)))
    return st;
  // every link pixel's weight (NaN: invalid), written by the first sweep
  if ((st = ensure_buf(ctx, "depth.weights", sizeof(float) * ((size_t)n_links * hw + 4), s,
                       &p_w)))
    return st;
  // every buffer may have moved if a later one grew
  PairState* state = (PairState*)ctx->bufs["depth.state"].ptr;
  double* partials = (double*)ctx->bufs["depth.partials"].ptr;
  int32_t* link_pair = (int32_t*)ctx->bufs["depth.link_pair"].ptr;
  LinkState* links = (LinkState*)ctx->bufs["depth.links"].ptr;
  float* weights = (float*)ctx->bufs["depth.weights"].ptr;
  const bool vec =
      (hw % 4 == 0) && ((uintptr_t)d_depth % 16 == 0) && ((uintptr_t)d_conf % 16 == 0);
  const ec3r_align_opts o = *opts;
  const std::string key = key_of(
      "align_depth", {(uint64_t)d_depth, (uint64_t)d_conf, (uint64_t)d_cams, (uint64_t)n_frames,
                      (uint64_t)H, (uint64_t)W, (uint64_t)n_pairs, (uint64_t)n_links,
                      (uint64_t)d_link_off, (uint64_t)d_src, (uint64_t)d_tgt,
                      (uint64_t)d_pair_conf_min, fbits(o.huber_delta), (uint64_t)o.iters,
                      fbits(o.conf_min), (uint64_t)o.weight_rule, (uint64_t)o.want_cost,
                      (uint64_t)d_out, (uint64_t)d_pair_status, (uint64_t)d_pair_cost});
  return run_graph(ctx, key, s, [&](cudaStream_t cs) -> ec3r_status {
    EC3R_CUDA_TRY(ctx, cudaMemsetAsync(link_pair, 0xff, sizeof(int32_t) * (size_t)(n_links + 1),
                                       cs));
    int32_t* malformed = link_pair + n_links + 1;
    traced(ctx, cs, "depth_setup", [&] {
      k_check_offsets<<<1, 1024, 0, cs>>>(d_link_off, n_pairs, n_links, malformed);
      k_setup_depth<<<n_pairs, THREADS, 0, cs>>>(d_depth, d_conf, d_cams, n_frames, W, hw,
                                                 n_pairs, n_links, d_link_off, d_src, d_tgt,
                                                 d_pair_conf_min, o.conf_min, link_pair,
                                                 malformed, state, links, ctx->d_flags);
    });
    for (int it = 1; it <= o.iters + (o.want_cost ? 1 : 0); ++it) {
      const int kind = it == 1 ? FIRST : (it > o.iters ? COST : IRLS);
      // the cost of a single solve uses h = 1, which a huge delta reproduces
      const float dl = (kind == COST && o.iters == 1) ? FLT_MAX : o.huber_delta;
      if (n_tiles > 0)
        traced(ctx, cs, "depth_sweep", [&] {
          if (vec)
            launch_sweep_depth<true>(kind, n_tiles, cs, d_depth, d_conf, W, hw, (int)tpl, d_src,
                                     d_tgt, link_pair, state, links, dl, o.weight_rule,
                                     partials, weights);
          else
            launch_sweep_depth<false>(kind, n_tiles, cs, d_depth, d_conf, W, hw, (int)tpl, d_src,
                                      d_tgt, link_pair, state, links, dl, o.weight_rule,
                                      partials, weights);
        });
      if (kind == COST)
        traced(ctx, cs, "depth_cost", [&] {
          k_cost<<<n_pairs, 32, 0, cs>>>(n_pairs, d_link_off, (int)tpl, partials, state,
                                         d_pair_cost, nullptr);
        });
      else
        traced(ctx, cs, "depth_solve", [&] {
          // one warp per CTA: pairs spread over all SMs' FP64 pipes
          k_solve_depth<<<n_pairs, 32, 0, cs>>>(n_pairs, d_link_off, (int)tpl, partials, d_src,
                                                d_tgt, d_cams, state, links, d_out,
                                                d_pair_status, it == o.iters);
        });
    }
    EC3R_CUDA_TRY(ctx, cudaGetLastError());
    return EC3R_OK;
  });
}
