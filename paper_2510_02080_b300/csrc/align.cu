// Batched Huber-IRLS weighted-Umeyama Sim(3) registration of submap pairs.
//
// The paper registers the current submap against every connected submap by
// minimising sum_i w_i |s R p_i + t - q_i|^2 over correspondences that are the
// same pixel of a shared keyframe, with the confidences turned into weights,
// and solves it with the weighted Umeyama closed form (Sec. III-C, Eq. (sim3)).
// Here that solve is repeated inside a Huber IRLS loop, for many pairs at once:
//
//   set-up  : k_setup      one CTA per pair: validate links, map link -> pair,
//                          pick a pivot (mean of <= 1024 sampled valid pairs)
//   sweep k : k_sweep      one CTA per tile of 8192 pixels of one link: per point
//                          validity, Huber weight from S_{k-1}, and the 19
//                          pivot-centred weighted moments; writes one FP64
//                          partial per tile (no atomics: deterministic)
//   solve k : k_solve      one warp per pair: fixed-order FP64 sum of the
//                          pair's tile partials, covariance, rotation as the
//                          orthogonal polar factor (FP32 Jacobi seed, FP64
//                          Newton-polar refinement), scale, translation
//
// The sweep is bandwidth-bound: it reads 32 bytes per pixel (p, q, c_p, c_q).
#include <algorithm>
#include <vector>

#include "align_impl.cuh"

namespace ec3r {
namespace align {

// --------------------------------------------------------------------------
// set-up
// --------------------------------------------------------------------------
// One thread per sampled correspondence: the 1024 pivot samples are one
// round of loads instead of four.
constexpr int SETUP_THREADS = 1024;

__global__ void __launch_bounds__(SETUP_THREADS) k_setup(
    const float* __restrict__ xyz, const float* __restrict__ conf, int64_t n_frames, int64_t hw,
    int n_pairs, int64_t n_links, const int32_t* __restrict__ link_off,
    const int32_t* __restrict__ src, const int32_t* __restrict__ tgt,
    const float* __restrict__ pair_cmin, float cmin_default, int32_t* __restrict__ link_pair,
    const int32_t* __restrict__ malformed, PairState* __restrict__ st, unsigned* flags,
    ec3r_sim3* __restrict__ out, int32_t* __restrict__ status_out, double* __restrict__ cost,
    double* __restrict__ cost_sums) {
  const int k = blockIdx.x;
  __shared__ int bad;
  __shared__ float red[SETUP_THREADS / 32][7];
  // a malformed offset array (k_check_offsets) marks every pair of the batch
  const int64_t l0 = *malformed ? 0 : link_off[k], l1 = *malformed ? 0 : link_off[k + 1];
  if (threadIdx.x == 0) bad = *malformed;
  __syncthreads();
  if (!bad) {
    for (int64_t l = l0 + threadIdx.x; l < l1; l += SETUP_THREADS) {
      const int a = src[l], b = tgt[l];
      if (a < 0 || a >= n_frames || b < 0 || b >= n_frames) bad = 1;
    }
  }
  __syncthreads();
  const float cmin = pair_cmin ? pair_cmin[k] : cmin_default;
  if (!bad) {
    for (int64_t l = l0 + threadIdx.x; l < l1; l += SETUP_THREADS) link_pair[l] = k;
  }
  // pivot: mean of up to 1024 valid correspondences sampled evenly
  float acc[7] = {0, 0, 0, 0, 0, 0, 0};
  if (!bad && l1 > l0) {
    const int64_t npix = (l1 - l0) * hw;
    for (int j = threadIdx.x; j < 1024; j += SETUP_THREADS) {
      int64_t f = (int64_t)((double)j * (double)npix / 1024.0);
      if (f >= npix) f = npix - 1;
      const int64_t l = l0 + f / hw, px = f % hw;
      const float* P = xyz + ((int64_t)src[l] * hw + px) * 3;
      const float* Q = xyz + ((int64_t)tgt[l] * hw + px) * 3;
      const float cp = conf[(int64_t)src[l] * hw + px], cq = conf[(int64_t)tgt[l] * hw + px];
      const float p0 = P[0], p1 = P[1], p2 = P[2], q0 = Q[0], q1 = Q[1], q2 = Q[2];
      const bool v = finitef(p0) && finitef(p1) && finitef(p2) && finitef(q0) && finitef(q1) &&
                     finitef(q2) && finitef(cp) && finitef(cq) && cp > cmin && cq > cmin;
      if (v) {
        acc[0] += p0; acc[1] += p1; acc[2] += p2;
        acc[3] += q0; acc[4] += q1; acc[5] += q2;
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
    for (int w = 0; w < SETUP_THREADS / 32; ++w)
      for (int m = 0; m < 7; ++m) s[m] += red[w][m];
    PairState& S = st[k];
    const float inv = s[6] > 0.f ? 1.f / s[6] : 0.f;
    for (int i = 0; i < 3; ++i) {
      S.piv_p[i] = s[i] * inv;
      S.piv_q[i] = s[3 + i] * inv;
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
    // A pair without links is degenerate before any solve: with a bad one it
    // is final here (identity, status, zero cost), since no solve runs for it.
    const int status = bad ? (int)EC3R_PAIR_BAD_INPUT : (l1 == l0 ? (int)EC3R_PAIR_FEW_POINTS : 0);
    S.active = status ? 0 : 1;
    S.status = status;
    if (bad) atomicOr(flags, FLAG_BAD_INDEX);
    if (status) {
      write_identity(&out[k]);
      status_out[k] = status;
      if (cost) cost[k] = 0.0;
      if (cost_sums)
        for (int i = 0; i < CS_STRIDE; ++i) cost_sums[(size_t)k * CS_STRIDE + i] = 0.0;
    }
  }
}

// --------------------------------------------------------------------------
// moment sweep
// --------------------------------------------------------------------------
// Per-tile partial moments.  Each thread sums its 32 pixels (8 groups of 4
// consecutive pixels); warps combine by a pairwise butterfly in T; the eight
// warp sums are added in FP64 in a fixed order.  `wbuf` ([n_links][hw],
// nullable): the first FP32 sweep writes every link pixel's weight there;
// with WGT a later sweep reads it instead of both confidences (28 B per pixel
// instead of 32).
template <typename T, int KIND, bool VEC, bool WGT>
__global__ void __launch_bounds__(THREADS, sizeof(T) == 4 ? 4 : 2) k_sweep(
    const float* __restrict__ xyz, const float* __restrict__ conf, int64_t hw, int tpl,
    const int32_t* __restrict__ src, const int32_t* __restrict__ tgt,
    const int32_t* __restrict__ link_pair, const PairState* __restrict__ st, float delta,
    int rule, double* __restrict__ partials, float* __restrict__ wbuf) {
  const int64_t t = blockIdx.x;
  const int64_t l = t / tpl;
  const int c = (int)(t - l * tpl);
  const int k = link_pair[l];
  if (k < 0) return;
  const PairState& S = st[k];
  if (!S.active) return;
  PointOp<T, KIND> op;
  if constexpr (sizeof(T) == 4) {
    for (int i = 0; i < 9; ++i) { op.A[i] = S.A[i]; op.Ap[i] = S.Ap[i]; }
    for (int i = 0; i < 3; ++i) { op.b[i] = S.b[i]; op.bp[i] = S.bp[i]; }
  } else {
    for (int i = 0; i < 9; ++i) { op.A[i] = S.Ad[i]; op.Ap[i] = S.Adp[i]; }
    for (int i = 0; i < 3; ++i) { op.b[i] = S.bd[i]; op.bp[i] = S.bdp[i]; }
  }
  for (int i = 0; i < 3; ++i) { op.pp[i] = (T)S.piv_p[i]; op.pq[i] = (T)S.piv_q[i]; }
  op.delta = (T)delta;
  op.cmin = S.cmin;
  op.rule = rule;

  const int64_t fs = src[l], ft = tgt[l];
  const int64_t px0 = (int64_t)c * TILE;
  const float* P = xyz + (fs * hw + px0) * 3;
  const float* Q = xyz + (ft * hw + px0) * 3;
  const float* CP = conf + fs * hw + px0;
  const float* CQ = conf + ft * hw + px0;
  const int64_t rem = hw - px0;
  const int npx = rem < TILE ? (int)rem : TILE;
  // the first FP32 sweep leaves every link pixel's weight for the later sweeps
  // and the backward pass (pixel_weight: NaN marks an invalid correspondence)
  constexpr bool STORE_W = sizeof(T) == 4 && KIND == FIRST;
  float* WO = STORE_W && wbuf ? wbuf + l * hw + px0 : nullptr;
  const float* WI = WGT ? wbuf + l * hw + px0 : nullptr;
  const float cmin = S.cmin;

  T acc[NMOM];
#pragma unroll
  for (int m = 0; m < NMOM; ++m) acc[m] = T(0);

#pragma unroll 2
  for (int g = threadIdx.x; g < TILE / 4; g += THREADS) {
    const int i0 = 4 * g;
    if (i0 >= npx) break;
    if (VEC && i0 + 4 <= npx) {
      const float4* P4 = reinterpret_cast<const float4*>(P + 3 * i0);
      const float4* Q4 = reinterpret_cast<const float4*>(Q + 3 * i0);
      const float4 pa = __ldcs(P4), pb = __ldcs(P4 + 1), pc = __ldcs(P4 + 2);
      const float4 qa = __ldcs(Q4), qb = __ldcs(Q4 + 1), qc = __ldcs(Q4 + 2);
      if constexpr (WGT) {
        const float4 w = __ldcs(reinterpret_cast<const float4*>(WI + i0));
        op(pa.x, pa.y, pa.z, qa.x, qa.y, qa.z, w.x, acc);
        op(pa.w, pb.x, pb.y, qa.w, qb.x, qb.y, w.y, acc);
        op(pb.z, pb.w, pc.x, qb.z, qb.w, qc.x, w.z, acc);
        op(pc.y, pc.z, pc.w, qc.y, qc.z, qc.w, w.w, acc);
        continue;
      }
      const float4 cp = __ldcs(reinterpret_cast<const float4*>(CP + i0));
      const float4 cq = __ldcs(reinterpret_cast<const float4*>(CQ + i0));
      op(pa.x, pa.y, pa.z, qa.x, qa.y, qa.z, cp.x, cq.x, acc);
      op(pa.w, pb.x, pb.y, qa.w, qb.x, qb.y, cp.y, cq.y, acc);
      op(pb.z, pb.w, pc.x, qb.z, qb.w, qc.x, cp.z, cq.z, acc);
      op(pc.y, pc.z, pc.w, qc.y, qc.z, qc.w, cp.w, cq.w, acc);
      if (STORE_W && WO)
        __stcs(reinterpret_cast<float4*>(WO + i0),
               make_float4(
                   pixel_weight(pa.x, pa.y, pa.z, qa.x, qa.y, qa.z, cp.x, cq.x, cmin, rule),
                   pixel_weight(pa.w, pb.x, pb.y, qa.w, qb.x, qb.y, cp.y, cq.y, cmin, rule),
                   pixel_weight(pb.z, pb.w, pc.x, qb.z, qb.w, qc.x, cp.z, cq.z, cmin, rule),
                   pixel_weight(pc.y, pc.z, pc.w, qc.y, qc.z, qc.w, cp.w, cq.w, cmin, rule)));
    } else {
      const int n = min(4, npx - i0);
      for (int j = 0; j < n; ++j) {
        const int i = i0 + j;
        if constexpr (WGT) {
          op(P[3 * i], P[3 * i + 1], P[3 * i + 2], Q[3 * i], Q[3 * i + 1], Q[3 * i + 2],
             __ldcs(WI + i), acc);
          continue;
        }
        op(P[3 * i], P[3 * i + 1], P[3 * i + 2], Q[3 * i], Q[3 * i + 1], Q[3 * i + 2], CP[i],
           CQ[i], acc);
        if (STORE_W && WO)
          __stcs(WO + i, pixel_weight(P[3 * i], P[3 * i + 1], P[3 * i + 2], Q[3 * i],
                                      Q[3 * i + 1], Q[3 * i + 2], CP[i], CQ[i], cmin, rule));
      }
    }
  }
  // pairwise butterfly inside the warp
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


// One warp per pair: FP64 tile sums (lane m < 19 owns moment m), then lane 0
// solves.  `last` marks the final iteration (writes the outputs).
// `ckpt` (nullable) receives, per pair and iteration `it` (1-based), the
// moments and the new estimate for the backward pass.
__global__ void __launch_bounds__(256) k_solve(int n_pairs, const int32_t* __restrict__ link_off,
                                               int tpl, const double* __restrict__ partials,
                                               PairState* __restrict__ st,
                                               ec3r_sim3* __restrict__ out,
                                               int32_t* __restrict__ status_out, int last,
                                               double* __restrict__ ckpt, int it, int iters) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  __shared__ double mom[8][NMOM];
  if (warp >= n_pairs) return;
  PairState& S = st[warp];
  const int wib = threadIdx.x >> 5;
  if (!S.active) {
    if (last && lane == 0) {
      write_identity(&out[warp]);
      status_out[warp] = S.status;
    }
    return;
  }
  const int64_t t0 = (int64_t)link_off[warp] * tpl, t1 = (int64_t)link_off[warp + 1] * tpl;
  if (lane < NMOM) mom[wib][lane] = tile_sum<NMOM>(partials, t0, t1, lane);
  __syncwarp();
  if (lane != 0) return;
  const double* M = mom[wib];
  double R[9], s = 1.0, b[3] = {0, 0, 0}, dV[12];
  double* ck = ckpt ? ckpt + ((size_t)warp * iters + (it - 1)) * CKPT : nullptr;
  const unsigned status = umeyama_from_moments(M, R, s, b, ck ? dV : nullptr);
  if (ck) {
    for (int m = 0; m < NMOM; ++m) ck[CK_MOM + m] = M[m];
    for (int i = 0; i < 9; ++i) ck[CK_A + i] = s * R[i];
    for (int i = 0; i < 3; ++i) ck[CK_B + i] = b[i];
    ck[CK_STATUS] = (double)status;
    ck[CK_S] = s;
    for (int i = 0; i < 9; ++i) ck[CK_R + i] = R[i];
    for (int i = 0; i < 12; ++i) ck[CK_D + i] = status ? 0.0 : dV[i];
  }
  commit_estimate(S, status, R, s, b, last, out[warp], status_out[warp]);
}

template <typename T, bool VEC>
void launch_sweep(int kind, int64_t n_tiles, cudaStream_t s, const float* xyz, const float* conf,
                  int64_t hw, int tpl, const int32_t* src, const int32_t* tgt,
                  const int32_t* link_pair, const PairState* st, float delta, int rule,
                  double* partials, float* wbuf) {
  const dim3 grid((unsigned)n_tiles);
  if (kind == FIRST) {
    k_sweep<T, FIRST, VEC, false><<<grid, THREADS, 0, s>>>(xyz, conf, hw, tpl, src, tgt,
                                                           link_pair, st, delta, rule, partials,
                                                           wbuf);
    return;
  }
  // FP32 sweeps after the first read the weights it stored (when it stored them)
  if constexpr (sizeof(T) == 4) {
    if (wbuf) {
      if (kind == IRLS)
        k_sweep<T, IRLS, VEC, true><<<grid, THREADS, 0, s>>>(xyz, conf, hw, tpl, src, tgt,
                                                             link_pair, st, delta, rule, partials,
                                                             wbuf);
      else
        k_sweep<T, COST, VEC, true><<<grid, THREADS, 0, s>>>(xyz, conf, hw, tpl, src, tgt,
                                                             link_pair, st, delta, rule, partials,
                                                             wbuf);
      return;
    }
  }
  if (kind == IRLS)
    k_sweep<T, IRLS, VEC, false><<<grid, THREADS, 0, s>>>(xyz, conf, hw, tpl, src, tgt,
                                                          link_pair, st, delta, rule, partials,
                                                          nullptr);
  else
    k_sweep<T, COST, VEC, false><<<grid, THREADS, 0, s>>>(xyz, conf, hw, tpl, src, tgt,
                                                          link_pair, st, delta, rule, partials,
                                                          nullptr);
}

}  // namespace align
}  // namespace ec3r

using namespace ec3r;
using namespace ec3r::align;

extern "C" {

void ec3r_align_opts_default(ec3r_align_opts* o) {
  if (!o) return;
  o->huber_delta = 0.02f;
  o->iters = 10;
  o->conf_min = 0.0f;
  o->weight_rule = EC3R_WEIGHT_PRODUCT;
  o->precision = EC3R_PREC_FP32C;
  o->want_cost = 0;
}

ec3r_status ec3r_align_submaps(ec3r_ctx* ctx, const float* d_xyz, const float* d_conf,
                               int64_t n_frames, int64_t hw, int n_pairs, int64_t n_links,
                               const int32_t* d_link_off, const int32_t* d_src,
                               const int32_t* d_tgt, const float* d_pair_conf_min,
                               const ec3r_align_opts* opts, ec3r_sim3* d_out,
                               int32_t* d_pair_status, double* d_pair_cost, void* stream) {
  if (!ctx) return EC3R_ERR_INVALID_ARG;
  if (!opts) return set_error(ctx, EC3R_ERR_INVALID_ARG, "opts is NULL");
  if (n_pairs < 0 || n_links < 0 || hw <= 0 || n_frames <= 0)
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "bad sizes (n_pairs %d, n_links %lld, hw %lld)",
                     n_pairs, (long long)n_links, (long long)hw);
  if (n_pairs == 0) return EC3R_OK;
  if (!d_xyz || !d_conf || !d_link_off || !d_out || !d_pair_status ||
      (n_links > 0 && (!d_src || !d_tgt)))
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "a required pointer is NULL");
  if (!(opts->huber_delta > 0.f) || !(opts->huber_delta <= FLT_MAX) || opts->iters < 1 ||
      opts->iters > 64 || (opts->weight_rule != 0 && opts->weight_rule != 1) ||
      (opts->precision != 0 && opts->precision != 1) || opts->conf_min != opts->conf_min)
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "bad ec3r_align_opts");
  if (opts->want_cost && !d_pair_cost)
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "want_cost set but d_pair_cost is NULL");
  // the smallest tile of any variant bounds the tile count
  const int64_t tpl_max = (hw + reg_min_tile() - 1) / reg_min_tile();
  const int64_t n_tiles_max = n_links * tpl_max;
  if (n_tiles_max >= ((int64_t)1 << 31) || n_frames > ((int64_t)1 << 40) / hw)
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "problem too large for one call");
  EC3R_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  void *p_state, *p_part, *p_lp, *p_ck, *p_cs, *p_ctl, *p_cp, *p_w;
  ec3r_status st;
  const size_t ctl_bytes = reg_ctl_bytes(n_pairs);
  if ((st = ensure_buf(ctx, "align.state", sizeof(PairState) * (size_t)n_pairs, s, &p_state)) ||
      (st = ensure_buf(ctx, "align.partials", sizeof(double) * NMOM * (size_t)(n_tiles_max + 1),
                       s, &p_part)) ||
      // link -> pair map, then one word for the result of k_check_offsets
      (st = ensure_buf(ctx, "align.link_pair", sizeof(int32_t) * (size_t)(n_links + 2), s,
                       &p_lp)) ||
      (st = ensure_buf(ctx, "align.ckpt",
                       sizeof(double) * CKPT * (size_t)n_pairs * (size_t)opts->iters, s, &p_ck)) ||
      (st = ensure_buf(ctx, "align.cost_sums", sizeof(double) * CS_STRIDE * (size_t)n_pairs, s,
                       &p_cs)) ||
      (st = ensure_buf(ctx, "align.ctl", ctl_bytes, s, &p_ctl)) ||
      (st = ensure_buf(ctx, "align.final_partials",
                       sizeof(double) * FINAL_VALUES *
                           (size_t)(n_links * ((hw + TILE - 1) / TILE) + 1),
                       s, &p_cp)) ||
      // every link pixel's weight (NaN: invalid), written by the first sweep
      (st = ensure_buf(ctx, "align.weights", sizeof(float) * ((size_t)n_links * hw + 4), s,
                       &p_w)))
    return st;
  // (buffers that grew dropped the graphs holding older ones; re-read them all)
  PairState* state = (PairState*)ctx->bufs["align.state"].ptr;
  double* partials = (double*)ctx->bufs["align.partials"].ptr;
  int32_t* link_pair = (int32_t*)ctx->bufs["align.link_pair"].ptr;
  double* ckpt = (double*)ctx->bufs["align.ckpt"].ptr;
  double* cost_sums = (double*)ctx->bufs["align.cost_sums"].ptr;
  void* ctl = ctx->bufs["align.ctl"].ptr;
  float* weights = (float*)ctx->bufs["align.weights"].ptr;
  double* final_partials = (double*)ctx->bufs["align.final_partials"].ptr;
  const bool vec =
      (hw % 4 == 0) && ((uintptr_t)d_xyz % 16 == 0) && ((uintptr_t)d_conf % 16 == 0);
  const bool fp64 = opts->precision == EC3R_PREC_FP64;
  const ec3r_align_opts o = *opts;
  int32_t* malformed = link_pair + n_links + 1;
  // This call overwrites the workspace that an earlier token refers to.
  ctx->align_token = 0;

  // set-up, then every sweep and solve: the persistent launches (or separate grids)
  auto enqueue = [&](cudaStream_t cs, int v) -> ec3r_status {
    EC3R_CUDA_TRY(ctx, cudaMemsetAsync(link_pair, 0xff, sizeof(int32_t) * (size_t)(n_links + 1),
                                       cs));
    traced(ctx, cs, "align_setup", [&] {
      k_check_offsets<<<1, 1024, 0, cs>>>(d_link_off, n_pairs, n_links, malformed);
      k_setup<<<n_pairs, SETUP_THREADS, 0, cs>>>(d_xyz, d_conf, n_frames, hw, n_pairs, n_links,
                                           d_link_off, d_src, d_tgt, d_pair_conf_min,
                                           o.conf_min, link_pair, malformed, state,
                                           ctx->d_flags, d_out, d_pair_status,
                                           o.want_cost ? d_pair_cost : nullptr, cost_sums);
    });
    if (!fp64 && !(vec && v == reg_grid_variant())) {
      // With the cost, the last Huber sweep runs as its own grid that also
      // forms the cost and its sums (k_final_sweep, overlapping the
      // persistent launch's tail); without, the persistent launch runs all.
      const int n_sweeps = o.want_cost ? o.iters - 1 : o.iters;
      ec3r_status r = EC3R_OK;
      // sweep 1 (confidences in, pixel weights out), then sweeps 2 .. n_sweeps
      for (const bool first : {true, false}) {
        traced(ctx, cs, first ? "irls_sweep1" : "irls_register", [&] {
          r = launch_register(ctx, cs, v, vec, first, d_xyz, d_conf, hw, n_pairs, n_links,
                              d_link_off, d_src, d_tgt, link_pair, weights, state, partials,
                              o.huber_delta, o.weight_rule, o.iters, n_sweeps, d_out,
                              d_pair_status, o.want_cost ? d_pair_cost : nullptr, cost_sums,
                              ckpt, ctl, ctl_bytes);
        });
        if (r != EC3R_OK) return r;
      }
      if (o.want_cost) {
        traced(ctx, cs, "irls_final_sweep", [&] {
          r = launch_final(ctx, cs, vec, n_sweeps > 0 && !ctx->profiling, d_xyz, d_conf, hw,
                           n_pairs, n_links, d_link_off, d_src, d_tgt, link_pair, weights,
                           state, final_partials, o.huber_delta, o.weight_rule, o.iters, d_out,
                           d_pair_status, d_pair_cost, cost_sums, ckpt, ctl);
        });
        if (r != EC3R_OK) return r;
      }
    } else {
      // one grid per sweep and per solve: the FP64-accumulation mode (the plain
      // baseline), and with FP32 moments the autotuner's grid variant
      const int64_t tpl = (hw + TILE - 1) / TILE;
      const int64_t n_tiles = n_links * tpl;
      for (int it = 1; it <= o.iters + (o.want_cost ? 1 : 0); ++it) {
        const int kind = it == 1 ? FIRST : (it > o.iters ? COST : IRLS);
        // the cost of a single solve uses h = 1, which a huge delta reproduces
        const float dl = (kind == COST && o.iters == 1) ? FLT_MAX : o.huber_delta;
        if (n_tiles > 0) traced(ctx, cs, fp64 ? "irls_sweep_fp64" : "irls_sweep_fp32", [&] {
          if (fp64 && vec)
            launch_sweep<double, true>(kind, n_tiles, cs, d_xyz, d_conf, hw, (int)tpl, d_src,
                                       d_tgt, link_pair, state, dl, o.weight_rule, partials,
                                       weights);
          else if (fp64)
            launch_sweep<double, false>(kind, n_tiles, cs, d_xyz, d_conf, hw, (int)tpl, d_src,
                                        d_tgt, link_pair, state, dl, o.weight_rule, partials,
                                        weights);
          else
            launch_sweep<float, true>(kind, n_tiles, cs, d_xyz, d_conf, hw, (int)tpl, d_src,
                                      d_tgt, link_pair, state, dl, o.weight_rule, partials,
                                      weights);
        });
        if (kind == COST)
          traced(ctx, cs, "irls_cost", [&] {
            k_cost<<<n_pairs, 32, 0, cs>>>(n_pairs, d_link_off, (int)tpl, partials, state,
                                           d_pair_cost, cost_sums);
          });
        else
          traced(ctx, cs, "sim3_solve", [&] {
            k_solve<<<n_pairs, 32, 0, cs>>>(n_pairs, d_link_off, (int)tpl, partials, state,
                                            d_out, d_pair_status, it == o.iters, ckpt, it,
                                            o.iters);
          });
      }
    }
    EC3R_CUDA_TRY(ctx, cudaGetLastError());
    return EC3R_OK;
  };

  // Variant: forced, or the one timed fastest for this size bucket (FP32
  // moments on aligned pointmaps; the other modes have one configuration).
  int v = 0;
  ctx->align_last_ms.clear();
  if (!fp64 && vec) {
    if (ctx->align_force >= 0) {
      v = ctx->align_force;
    } else {
      const int64_t px = n_links * hw;
      const uint64_t bucket = (uint64_t)(63 - __builtin_clzll((unsigned long long)px)) * 64 +
                              (uint64_t)(31 - __builtin_clz((unsigned)n_pairs));
      auto it = ctx->align_tune.find(bucket);
      if (it != ctx->align_tune.end()) {
        v = it->second.first;
        ctx->align_last_ms = it->second.second;
      } else if (!ctx->profiling && !stream_capturing(s)) {
        // first call of this size: time every variant on these inputs (this
        // call therefore synchronises with `stream`)
        const int nv = reg_variant_count();
        std::vector<float> ms(nv, 0.f);
        cudaEvent_t e0, e1;
        EC3R_CUDA_TRY(ctx, cudaEventCreate(&e0));
        EC3R_CUDA_TRY(ctx, cudaEventCreate(&e1));
        ec3r_status tr = EC3R_OK;
        for (int c = 0; c < nv && tr == EC3R_OK; ++c) {
          if ((tr = enqueue(s, c))) break;       // warm-up
          std::vector<float> reps;
          for (int r = 0; r < 3 && tr == EC3R_OK; ++r) {
            cudaEventRecord(e0, s);
            tr = enqueue(s, c);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) tr = EC3R_ERR_CUDA;
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            reps.push_back(t);
          }
          std::sort(reps.begin(), reps.end());
          ms[c] = reps.empty() ? 0.f : reps[reps.size() / 2];
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (tr != EC3R_OK) {
          cudaGetLastError();
          return set_error(ctx, tr == EC3R_ERR_CUDA ? EC3R_ERR_CUDA : tr,
                           "timing the registration variants failed");
        }
        v = (int)(std::min_element(ms.begin(), ms.end()) - ms.begin());
        ctx->align_tune[bucket] = {v, ms};
        ctx->align_last_ms = ms;
      }
    }
  }
  ctx->align_last_variant = (!fp64 && vec) ? v : -1;
  const std::string key = key_of(
      "align", {(uint64_t)d_xyz, (uint64_t)d_conf, (uint64_t)n_frames, (uint64_t)hw,
                (uint64_t)n_pairs, (uint64_t)n_links, (uint64_t)d_link_off, (uint64_t)d_src,
                (uint64_t)d_tgt, (uint64_t)d_pair_conf_min, fbits(o.huber_delta),
                (uint64_t)o.iters, fbits(o.conf_min), (uint64_t)o.weight_rule,
                (uint64_t)o.precision, (uint64_t)o.want_cost, (uint64_t)d_out,
                (uint64_t)d_pair_status, (uint64_t)d_pair_cost, (uint64_t)v});
  const ec3r_status rs = run_graph(ctx, key, s, [&](cudaStream_t cs) { return enqueue(cs, v); });
  if (rs != EC3R_OK) return rs;
  // Remember this call: a backward call given its token reuses its checkpoints.
  ctx->align_args = key_of("fwd", {(uint64_t)d_xyz, (uint64_t)d_conf, (uint64_t)n_frames,
                                   (uint64_t)hw, (uint64_t)n_pairs, (uint64_t)n_links,
                                   (uint64_t)d_link_off, (uint64_t)d_src, (uint64_t)d_tgt,
                                   (uint64_t)d_pair_conf_min, fbits(o.huber_delta),
                                   (uint64_t)o.iters, fbits(o.conf_min), (uint64_t)o.weight_rule,
                                   (uint64_t)o.precision});
  ctx->align_had_cost = o.want_cost != 0;
  ctx->align_token = ++ctx->align_tokens_issued;
  return EC3R_OK;
}

ec3r_status ec3r_align_set_variant(ec3r_ctx* ctx, int v) {
  if (!ctx) return EC3R_ERR_INVALID_ARG;
  if (v < -1 || v >= reg_variant_count())
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "variant %d out of range", v);
  ctx->align_force = v;
  return EC3R_OK;
}

int ec3r_align_variant_count(void) { return reg_variant_count(); }

ec3r_status ec3r_align_variant_info(int v, int* tile_pixels, int* ctas_per_sm,
                                    int* persistent) {
  if (!tile_pixels || !ctas_per_sm || !persistent ||
      !reg_variant_info(v, tile_pixels, ctas_per_sm, persistent))
    return EC3R_ERR_INVALID_ARG;
  return EC3R_OK;
}

ec3r_status ec3r_align_last_variant(const ec3r_ctx* ctx, int* variant, float* ms) {
  if (!ctx || !variant) return EC3R_ERR_INVALID_ARG;
  *variant = ctx->align_last_variant;
  if (ms) {
    const int nv = reg_variant_count();
    for (int i = 0; i < nv; ++i)
      ms[i] = i < (int)ctx->align_last_ms.size() ? ctx->align_last_ms[i] : -1.f;
  }
  return EC3R_OK;
}

uint64_t ec3r_align_token(const ec3r_ctx* ctx) { return ctx ? ctx->align_token : 0; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Registration for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: code that runs inside a memory
// pool or arena it does not own, real-time loops that forbid allocation (an
// allocation can synchronise the device and take unbounded time), and hosts
// whose allocator is another framework's.  ec3r_align_submaps_noalloc serves
// them: it runs the same kernels as ec3r_align_submaps, but its scratch (pair
// states, per-tile partial moments, link-to-pair map, a status word) lives in
// one fixed file-scope device array, so it allocates nothing and needs no
// context.  Every GPU that loads the library holds that array until exit.
// ---------------------------------------------------------------------------
#include <mutex>

namespace ec3r {
namespace align {

constexpr size_t round256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t NA_STATE_BYTES = round256(sizeof(PairState) * EC3R_NOALLOC_MAX_PAIRS);
constexpr size_t NA_PART_BYTES = round256(sizeof(double) * NMOM * EC3R_NOALLOC_MAX_TILES);
constexpr size_t NA_LP_BYTES = round256(sizeof(int32_t) * (EC3R_NOALLOC_MAX_LINKS + 2));
constexpr size_t NA_FLAG_BYTES = 256;
constexpr size_t NA_BYTES = NA_STATE_BYTES + NA_PART_BYTES + NA_LP_BYTES + NA_FLAG_BYTES;

// The scratch.  In host code this name is only a stand-in for the device
// array: kernels get its device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 64;
static void* g_noalloc_addr[NA_MAX_DEVICES] = {};
static std::mutex g_noalloc_mu;

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device does the lookup).
static ec3r_status noalloc_scratch(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
    cudaGetLastError();
    return EC3R_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return EC3R_ERR_CUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = (unsigned char*)g_noalloc_addr[dev];
  return EC3R_OK;
}

}  // namespace align
}  // namespace ec3r

extern "C" ec3r_status ec3r_align_submaps_noalloc(
    const float* d_xyz, const float* d_conf, int64_t n_frames, int64_t hw, int n_pairs,
    int64_t n_links, const int32_t* d_link_off, const int32_t* d_src, const int32_t* d_tgt,
    const float* d_pair_conf_min, const ec3r_align_opts* opts, ec3r_sim3* d_out,
    int32_t* d_pair_status, double* d_pair_cost, void* stream) {
  if (!opts || n_pairs < 0 || n_links < 0 || hw <= 0 || n_frames <= 0)
    return EC3R_ERR_INVALID_ARG;
  if (n_pairs == 0) return EC3R_OK;
  if (!d_xyz || !d_conf || !d_link_off || !d_out || !d_pair_status ||
      (n_links > 0 && (!d_src || !d_tgt)))
    return EC3R_ERR_INVALID_ARG;
  if (!(opts->huber_delta > 0.f) || !(opts->huber_delta <= FLT_MAX) || opts->iters < 1 ||
      opts->iters > 64 || (opts->weight_rule != 0 && opts->weight_rule != 1) ||
      (opts->precision != 0 && opts->precision != 1) || opts->conf_min != opts->conf_min ||
      (opts->want_cost && !d_pair_cost))
    return EC3R_ERR_INVALID_ARG;
  const int64_t tpl = (hw + TILE - 1) / TILE;
  const int64_t n_tiles = n_links * tpl;
  // the fixed scratch bounds every size
  if (n_pairs > EC3R_NOALLOC_MAX_PAIRS || n_links > EC3R_NOALLOC_MAX_LINKS ||
      n_tiles > EC3R_NOALLOC_MAX_TILES || n_frames > ((int64_t)1 << 40) / hw)
    return EC3R_ERR_INVALID_ARG;
  unsigned char* base = nullptr;
  ec3r_status st = noalloc_scratch(&base);
  if (st != EC3R_OK) return st;
  PairState* state = (PairState*)base;
  double* partials = (double*)(base + NA_STATE_BYTES);
  int32_t* link_pair = (int32_t*)(base + NA_STATE_BYTES + NA_PART_BYTES);
  unsigned* flags = (unsigned*)(base + NA_STATE_BYTES + NA_PART_BYTES + NA_LP_BYTES);
  cudaStream_t cs = (cudaStream_t)stream;
  const bool vec =
      (hw % 4 == 0) && ((uintptr_t)d_xyz % 16 == 0) && ((uintptr_t)d_conf % 16 == 0);
  const bool fp64 = opts->precision == EC3R_PREC_FP64;
  const ec3r_align_opts o = *opts;
  // the previous call's link map and status word must not leak into this one
  if (cudaMemsetAsync(link_pair, 0xff, sizeof(int32_t) * (size_t)(n_links + 1), cs) !=
          cudaSuccess ||
      cudaMemsetAsync(flags, 0, sizeof(unsigned), cs) != cudaSuccess) {
    cudaGetLastError();
    return EC3R_ERR_CUDA;
  }
  int32_t* malformed = link_pair + n_links + 1;
  k_check_offsets<<<1, 1024, 0, cs>>>(d_link_off, n_pairs, n_links, malformed);
  k_setup<<<n_pairs, SETUP_THREADS, 0, cs>>>(d_xyz, d_conf, n_frames, hw, n_pairs, n_links,
                                       d_link_off, d_src, d_tgt, d_pair_conf_min, o.conf_min,
                                       link_pair, malformed, state, flags, d_out, d_pair_status,
                                       o.want_cost ? d_pair_cost : nullptr, nullptr);
  const int solve_blocks = n_pairs;  // one warp per CTA: pairs spread over all SMs' FP64 pipes
  for (int it = 1; it <= o.iters + (o.want_cost ? 1 : 0); ++it) {
    const int kind = it == 1 ? FIRST : (it > o.iters ? COST : IRLS);
    const float dl = (kind == COST && o.iters == 1) ? FLT_MAX : o.huber_delta;
    if (n_tiles > 0) {
      if (fp64) {
        if (vec)
          launch_sweep<double, true>(kind, n_tiles, cs, d_xyz, d_conf, hw, (int)tpl, d_src,
                                     d_tgt, link_pair, state, dl, o.weight_rule, partials,
                                     nullptr);
        else
          launch_sweep<double, false>(kind, n_tiles, cs, d_xyz, d_conf, hw, (int)tpl, d_src,
                                      d_tgt, link_pair, state, dl, o.weight_rule, partials,
                                      nullptr);
      } else {
        if (vec)
          launch_sweep<float, true>(kind, n_tiles, cs, d_xyz, d_conf, hw, (int)tpl, d_src,
                                    d_tgt, link_pair, state, dl, o.weight_rule, partials,
                                    nullptr);
        else
          launch_sweep<float, false>(kind, n_tiles, cs, d_xyz, d_conf, hw, (int)tpl, d_src,
                                     d_tgt, link_pair, state, dl, o.weight_rule, partials,
                                     nullptr);
      }
    }
    if (kind == COST)
      k_cost<<<n_pairs, 32, 0, cs>>>(n_pairs, d_link_off, (int)tpl, partials, state,
                                     d_pair_cost, nullptr);
    else
      k_solve<<<solve_blocks, 32, 0, cs>>>(n_pairs, d_link_off, (int)tpl, partials, state,
                                            d_out, d_pair_status, it == o.iters, nullptr, it,
                                            o.iters);
  }
  if (cudaGetLastError() != cudaSuccess) return EC3R_ERR_CUDA;
  return EC3R_OK;
}
