// Reverse-mode derivative (adjoint) of the batched Huber-IRLS registration.
//
// The forward pass (align.cu) checkpoints, per pair and iteration, the 19
// moments, the estimate (A = s R, b), s and R, and the singular values and
// right singular vectors of the cross-covariance; the backward call reuses the last
// forward call's checkpoints when its inputs match, else re-runs it.  The
// loss gradient then flows backwards through every iteration: the Huber
// weights of solve k depend on estimate k-1, so each solve is differentiated
// and the weights' dependence is carried into the previous estimate.
//
//   k_adj_init     per pair: upstream dL/d(s, R, t) -> pivot-relative (s, R, b)
//   cost term      (dL/dcost != 0) sum om e p'^T, sum om e at the last
//                  estimate: accumulated by the forward's last sweep
//   k_adj_solve    one warp per pair: back through one weighted-Umeyama solve
//                  (covariance, polar rotation with the (d_i + d_j) form from
//                  the checkpointed d, V, scale, translation) to the gradient
//                  of its moments; writes the pair's FP32 parameters of the
//                  next reduce sweep
//   reduce sweep   per point: the moments' gradient gives dL/d omega_i; through
//                  h_i = min(1, delta/r_i) it gives dL/d(A, b) of the previous
//                  estimate, reduced per pair (fixed-order FP64 partials)
//   scatter sweep  per point, all iterations at once: dL/dp, dL/dq, dL/dc_p,
//                  dL/dc_q of every correspondence (link layout)
//   k_adj_frames   per pixel, links in order: accumulate into the frame bank
//                  (deterministic: no atomics)
#include "align_impl.cuh"

namespace ec3r {
namespace align {

constexpr int NRED = 12;  // reduced values: sum g p'^T (9) + sum g (3)
constexpr int NGM = 17;   // gradient of the moments W, Sp(3), Sq(3), Spp, Sqp(9)
enum { G_W = 0, G_SP = 1, G_SQ = 4, G_PP = 7, G_QP = 8 };

struct AdjState {
  double gs, gR[9], gb[3];  // adjoint of the current estimate (s, R, b)
  double gJ, gOm;           // cost = J / Om: dL/dJ and dL/dOm
  int active;
  int pad;
};

// FP32 parameters of one pair for the next reduction sweep, written once per
// pair by the kernel before it (so that no sweep thread converts FP64
// checkpoints): "prev" estimate (weights), "cur" estimate (cost residual),
// the moments' gradient, dL/dJ, dL/dOm, pivots, confidence floor and the
// Huber threshold of that iteration.
struct RedParams {
  float Ap[9], bp[3], Ac[9], bc[3], G[NGM];
  float gJ, gOm, pp[3], pq[3], cmin, dl;
  int active;
  int pad[3];
};

__device__ inline void ck_sR(const double* ck, double* s, double* R) {
  *s = ck[CK_S];
  for (int i = 0; i < 9; ++i) R[i] = ck[CK_R + i];
}

// Everything the forward left for the backward is context-owned: a pair was
// solved iff its state is still active after the last solve, and its cost sits
// in its cost record (never the caller's output buffers, which may be gone).
__global__ void k_adj_init(int n_pairs, int iters, const double* __restrict__ ckpt,
                           const PairState* __restrict__ st,
                           const double* __restrict__ cost_rec, const double* __restrict__ gS,
                           const double* __restrict__ gcost, AdjState* __restrict__ adj,
                           RedParams* __restrict__ rp) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_pairs) return;
  AdjState& a = adj[k];
  a.active = st[k].active ? 1 : 0;
  rp[k].active = a.active;
  a.gs = 0.0;
  for (int i = 0; i < 9; ++i) a.gR[i] = 0.0;
  for (int i = 0; i < 3; ++i) a.gb[i] = 0.0;
  a.gJ = a.gOm = 0.0;
  if (!a.active) return;
  const double* ck = ckpt + ((size_t)k * iters + (iters - 1)) * CKPT;
  double s, R[9];
  ck_sR(ck, &s, R);
  const double pp[3] = {st[k].piv_p[0], st[k].piv_p[1], st[k].piv_p[2]};
  const double* g = gS + (size_t)k * 13;
  // t = b + piv_q - s R piv_p
  double Rp[3];
  for (int i = 0; i < 3; ++i)
    Rp[i] = R[3 * i] * pp[0] + R[3 * i + 1] * pp[1] + R[3 * i + 2] * pp[2];
  a.gs = g[0] - (g[10] * Rp[0] + g[11] * Rp[1] + g[12] * Rp[2]);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) a.gR[3 * i + j] = g[1 + 3 * i + j] - s * g[10 + i] * pp[j];
  for (int i = 0; i < 3; ++i) a.gb[i] = g[10 + i];
  if (gcost) {
    const double W = ck[CK_MOM + M_W];
    a.gJ = gcost[k] / W;
    a.gOm = -gcost[k] * cost_rec[(size_t)k * CS_STRIDE + CS_COST] / W;
  }
}

// Reduction sweep of the Huber path of iteration k (S_{k-1} and the
// moments' gradient of k).  (The cost term's sums come from the forward's
// last sweep.)  The pixels' weights are the ones the forward's first sweep
// stored (NaN: invalid), so a pixel costs 28 bytes, not 32.  One tile of it:
// the tile's 12 partial sums go to slot t.
template <bool LASTK, bool VEC>
__device__ __forceinline__ void reduce_tile(
    const float* __restrict__ xyz, const float* __restrict__ weights, int64_t hw, int tpl,
    const int32_t* __restrict__ src, const int32_t* __restrict__ tgt,
    const int32_t* __restrict__ link_pair, const RedParams* __restrict__ rp,
    double* __restrict__ partials, int64_t t, double (*red)[NRED]) {
  const int64_t l = t / tpl;
  const int c = (int)(t - l * tpl);
  const int k = link_pair[l];
  if (k < 0) return;
  const RedParams& RP = rp[k];
  if (!RP.active) return;
  // estimates: "prev" = S_{k_it-1} (weights), "cur" = S_{k_it} (cost residual)
  float Ap[9], bp[3], Ac[9], bc[3], G[NGM];
  for (int i = 0; i < 9; ++i) {
    Ap[i] = RP.Ap[i];
    Ac[i] = LASTK ? RP.Ac[i] : 0.f;
  }
  for (int i = 0; i < 3; ++i) {
    bp[i] = RP.bp[i];
    bc[i] = LASTK ? RP.bc[i] : 0.f;
  }
  for (int i = 0; i < NGM; ++i) G[i] = RP.G[i];
  const float gJ = RP.gJ, gOm = RP.gOm;
  constexpr bool lastk = LASTK;  // the cost residual at S_K enters the last Huber sweep
  const float pp0 = RP.pp[0], pp1 = RP.pp[1], pp2 = RP.pp[2];
  const float pq0 = RP.pq[0], pq1 = RP.pq[1], pq2 = RP.pq[2];
  const float dl = RP.dl;

  const int64_t fs = src[l], ft = tgt[l];
  const int64_t px0 = (int64_t)c * TILE;
  const float* P = xyz + (fs * hw + px0) * 3;
  const float* Q = xyz + (ft * hw + px0) * 3;
  const float* WL = weights + l * hw + px0;
  const int64_t rem = hw - px0;
  const int npx = rem < TILE ? (int)rem : TILE;
  float acc[NRED];
#pragma unroll
  for (int m = 0; m < NRED; ++m) acc[m] = 0.f;

  auto point = [&](float p0, float p1, float p2, float q0, float q1, float q2, float w) {
    if (!(w == w)) return;
    const float x0 = p0 - pp0, x1 = p1 - pp1, x2 = p2 - pp2;
    const float y0 = q0 - pq0, y1 = q1 - pq1, y2 = q2 - pq2;
    const float e0 = Ap[0] * x0 + Ap[1] * x1 + Ap[2] * x2 + bp[0] - y0;
    const float e1 = Ap[3] * x0 + Ap[4] * x1 + Ap[5] * x2 + bp[1] - y1;
    const float e2 = Ap[6] * x0 + Ap[7] * x1 + Ap[8] * x2 + bp[2] - y2;
    const float rr = e0 * e0 + e1 * e1 + e2 * e2;
    float g0, g1, g2;
    {
      float gom = G[G_W] + G[G_SP] * x0 + G[G_SP + 1] * x1 + G[G_SP + 2] * x2 +
                  G[G_SQ] * y0 + G[G_SQ + 1] * y1 + G[G_SQ + 2] * y2 +
                  G[G_PP] * (x0 * x0 + x1 * x1 + x2 * x2) +
                  y0 * (G[G_QP] * x0 + G[G_QP + 1] * x1 + G[G_QP + 2] * x2) +
                  y1 * (G[G_QP + 3] * x0 + G[G_QP + 4] * x1 + G[G_QP + 5] * x2) +
                  y2 * (G[G_QP + 6] * x0 + G[G_QP + 7] * x1 + G[G_QP + 8] * x2);
      if constexpr (lastk) {
        const float f0 = Ac[0] * x0 + Ac[1] * x1 + Ac[2] * x2 + bc[0] - y0;
        const float f1 = Ac[3] * x0 + Ac[4] * x1 + Ac[5] * x2 + bc[1] - y1;
        const float f2 = Ac[6] * x0 + Ac[7] * x1 + Ac[8] * x2 + bc[2] - y2;
        gom += gJ * (f0 * f0 + f1 * f1 + f2 * f2) + gOm;
      }
      // h = delta / r on the outer branch: dh/de = -delta e / r^3
      const float rs = rsqrtf(rr);
      const float f = rr > dl * dl ? -(gom * w) * dl * rs * rs * rs : 0.f;
      g0 = f * e0; g1 = f * e1; g2 = f * e2;
    }
    acc[0] += g0 * x0; acc[1] += g0 * x1; acc[2] += g0 * x2;
    acc[3] += g1 * x0; acc[4] += g1 * x1; acc[5] += g1 * x2;
    acc[6] += g2 * x0; acc[7] += g2 * x1; acc[8] += g2 * x2;
    acc[9] += g0; acc[10] += g1; acc[11] += g2;
  };

#pragma unroll 2
  for (int g = threadIdx.x; g < TILE / 4; g += THREADS) {
    const int i0 = 4 * g;
    if (i0 >= npx) break;
    if (VEC && i0 + 4 <= npx) {
      const float4* P4 = reinterpret_cast<const float4*>(P + 3 * i0);
      const float4* Q4 = reinterpret_cast<const float4*>(Q + 3 * i0);
      const float4 pa = __ldcs(P4), pb = __ldcs(P4 + 1), pc = __ldcs(P4 + 2);
      const float4 qa = __ldcs(Q4), qb = __ldcs(Q4 + 1), qc = __ldcs(Q4 + 2);
      const float4 w = __ldcs(reinterpret_cast<const float4*>(WL + i0));
      point(pa.x, pa.y, pa.z, qa.x, qa.y, qa.z, w.x);
      point(pa.w, pb.x, pb.y, qa.w, qb.x, qb.y, w.y);
      point(pb.z, pb.w, pc.x, qb.z, qb.w, qc.x, w.z);
      point(pc.y, pc.z, pc.w, qc.y, qc.z, qc.w, w.w);
    } else {
      const int n = min(4, npx - i0);
      for (int j = 0; j < n; ++j) {
        const int i = i0 + j;
        point(P[3 * i], P[3 * i + 1], P[3 * i + 2], Q[3 * i], Q[3 * i + 1], Q[3 * i + 2], WL[i]);
      }
    }
  }
#pragma unroll
  for (int m = 0; m < NRED; ++m)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], o);
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int m = 0; m < NRED; ++m) red[warp][m] = (double)acc[m];
  __syncthreads();
  if (threadIdx.x < NRED) {
    double s = 0.0;
    for (int w = 0; w < THREADS / 32; ++w) s += red[w][threadIdx.x];
    partials[t * NRED + threadIdx.x] = s;
  }
}

// The sweep: a CTA per tile (grid = the tile count), or ctas_per_sm CTAs per
// SM striding over the tiles (ec3r_align_backward_set_ctas_per_sm).
template <bool LASTK, bool VEC>
__global__ void __launch_bounds__(THREADS, 4) k_adj_reduce(
    const float* __restrict__ xyz, const float* __restrict__ weights, int64_t hw, int tpl,
    const int32_t* __restrict__ src, const int32_t* __restrict__ tgt,
    const int32_t* __restrict__ link_pair, const RedParams* __restrict__ rp,
    double* __restrict__ partials, int64_t n_tiles) {
  __shared__ double red[THREADS / 32][NRED];
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    reduce_tile<LASTK, VEC>(xyz, weights, hw, tpl, src, tgt, link_pair, rp, partials, t, red);
    __syncthreads();  // red is reused by the CTA's next tile
  }
}

// One warp per pair (one warp per CTA).  First folds the reduced sums (scaled
// by `scale`: 2 dL/dJ for the cost term, 1 for a Huber sweep) into the adjoint
// of estimate j as dL/dA and dL/db, then differentiates solve j and stores the
// gradient of its moments in gM[j].
//
// On B300 a dependent FP64 operation takes about the same time whether one
// lane or a few carry it, so the 3x3 algebra runs element-parallel: lane e < 9
// (and its copy e + 16) owns element (e / 3, e % 3) of each matrix, the
// matrices pass between products through shared memory, and 9-term sums are
// fixed-order butterflies over the 16-lane half-warp (lanes 9..15 add zeros).
// Scalars every lane needs are computed redundantly by all lanes, one
// instruction each.
__device__ __forceinline__ double half_warp_sum(double x) {
  x += __shfl_xor_sync(0xffffffffu, x, 8);
  x += __shfl_xor_sync(0xffffffffu, x, 4);
  x += __shfl_xor_sync(0xffffffffu, x, 2);
  x += __shfl_xor_sync(0xffffffffu, x, 1);
  return x;
}

__device__ __forceinline__ double pick3(int i, double a0, double a1, double a2) {
  return i == 0 ? a0 : (i == 1 ? a1 : a2);
}

static_assert(sizeof(AdjState) == 16 * sizeof(double), "AdjState is 15 doubles + 2 ints");
enum { AG_S = 0, AG_R = 1, AG_B = 10, AG_J = 13, AG_OM = 14, AG_N = 15 };

__global__ void __launch_bounds__(32) k_adj_solve(int n_pairs, int iters, int j,
                                                  const int32_t* __restrict__ link_off, int tpl,
                                                  const double* __restrict__ partials,
                                                  int have_partials, int scale_by_gJ,
                                                  const double* __restrict__ ckpt,
                                                  AdjState* __restrict__ adj,
                                                  double* __restrict__ gM,
                                                  const PairState* __restrict__ st,
                                                  float delta, RedParams* __restrict__ rp,
                                                  const double* __restrict__ pair_sums) {
  const int k = blockIdx.x;
  const int lane = threadIdx.x;
  if (k >= n_pairs) return;
  if (!adj[k].active) return;
  __shared__ double ck[CKPT];   // checkpoint of solve j: moments, A, b, s, R, d, V
  __shared__ double ckp[12];    // A, b of estimate j - 1 (the next sweep's weights)
  __shared__ double ag[AG_N];   // adjoint state: gs, gR, gb, gJ, gOm
  __shared__ double red[NRED];  // reduced sums of the sweep that ran last
  __shared__ double X[9], Y[9], Z[9];
  const double* ckb = ckpt + (size_t)k * iters * CKPT;
  for (int i = lane; i < CKPT; i += 32) ck[i] = ckb[(size_t)(j - 1) * CKPT + i];
  if (j >= 2 && lane < 12) ckp[lane] = ckb[(size_t)(j - 2) * CKPT + CK_A + lane];
  double* agd = reinterpret_cast<double*>(adj + k);
  if (lane < AG_N) ag[lane] = agd[lane];
  if (have_partials && lane < NRED) {
    if (pair_sums) {  // summed per pair already (the forward's last sweep)
      red[lane] = pair_sums[(size_t)k * CS_STRIDE + lane];
    } else {
      const int64_t t0 = (int64_t)link_off[k] * tpl, t1 = (int64_t)link_off[k + 1] * tpl;
      red[lane] = tile_sum<NRED>(partials, t0, t1, lane);
    }
  }
  __syncwarp();
  const int e = lane & 15;
  const bool own = e < 9;
  const int r = own ? e / 3 : 0, c = own ? e % 3 : 0;
  const double* M = ck + CK_MOM;
  const double* R = ck + CK_R;
  const double* V = ck + CK_V;
  const double s = ck[CK_S];
  const double W = M[M_W], iw = 1.0 / W;
  // this lane's reciprocal of the polar factor's derivative: 1/(d_r + d_c)
  const int da = r < c ? r : c, db = r < c ? c : r;
  const double idd = 1.0 / (ck[CK_D + (own && r != c ? da : 0)] +
                            ck[CK_D + (own && r != c ? db : 1)]);
  const double Re = R[3 * r + c];
  // dL/dA = f X, dL/db = f y; A = s R -> dL/ds = <dL/dA, R>, dL/dR = s dL/dA
  double gs = ag[AG_S];
  double gRe = own ? ag[AG_R + e] : 0.0;
  double gb0 = ag[AG_B], gb1 = ag[AG_B + 1], gb2 = ag[AG_B + 2];
  if (have_partials) {
    const double f = scale_by_gJ ? 2.0 * ag[AG_J] : 1.0;
    const double gA = f * red[3 * r + c];
    gRe = own ? fma(s, gA, gRe) : 0.0;
    gb0 = fma(f, red[9], gb0);
    gb1 = fma(f, red[10], gb1);
    gb2 = fma(f, red[11], gb2);
    gs += half_warp_sum(own ? gA * Re : 0.0);
  }
  // forward quantities of solve j from its moments
  const double mp0 = M[M_SP] * iw, mp1 = M[M_SP + 1] * iw, mp2 = M[M_SP + 2] * iw;
  const double mq0 = M[M_SQ] * iw, mq1 = M[M_SQ + 1] * iw, mq2 = M[M_SQ + 2] * iw;
  const double mpc = pick3(c, mp0, mp1, mp2), mqr = pick3(r, mq0, mq1, mq2);
  const double gbr = pick3(r, gb0, gb1, gb2);
  const double Sige = fma(-mqr, mpc, M[M_QP + 3 * r + c] * iw);
  const double var = M[M_PP] * iw - (mp0 * mp0 + mp1 * mp1 + mp2 * mp2);
  // tau = tr(R^T Sig), the scale's numerator
  const double tau = half_warp_sum(own ? Re * Sige : 0.0);
  // b = mq - s R mp: dL/ds -= gb^T R mp, dL/dR -= s gb mp^T,
  // dL/dmp = -s R^T gb, dL/dmq = gb
  gs -= half_warp_sum(own ? gbr * Re * mpc : 0.0);
  const double gR2 = own ? gRe - s * gbr * mpc : 0.0;
  // s = tau / var, d tau / dSig = R
  const double ivar = 1.0 / var;
  const double gtau = gs * ivar;
  const double gvar = -gs * tau * ivar * ivar;
  double gSig = gtau * Re;
  // R = U' V^T, U' = R V: dL/dSig += U' K V^T, K_ab = (G'_ab - G'_ba) / (d_a + d_b)
  if (lane < 9) {
    X[e] = R[3 * r] * V[c] + R[3 * r + 1] * V[3 + c] + R[3 * r + 2] * V[6 + c];  // U
    Y[e] = gR2;
  }
  __syncwarp();
  if (lane < 9) Z[e] = X[r] * Y[c] + X[3 + r] * Y[3 + c] + X[6 + r] * Y[6 + c];  // U^T gR
  __syncwarp();
  if (lane < 9) Y[e] = Z[3 * r] * V[c] + Z[3 * r + 1] * V[3 + c] + Z[3 * r + 2] * V[6 + c];  // G2
  __syncwarp();
  if (lane < 9) Z[e] = r == c ? 0.0 : (Y[e] - Y[3 * c + r]) * idd;  // K
  __syncwarp();
  if (lane < 9) Y[e] = X[3 * r] * Z[c] + X[3 * r + 1] * Z[3 + c] + X[3 * r + 2] * Z[6 + c];  // U K
  __syncwarp();
  gSig += Y[3 * r] * V[3 * c] + Y[3 * r + 1] * V[3 * c + 1] + Y[3 * r + 2] * V[3 * c + 2];
  if (lane < 9) X[e] = gSig;
  __syncwarp();
  // Sig = Sqp/W - mq mp^T, var = Spp/W - |mp|^2, mp = Sp/W, mq = Sq/W.
  // Lanes 0-2: dL/dmq_i (row i of gSig against mp); lanes 3-5: dL/dmp_m
  // (column m against mq, the b and var terms).
  double gv = 0.0;
  if (e < 3) {
    gv = pick3(e, gb0, gb1, gb2) - (X[3 * e] * mp0 + X[3 * e + 1] * mp1 + X[3 * e + 2] * mp2);
  } else if (e < 6) {
    const int m = e - 3;
    const double mpm = pick3(m, mp0, mp1, mp2);
    gv = -s * (R[m] * gb0 + R[3 + m] * gb1 + R[6 + m] * gb2) -
         (X[m] * mq0 + X[3 + m] * mq1 + X[6 + m] * mq2) - 2.0 * gvar * mpm;
  }
  // dL/dW = -(sum gSig Sqp + gvar Spp + gmp Sp + gmq Sq) / W^2
  double cw = own ? gSig * M[M_QP + e] : 0.0;
  if (e < 3) cw += gv * M[M_SQ + e];
  else if (e < 6) cw += gv * M[M_SP + e - 3];
  const double gW = -(half_warp_sum(cw) + gvar * M[M_PP]) * iw * iw;
  double* out = gM + ((size_t)k * iters + (j - 1)) * NGM;
  // The Huber sweep of iteration j rebuilds the adjoint of estimate j-1 from
  // these parameters; iteration 1 starts from the identity with unit weights
  // and has none.
  RedParams& P = rp[k];
  const bool params = j >= 2;
  if (lane < 9) {
    const double o = gSig * iw;
    out[G_QP + e] = o;
    if (params) P.G[G_QP + e] = (float)o;
  }
  if (e < 6 && lane < 16) {
    const double o = gv * iw;
    const int slot = e < 3 ? G_SQ + e : G_SP + e - 3;
    out[slot] = o;
    if (params) P.G[slot] = (float)o;
  }
  if (lane == 16) {
    out[G_PP] = gvar * iw;
    out[G_W] = gW;
    if (params) {
      P.G[G_PP] = (float)(gvar * iw);
      P.G[G_W] = (float)gW;
    }
  }
  if (params) {
    const bool cur = j == iters;
    if (lane < 9) {
      P.Ap[lane] = (float)ckp[lane];
      P.Ac[lane] = cur ? (float)ck[CK_A + lane] : 0.f;
    } else if (lane < 12) {
      P.bp[lane - 9] = (float)ckp[lane];
      P.bc[lane - 9] = cur ? (float)ck[CK_A + lane] : 0.f;
    } else if (lane < 15) {
      P.pp[lane - 12] = st[k].piv_p[lane - 12];
      P.pq[lane - 12] = st[k].piv_q[lane - 12];
    } else if (lane == 15) {
      P.gJ = (float)ag[AG_J];
      P.gOm = (float)ag[AG_OM];
      P.cmin = st[k].cmin;
      P.dl = delta;
    }
  }
  // the adjoint of estimate j-1 is rebuilt by the next Huber sweep
  if (lane < AG_J) agd[lane] = 0.0;
}

// Per-correspondence gradients, all iterations in one pass (link layout,
// 8 floats per pixel: dp(3), dq(3), dc_p, dc_q).
// A side whose frame no other link references writes straight into the frame
// gradients; a shared frame's side goes to the link buffer and is summed by
// k_adj_frames in link order.  Invalid pixels carry zero weight and zero
// coordinates, so every term they add is zero.
//
// Iteration k's moments are sums of om_k phi(p, q) with phi = (1, p, q, |p|^2,
// q p^T) and om_k = w h_k(r_k).  The part of the gradient that holds om_k fixed
// is linear in the moment adjoints, so it is accumulated as one 17-vector
// Gt = sum_k om_k gM_k and differentiated once at the end; per iteration a
// pixel only evaluates gom_k = <gM_k, phi> (for the weight and the Huber
// branch) and adds om_k gM_k to Gt.
//
// Each thread owns 2 consecutive pixels and carries them as the two lanes of
// packed FP32 pairs (one f32x2 instruction does both pixels' multiply-adds, each
// lane rounded exactly like the scalar operation).  The per-iteration constants
// sit in shared memory as duplicated pairs, so a 16-byte load yields two
// broadcast operands.
constexpr int SC_PAIRS = 32;  // float2 per iteration: A 9, b 3, gM 17, 3 pad

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// One iteration of the scatter for a packed pixel pair.  S: estimate it-1
// (A, b) and gM of iteration it; Sp: the estimate whose residual weights
// iteration it (HUBER: it > 1; iteration 1 has h = 1); COSTK: the last
// iteration, which also carries the cost terms of the returned estimate.
template <bool HUBER, bool COSTK>
__device__ __forceinline__ void scatter_iter(const float2* S, const float2* Sp, const float2 (&X)[3],
                                             const float2 (&Y)[3], const float2 (&nY)[3],
                                             float2 W, float2 XX, float delta, float d2,
                                             float gJ, float gOm, float2 (&gp)[3],
                                             float2 (&gq)[3], float2& gw, float2 (&Gt)[NGM]) {
  float2 h = f2(1.f), e[3] = {f2(0.f), f2(0.f), f2(0.f)}, rr = f2(0.f), rs = f2(0.f);
  if (HUBER) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
      e[r] = fma2(Sp[3 * r], X[0],
                  fma2(Sp[3 * r + 1], X[1], fma2(Sp[3 * r + 2], X[2], add2(Sp[9 + r], nY[r]))));
    rr = fma2(e[0], e[0], fma2(e[1], e[1], mul2(e[2], e[2])));
    rs = make_float2(rsqrtf(rr.x), rsqrtf(rr.y));
    const float2 dr = mul2(f2(delta), rs);
    h = make_float2(fminf(1.f, dr.x), fminf(1.f, dr.y));
  }
  const float2 om = mul2(W, h);
  const float2* G = S + 12;
  float2 gom = fma2(G[G_PP], XX, G[G_W]);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float2 Gx = fma2(G[G_QP + 3 * r], X[0],
                           fma2(G[G_QP + 3 * r + 1], X[1], fma2(G[G_QP + 3 * r + 2], X[2], G[G_SQ + r])));
    gom = fma2(G[G_SP + r], X[r], gom);
    gom = fma2(Y[r], Gx, gom);
  }
#pragma unroll
  for (int i = 0; i < NGM; ++i) Gt[i] = fma2(om, G[i], Gt[i]);
  if (COSTK) {  // cost terms of the returned estimate
    float2 f[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
      f[r] = fma2(S[3 * r], X[0],
                  fma2(S[3 * r + 1], X[1], fma2(S[3 * r + 2], X[2], add2(S[9 + r], nY[r]))));
    const float2 ff = fma2(f[0], f[0], fma2(f[1], f[1], mul2(f[2], f[2])));
    gom = add2(gom, fma2(f2(gJ), ff, f2(gOm)));
    const float2 s2 = mul2(f2(2.f * gJ), om);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float2 ge = mul2(s2, f[r]);
      gq[r] = fma2(f2(-1.f), ge, gq[r]);
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) gp[cc] = fma2(S[3 * r + cc], ge, gp[cc]);
    }
  }
  gw = fma2(gom, h, gw);
  if (HUBER) {
    // Huber branch (|r| > delta): d h / d e = -delta e / |r|^3
    float2 u = mul2(mul2(gom, W), mul2(f2(-delta), mul2(rs, mul2(rs, rs))));
    u.x = rr.x > d2 ? u.x : 0.f;
    u.y = rr.y > d2 ? u.y : 0.f;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float2 ge = mul2(u, e[r]);
      gq[r] = fma2(f2(-1.f), ge, gq[r]);
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) gp[cc] = fma2(Sp[3 * r + cc], ge, gp[cc]);
    }
  }
}

// The frame zeroing that the scatter's CTAs share: the frame bank's pixels
// (frame-major, n_frames x hw) split into equal runs of a multiple of four
// pixels, one per CTA, and each run into ZS slices, one per trip of the
// CTA's pixel loop; a slice's pixels of a frame that no scatter writes
// directly (references 0 or > 1) are zeroed.  The stores drain while the
// CTA computes: the scatter is bound by FP32 latency, not by HBM.
constexpr int ZS = TILE / 2 / THREADS;  // trips of the scatter's pixel loop

template <bool VEC>
__device__ __forceinline__ void zero_slice(int64_t n_frames, int64_t hw, int slice,
                                           const int32_t* __restrict__ refs,
                                           float* __restrict__ gxyz, float* __restrict__ gconf) {
  const int64_t U = n_frames * hw, G = gridDim.x;
  const int64_t per = (((U + G - 1) / G) + 3) & ~(int64_t)3;
  const int64_t r0 = min(U, (int64_t)blockIdx.x * per), r1 = min(U, r0 + per);
  const int64_t sub = (((r1 - r0) / 4 + ZS - 1) / ZS) * 4;
  int64_t u0 = min(r1, r0 + slice * sub);
  const int64_t u1 = min(r1, u0 + sub);
  while (u0 < u1) {
    const int64_t f = u0 / hw;
    const int64_t fe = min(u1, (f + 1) * hw);
    if (refs[f] != 1) {
      if (VEC) {  // hw and the slice boundaries are multiples of 4 pixels
        float4* x4 = reinterpret_cast<float4*>(gxyz + 3 * u0);
        float4* c4 = reinterpret_cast<float4*>(gconf + u0);
        const int64_t n4 = (fe - u0) / 4;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int64_t i = threadIdx.x; i < 3 * n4; i += THREADS) __stcs(x4 + i, z);
        for (int64_t i = threadIdx.x; i < n4; i += THREADS) __stcs(c4 + i, z);
      } else {
        for (int64_t i = 3 * u0 + threadIdx.x; i < 3 * fe; i += THREADS) gxyz[i] = 0.f;
        for (int64_t i = u0 + threadIdx.x; i < fe; i += THREADS) gconf[i] = 0.f;
      }
    }
    u0 = fe;
  }
}

template <bool VEC>
__global__ void __launch_bounds__(THREADS, 2) k_adj_scatter(
    const float* __restrict__ xyz, const float* __restrict__ conf, int64_t n_frames, int64_t hw,
    int tpl, const int32_t* __restrict__ src, const int32_t* __restrict__ tgt,
    const int32_t* __restrict__ link_pair, const PairState* __restrict__ st,
    const AdjState* __restrict__ adj, const double* __restrict__ ckpt,
    const double* __restrict__ gM, int iters, float delta, int rule, float* __restrict__ lg,
    const int32_t* __restrict__ refs, float* __restrict__ gxyz, float* __restrict__ gconf) {
  const int64_t t = blockIdx.x;
  const int64_t l = t / tpl;
  const int c = (int)(t - l * tpl);
  const int k = link_pair[l];
  if (k < 0) {  // pair rejected at set-up: its frames were not counted
    for (int z = 0; z < ZS; ++z) zero_slice<VEC>(n_frames, hw, z, refs, gxyz, gconf);
    return;
  }
  const int64_t px0 = (int64_t)c * TILE;
  const int64_t rem = hw - px0;
  const int npx = rem < TILE ? (int)rem : TILE;
  const int64_t fs = src[l], ft = tgt[l];
  const bool ds = refs[fs] == 1, dt = refs[ft] == 1;  // direct writes
  float* out = lg + (l * hw + px0) * 8;
  float* gxs = gxyz + (fs * hw + px0) * 3;
  float* gxt = gxyz + (ft * hw + px0) * 3;
  float* gcs = gconf + fs * hw + px0;
  float* gct = gconf + ft * hw + px0;
  const bool active = adj[k].active;
  extern __shared__ float4 sh4[];
  float2* sh2 = reinterpret_cast<float2*>(sh4);
  if (active) {
    const double* ckb = ckpt + (size_t)k * iters * CKPT;
    for (int i = threadIdx.x; i < iters * SC_PAIRS; i += THREADS) {
      const int it = i / SC_PAIRS, f = i % SC_PAIRS;
      float v = 0.f;
      if (f < 9) v = (float)ckb[it * CKPT + CK_A + f];
      else if (f < 12) v = (float)ckb[it * CKPT + CK_B + (f - 9)];
      else if (f < 12 + NGM) v = (float)gM[((size_t)k * iters + it) * NGM + (f - 12)];
      sh2[i] = f2(v);
    }
  }
  __syncthreads();
  const float gJ = active ? (float)adj[k].gJ : 0.f, gOm = active ? (float)adj[k].gOm : 0.f;
  const float piv[6] = {st[k].piv_p[0], st[k].piv_p[1], st[k].piv_p[2],
                        st[k].piv_q[0], st[k].piv_q[1], st[k].piv_q[2]};
  const float cmin = st[k].cmin;
  const float d2 = delta * delta;
  const float* P = xyz + (fs * hw + px0) * 3;
  const float* Q = xyz + (ft * hw + px0) * 3;
  const float* CP = conf + fs * hw + px0;
  const float* CQ = conf + ft * hw + px0;
  int zs = 0;  // zeroing slices done by this thread
  for (int g = threadIdx.x; g < TILE / 2; g += THREADS) {
    const int i0 = 2 * g;
    if (i0 >= npx) break;
    zero_slice<VEC>(n_frames, hw, zs++, refs, gxyz, gconf);
    const int n = min(2, npx - i0);
    float pr[6], qr[6], cpr[2], cqr[2];
    if (VEC && n == 2) {
      const float2* P2 = reinterpret_cast<const float2*>(P + 3 * i0);
      const float2* Q2 = reinterpret_cast<const float2*>(Q + 3 * i0);
      const float2 a = __ldcs(P2), b = __ldcs(P2 + 1), cc = __ldcs(P2 + 2);
      const float2 d = __ldcs(Q2), e = __ldcs(Q2 + 1), f = __ldcs(Q2 + 2);
      const float2 u = __ldcs(reinterpret_cast<const float2*>(CP + i0));
      const float2 v = __ldcs(reinterpret_cast<const float2*>(CQ + i0));
      pr[0] = a.x; pr[1] = a.y; pr[2] = b.x; pr[3] = b.y; pr[4] = cc.x; pr[5] = cc.y;
      qr[0] = d.x; qr[1] = d.y; qr[2] = e.x; qr[3] = e.y; qr[4] = f.x; qr[5] = f.y;
      cpr[0] = u.x; cpr[1] = u.y;
      cqr[0] = v.x; cqr[1] = v.y;
    } else {
      for (int j = 0; j < 2; ++j) {
        const bool in = j < n;
        for (int dd = 0; dd < 3; ++dd) {
          pr[3 * j + dd] = in ? P[3 * (i0 + j) + dd] : 0.f;
          qr[3 * j + dd] = in ? Q[3 * (i0 + j) + dd] : 0.f;
        }
        cpr[j] = in ? CP[i0 + j] : 0.f;
        cqr[j] = in ? CQ[i0 + j] : 0.f;
      }
    }
    // lane j of every pair is pixel i0 + j
    float2 X[3], Y[3], W, XX;
    bool val[2];
    {
      float xs[2][3], ys[2][3], ws[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const bool v = active && j < n && finitef(pr[3 * j]) && finitef(pr[3 * j + 1]) &&
                       finitef(pr[3 * j + 2]) && finitef(qr[3 * j]) && finitef(qr[3 * j + 1]) &&
                       finitef(qr[3 * j + 2]) && finitef(cpr[j]) && finitef(cqr[j]) &&
                       cpr[j] > cmin && cqr[j] > cmin;
        val[j] = v;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          xs[j][r] = v ? pr[3 * j + r] - piv[r] : 0.f;
          ys[j][r] = v ? qr[3 * j + r] - piv[3 + r] : 0.f;
        }
        ws[j] = v ? (rule == 0 ? cpr[j] * cqr[j] : cpr[j]) : 0.f;
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        X[r] = make_float2(xs[0][r], xs[1][r]);
        Y[r] = make_float2(ys[0][r], ys[1][r]);
      }
      W = make_float2(ws[0], ws[1]);
      XX = fma2(X[0], X[0], fma2(X[1], X[1], mul2(X[2], X[2])));
    }
    const float2 nY[3] = {make_float2(-Y[0].x, -Y[0].y), make_float2(-Y[1].x, -Y[1].y),
                          make_float2(-Y[2].x, -Y[2].y)};
    float2 gp[3] = {f2(0.f), f2(0.f), f2(0.f)}, gq[3] = {f2(0.f), f2(0.f), f2(0.f)};
    float2 gw = f2(0.f), Gt[NGM];
#pragma unroll
    for (int i = 0; i < NGM; ++i) Gt[i] = f2(0.f);
    if (active) {
      // iteration 1 (unit Huber weights) and the last one (cost terms) peeled,
      // so that the iterations between run without branches, two per trip
      // (the next one's shared-memory constants load while this one computes)
      if (iters == 1) {
        scatter_iter<false, true>(sh2, sh2, X, Y, nY, W, XX, delta, d2, gJ, gOm, gp, gq, gw, Gt);
      } else {
        scatter_iter<false, false>(sh2, sh2, X, Y, nY, W, XX, delta, d2, gJ, gOm, gp, gq, gw,
                                   Gt);
#pragma unroll 2
        for (int it = 2; it < iters; ++it) {
          const float2* S = sh2 + (it - 1) * SC_PAIRS;
          scatter_iter<true, false>(S, S - SC_PAIRS, X, Y, nY, W, XX, delta, d2, gJ, gOm, gp, gq,
                                    gw, Gt);
        }
        const float2* S = sh2 + (iters - 1) * SC_PAIRS;
        scatter_iter<true, true>(S, S - SC_PAIRS, X, Y, nY, W, XX, delta, d2, gJ, gOm, gp, gq, gw,
                                 Gt);
      }
      // the fixed-weight part: d<Gt, phi>/dp and d<Gt, phi>/dq
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        gq[r] = add2(gq[r], fma2(Gt[G_QP + 3 * r], X[0],
                                 fma2(Gt[G_QP + 3 * r + 1], X[1],
                                      fma2(Gt[G_QP + 3 * r + 2], X[2], Gt[G_SQ + r]))));
        gp[r] = add2(gp[r], fma2(mul2(f2(2.f), Gt[G_PP]), X[r],
                                 fma2(Gt[G_QP + r], Y[0],
                                      fma2(Gt[G_QP + 3 + r], Y[1],
                                           fma2(Gt[G_QP + 6 + r], Y[2], Gt[G_SP + r])))));
      }
    }
    float gpo[2][3], gqo[2][3], gcp[2], gcq[2];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      gpo[0][r] = gp[r].x; gpo[1][r] = gp[r].y;
      gqo[0][r] = gq[r].x; gqo[1][r] = gq[r].y;
    }
    const float gws[2] = {gw.x, gw.y};
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      gcp[j] = val[j] ? (rule == 0 ? gws[j] * cqr[j] : gws[j]) : 0.f;
      gcq[j] = val[j] ? (rule == 0 ? gws[j] * cpr[j] : 0.f) : 0.f;
    }
    if (VEC && n == 2 && ds) {
      float2* o = reinterpret_cast<float2*>(gxs + 3 * i0);
      o[0] = make_float2(gpo[0][0], gpo[0][1]);
      o[1] = make_float2(gpo[0][2], gpo[1][0]);
      o[2] = make_float2(gpo[1][1], gpo[1][2]);
      *reinterpret_cast<float2*>(gcs + i0) = make_float2(gcp[0], gcp[1]);
    } else {
      for (int j = 0; j < n; ++j) {
        const int i = i0 + j;
        if (ds) {
          gxs[3 * i] = gpo[j][0]; gxs[3 * i + 1] = gpo[j][1]; gxs[3 * i + 2] = gpo[j][2];
          gcs[i] = gcp[j];
        } else {
          out[8 * i] = gpo[j][0]; out[8 * i + 1] = gpo[j][1]; out[8 * i + 2] = gpo[j][2];
          out[8 * i + 6] = gcp[j];
        }
      }
    }
    if (VEC && n == 2 && dt) {
      float2* o = reinterpret_cast<float2*>(gxt + 3 * i0);
      o[0] = make_float2(gqo[0][0], gqo[0][1]);
      o[1] = make_float2(gqo[0][2], gqo[1][0]);
      o[2] = make_float2(gqo[1][1], gqo[1][2]);
      *reinterpret_cast<float2*>(gct + i0) = make_float2(gcq[0], gcq[1]);
    } else {
      for (int j = 0; j < n; ++j) {
        const int i = i0 + j;
        if (dt) {
          gxt[3 * i] = gqo[j][0]; gxt[3 * i + 1] = gqo[j][1]; gxt[3 * i + 2] = gqo[j][2];
          gct[i] = gcq[j];
        } else {
          out[8 * i + 3] = gqo[j][0]; out[8 * i + 4] = gqo[j][1]; out[8 * i + 5] = gqo[j][2];
          out[8 * i + 7] = gcq[j];
        }
      }
    }
  }
  // the slices of the trips a ragged tile does not make
  for (; zs < ZS; ++zs) zero_slice<VEC>(n_frames, hw, zs, refs, gxyz, gconf);
}

// References of every frame by the links of valid pairs.
__global__ void k_adj_refcount(int64_t n_links, int64_t n_frames,
                               const int32_t* __restrict__ src, const int32_t* __restrict__ tgt,
                               const int32_t* __restrict__ link_pair, int32_t* refs,
                               int32_t* any_shared) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n_links || link_pair[l] < 0) return;
  const int a = src[l], b = tgt[l];
  if (atomicAdd(&refs[a], 1) >= 1) atomicExch(any_shared, 1);
  if (atomicAdd(&refs[b], 1) >= 1) atomicExch(any_shared, 1);
}

// Zero the gradients of frames that no scatter writes directly (references 0
// or > 1).  One CTA per frame.
__global__ void k_adj_zero_frames(int64_t hw, const int32_t* __restrict__ refs,
                                  float* __restrict__ gxyz, float* __restrict__ gconf) {
  const int64_t f = blockIdx.x;
  if (refs[f] == 1) return;
  float* gx = gxyz + f * hw * 3;
  float* gc = gconf + f * hw;
  for (int64_t i = threadIdx.x; i < hw * 3; i += blockDim.x) gx[i] = 0.f;
  for (int64_t i = threadIdx.x; i < hw; i += blockDim.x) gc[i] = 0.f;
}

// Frame-bank gradients: one thread per pixel index, links in order.
__global__ void k_adj_frames(int64_t hw, int64_t n_links, const int32_t* __restrict__ src,
                             const int32_t* __restrict__ tgt,
                             const int32_t* __restrict__ link_pair,
                             const int32_t* __restrict__ refs,
                             const int32_t* __restrict__ any_shared, const float* __restrict__ lg,
                             float* __restrict__ gxyz, float* __restrict__ gconf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= hw || !*any_shared) return;
  for (int64_t l = 0; l < n_links; ++l) {
    if (link_pair[l] < 0) continue;
    const float* g = lg + (l * hw + i) * 8;
    const int64_t a = src[l], b = tgt[l];
    if (refs[a] > 1) {
      float* ga = gxyz + (a * hw + i) * 3;
      ga[0] += g[0]; ga[1] += g[1]; ga[2] += g[2];
      gconf[a * hw + i] += g[6];
    }
    if (refs[b] > 1) {
      float* gb = gxyz + (b * hw + i) * 3;
      gb[0] += g[3]; gb[1] += g[4]; gb[2] += g[5];
      gconf[b * hw + i] += g[7];
    }
  }
}

}  // namespace align
}  // namespace ec3r

using namespace ec3r;
using namespace ec3r::align;

extern "C" ec3r_status ec3r_align_submaps_backward(
    ec3r_ctx* ctx, const float* d_xyz, const float* d_conf, int64_t n_frames, int64_t hw,
    int n_pairs, int64_t n_links, const int32_t* d_link_off, const int32_t* d_src,
    const int32_t* d_tgt, const float* d_pair_conf_min, const ec3r_align_opts* opts,
    uint64_t fwd_token, const double* d_grad_S, const double* d_grad_cost, float* d_grad_xyz,
    float* d_grad_conf, void* stream) {
  if (!ctx) return EC3R_ERR_INVALID_ARG;
  if (!opts || (n_pairs > 0 && !d_grad_S) || !d_grad_xyz || !d_grad_conf)
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "a required pointer is NULL");
  if (opts->precision != EC3R_PREC_FP32C)
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "the backward pass supports FP32 moments only");
  if (n_pairs < 0) return set_error(ctx, EC3R_ERR_INVALID_ARG, "n_pairs < 0");
  cudaStream_t s = (cudaStream_t)stream;
  if (n_pairs == 0) {  // no pair: every point's gradient is zero
    if (n_frames < 0 || hw < 0)
      return set_error(ctx, EC3R_ERR_INVALID_ARG, "negative frame bank size");
    const size_t px = (size_t)n_frames * (size_t)hw;
    EC3R_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    EC3R_CUDA_TRY(ctx, cudaMemsetAsync(d_grad_xyz, 0, sizeof(float) * 3 * px, s));
    EC3R_CUDA_TRY(ctx, cudaMemsetAsync(d_grad_conf, 0, sizeof(float) * px, s));
    return EC3R_OK;
  }
  // the forward that the caller's call would be: with the cost only when the
  // cost has a gradient (the last sweep and solve then run in another kernel,
  // so the two differ at FP32 rounding level)
  ec3r_align_opts fo = *opts;
  fo.want_cost = d_grad_cost ? 1 : 0;
  ec3r_status st;
  if (fwd_token != 0) {
    // Reuse the checkpoints of the forward call that issued this token: it must
    // be the last registration call on this context, with these inputs and
    // options, and with the cost if the cost has a gradient.
    const std::string want = key_of(
        "fwd", {(uint64_t)d_xyz, (uint64_t)d_conf, (uint64_t)n_frames, (uint64_t)hw,
                (uint64_t)n_pairs, (uint64_t)n_links, (uint64_t)d_link_off, (uint64_t)d_src,
                (uint64_t)d_tgt, (uint64_t)d_pair_conf_min, fbits(fo.huber_delta),
                (uint64_t)fo.iters, fbits(fo.conf_min), (uint64_t)fo.weight_rule,
                (uint64_t)fo.precision});
    if (fwd_token != ctx->align_token)
      return set_error(ctx, EC3R_ERR_INVALID_ARG,
                       "fwd_token %llu is not the token of the last registration call (%llu)",
                       (unsigned long long)fwd_token, (unsigned long long)ctx->align_token);
    if (ctx->align_args != want)
      return set_error(ctx, EC3R_ERR_INVALID_ARG,
                       "fwd_token's registration call had other inputs or options");
    if (d_grad_cost && !ctx->align_had_cost)
      return set_error(ctx, EC3R_ERR_INVALID_ARG,
                       "d_grad_cost given but fwd_token's call ran without want_cost");
  } else {
    // No token: run the forward pass here, into context-owned outputs.
    void *p_out, *p_st, *p_cost;
    if ((st = ensure_buf(ctx, "adj.out", sizeof(ec3r_sim3) * (size_t)n_pairs, s, &p_out)))
      return st;
    if ((st = ensure_buf(ctx, "adj.status", sizeof(int32_t) * (size_t)n_pairs, s, &p_st)))
      return st;
    if ((st = ensure_buf(ctx, "adj.cost", sizeof(double) * (size_t)n_pairs, s, &p_cost)))
      return st;
    if ((st = ec3r_align_submaps(ctx, d_xyz, d_conf, n_frames, hw, n_pairs, n_links, d_link_off,
                                 d_src, d_tgt, d_pair_conf_min, &fo, (ec3r_sim3*)p_out,
                                 (int32_t*)p_st, (double*)p_cost, stream)))
      return st;
  }
  const int iters = opts->iters;
  const int64_t tpl = (hw + TILE - 1) / TILE;
  const int64_t n_tiles = n_links * tpl;
  void *p_adj, *p_gm, *p_part, *p_lg;
  if ((st = ensure_buf(ctx, "adj.state", sizeof(AdjState) * (size_t)n_pairs, s, &p_adj))) return st;
  void* p_rp;
  if ((st = ensure_buf(ctx, "adj.red_params", sizeof(RedParams) * (size_t)n_pairs, s, &p_rp)))
    return st;
  if ((st = ensure_buf(ctx, "adj.gM", sizeof(double) * NGM * (size_t)n_pairs * iters, s, &p_gm)))
    return st;
  if ((st = ensure_buf(ctx, "adj.partials", sizeof(double) * NRED * (size_t)(n_tiles + 1), s,
                       &p_part)))
    return st;
  if ((st = ensure_buf(ctx, "adj.link_grads", sizeof(float) * 8 * (size_t)(n_links * hw + 1), s,
                       &p_lg)))
    return st;
  // pointers of the forward workspace (stable: the forward call above sized them)
  PairState* state = (PairState*)ctx->bufs["align.state"].ptr;
  double* ckpt = (double*)ctx->bufs["align.ckpt"].ptr;
  int32_t* link_pair = (int32_t*)ctx->bufs["align.link_pair"].ptr;
  const float* weights = (const float*)ctx->bufs["align.weights"].ptr;
  AdjState* adj = (AdjState*)p_adj;
  RedParams* rp = (RedParams*)p_rp;
  double* gM = (double*)p_gm;
  double* part = (double*)p_part;
  float* lg = (float*)p_lg;
  const bool vec =
      (hw % 4 == 0) && ((uintptr_t)d_xyz % 16 == 0) && ((uintptr_t)d_conf % 16 == 0);
  const float delta = opts->huber_delta;
  const int rule = opts->weight_rule;
  const dim3 grid((unsigned)(n_tiles > 0 ? n_tiles : 1));
  // the reduction sweeps' grid: one CTA per tile, or a share of the SMs
  const int64_t cap = (int64_t)ctx->bwd_ctas_per_sm * ctx->sm_count;
  const dim3 grid_red((unsigned)(cap > 0 && cap < n_tiles ? cap : (n_tiles > 0 ? n_tiles : 1)));
  const int solve_blocks = n_pairs;  // one warp per CTA: pairs spread over all SMs' FP64 pipes
  void* p_refs;
  if ((st = ensure_buf(ctx, "adj.refs", sizeof(int32_t) * (size_t)(n_frames + 1), s, &p_refs)))
    return st;
  int32_t* refs = (int32_t*)p_refs;
  int32_t* any_shared = refs + n_frames;
  const double* gcost = d_grad_cost;
  const std::string gkey =
      key_of("adj", {(uint64_t)d_xyz, (uint64_t)d_conf, (uint64_t)n_frames, (uint64_t)hw,
                     (uint64_t)n_pairs, (uint64_t)n_links, (uint64_t)d_link_off, (uint64_t)d_src,
                     (uint64_t)d_tgt, fbits(delta), (uint64_t)iters, (uint64_t)rule,
                     (uint64_t)d_grad_S, (uint64_t)gcost, (uint64_t)d_grad_xyz,
                     (uint64_t)d_grad_conf, (uint64_t)vec, (uint64_t)grid_red.x});
  // the cost term's sums (sum g p'^T, sum g at the returned estimate with the
  // last weights) and the cost come from the forward's last sweep, per pair
  const double* cost_sums = (const double*)ctx->bufs["align.cost_sums"].ptr;
  return run_graph(ctx, gkey, s, [&](cudaStream_t cs) -> ec3r_status {
    traced(ctx, cs, "adj_init", [&] {
      k_adj_init<<<(n_pairs + 127) / 128, 128, 0, cs>>>(n_pairs, iters, ckpt, state, cost_sums,
                                                      d_grad_S, d_grad_cost, adj, rp);
    });
    const bool cost_path = d_grad_cost != nullptr;
    traced(ctx, cs, "adj_solve", [&] {
      k_adj_solve<<<solve_blocks, 32, 0, cs>>>(n_pairs, iters, iters, d_link_off, (int)tpl, part,
                                               cost_path && n_tiles > 0, 1, ckpt, adj, gM, state,
                                               delta, rp, cost_sums);
    });
    for (int k = iters; k >= 2; --k) {
      if (n_tiles > 0)
        traced(ctx, cs, "adj_reduce", [&] {
          const bool last = k == iters;
          if (vec && last)
            k_adj_reduce<true, true><<<grid_red, THREADS, 0, cs>>>(
                d_xyz, weights, hw, (int)tpl, d_src, d_tgt, link_pair, rp, part, n_tiles);
          else if (vec)
            k_adj_reduce<false, true><<<grid_red, THREADS, 0, cs>>>(
                d_xyz, weights, hw, (int)tpl, d_src, d_tgt, link_pair, rp, part, n_tiles);
          else if (last)
            k_adj_reduce<true, false><<<grid_red, THREADS, 0, cs>>>(
                d_xyz, weights, hw, (int)tpl, d_src, d_tgt, link_pair, rp, part, n_tiles);
          else
            k_adj_reduce<false, false><<<grid_red, THREADS, 0, cs>>>(
                d_xyz, weights, hw, (int)tpl, d_src, d_tgt, link_pair, rp, part, n_tiles);
        });
      traced(ctx, cs, "adj_solve", [&] {
        k_adj_solve<<<solve_blocks, 32, 0, cs>>>(n_pairs, iters, k - 1, d_link_off, (int)tpl,
                                                 part, n_tiles > 0, 0, ckpt, adj, gM, state,
                                                 delta, rp, nullptr);
      });
    }
    EC3R_CUDA_TRY(ctx, cudaMemsetAsync(refs, 0, sizeof(int32_t) * (size_t)(n_frames + 1), cs));
    if (n_links > 0)
      traced(ctx, cs, "adj_refcount", [&] {
        k_adj_refcount<<<(unsigned)((n_links + 255) / 256), 256, 0, cs>>>(
            n_links, n_frames, d_src, d_tgt, link_pair, refs, any_shared);
      });
    // The scatter writes the frames that exactly one link references; its CTAs
    // also zero every other frame (zero_slice: HBM stores beside FP32-bound
    // work, where a separate zeroing kernel could not run beside the scatter,
    // whose two CTAs per SM hold the whole register file).
    if (n_tiles > 0) {
      const size_t shm = sizeof(float2) * SC_PAIRS * (size_t)iters;
      const bool vz = vec && ((uintptr_t)d_grad_xyz % 16 == 0) &&
                      ((uintptr_t)d_grad_conf % 16 == 0);
      traced(ctx, cs, "adj_scatter", [&] {
        if (vz)
          k_adj_scatter<true><<<grid, THREADS, shm, cs>>>(
              d_xyz, d_conf, n_frames, hw, (int)tpl, d_src, d_tgt, link_pair, state, adj, ckpt,
              gM, iters, delta, rule, lg, refs, d_grad_xyz, d_grad_conf);
        else
          k_adj_scatter<false><<<grid, THREADS, shm, cs>>>(
              d_xyz, d_conf, n_frames, hw, (int)tpl, d_src, d_tgt, link_pair, state, adj, ckpt,
              gM, iters, delta, rule, lg, refs, d_grad_xyz, d_grad_conf);
      });
    } else {
      traced(ctx, cs, "adj_zero_frames", [&] {
        k_adj_zero_frames<<<(unsigned)n_frames, 512, 0, cs>>>(hw, refs, d_grad_xyz, d_grad_conf);
      });
    }
    if (n_tiles > 0)
      traced(ctx, cs, "adj_frames", [&] {
        k_adj_frames<<<(unsigned)((hw + 255) / 256), 256, 0, cs>>>(hw, n_links, d_src, d_tgt,
                                                                  link_pair, refs, any_shared, lg,
                                                                  d_grad_xyz, d_grad_conf);
      });
    EC3R_CUDA_TRY(ctx, cudaGetLastError());
    return EC3R_OK;
  });
}
