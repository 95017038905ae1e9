// Batched Huber-IRLS registration as persistent launches.
//
// The registration of Sec. III-C (Eq. (sim3), weighted Umeyama in Huber IRLS)
// alternates an HBM-bound moment sweep over every correspondence with a
// latency-bound FP64 solve per pair.  Launched as separate grids, every solve
// is a barrier across all pairs: the whole GPU waits for the slowest pair's
// FP64 solve ten times per call.  Here the sweeps of all iterations are one
// stream of work items (iteration j, tile t), handed out in that order by an
// atomic counter to a grid of resident CTAs:
//
//   * a CTA sweeps its tile with the pair's current estimate and writes the
//     tile's 19 FP64 partial moments (fixed slots: deterministic);
//   * it counts the tile in the pair's completion counter; the CTA that
//     completes the pair's last tile of iteration j sums the pair's partials
//     in fixed order and solves (FP64 polar factor, scale, translation), then
//     publishes the pair's epoch j with a release store;
//   * a tile of iteration j + 1 first waits (acquire) for its own pair's epoch
//     j, which its pair's tiles of iteration j - all handed out earlier, to
//     running CTAs - complete; no CTA ever waits for a CTA that has not started.
//
// So each pair's solve runs while other pairs' tiles stream, and only the
// last pair's last solve is exposed.  Sweep 1 runs as a launch of its own: it
// reads both confidences and stores every correspondence's weight (c_p c_q or
// c_p, NaN where the correspondence is invalid); the launch of the later
// sweeps follows it (programmatic dependent launch, same work-item scheme)
// and reads that weight instead: 28 B per pixel and sweep instead of 32.
// Every wait is bounded: past the limit the CTA raises FLAG_TIMEOUT and skips
// its tile.  When the cost is wanted, the last sweep runs after these
// launches as its own grid (k_final_sweep): it
// also accumulates the sums from which the cost under the last solve follows
// exactly (37 sums per pixel instead of 19, which would not fit the persistent
// loop's register budget of four CTAs per SM).
//
// Variants (tile pixels x CTAs per SM) are instantiated for the autotuner;
// the tile size groups the FP32 sums, so variants differ at FP32 rounding
// level; each is deterministic (tile partials have fixed slots and are summed
// in a fixed order, whichever CTA computed them).
#include "align_impl.cuh"

namespace ec3r {
namespace align {

// The weighted moments of one point (om its IRLS weight, x = p - piv_p,
// y = q - piv_q; v: the point is valid): W, Sp, Sq, Spp, Sqp and the count.
__device__ __forceinline__ void add_moments(float om, bool v, float x0, float x1, float x2,
                                            float y0, float y1, float y2, float* acc) {
  acc[M_W] += om;
  acc[M_CNT] += v ? 1.f : 0.f;
  const float wx0 = om * x0, wx1 = om * x1, wx2 = om * x2;
  const float wy0 = om * y0, wy1 = om * y1, wy2 = om * y2;
  acc[M_SP + 0] += wx0; acc[M_SP + 1] += wx1; acc[M_SP + 2] += wx2;
  acc[M_SQ + 0] += wy0; acc[M_SQ + 1] += wy1; acc[M_SQ + 2] += wy2;
  acc[M_PP] += wx0 * x0 + wx1 * x1 + wx2 * x2;
  acc[M_QP + 0] += wy0 * x0; acc[M_QP + 1] += wy0 * x1; acc[M_QP + 2] += wy0 * x2;
  acc[M_QP + 3] += wy1 * x0; acc[M_QP + 4] += wy1 * x1; acc[M_QP + 5] += wy1 * x2;
  acc[M_QP + 6] += wy2 * x0; acc[M_QP + 7] += wy2 * x1; acc[M_QP + 8] += wy2 * x2;
}

// One point's contribution to the moments of Huber-IRLS sweep j >= 2: weights
// from the current estimate S_{j-1} (A, b) around the pair's pivots (the
// solve uses no cost moment).  wv: the pixel's weight as pixel_weight gives
// it (NaN: invalid).
struct HuberOp {
  static constexpr int NV = NMOM;
  float A[9], b[3], pp[3], pq[3], delta, cmin;
  int rule;

  __device__ __forceinline__ void operator()(float p0, float p1, float p2, float q0, float q1,
                                             float q2, float wv, float* acc) const {
    const bool v = wv == wv;
    const float x0 = v ? p0 - pp[0] : 0.f, x1 = v ? p1 - pp[1] : 0.f, x2 = v ? p2 - pp[2] : 0.f;
    const float y0 = v ? q0 - pq[0] : 0.f, y1 = v ? q1 - pq[1] : 0.f, y2 = v ? q2 - pq[2] : 0.f;
    const float w = v ? wv : 0.f;
    const float e0 = A[0] * x0 + A[1] * x1 + A[2] * x2 + b[0] - y0;
    const float e1 = A[3] * x0 + A[4] * x1 + A[5] * x2 + b[1] - y1;
    const float e2 = A[6] * x0 + A[7] * x1 + A[8] * x2 + b[2] - y2;
    const float rr = e0 * e0 + e1 * e1 + e2 * e2;
    add_moments(w * fminf(1.f, delta * rsqrtf(rr)), v, x0, x1, x2, y0, y1, y2, acc);
  }
};

// Sweep 1 starts from the identity with h = 1: the IRLS weight is the pixel
// weight itself.  (HuberOp with delta = +inf gives the same om bit for bit:
// min(1, inf * rsqrt(r^2)) is 1 for every r^2, NaN included, since fminf
// drops a NaN operand; without the residual the loop holds fewer registers.)
struct FirstOp {
  static constexpr int NV = NMOM;
  float pp[3], pq[3], cmin;
  int rule;

  __device__ __forceinline__ void operator()(float p0, float p1, float p2, float q0, float q1,
                                             float q2, float wv, float* acc) const {
    const bool v = wv == wv;
    const float x0 = v ? p0 - pp[0] : 0.f, x1 = v ? p1 - pp[1] : 0.f, x2 = v ? p2 - pp[2] : 0.f;
    const float y0 = v ? q0 - pq[0] : 0.f, y1 = v ? q1 - pq[1] : 0.f, y2 = v ? q2 - pq[2] : 0.f;
    add_moments(v ? wv : 0.f, v, x0, x1, x2, y0, y1, y2, acc);
  }
};

// The pair's estimate as the operator of sweep j >= 2.  The state changes
// during the launch (other CTAs solve), so it is read from L2
// (ld.global.cg), never from a possibly stale L1 line.
__device__ __forceinline__ void load_op(const PairState* S, float delta, int rule, HuberOp& op) {
#pragma unroll
  for (int i = 0; i < 9; ++i) op.A[i] = __ldcg(&S->A[i]);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    op.b[i] = __ldcg(&S->b[i]);
    op.pp[i] = __ldcg(&S->piv_p[i]);
    op.pq[i] = __ldcg(&S->piv_q[i]);
  }
  op.delta = delta;
  op.cmin = __ldcg(&S->cmin);
  op.rule = rule;
}

__device__ __forceinline__ void load_first(const PairState* S, int rule, FirstOp& op) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    op.pp[i] = __ldcg(&S->piv_p[i]);
    op.pq[i] = __ldcg(&S->piv_q[i]);
  }
  op.cmin = __ldcg(&S->cmin);
  op.rule = rule;
}

// Pairwise butterfly of a thread's sums inside the warp; lane 0 of warp w
// leaves the warp's sums in red[w] (the caller adds the warps in FP64).
template <int NV>
__device__ __forceinline__ void warp_sums(float* acc, double (*red)[NV]) {
#pragma unroll
  for (int m = 0; m < NV; ++m)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], o);
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int m = 0; m < NV; ++m) red[warp][m] = (double)acc[m];
}

// The first sweep's tile of TP pixels of one link: per-thread sums of 4
// consecutive pixels at a time (p, q and both confidences read), and every
// pixel's weight stored for the later sweeps (WO: the tile's slice of the
// link's weights).
template <bool VEC, int TP, class OP, int UNROLL = 2>
__device__ __forceinline__ void tile_first(const OP& op, const float* __restrict__ P,
                                           const float* __restrict__ Q,
                                           const float* __restrict__ CP,
                                           const float* __restrict__ CQ, float* __restrict__ WO,
                                           int npx, double (*red)[OP::NV]) {
  constexpr int NV = OP::NV;
  float acc[NV];
#pragma unroll
  for (int m = 0; m < NV; ++m) acc[m] = 0.f;
  const float cmin = op.cmin;
  const int rule = op.rule;
#pragma unroll UNROLL
  for (int g = threadIdx.x; g < TP / 4; g += THREADS) {
    const int i0 = 4 * g;
    if (i0 >= npx) break;
    if (VEC && i0 + 4 <= npx) {
      const float4* P4 = reinterpret_cast<const float4*>(P + 3 * i0);
      const float4* Q4 = reinterpret_cast<const float4*>(Q + 3 * i0);
      const float4 pa = __ldcs(P4), pb = __ldcs(P4 + 1), pc = __ldcs(P4 + 2);
      const float4 qa = __ldcs(Q4), qb = __ldcs(Q4 + 1), qc = __ldcs(Q4 + 2);
      const float4 cp = __ldcs(reinterpret_cast<const float4*>(CP + i0));
      const float4 cq = __ldcs(reinterpret_cast<const float4*>(CQ + i0));
      // pixel by pixel, so that each pixel's loads die after its use
      float4 w;
      w.x = pixel_weight(pa.x, pa.y, pa.z, qa.x, qa.y, qa.z, cp.x, cq.x, cmin, rule);
      op(pa.x, pa.y, pa.z, qa.x, qa.y, qa.z, w.x, acc);
      w.y = pixel_weight(pa.w, pb.x, pb.y, qa.w, qb.x, qb.y, cp.y, cq.y, cmin, rule);
      op(pa.w, pb.x, pb.y, qa.w, qb.x, qb.y, w.y, acc);
      w.z = pixel_weight(pb.z, pb.w, pc.x, qb.z, qb.w, qc.x, cp.z, cq.z, cmin, rule);
      op(pb.z, pb.w, pc.x, qb.z, qb.w, qc.x, w.z, acc);
      w.w = pixel_weight(pc.y, pc.z, pc.w, qc.y, qc.z, qc.w, cp.w, cq.w, cmin, rule);
      op(pc.y, pc.z, pc.w, qc.y, qc.z, qc.w, w.w, acc);
      __stcs(reinterpret_cast<float4*>(WO + i0), w);
    } else {
      const int n = min(4, npx - i0);
      for (int j = 0; j < n; ++j) {
        const int i = i0 + j;
        const float w = pixel_weight(P[3 * i], P[3 * i + 1], P[3 * i + 2], Q[3 * i],
                                     Q[3 * i + 1], Q[3 * i + 2], CP[i], CQ[i], cmin, rule);
        __stcs(WO + i, w);
        op(P[3 * i], P[3 * i + 1], P[3 * i + 2], Q[3 * i], Q[3 * i + 1], Q[3 * i + 2], w, acc);
      }
    }
  }
  warp_sums<NV>(acc, red);
}

// A later sweep's tile: p, q and the stored weights (28 B per pixel instead
// of 32).  The weights come from the sweep-1 launch, and a tile reads them
// only after acquiring its pair's epoch (>= 1): no CTA of the reading launch
// writes them, so they stream like p and q (evict-first: about as large as
// L2, at normal priority they would displace the p, q lines in flight).
template <bool VEC, int TP, class OP, int UNROLL = 2>
__device__ __forceinline__ void tile_w(const OP& op, const float* __restrict__ P,
                                       const float* __restrict__ Q, const float* WI, int npx,
                                       double (*red)[OP::NV]) {
  constexpr int NV = OP::NV;
  float acc[NV];
#pragma unroll
  for (int m = 0; m < NV; ++m) acc[m] = 0.f;
#pragma unroll UNROLL
  for (int g = threadIdx.x; g < TP / 4; g += THREADS) {
    const int i0 = 4 * g;
    if (i0 >= npx) break;
    if (VEC && i0 + 4 <= npx) {
      const float4* P4 = reinterpret_cast<const float4*>(P + 3 * i0);
      const float4* Q4 = reinterpret_cast<const float4*>(Q + 3 * i0);
      const float4 pa = __ldcs(P4), pb = __ldcs(P4 + 1), pc = __ldcs(P4 + 2);
      const float4 qa = __ldcs(Q4), qb = __ldcs(Q4 + 1), qc = __ldcs(Q4 + 2);
      const float4 w = __ldcs(reinterpret_cast<const float4*>(WI + i0));
      op(pa.x, pa.y, pa.z, qa.x, qa.y, qa.z, w.x, acc);
      op(pa.w, pb.x, pb.y, qa.w, qb.x, qb.y, w.y, acc);
      op(pb.z, pb.w, pc.x, qb.z, qb.w, qc.x, w.z, acc);
      op(pc.y, pc.z, pc.w, qc.y, qc.z, qc.w, w.w, acc);
    } else {
      const int n = min(4, npx - i0);
      for (int j = 0; j < n; ++j) {
        const int i = i0 + j;
        op(P[3 * i], P[3 * i + 1], P[3 * i + 2], Q[3 * i], Q[3 * i + 1], Q[3 * i + 2],
           __ldcs(WI + i), acc);
      }
    }
  }
  warp_sums<NV>(acc, red);
}

struct RegArgs {
  const float* xyz;
  const float* conf;
  int64_t hw;
  int tpl;             // tiles per link
  int64_t n_tiles;     // tiles per sweep
  float* wt;           // [n_links][hw] link pixel weights: written by sweep 1, read after
  const int32_t* link_off;
  const int32_t* src;
  const int32_t* tgt;
  const int32_t* link_pair;
  PairState* st;
  double* partials;    // [n_tiles][NMOM]
  float delta;
  int rule;
  int iters;           // Huber-IRLS solves of the call
  int n_sweeps;        // sweeps of this launch: iters, or iters - 1 before k_final_sweep
  ec3r_sim3* out;
  int32_t* status_out;
  double* cost;        // nullable: zeroed for pairs that turn degenerate
  double* cost_sums;   // [n_pairs][CS_STRIDE], zeroed likewise
  double* ckpt;        // [n_pairs][iters][CKPT]
  unsigned long long* next;   // work items handed out (sweep 1)
  unsigned long long* next2;  // work items handed out (sweeps 2 .. n_sweeps)
  unsigned* abort;            // set when a wait gave up: every CTA stops
  unsigned long long* done;   // per pair: tiles completed, over all sweeps
  unsigned* epoch;            // per pair: solves completed (EPOCH_DONE: degenerate)
  unsigned* flags;
  long long wait_cycles;
  int no_epoch;        // test injection: solves publish no epoch
};

// Warp 0 of the CTA that completed pair k's sweep j: the solve of iteration j,
// then the pair's epoch j (EPOCH_DONE if the pair turned degenerate).
__device__ __noinline__ void finish_pair(const RegArgs& a, int k, int j, double* mom) {
  const int lane = threadIdx.x & 31;
  __threadfence();
  const int64_t t0 = (int64_t)a.link_off[k] * a.tpl, t1 = (int64_t)a.link_off[k + 1] * a.tpl;
  if (lane < NMOM) mom[lane] = tile_sum_cg<NMOM>(a.partials, t0, t1, lane);
  __syncwarp();
  if (lane == 0) {
    double R[9], s = 1.0, b[3] = {0, 0, 0}, dV[12];
    const unsigned status = umeyama_from_moments(mom, R, s, b, dV);
    double* ck = a.ckpt + ((size_t)k * a.iters + (j - 1)) * CKPT;
    for (int m = 0; m < NMOM; ++m) ck[CK_MOM + m] = mom[m];
    for (int i = 0; i < 9; ++i) ck[CK_A + i] = s * R[i];
    for (int i = 0; i < 3; ++i) ck[CK_B + i] = b[i];
    ck[CK_STATUS] = (double)status;
    ck[CK_S] = s;
    for (int i = 0; i < 9; ++i) ck[CK_R + i] = R[i];
    for (int i = 0; i < 12; ++i) ck[CK_D + i] = status ? 0.0 : dV[i];
    commit_estimate(a.st[k], status, R, s, b, j == a.iters, a.out[k], a.status_out[k]);
    if (status && a.cost) {  // a degenerate pair reports no cost
      a.cost[k] = 0.0;
      double* cs = a.cost_sums + (size_t)k * CS_STRIDE;
      for (int i = 0; i < CS_STRIDE; ++i) cs[i] = 0.0;
    }
    __threadfence();
    // a pair that turned degenerate is skipped by every later sweep
    if (!a.no_epoch) st_release_u32(a.epoch + k, status ? EPOCH_DONE : (unsigned)j);
  }
}

// FIRSTP: sweep 1 alone (confidences in, pixel weights out); otherwise
// sweeps 2 .. n_sweeps, which read the weights.  The two are separate
// launches so that each loop has the registers to itself (one kernel holding
// both tile paths spills under the 64 registers of four CTAs per SM); the
// second is a programmatic dependent launch whose tiles wait per pair on
// epoch 1 like any later sweep, so it starts as the first one's CTAs retire.
template <bool VEC, int TP, int MINB, bool FIRSTP>
__global__ void __launch_bounds__(THREADS, MINB) k_register(const __grid_constant__ RegArgs a) {
  // the next launch (programmatic dependent) may be scheduled as soon as this
  // grid's CTAs are resident: it waits per pair on the epochs
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  constexpr int J0 = FIRSTP ? 1 : 2;  // the launch's first sweep
  unsigned long long* next = FIRSTP ? a.next : a.next2;
  __shared__ double red[THREADS / 32][NMOM];
  __shared__ double mom[NMOM];
  __shared__ long long s_item;
  __shared__ int s_k, s_go, s_last;
  __shared__ long long s_pre;  // the next item, fetched while this one is reduced
  const long long total = FIRSTP ? a.n_tiles : (long long)(a.n_sweeps - 1) * a.n_tiles;
  if (threadIdx.x == 0) s_pre = -1;
  for (;;) {
    if (threadIdx.x == 0) {
      // after a timeout anywhere, hand out nothing more
      const long long item = ld_acquire_u32(a.abort) ? total
                             : s_pre >= 0            ? s_pre
                                                     : (long long)atomicAdd(next, 1ull);
      s_pre = -1;
      int k = -1, go = 0;
      if (item < total) {
        const int j = (int)(item / a.n_tiles) + J0;
        const int64_t t = item - (long long)(j - J0) * a.n_tiles;
        k = a.link_pair[t / a.tpl];
        if (k >= 0) {
          go = FIRSTP ? 1 : (int)wait_epoch(a.epoch + k, (unsigned)(j - 1), a.abort, a.flags,
                                            a.wait_cycles);
          if (go) go = __ldcg(&a.st[k].active);
        }
      }
      s_item = item;
      s_k = k;
      s_go = go;
    }
    __syncthreads();
    const long long item = s_item;
    if (item >= total) break;
    if (s_go) {
      {
        const int k = s_k;
        const int j = (int)(item / a.n_tiles) + J0;
        const int64_t t = item - (long long)(j - J0) * a.n_tiles;
        const int64_t l = t / a.tpl;
        const int c = (int)(t - l * a.tpl);
        const int64_t fs = a.src[l], ft = a.tgt[l];
        const int64_t px0 = (int64_t)c * TP;
        const int64_t rem = a.hw - px0;
        const int npx = rem < TP ? (int)rem : TP;
        const float* P = a.xyz + (fs * a.hw + px0) * 3;
        const float* Q = a.xyz + (ft * a.hw + px0) * 3;
        float* wt = a.wt + l * a.hw + px0;
        if (FIRSTP) {
          FirstOp op;
          load_first(a.st + k, a.rule, op);
          tile_first<VEC, TP, FirstOp>(op, P, Q, a.conf + fs * a.hw + px0,
                                       a.conf + ft * a.hw + px0, wt, npx, red);
          // the weights are published with the tile's count (below)
          __threadfence();
        } else {
          HuberOp op;
          load_op(a.st + k, a.delta, a.rule, op);
          tile_w<VEC, TP, HuberOp>(op, P, Q, wt, npx, red);
        }
      }
      // the next item's round trip to the counter overlaps this one's reduction
      if (threadIdx.x == 0) s_pre = (long long)atomicAdd(next, 1ull);
      __syncthreads();
      // the item again from shared memory, so that nothing of it stays live
      // across the sweep (registers)
      const long long it = *(volatile long long*)&s_item;
      const int k = *(volatile int*)&s_k;
      const int j = (int)(it / a.n_tiles) + J0;
      const int64_t t = it - (long long)(j - J0) * a.n_tiles;
      if (threadIdx.x < NMOM) {  // the tile's moments: FP64 over the warps, fixed order
        double sum = 0.0;
#pragma unroll
        for (int w = 0; w < THREADS / 32; ++w) sum += red[w][threadIdx.x];
        a.partials[t * NMOM + threadIdx.x] = sum;
        __threadfence();
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        const unsigned long long nt =
            (unsigned long long)(a.link_off[k + 1] - a.link_off[k]) * (unsigned long long)a.tpl;
        const unsigned long long old = atomicAdd(a.done + k, 1ull);
        s_last = old + 1ull == (unsigned long long)j * nt;
        if (s_last) __threadfence();
      }
      __syncthreads();
      if (s_last && threadIdx.x < 32) finish_pair(a, k, j, mom);
    }
    __syncthreads();
  }
  // the sweeps after the first end only once sweep 1's launch has completed,
  // so that work ordered after this launch in the stream also follows that one
  if (!FIRSTP) asm volatile("griddepcontrol.wait;" ::: "memory");
}

// --------------------------------------------------------------------------
// the last Huber sweep with the cost, overlapping the persistent launch's tail
// --------------------------------------------------------------------------
// The cost the adjoint needs, J = sum om |r_K|^2 / sum om (weights om of the
// last sweep, from S_{K-1}; residual r_K under the returned S_K), and its
// sums sum om r_K p'^T, sum om r_K, come out of the last Huber sweep itself
// instead of one more pass over every correspondence.  With r = r_{K-1} and
// D = S_K - S_{K-1} in the (A, b) form, r_K = r + D_A p' + D_b exactly, so
//   sum om |r_K|^2 = E + 2 <D_A, G> + 2 D_b . g + <D_A C, D_A> + 2 D_b . D_A Sp + W |D_b|^2
//   sum om r_K p'^T = G + D_A C + D_b Sp^T,     sum om r_K = g + D_A Sp + W D_b
// with E = sum om |r|^2, G = sum om r p'^T, g = sum om r, C = sum om p' p'^T
// accumulated by the sweep beside the moments (Sp = sum om p', W = sum om).
// Once the IRLS has settled D is small, so the terms that carry it are
// corrections to sums accumulated directly (no cancellation of large terms).
constexpr int F_G = NMOM;        // G, row-major (9)
constexpr int F_GV = NMOM + 9;   // g (3)
constexpr int F_C = NMOM + 12;   // C: xx, xy, xz, yy, yz, zz (6)
constexpr int NFIN = FINAL_VALUES;

struct FinalOp {
  static constexpr int NV = NFIN;
  float A[9], b[3], pp[3], pq[3], delta, cmin;
  int rule;

  // the moments exactly as HuberOp forms them, then E (in the M_COST slot), G, g, C
  __device__ __forceinline__ void operator()(float p0, float p1, float p2, float q0, float q1,
                                             float q2, float wv, float* acc) const {
    const bool v = wv == wv;
    const float x0 = v ? p0 - pp[0] : 0.f, x1 = v ? p1 - pp[1] : 0.f, x2 = v ? p2 - pp[2] : 0.f;
    const float y0 = v ? q0 - pq[0] : 0.f, y1 = v ? q1 - pq[1] : 0.f, y2 = v ? q2 - pq[2] : 0.f;
    const float w = v ? wv : 0.f;
    const float e0 = A[0] * x0 + A[1] * x1 + A[2] * x2 + b[0] - y0;
    const float e1 = A[3] * x0 + A[4] * x1 + A[5] * x2 + b[1] - y1;
    const float e2 = A[6] * x0 + A[7] * x1 + A[8] * x2 + b[2] - y2;
    const float rr = e0 * e0 + e1 * e1 + e2 * e2;
    const float om = w * fminf(1.f, delta * rsqrtf(rr));
    add_moments(om, v, x0, x1, x2, y0, y1, y2, acc);
    acc[M_COST] += om * rr;
    const float wx0 = om * x0, wx1 = om * x1, wx2 = om * x2;
    const float g0 = om * e0, g1 = om * e1, g2 = om * e2;
    acc[F_G + 0] += g0 * x0; acc[F_G + 1] += g0 * x1; acc[F_G + 2] += g0 * x2;
    acc[F_G + 3] += g1 * x0; acc[F_G + 4] += g1 * x1; acc[F_G + 5] += g1 * x2;
    acc[F_G + 6] += g2 * x0; acc[F_G + 7] += g2 * x1; acc[F_G + 8] += g2 * x2;
    acc[F_GV + 0] += g0; acc[F_GV + 1] += g1; acc[F_GV + 2] += g2;
    acc[F_C + 0] += wx0 * x0; acc[F_C + 1] += wx0 * x1; acc[F_C + 2] += wx0 * x2;
    acc[F_C + 3] += wx1 * x1; acc[F_C + 4] += wx1 * x2; acc[F_C + 5] += wx2 * x2;
  }
};

struct FinalArgs {
  const float* xyz;
  const float* conf;
  int64_t hw;
  int tpl;              // tiles of TILE pixels per link
  const int32_t* link_off;
  const int32_t* src;
  const int32_t* tgt;
  const int32_t* link_pair;
  float* wt;            // [n_links][hw] link pixel weights (written here when iters = 1)
  PairState* st;
  double* partials;     // [n_tiles][NFIN], its own buffer
  float delta;
  int rule;
  int iters;
  ec3r_sim3* out;
  int32_t* status_out;
  double* cost;         // [n_pairs]
  double* cost_sums;    // [n_pairs][CS_STRIDE]
  double* ckpt;
  unsigned long long* done;  // per pair: final tiles completed
  const unsigned* epoch;     // the persistent launch's per-pair epochs
  unsigned* abort;
  unsigned* flags;
  long long wait_cycles;
};

// Warp 0 of the CTA that completed pair k's final tiles: the last solve (as
// finish_pair), then the cost and the cost term's sums from the identities above.
__device__ __noinline__ void finish_final(const FinalArgs& a, int k, double* f) {
  const int lane = threadIdx.x & 31;
  __threadfence();
  const int64_t t0 = (int64_t)a.link_off[k] * a.tpl, t1 = (int64_t)a.link_off[k + 1] * a.tpl;
  f[lane] = tile_sum_cg<NFIN>(a.partials, t0, t1, lane);
  if (lane + 32 < NFIN) f[lane + 32] = tile_sum_cg<NFIN>(a.partials, t0, t1, lane + 32);
  __syncwarp();
  if (lane != 0) return;
  double R[9], s = 1.0, b[3] = {0, 0, 0}, dV[12];
  const unsigned status = umeyama_from_moments(f, R, s, b, dV);
  double* ck = a.ckpt + ((size_t)k * a.iters + (a.iters - 1)) * CKPT;
  for (int m = 0; m < NMOM; ++m) ck[CK_MOM + m] = f[m];
  for (int i = 0; i < 9; ++i) ck[CK_A + i] = s * R[i];
  for (int i = 0; i < 3; ++i) ck[CK_B + i] = b[i];
  ck[CK_STATUS] = (double)status;
  ck[CK_S] = s;
  for (int i = 0; i < 9; ++i) ck[CK_R + i] = R[i];
  for (int i = 0; i < 12; ++i) ck[CK_D + i] = status ? 0.0 : dV[i];
  PairState& S = a.st[k];
  commit_estimate(S, status, R, s, b, true, a.out[k], a.status_out[k]);
  double* cs = a.cost_sums + (size_t)k * CS_STRIDE;
  if (status) {  // a degenerate pair reports no cost
    a.cost[k] = 0.0;
    for (int i = 0; i < CS_STRIDE; ++i) cs[i] = 0.0;
    return;
  }
  // D between the FP32 estimates that the residuals use (S_K now in A, b;
  // S_{K-1}, which weighted this sweep, in Ap, bp)
  double DA[9], Db[3], C[9];
  for (int i = 0; i < 9; ++i) DA[i] = (double)S.A[i] - (double)S.Ap[i];
  for (int i = 0; i < 3; ++i) Db[i] = (double)S.b[i] - (double)S.bp[i];
  C[0] = f[F_C + 0]; C[1] = C[3] = f[F_C + 1]; C[2] = C[6] = f[F_C + 2];
  C[4] = f[F_C + 3]; C[5] = C[7] = f[F_C + 4]; C[8] = f[F_C + 5];
  const double W = f[M_W];
  const double* Sp = f + M_SP;
  double J = f[M_COST];
  for (int i = 0; i < 3; ++i) {
    const double dAs = DA[3 * i] * Sp[0] + DA[3 * i + 1] * Sp[1] + DA[3 * i + 2] * Sp[2];
    double gi = f[F_GV + i] + dAs + W * Db[i];
    J += 2.0 * Db[i] * (f[F_GV + i] + dAs) + W * Db[i] * Db[i];
    for (int j = 0; j < 3; ++j) {
      const double dAC = DA[3 * i] * C[j] + DA[3 * i + 1] * C[3 + j] + DA[3 * i + 2] * C[6 + j];
      const double G = f[F_G + 3 * i + j];
      J += DA[3 * i + j] * (2.0 * G + dAC);
      cs[3 * i + j] = G + dAC + Db[i] * Sp[j];
    }
    cs[9 + i] = gi;
  }
  const double v = W > 0.0 ? J / W : 0.0;
  a.cost[k] = v;
  cs[CS_COST] = v;
}

// One CTA per tile of TILE pixels (a programmatic dependent launch after
// k_register, which ran sweeps 1 .. K-1): waits for its pair's solve K-1
// (epoch K-1), runs the pair's last Huber sweep with the cost sums, and the
// CTA that completes a pair's tiles solves, checkpoints and commits S_K and
// forms the cost.  Every CTA ends by waiting for k_register to complete, so
// that the work after this launch in the stream also follows k_register.
// (37 accumulators: three CTAs of 256 threads per SM, 80 registers)
constexpr int FIN_MINB = 3, FIN_UNROLL = 2;

// FIRSTW: a single solve (iters = 1), whose only sweep reads the
// confidences and stores the pixel weights.
template <bool VEC, bool FIRSTW>
__global__ void __launch_bounds__(THREADS, FIN_MINB)
    k_final_sweep(const __grid_constant__ FinalArgs a) {
  __shared__ double red[THREADS / 32][NFIN];
  __shared__ double fin[NFIN];
  __shared__ int s_go, s_last;
  const int64_t t = blockIdx.x;
  const int64_t l = t / a.tpl;
  const int c = (int)(t - l * a.tpl);
  const int k = a.link_pair[l];
  if (threadIdx.x == 0) {
    int go = 0;
    if (k >= 0) {
      go = a.iters < 2 ? 1
                       : (int)wait_epoch(a.epoch + k, (unsigned)(a.iters - 1), a.abort, a.flags,
                                         a.wait_cycles);
      if (go) go = __ldcg(&a.st[k].active);
    }
    s_go = go;
  }
  __syncthreads();
  if (s_go) {
    const PairState* S = a.st + k;
    FinalOp op;
#pragma unroll
    for (int i = 0; i < 9; ++i) op.A[i] = __ldcg(&S->A[i]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      op.b[i] = __ldcg(&S->b[i]);
      op.pp[i] = __ldcg(&S->piv_p[i]);
      op.pq[i] = __ldcg(&S->piv_q[i]);
    }
    // a single solve has unit Huber weights (its sweep starts from the identity)
    op.delta = a.iters == 1 ? INFINITY : a.delta;
    op.cmin = __ldcg(&S->cmin);
    op.rule = a.rule;
    const int64_t fs = a.src[l], ft = a.tgt[l];
    const int64_t px0 = (int64_t)c * TILE;
    const int64_t rem = a.hw - px0;
    const float* P = a.xyz + (fs * a.hw + px0) * 3;
    const float* Q = a.xyz + (ft * a.hw + px0) * 3;
    float* wt = a.wt + l * a.hw + px0;
    const int npx = rem < TILE ? (int)rem : TILE;
    if (FIRSTW)  // the only sweep: weights from the confidences, stored for the adjoint
      tile_first<VEC, TILE, FinalOp, FIN_UNROLL>(op, P, Q, a.conf + fs * a.hw + px0,
                                                 a.conf + ft * a.hw + px0, wt, npx, red);
    else  // sweep 1 of k_register wrote them before the pair's epoch 1
      tile_w<VEC, TILE, FinalOp, FIN_UNROLL>(op, P, Q, wt, npx, red);
    __syncthreads();
    for (int m = threadIdx.x; m < NFIN; m += THREADS) {
      double sum = 0.0;
#pragma unroll
      for (int w = 0; w < THREADS / 32; ++w) sum += red[w][m];
      a.partials[t * NFIN + m] = sum;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned long long nt =
          (unsigned long long)(a.link_off[k + 1] - a.link_off[k]) * (unsigned long long)a.tpl;
      s_last = atomicAdd(a.done + k, 1ull) + 1ull == nt;
      if (s_last) __threadfence();
    }
    __syncthreads();
    if (s_last && threadIdx.x < 32) finish_final(a, k, fin);
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// --------------------------------------------------------------------------
// host side: variants, occupancy, launch
// --------------------------------------------------------------------------
typedef void (*RegKernel)(const RegArgs);

struct RegVariant {
  int tile, ctas;
  RegKernel first;  // sweep 1
  RegKernel fn;     // sweeps 2 .. n
};

#define EC3R_REG_VARIANT(VEC, TP, MINB) \
  { TP, MINB, k_register<VEC, TP, MINB, true>, k_register<VEC, TP, MINB, false> }

// 16-byte aligned pointmaps: the autotuner's persistent candidates (tile
// pixels, CTAs per SM; 64, 80 and 128 registers per thread).  One more
// variant, the last, runs every sweep and solve as separate grids (align.cu).
static const RegVariant kTuned[] = {
    EC3R_REG_VARIANT(true, 8192, 4),  EC3R_REG_VARIANT(true, 8192, 3),
    EC3R_REG_VARIANT(true, 8192, 2),  EC3R_REG_VARIANT(true, 4096, 4),
    EC3R_REG_VARIANT(true, 4096, 3),  EC3R_REG_VARIANT(true, 4096, 2),
    EC3R_REG_VARIANT(true, 16384, 4), EC3R_REG_VARIANT(true, 16384, 3),
    EC3R_REG_VARIANT(true, 16384, 2), EC3R_REG_VARIANT(true, 32768, 4),
    EC3R_REG_VARIANT(true, 32768, 3), EC3R_REG_VARIANT(true, 32768, 2),
};
constexpr int N_TUNED = sizeof(kTuned) / sizeof(kTuned[0]);
// Unaligned pointmaps or hw not a multiple of 4: scalar loads, one configuration.
static const RegVariant kScalar = EC3R_REG_VARIANT(false, 8192, 3);
#undef EC3R_REG_VARIANT

int reg_variant_count() { return N_TUNED + 1; }

int reg_grid_variant() { return N_TUNED; }

bool reg_variant_info(int v, int* tile, int* ctas, int* persistent) {
  if (v == N_TUNED) {  // separate grids: k_sweep and k_solve
    *tile = TILE;
    *ctas = 4;
    *persistent = 0;
    return true;
  }
  if (v < 0 || v >= N_TUNED) return false;
  *tile = kTuned[v].tile;
  *ctas = kTuned[v].ctas;
  *persistent = 1;
  return true;
}

int reg_min_tile() { return 4096; }

static const RegVariant& pick(int v, bool vec) {
  if (!vec) return kScalar;
  return kTuned[(v >= 0 && v < N_TUNED) ? v : 0];
}

// Resident CTAs of a kernel of a variant on this device (the persistent grid's size).
static int resident_ctas(RegKernel fn, int sm_count) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, THREADS, 0) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return per_sm * sm_count;
}

// Enqueues a persistent launch of variant v on `s`: with `first`, sweep 1
// (after clearing `ctl`, inside the caller's graph, so every call starts from
// zero); otherwise sweeps 2 .. n_sweeps, a programmatic dependent launch that
// must directly follow the first in the stream.  `ctl` holds the first work
// counter, the abort word, the per-pair completion counters and epochs, and
// the second work counter (reg_ctl_bytes).
ec3r_status launch_register(ec3r_ctx* ctx, cudaStream_t s, int v, bool vec, bool first,
                            const float* xyz, const float* conf, int64_t hw, int n_pairs,
                            int64_t n_links, const int32_t* link_off, const int32_t* src,
                            const int32_t* tgt, const int32_t* link_pair, float* weights,
                            PairState* st, double* partials, float delta, int rule, int iters,
                            int n_sweeps, ec3r_sim3* out, int32_t* status_out, double* cost,
                            double* cost_sums, double* ckpt, void* ctl, size_t ctl_bytes) {
  const RegVariant& rv = pick(v, vec);
  const int64_t tpl = (hw + rv.tile - 1) / rv.tile;
  RegArgs a;
  a.xyz = xyz;
  a.conf = conf;
  a.hw = hw;
  a.tpl = (int)tpl;
  a.n_tiles = n_links * tpl;
  a.wt = weights;
  a.link_off = link_off;
  a.src = src;
  a.tgt = tgt;
  a.link_pair = link_pair;
  a.st = st;
  a.partials = partials;
  a.delta = delta;
  a.rule = rule;
  a.iters = iters;
  a.n_sweeps = n_sweeps;
  a.out = out;
  a.status_out = status_out;
  a.cost = cost;
  a.cost_sums = cost_sums;
  a.ckpt = ckpt;
  unsigned long long* c = (unsigned long long*)ctl;
  a.next = c;
  a.abort = (unsigned*)(c + 1);
  a.done = c + 2;
  a.epoch = (unsigned*)(c + 2 + n_pairs);
  a.next2 = (unsigned long long*)((unsigned*)(c + 2 + n_pairs) + n_pairs + (n_pairs & 1)) +
            n_pairs;
  a.flags = ctx->d_flags;
  a.wait_cycles = wait_limit_cycles(ctx);
  a.no_epoch = (ctx->inject & EC3R_INJECT_ALIGN_NO_EPOCH) ? 1 : 0;
  if (first) {
    EC3R_CUDA_TRY(ctx, cudaMemsetAsync(ctl, 0, ctl_bytes, s));
    if (n_sweeps == 0 || a.n_tiles == 0) return EC3R_OK;
    const long long grid =
        std::min<long long>(resident_ctas(rv.first, ctx->sm_count), a.n_tiles);
    rv.first<<<(unsigned)grid, THREADS, 0, s>>>(a);
    EC3R_CUDA_TRY(ctx, cudaGetLastError());
    return EC3R_OK;
  }
  if (n_sweeps <= 1 || a.n_tiles == 0) return EC3R_OK;
  const long long rest = (long long)(n_sweeps - 1) * a.n_tiles;
  const long long grid = std::min<long long>(resident_ctas(rv.fn, ctx->sm_count), rest);
  // (under per-kernel profiling, a plain launch: the two do not overlap)
  if (ctx->profiling)
    rv.fn<<<(unsigned)grid, THREADS, 0, s>>>(a);
  else
    EC3R_CUDA_TRY(ctx, launch_pdl(rv.fn, dim3((unsigned)grid), dim3(THREADS), 0, s, a));
  EC3R_CUDA_TRY(ctx, cudaGetLastError());
  return EC3R_OK;
}

// The final sweep as a programmatic dependent launch after launch_register's
// (same stream, same control block; a plain launch when `after_register` is
// false, i.e. no sweep ran before it): its tiles start as the persistent CTAs
// retire and wait only for their own pair's solve K-1.
ec3r_status launch_final(ec3r_ctx* ctx, cudaStream_t s, bool vec, bool after_register,
                         const float* xyz, const float* conf, int64_t hw, int n_pairs,
                         int64_t n_links, const int32_t* link_off, const int32_t* src,
                         const int32_t* tgt, const int32_t* link_pair, float* weights,
                         PairState* st, double* partials, float delta, int rule, int iters,
                         ec3r_sim3* out,
                         int32_t* status_out, double* cost, double* cost_sums, double* ckpt,
                         void* ctl) {
  const int64_t tpl = (hw + TILE - 1) / TILE;
  const int64_t n_tiles = n_links * tpl;
  if (n_tiles == 0) return EC3R_OK;
  FinalArgs a;
  a.xyz = xyz;
  a.conf = conf;
  a.hw = hw;
  a.tpl = (int)tpl;
  a.link_off = link_off;
  a.src = src;
  a.tgt = tgt;
  a.link_pair = link_pair;
  a.wt = weights;
  a.st = st;
  a.partials = partials;
  a.delta = delta;
  a.rule = rule;
  a.iters = iters;
  a.out = out;
  a.status_out = status_out;
  a.cost = cost;
  a.cost_sums = cost_sums;
  a.ckpt = ckpt;
  unsigned long long* c = (unsigned long long*)ctl;
  a.abort = (unsigned*)(c + 1);
  a.epoch = (const unsigned*)(c + 2 + n_pairs);
  a.done = (unsigned long long*)((unsigned*)(c + 2 + n_pairs) + n_pairs + (n_pairs & 1));
  a.flags = ctx->d_flags;
  a.wait_cycles = wait_limit_cycles(ctx);
  const dim3 grid((unsigned)n_tiles), block(THREADS);
  cudaError_t e;
  // (after_register implies iters >= 2: sweeps ran before this one)
  if (after_register)
    e = vec ? launch_pdl(k_final_sweep<true, false>, grid, block, 0, s, a)
            : launch_pdl(k_final_sweep<false, false>, grid, block, 0, s, a);
  else {
    if (iters == 1 && vec)
      k_final_sweep<true, true><<<grid, block, 0, s>>>(a);
    else if (iters == 1)
      k_final_sweep<false, true><<<grid, block, 0, s>>>(a);
    else if (vec)
      k_final_sweep<true, false><<<grid, block, 0, s>>>(a);
    else
      k_final_sweep<false, false><<<grid, block, 0, s>>>(a);
    e = cudaGetLastError();
  }
  EC3R_CUDA_TRY(ctx, e);
  return EC3R_OK;
}

// Sweep 1's work counter, abort word, per pair the completion counters and
// epochs of the persistent launches, then (8-byte aligned) the final sweep's
// completion counters and the later sweeps' work counter.
size_t reg_ctl_bytes(int n_pairs) {
  return sizeof(unsigned long long) * (2 + (size_t)n_pairs) +
         sizeof(unsigned) * ((size_t)n_pairs + (size_t)(n_pairs & 1)) +
         sizeof(unsigned long long) * ((size_t)n_pairs + 1);
}

}  // namespace align
}  // namespace ec3r
