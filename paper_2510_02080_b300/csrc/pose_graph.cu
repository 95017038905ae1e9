// Sim(3) pose-graph correction of submap poses (Sec. III-E).
//
// Nodes are submap poses T_t (submap -> world), an edge (i, j) carries the
// relative transform T_ij from registration, its error is
// e_ij = log(T_ij^-1 T_i^-1 T_j) and the energy chi^2 = sum e^T Omega e.  The
// poses are initialised by chaining the relative transforms and refined by
// Gauss-Newton (optionally damped: H + lambda I) with right perturbations
// T <- T Exp(delta) and one node held fixed.
//
// Host (once per graph structure, cached in the context): an ordering of the
// free nodes (nested dissection or minimum degree, whichever a cost estimate
// prefers), the block fill of the Cholesky factor, its elimination-tree
// levels, the trailing dense supernode, the left-looking update lists and the
// assembly lists.
// Device, per Gauss-Newton iteration, all FP64:
//   k_pg_linearize   two warps per edge (the adjoint beside the logarithm):
//                    e, J_i = -Jr^-1(e) Ad(T_j^-1 T_i),
//                    J_j = Jr^-1(e) (Jr^-1 from its Bernoulli series), and the
//                    blocks J^T Omega J, J^T Omega e, e^T Omega e
//   k_pg_assemble    one warp per factor block: fixed-order sums of the edge
//                    blocks (deterministic, no atomics); g; chi^2
//   k_pg_factor      one launch per tree level, four warps per 7x7 block
//                    column: left-looking updates into the column staged in
//                    shared memory, dense 7x7 Cholesky, off-diagonal triangular
//                    solves, forward substitution (its products formed in
//                    parallel with the updates)
//   k_pg_backsolve   one launch per level, root to leaves, one warp per column
//   k_pg_update      one thread per node: T <- T Exp(delta)
// The trailing dense supernode (the top of the elimination tree):
//   k_pg_sn_assemble      updates of its blocks by the sparse columns
//   k_pg_sn_panel_first   7x7 Cholesky, its inverse and the triangular solves
//                         of its first column
//   k_pg_sn_update_panel  per column: the right-looking update of the
//                         remaining blocks over all SMs, and the next column's
//                         panel in the CTA that completes that column
//   k_pg_sn_rhs           the sparse columns' terms of its right-hand side
//   k_pg_sn_dense_solve   one CTA: forward and back substitution, right-looking
// Adaptive LM (lm_adaptive): k_pg_lm_start, k_pg_backup, k_pg_decide.
#include <algorithm>
#include <cmath>
#include <functional>
#include <map>
#include <queue>
#include <set>
#include <vector>

#include "common.cuh"
#include "sim3_math.cuh"

namespace ec3r {
namespace pg {

constexpr int NB = 49;
constexpr int NBERN = 24;
constexpr int SN_MIN = 8;  // smallest trailing supernode factored right-looking
__constant__ double c_bern[NBERN];  // B_2k / (2k)!, k = 1..24

// --------------------------------------------------------------------------
// device helpers: 7x7 blocks in shared memory, one warp
// --------------------------------------------------------------------------
// C = op(A) op(B) (C distinct from A and B); each lane computes entries lane
// and lane + 32, their FMA chains interleaved.
__device__ __forceinline__ void warp_mm7(const double* A, bool tA, const double* B, bool tB,
                                         double* C, int lane) {
  const int i1 = lane + 32;
  const bool two = i1 < NB;
  const int r0 = lane / 7, c0 = lane % 7;
  const int r1 = two ? i1 / 7 : 0, c1 = two ? i1 % 7 : 0;  // lanes >= 17: a dummy entry
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;  // independent partial sums: short FP64 chains
  double t0 = 0.0, t1 = 0.0, t2 = 0.0;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const double a0 = tA ? A[7 * k + r0] : A[7 * r0 + k];
    const double b0 = tB ? B[7 * c0 + k] : B[7 * k + c0];
    const double a1 = tA ? A[7 * k + r1] : A[7 * r1 + k];
    const double b1 = tB ? B[7 * c1 + k] : B[7 * k + c1];
    if (k % 3 == 0) {
      s0 = fma(a0, b0, s0);
      t0 = fma(a1, b1, t0);
    } else if (k % 3 == 1) {
      s1 = fma(a0, b0, s1);
      t1 = fma(a1, b1, t1);
    } else {
      s2 = fma(a0, b0, s2);
      t2 = fma(a1, b1, t2);
    }
  }
  C[lane] = (s0 + s1) + s2;
  if (two) C[i1] = (t0 + t1) + t2;
  __syncwarp();
}

// Adjoint of T = (s, R, t) in (rho, phi, sigma) coordinates:
// [[sR, t^ R, -t], [0, R, 0], [0, 0, 1]].
__device__ void adjoint7(const s3::Sim3d& T, double* A) {
  for (int i = 0; i < NB; ++i) A[i] = 0.0;
  const double* R = T.R;
  const double* t = T.t;
  const double th[9] = {0.0, -t[2], t[1], t[2], 0.0, -t[0], -t[1], t[0], 0.0};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      A[7 * i + j] = T.s * R[3 * i + j];
      A[7 * (i + 3) + (j + 3)] = R[3 * i + j];
      double v = 0.0;
      for (int k = 0; k < 3; ++k) v += th[3 * i + k] * R[3 * k + j];
      A[7 * i + (j + 3)] = v;
    }
  for (int i = 0; i < 3; ++i) A[7 * i + 6] = -t[i];
  A[48] = 1.0;
}

// ad of xi = (rho, phi, sigma): [[phi^ + sigma I, rho^, -rho], [0, phi^, 0], [0, 0, 0]].
__device__ void small_ad7(const double* xi, double* A) {
  for (int i = 0; i < NB; ++i) A[i] = 0.0;
  const double* r = xi;
  const double* p = xi + 3;
  const double ph[9] = {0.0, -p[2], p[1], p[2], 0.0, -p[0], -p[1], p[0], 0.0};
  const double rh[9] = {0.0, -r[2], r[1], r[2], 0.0, -r[0], -r[1], r[0], 0.0};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      A[7 * i + j] = ph[3 * i + j] + (i == j ? xi[6] : 0.0);
      A[7 * i + j + 3] = rh[3 * i + j];
      A[7 * (i + 3) + j + 3] = ph[3 * i + j];
    }
  for (int i = 0; i < 3; ++i) A[7 * i + 6] = -r[i];
}

__device__ __forceinline__ s3::Sim3d edge_error_T(const s3::Sim3d& Ti, const s3::Sim3d& Tj,
                                                  const s3::Sim3d& Tij) {
  return s3::compose(s3::inverse(Tij), s3::compose(s3::inverse(Ti), Tj));
}

// --------------------------------------------------------------------------
// chaining initialisation: pointer jumping along the spanning tree (one CTA)
// --------------------------------------------------------------------------
// Programmatic dependent launch (PDL): every pose-graph kernel is launched so
// that the next can be scheduled before it finishes.  Each kernel first waits
// for the previous one to complete (its results visible) - before any access
// to data that a launch writes; only the plan's static index arrays may be
// read earlier - and only then lets its own dependent launch, so that at most
// one kernel waits ahead (launched without the attribute, both are no-ops).
__device__ __forceinline__ void pdl_prologue() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__global__ void __launch_bounds__(1024) k_pg_init(int n, int fixed, const int* __restrict__ parent,
                                                  const int* __restrict__ tedge,
                                                  const int* __restrict__ tdir,
                                                  const ec3r_sim3* __restrict__ Tij,
                                                  ec3r_sim3* nodes, ec3r_sim3* W0, ec3r_sim3* W1,
                                                  int* anc0, int* anc1, int rounds) {
  pdl_prologue();
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    s3::Sim3d w;
    int a = -1;
    if (v == fixed) {
      w = s3::load(nodes[v]);
    } else if (parent[v] < 0) {
      w = s3::identity();
    } else {
      const s3::Sim3d M = s3::load(Tij[tedge[v]]);
      w = tdir[v] > 0 ? M : s3::inverse(M);
      a = parent[v];
    }
    s3::store(w, W0[v]);
    anc0[v] = a;
  }
  __syncthreads();
  ec3r_sim3* Ws = W0;
  ec3r_sim3* Wd = W1;
  int* As = anc0;
  int* Ad = anc1;
  for (int r = 0; r < rounds; ++r) {
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
      const int a = As[v];
      if (a >= 0) {
        s3::store(s3::compose(s3::load(Ws[a]), s3::load(Ws[v])), Wd[v]);
        Ad[v] = As[a];
      } else {
        Wd[v] = Ws[v];
        Ad[v] = -1;
      }
    }
    __syncthreads();
    ec3r_sim3* tw = Ws; Ws = Wd; Wd = tw;
    int* ta = As; As = Ad; Ad = ta;
  }
  for (int v = threadIdx.x; v < n; v += blockDim.x)
    if (v != fixed) nodes[v] = Ws[v];
}

// --------------------------------------------------------------------------
// device view of a plan and of one call's data
// --------------------------------------------------------------------------
struct PgDev {
  int n, m, nf, n_blocks, sn0, nlev, n_sn_groups, iters;
  double lambda;
  const int *ei, *ej, *perm, *col_ptr, *off_row, *off_blk, *grp_ptr, *grp, *upd_ab, *sn_grp,
      *row_ptr, *row, *level_ptr, *level_cols, *asm_ptr, *asm_it, *g_ptr, *g_it;
  const int4* col_meta;  // per column in level order: ColMeta as two int4
  const int* grp_slot;   // per update group: its block's slot in the column (0: diagonal)
  double *L, *b, *contrib, *gvec, *chi2e, *idiag, *chi2;
  double* lm;           // adaptive LM: lambda, chi^2 at the step's start, after it (else null)
  ec3r_sim3* backup;    // adaptive LM: poses before the tentative step
  int* fail;
  unsigned* flags;
  const ec3r_sim3* Tij;
  const double* info;
  ec3r_sim3* nodes;
};

// Loads of values written by an earlier launch of the same solve: plain
// coherent loads, never the read-only data path.
__device__ __forceinline__ double ldc(const double* p) { return *p; }
__device__ __forceinline__ int ldc(const int* p) { return *p; }

// The plan's index arrays are written by the host before a call and by no
// kernel, so a launch may touch them before griddepcontrol.wait: it reads its
// column's metadata and prefetches the column's index ranges into L1 there,
// while the launch before it still runs.  Beside HBM-saturating work an L2
// round trip costs several times its unloaded latency, and the factor and
// back-substitution launches, one per tree level, are chains of such trips.
__device__ __forceinline__ void prefetch_bytes(const void* base, size_t bytes, int tid,
                                               int nthreads) {
  const uintptr_t a0 = (uintptr_t)base & ~(uintptr_t)127, a1 = (uintptr_t)base + bytes;
  for (uintptr_t a = a0 + (uintptr_t)tid * 128; a < a1; a += (uintptr_t)nthreads * 128)
    asm volatile("prefetch.global.L1 [%0];" ::"l"(a));
}
__device__ __forceinline__ void prefetch_range(const int* base, int n, int tid, int nthreads) {
  prefetch_bytes(base, sizeof(int) * (size_t)(n > 0 ? n : 0), tid, nthreads);
}

__device__ __forceinline__ s3::Sim3d load_cg(const ec3r_sim3* a) { return s3::load(*a); }

// Shared-memory scratch of one warp.
struct WarpScratch {
  double A[NB], B[NB], C[NB], J[NB], Ji[NB], O[NB], OJ[NB], OJj[NB];
  double e[7], inv[7], y[7];
  int K;
};

// --------------------------------------------------------------------------
// linearisation of one edge (one warp)
// --------------------------------------------------------------------------
// Warp 1 of the edge's CTA: Ad(T_j^-1 T_i) into w.B, independent of the error,
// while warp 0 takes the logarithm; barrier 1 joins the two warps.
__device__ __forceinline__ void pair_barrier() { asm volatile("bar.sync 1, 64;" ::: "memory"); }

__device__ void linearize_adjoint(int e, int lane, WarpScratch& w, const PgDev& p, int jacobians) {
  if (lane == 0 && jacobians) {
    const s3::Sim3d Ti = load_cg(p.nodes + p.ei[e]), Tj = load_cg(p.nodes + p.ej[e]);
    adjoint7(s3::compose(s3::inverse(Tj), Ti), w.B);
  }
  pair_barrier();
}

__device__ void linearize_edge(int e, int lane, WarpScratch& w, const PgDev& p, int jacobians) {
  if (lane == 0) {
    const s3::Sim3d Ti = load_cg(p.nodes + p.ei[e]), Tj = load_cg(p.nodes + p.ej[e]);
    const s3::Sim3d M = s3::load(p.Tij[e]);
    double xi[7];
    s3::log(edge_error_T(Ti, Tj, M), xi);
    for (int k = 0; k < 7; ++k) w.e[k] = xi[k];
    if (jacobians) {
      small_ad7(xi, w.A);                                // ad(e)
      // series length from the spectral radius of ad(e) and the size of rho
      const double nu = sqrt(xi[3] * xi[3] + xi[4] * xi[4] + xi[5] * xi[5] + xi[6] * xi[6]);
      const double rn = 1.0 + fabs(xi[0]) + fabs(xi[1]) + fabs(xi[2]);
      const double q = nu / (2.0 * 3.14159265358979323846);
      int K = 1;
      double qk = q * q;  // q^(2K)
      while (K < NBERN && 4.0 * (K + 1) * rn * qk * q * q > 1e-18) {
        ++K;
        qk *= q * q;
      }
      w.K = K;
    }
  }
  pair_barrier();  // w.e, w.A, w.K (warp 0) and w.B (warp 1)
  double ev[7];
  for (int k = 0; k < 7; ++k) ev[k] = w.e[k];
  // Omega (identity unless given)
  for (int idx = lane; idx < NB; idx += 32)
    w.O[idx] = p.info ? p.info[(size_t)e * NB + idx] : ((idx % 8 == 0) ? 1.0 : 0.0);
  __syncwarp();
  if (lane == 0) {
    double v[7];
    for (int r = 0; r < 7; ++r) {
      double s = 0.0;
      for (int c = 0; c < 7; ++c) s += w.O[7 * r + c] * ev[c];
      v[r] = s;
    }
    double x2 = 0.0;
    for (int r = 0; r < 7; ++r) x2 += ev[r] * v[r];
    p.chi2e[e] = x2;
  }
  if (!jacobians) {
    __syncwarp();
    return;
  }
  // Jr^-1(e) = I + ad/2 + sum_k c_k ad^{2k}; Horner in ad^2
  warp_mm7(w.A, false, w.A, false, w.C, lane);          // C = ad^2
  const int K = w.K;
  for (int idx = lane; idx < NB; idx += 32) w.J[idx] = (idx % 8 == 0) ? c_bern[K - 1] : 0.0;
  __syncwarp();
  for (int k = K - 1; k >= 1; --k) {
    warp_mm7(w.C, false, w.J, false, w.OJ, lane);       // OJ = ad^2 Q
    for (int idx = lane; idx < NB; idx += 32)
      w.J[idx] = w.OJ[idx] + ((idx % 8 == 0) ? c_bern[k - 1] : 0.0);
    __syncwarp();
  }
  warp_mm7(w.C, false, w.J, false, w.OJ, lane);         // OJ = P(ad^2)
  for (int idx = lane; idx < NB; idx += 32)
    w.J[idx] = ((idx % 8 == 0) ? 1.0 : 0.0) + 0.5 * w.A[idx] + w.OJ[idx];  // J = Jr^-1 = J_j
  __syncwarp();
  warp_mm7(w.J, false, w.B, false, w.Ji, lane);         // Jr^-1 Ad
  for (int idx = lane; idx < NB; idx += 32) w.Ji[idx] = -w.Ji[idx];     // J_i
  __syncwarp();
  double* out = p.contrib + (size_t)e * 3 * NB;
  const double* OJi = w.Ji;  // Omega J_i, Omega J_j (Omega = I unless given)
  const double* OJj = w.J;
  if (p.info) {
    warp_mm7(w.O, false, w.Ji, false, w.OJ, lane);
    warp_mm7(w.O, false, w.J, false, w.OJj, lane);
    OJi = w.OJ;
    OJj = w.OJj;
  }
  warp_mm7(w.Ji, true, OJi, false, w.A, lane);          // J_i^T Omega J_i
  warp_mm7(w.J, true, OJj, false, w.B, lane);           // J_j^T Omega J_j
  warp_mm7(w.Ji, true, OJj, false, w.C, lane);          // J_i^T Omega J_j
  for (int idx = lane; idx < NB; idx += 32) {
    out[idx] = w.A[idx];
    out[NB + idx] = w.B[idx];
    out[2 * NB + idx] = w.C[idx];
  }
  // g: J^T Omega e
  if (lane < 14) {
    const int side = lane / 7, r = lane % 7;
    const double* OJ = side == 0 ? OJi : OJj;
    double s = 0.0;
    for (int c = 0; c < 7; ++c) s += OJ[7 * c + r] * ev[c];
    p.gvec[(size_t)e * 14 + lane] = s;
  }
  __syncwarp();
}

// --------------------------------------------------------------------------
// assembly unit b (one warp): a factor block (b < n_blocks), a right-hand
// side block (then nf of them), or chi^2 (the last unit)
// --------------------------------------------------------------------------
__device__ void assemble_unit(int b, int lane, int n_blocks, int nf, const PgDev& p,
                              double* chi2_out, int trial) {
  if (b < n_blocks) {
    const int p0 = p.asm_ptr[b], p1 = p.asm_ptr[b + 1];
    const double lambda = p.lm ? ldc(p.lm) : p.lambda;
    for (int idx = lane; idx < NB; idx += 32) {
      const int r = idx / 7, c = idx % 7;
      double s = (b < nf && r == c) ? lambda : 0.0;
      for (int q = p0; q < p1; ++q) {
        const int it = p.asm_it[q];
        const int edge = it >> 2, kind = it & 3;
        const double* C = p.contrib + (size_t)edge * 3 * NB;
        s += kind == 3 ? ldc(C + 2 * NB + 7 * c + r) : ldc(C + kind * NB + idx);
      }
      p.L[(size_t)b * NB + idx] = s;
    }
  } else if (b < n_blocks + nf) {
    const int k = b - n_blocks;
    if (lane < 7) {
      double s = 0.0;
      for (int q = p.g_ptr[k]; q < p.g_ptr[k + 1]; ++q) {
        const int it = p.g_it[q];
        s += ldc(p.gvec + (size_t)(it >> 1) * 14 + 7 * (it & 1) + lane);
      }
      p.b[7 * k + lane] = -s;
    }
  } else {
    double s = 0.0;
    for (int e = lane; e < p.m; e += 32) s += ldc(p.chi2e + e);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      if (trial) {  // chi^2 after a tentative LM step; the step's fail flag stays
        p.lm[2] = s;
      } else {
        if (chi2_out) *chi2_out = s;
        if (p.lm) p.lm[1] = s;
        *p.fail = 0;
      }
    }
  }
}

// --------------------------------------------------------------------------
// numeric factorisation helpers
// --------------------------------------------------------------------------
// L[dst] -= sum over the group's updates of A B^T for the entries idx of this
// lane; four independent partial sums break the FP64 dependency chain.
__device__ __forceinline__ void apply_group(double* L, int dst, const int* __restrict__ ab, int n,
                                            int lane) {
  double* Dst = L + (size_t)dst * NB;
  for (int idx = lane; idx < NB; idx += 32) {
    const int r = idx / 7, c = idx % 7;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int q = 0; q < n; ++q) {
      const double* A = L + (size_t)ab[2 * q] * NB + 7 * r;
      const double* B = L + (size_t)ab[2 * q + 1] * NB + 7 * c;
      s0 = fma(ldc(A + 0), ldc(B + 0), s0);
      s1 = fma(ldc(A + 1), ldc(B + 1), s1);
      s2 = fma(ldc(A + 2), ldc(B + 2), s2);
      s3 = fma(ldc(A + 3), ldc(B + 3), s3);
      s0 = fma(ldc(A + 4), ldc(B + 4), s0);
      s1 = fma(ldc(A + 5), ldc(B + 5), s1);
      s2 = fma(ldc(A + 6), ldc(B + 6), s2);
    }
    Dst[idx] = ldc(Dst + idx) - ((s0 + s1) + (s2 + s3));
  }
}

// Entry idx of block dst after its group's updates (the arithmetic of
// apply_group), returned instead of stored.
__device__ __forceinline__ double group_entry(const double* L, int dst, const int* __restrict__ ab,
                                              int n, int idx) {
  const int r = idx / 7, c = idx % 7;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (int q = 0; q < n; ++q) {
    const double* A = L + (size_t)ab[2 * q] * NB + 7 * r;
    const double* B = L + (size_t)ab[2 * q + 1] * NB + 7 * c;
    s0 = fma(ldc(A + 0), ldc(B + 0), s0);
    s1 = fma(ldc(A + 1), ldc(B + 1), s1);
    s2 = fma(ldc(A + 2), ldc(B + 2), s2);
    s3 = fma(ldc(A + 3), ldc(B + 3), s3);
    s0 = fma(ldc(A + 4), ldc(B + 4), s0);
    s1 = fma(ldc(A + 5), ldc(B + 5), s1);
    s2 = fma(ldc(A + 6), ldc(B + 6), s2);
  }
  return ldc(L + (size_t)dst * NB + idx) - ((s0 + s1) + (s2 + s3));
}

// Dense 7x7 Cholesky (lower) of the block at Lkk into D (shared), reciprocal
// pivots (through rsqrt) into inv; writes the factor back and the reciprocal
// pivots to id.  One warp.  A non-positive or non-finite pivot raises NOT_SPD.
__device__ void chol7_core(double* Lkk, double* id, double* D, double* inv, int lane,
                           const PgDev& p) {
  bool bad = false;
  for (int c = 0; c < 7; ++c) {
    const double d = D[8 * c];
    if (!(d > 0.0) || !isfinite(d)) bad = true;
    const double ip = rsqrt(fmax(d, 1e-300));
    __syncwarp();
    if (lane == 0) {
      D[8 * c] = d * ip;
      inv[c] = ip;
    }
    if (lane > c && lane < 7) D[7 * lane + c] *= ip;
    __syncwarp();
    for (int idx = lane; idx < NB; idx += 32) {
      const int r = idx / 7, cc = idx % 7;
      if (r > c && cc > c && cc <= r) D[idx] -= D[7 * r + c] * D[7 * cc + c];
    }
    __syncwarp();
  }
  if (bad && lane == 0) {
    atomicOr(p.flags, FLAG_NOT_SPD);
    atomicExch(p.fail, 1);
  }
  for (int idx = lane; idx < NB; idx += 32) {
    if (idx % 7 > idx / 7) D[idx] = 0.0;
    Lkk[idx] = D[idx];
  }
  if (lane < 7) id[lane] = inv[lane];
  __syncwarp();
}

__device__ void chol7(double* Lkk, double* id, double* D, double* inv, int lane, const PgDev& p) {
  for (int idx = lane; idx < NB; idx += 32) D[idx] = ldc(Lkk + idx);
  __syncwarp();
  chol7_core(Lkk, id, D, inv, lane, p);
}

// One row of an off-diagonal block, in place: x <- x Lkk^-T.
__device__ __forceinline__ void row_solve7(double* X, const double* D, const double* inv) {
  double x[7];
  for (int c = 0; c < 7; ++c) {
    double s = ldc(X + c);
    for (int t = 0; t < c; ++t) s -= x[t] * D[7 * c + t];
    x[c] = s * inv[c];
  }
  for (int c = 0; c < 7; ++c) X[c] = x[c];
}

// y <- Lkk^-1 y and x <- Lkk^-T x on 7-vectors in shared memory (one thread).
__device__ __forceinline__ void lower_solve7(double* y, const double* D, const double* inv) {
  for (int c = 0; c < 7; ++c) {
    double s = y[c];
    for (int t = 0; t < c; ++t) s -= D[7 * c + t] * y[t];
    y[c] = s * inv[c];
  }
}
__device__ __forceinline__ void upper_solve7(double* x, const double* D, const double* inv) {
  for (int c = 6; c >= 0; --c) {  // x[c + 1], the latest, enters last: a short chain
    double s = x[c];
    for (int t = 6; t > c; --t) s -= D[7 * t + c] * x[t];
    x[c] = s * inv[c];
  }
}

template <int TW>
__device__ __forceinline__ void team_sync() {
  if constexpr (TW == 1) __syncwarp();
  else __syncthreads();
}

// Column k of the sparse part, by a team of TW warps (tid in [0, 32 TW)):
// left-looking updates (each destination block's group summed in a fixed
// order, so the result does not depend on scheduling), dense 7x7 Cholesky,
// off-diagonal triangular solves, forward substitution
// y_k = Lkk^-1 (b_k - sum_j L_kj y_j) over its descendants j.
template <int TW>
__device__ void factor_column(int k, int tid, double* D, double* inv, double* y, const PgDev& p) {
  const int lane = tid & 31, warp = tid >> 5;
  for (int g = p.grp_ptr[k] + warp; g < p.grp_ptr[k + 1]; g += TW)
    apply_group(p.L, p.grp[3 * g], p.upd_ab + 2 * p.grp[3 * g + 1], p.grp[3 * g + 2], lane);
  team_sync<TW>();
  if (warp == 0) chol7(p.L + (size_t)k * NB, p.idiag + 7 * k, D, inv, lane, p);
  team_sync<TW>();
  const int o0 = p.col_ptr[k], o1 = p.col_ptr[k + 1];
  for (int q = o0 * 7 + tid; q < o1 * 7; q += 32 * TW)
    row_solve7(p.L + (size_t)p.off_blk[q / 7] * NB + 7 * (q % 7), D, inv);
  if (warp == 0) {
    if (lane < 7) {
      double s = ldc(p.b + 7 * k + lane);
      for (int q = p.row_ptr[k]; q < p.row_ptr[k + 1]; ++q) {
        const int j = p.row[2 * q], blk = p.row[2 * q + 1];
        const double* Lkj = p.L + (size_t)blk * NB + 7 * lane;
        for (int t = 0; t < 7; ++t) s -= ldc(Lkj + t) * ldc(p.b + 7 * j + t);
      }
      y[lane] = s;
    }
    __syncwarp();
    if (lane == 0) lower_solve7(y, D, inv);
    __syncwarp();
    if (lane < 7) p.b[7 * k + lane] = y[lane];
  }
  team_sync<TW>();
}

// Back substitution of column k (one warp): x_k = Lkk^-T (y_k - sum_i L_ik^T x_i).
__device__ void backsolve_column(int k, int lane, double* x, const PgDev& p) {
  if (lane < 7) {
    double s0 = ldc(p.b + 7 * k + lane), s1 = 0.0;
    for (int q = p.col_ptr[k]; q < p.col_ptr[k + 1]; ++q) {
      const int i = p.off_row[q];
      const double* Lik = p.L + (size_t)p.off_blk[q] * NB + lane;
      const double* xi = p.b + 7 * i;
      s0 -= ldc(Lik + 0) * ldc(xi + 0) + ldc(Lik + 14) * ldc(xi + 2) +
            ldc(Lik + 28) * ldc(xi + 4) + ldc(Lik + 42) * ldc(xi + 6);
      s1 -= ldc(Lik + 7) * ldc(xi + 1) + ldc(Lik + 21) * ldc(xi + 3) + ldc(Lik + 35) * ldc(xi + 5);
    }
    x[lane] = s0 + s1;
  }
  __syncwarp();
  if (lane == 0) {
    const double* D = p.L + (size_t)k * NB;
    const double* id = p.idiag + 7 * k;
    for (int c = 6; c >= 0; --c) {
      double s = x[c];
      for (int t = c + 1; t < 7; ++t) s -= ldc(D + 7 * t + c) * x[t];
      x[c] = s * ldc(id + c);
    }
  }
  __syncwarp();
  if (lane < 7) p.b[7 * k + lane] = x[lane];
  __syncwarp();
}

__device__ __forceinline__ void update_node(int k, const PgDev& p) {
  double d[7];
  for (int i = 0; i < 7; ++i) d[i] = ldc(p.b + 7 * k + i);
  const int v = p.perm[k];
  s3::store(s3::compose(load_cg(p.nodes + v), s3::exp(d)), p.nodes[v]);
}

// --------------------------------------------------------------------------
// multi-launch schedule: one launch per phase and per tree level
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(64) k_pg_linearize(PgDev p, int jacobians) {
  {  // the edge's static data, before the wait
    const int e = blockIdx.x, t = threadIdx.x;
    prefetch_range(p.ei + e, 1, t, 64);
    prefetch_range(p.ej + e, 1, t, 64);
    prefetch_bytes(p.Tij + e, sizeof(ec3r_sim3), t, 64);
    if (p.info) prefetch_bytes(p.info + (size_t)e * NB, sizeof(double) * NB, t, 64);
  }
  pdl_prologue();
  __shared__ WarpScratch w;
  if (threadIdx.x < 32) linearize_edge(blockIdx.x, threadIdx.x, w, p, jacobians);
  else linearize_adjoint(blockIdx.x, threadIdx.x - 32, w, p, jacobians);
}

__global__ void __launch_bounds__(32) k_pg_assemble(PgDev p, int n_blocks, int nf,
                                                    double* chi2_out, int trial) {
  {  // the unit's static index ranges, before the wait
    const int b = blockIdx.x;
    if (b < n_blocks) {
      const int p0 = p.asm_ptr[b], p1 = p.asm_ptr[b + 1];
      prefetch_range(p.asm_it + p0, p1 - p0, threadIdx.x, 32);
    } else if (b < n_blocks + nf) {
      const int k = b - n_blocks, q0 = p.g_ptr[k], q1 = p.g_ptr[k + 1];
      prefetch_range(p.g_it + q0, q1 - q0, threadIdx.x, 32);
    }
  }
  pdl_prologue();
  assemble_unit(blockIdx.x, threadIdx.x, n_blocks, nf, p, chi2_out, trial);
}

// Adaptive Levenberg-Marquardt (Sec. III-E names LM): the damping starts at
// lambda0; a step is kept when the factorisation succeeded and chi^2 went
// down (lambda / 10), else the poses before it are restored (lambda x 10);
// lambda stays in [LM_MIN, LM_MAX].
constexpr double LM_MIN = 1e-10, LM_MAX = 1e10;

__global__ void k_pg_lm_start(PgDev p, double lambda0) {
  pdl_prologue();
  p.lm[0] = lambda0;
}

__global__ void k_pg_backup(PgDev p) {
  pdl_prologue();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < p.n) p.backup[k] = p.nodes[k];
}

__global__ void k_pg_decide(PgDev p) {
  pdl_prologue();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const bool accept = !ldc(p.fail) && ldc(p.lm + 2) < ldc(p.lm + 1);
  if (!accept && k < p.n) p.nodes[k] = p.backup[k];
  if (k == 0) p.lm[0] = accept ? fmax(ldc(p.lm) * 0.1, LM_MIN) : fmin(ldc(p.lm) * 10.0, LM_MAX);
}

constexpr int FWARPS = 4;   // warps per column in k_pg_factor
constexpr int CB_MAX = 96;  // staged blocks of a column: the diagonal + up to 95 below it
constexpr int FS_MAX = 64;  // staged forward-substitution terms of a column

// Per column (in level order), built on the host: the column, its update
// groups [g0, g1), its off-diagonal blocks [o0, o1), its forward-substitution
// terms [r0, r1), whether the column fits the staged schedule, and the slots
// filled by groups (slot s: bit s % 32 of filled[s / 32]).
struct ColMeta {
  int k, g0, g1, o0, o1, r0, r1, fast;
  unsigned filled[3];
};
constexpr int META_INTS = 12;  // three int4 per column

__device__ __forceinline__ ColMeta load_meta(const int4* m, int pos) {
  const int4 a = m[3 * pos], b = m[3 * pos + 1], c = m[3 * pos + 2];
  return ColMeta{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w,
                 {(unsigned)c.x, (unsigned)c.y, (unsigned)c.z}};
}

// Column c by a CTA of four warps (tid in [0, 128)), staged schedule (a
// column with at most 95 blocks below the diagonal and 64 forward-substitution
// terms), every dependent step spread over the team:
//   1. the column's blocks enter shared memory, either as stored or through
//      their update group (left-looking, group_entry); the products
//      L_kj y_j of the forward substitution are formed meanwhile, one row of
//      one term per thread;
//   2. warp 0 factors the diagonal block; warp 1 sums b_k - sum_j L_kj y_j;
//   3. warps 0..2 solve the rows of the off-diagonal blocks, warp 3 the
//      diagonal system of the forward substitution.
__device__ void factor_staged(const ColMeta& c, int tid, double* CB, double* fpart, double* inv,
                              double* y, const PgDev& p) {
  const int lane = tid & 31, warp = tid >> 5;
  const int k = c.k;
  const int nblk = c.o1 - c.o0, nrow = c.r1 - c.r0;
  for (int it = tid; it < (1 + nblk) * NB; it += 32 * FWARPS) {
    const int sl = it / NB;
    if ((c.filled[sl >> 5] >> (sl & 31)) & 1u) continue;
    const int blk = sl == 0 ? k : p.off_blk[c.o0 + sl - 1];
    CB[it] = ldc(p.L + (size_t)blk * NB + it % NB);
  }
  for (int it = tid; it < (c.g1 - c.g0) * NB; it += 32 * FWARPS) {
    const int g = c.g0 + it / NB, idx = it % NB;
    CB[p.grp_slot[g] * NB + idx] =
        group_entry(p.L, p.grp[3 * g], p.upd_ab + 2 * p.grp[3 * g + 1], p.grp[3 * g + 2], idx);
  }
  for (int it = tid; it < nrow * 7; it += 32 * FWARPS) {
    const int q = c.r0 + it / 7, r = it % 7;
    const double* Lkj = p.L + (size_t)p.row[2 * q + 1] * NB + 7 * r;
    const double* yj = p.b + 7 * p.row[2 * q];
    double s0 = ldc(Lkj) * ldc(yj), s1 = ldc(Lkj + 1) * ldc(yj + 1);
    double s2 = ldc(Lkj + 2) * ldc(yj + 2);
    s0 = fma(ldc(Lkj + 3), ldc(yj + 3), s0);
    s1 = fma(ldc(Lkj + 4), ldc(yj + 4), s1);
    s2 = fma(ldc(Lkj + 5), ldc(yj + 5), s2);
    s0 = fma(ldc(Lkj + 6), ldc(yj + 6), s0);
    fpart[it] = (s0 + s1) + s2;
  }
  if (tid >= 32 && tid < 39) y[tid - 32] = ldc(p.b + 7 * k + tid - 32);
  __syncthreads();
  if (warp == 0) {
    chol7_core(p.L + (size_t)k * NB, p.idiag + 7 * k, CB, inv, lane, p);
  } else if (warp == 1 && lane < 7) {
    double s = y[lane];
    for (int q = 0; q < nrow; ++q) s -= fpart[7 * q + lane];
    y[lane] = s;
  }
  __syncthreads();
  if (warp == FWARPS - 1) {
    if (lane == 0) lower_solve7(y, CB, inv);
    __syncwarp();
    if (lane < 7) p.b[7 * k + lane] = y[lane];
  } else {
    for (int it = tid; it < nblk * 7; it += 32 * (FWARPS - 1)) {
      const int sl = 1 + it / 7, r = it % 7;
      const double* X = CB + sl * NB + 7 * r;
      double x[7];
      for (int cc = 0; cc < 7; ++cc) {
        double v = X[cc];
        for (int t = 0; t < cc; ++t) v -= x[t] * CB[7 * cc + t];
        x[cc] = v * inv[cc];
      }
      double* out = p.L + (size_t)p.off_blk[c.o0 + sl - 1] * NB + 7 * r;
      for (int cc = 0; cc < 7; ++cc) out[cc] = x[cc];
    }
  }
}

// One column per CTA: the staged schedule, else factor_column.
__global__ void __launch_bounds__(32 * FWARPS) k_pg_factor(PgDev p, int lstart) {
  __shared__ double CB[CB_MAX * NB], fpart[FS_MAX * 7], inv[7], y[7];
  const ColMeta c = load_meta(p.col_meta, lstart + blockIdx.x);  // static: before the wait
  if (c.fast) {
    const int t = threadIdx.x, nt = blockDim.x;
    prefetch_range(p.off_blk + c.o0, c.o1 - c.o0, t, nt);
    prefetch_range(p.grp + 3 * c.g0, 3 * (c.g1 - c.g0), t, nt);
    prefetch_range(p.grp_slot + c.g0, c.g1 - c.g0, t, nt);
    prefetch_range(p.row + 2 * c.r0, 2 * (c.r1 - c.r0), t, nt);
  }
  pdl_prologue();
  if (c.fast) factor_staged(c, threadIdx.x, CB, fpart, inv, y, p);
  else factor_column<FWARPS>(c.k, threadIdx.x, CB, inv, y, p);
}

constexpr int BS_MAX = 64;  // staged back-substitution terms of a column (x 7 rows)

// Column c by one warp: x_k = Lkk^-T (y_k - sum_i L_ik^T x_i).  The terms
// L_ik^T x_i (one row of one block per lane) are formed in parallel while the
// diagonal block is staged; a column with more than BS_MAX blocks below the
// diagonal takes backsolve_column.
__device__ void backsolve_staged(const ColMeta& c, int lane, double* D, double* part, double* id,
                                 double* x, const PgDev& p) {
  const int k = c.k, nblk = c.o1 - c.o0;
  if (nblk > BS_MAX) {
    backsolve_column(k, lane, x, p);
    return;
  }
  for (int it = lane; it < nblk * 7; it += 32) {
    const int q = c.o0 + it / 7, r = it % 7;
    const double* Lik = p.L + (size_t)p.off_blk[q] * NB + r;
    const double* xi = p.b + 7 * p.off_row[q];
    double s0 = ldc(Lik) * ldc(xi), s1 = ldc(Lik + 7) * ldc(xi + 1);
    double s2 = ldc(Lik + 14) * ldc(xi + 2);
    s0 = fma(ldc(Lik + 21), ldc(xi + 3), s0);
    s1 = fma(ldc(Lik + 28), ldc(xi + 4), s1);
    s2 = fma(ldc(Lik + 35), ldc(xi + 5), s2);
    s0 = fma(ldc(Lik + 42), ldc(xi + 6), s0);
    part[it] = (s0 + s1) + s2;
  }
  for (int idx = lane; idx < NB; idx += 32) D[idx] = ldc(p.L + (size_t)k * NB + idx);
  if (lane < 7) {
    id[lane] = ldc(p.idiag + 7 * k + lane);
    x[lane] = ldc(p.b + 7 * k + lane);
  }
  __syncwarp();
  if (lane < 7) {
    double s = x[lane];
    for (int q = 0; q < nblk; ++q) s -= part[7 * q + lane];
    x[lane] = s;
  }
  __syncwarp();
  if (lane == 0) upper_solve7(x, D, id);
  __syncwarp();
  if (lane < 7) p.b[7 * k + lane] = x[lane];
  __syncwarp();
}

struct WarpSolve {
  double D[NB], part[BS_MAX * 7], id[7], x[7];
};

// One column per warp (one warp per CTA).
__global__ void __launch_bounds__(32) k_pg_backsolve(PgDev p, int lstart) {
  __shared__ WarpSolve w;
  const ColMeta c = load_meta(p.col_meta, lstart + blockIdx.x);  // static: before the wait
  prefetch_range(p.off_blk + c.o0, c.o1 - c.o0, threadIdx.x, 32);
  prefetch_range(p.off_row + c.o0, c.o1 - c.o0, threadIdx.x, 32);
  pdl_prologue();
  backsolve_staged(c, threadIdx.x, w.D, w.part, w.id, w.x, p);
}

__global__ void k_pg_update(PgDev p) {
  pdl_prologue();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= p.nf || ldc(p.fail)) return;
  update_node(k, p);
}

// --------------------------------------------------------------------------
// trailing dense supernode (the last ns columns, whose factor columns are full)
// --------------------------------------------------------------------------
// Updates of the supernode's blocks by the sparse columns below it: one warp
// per destination block.
__global__ void __launch_bounds__(32) k_pg_sn_assemble(const int* __restrict__ grp,
                                                       const int* __restrict__ upd_ab, double* L) {
  pdl_prologue();
  const int g = blockIdx.x;
  apply_group(L, grp[3 * g], upd_ab + 2 * grp[3 * g + 1], grp[3 * g + 2], threadIdx.x);
}

__device__ __forceinline__ int sn_block(const int* col_ptr, const int* off_blk, int i, int j) {
  return i == j ? j : off_blk[col_ptr[j] + (i - j - 1)];
}

// Panel work of supernode column k by a CTA of SN_UPD_THREADS threads: 7x7
// Cholesky of the diagonal block and its inverse (warp 0; lane j forms column
// j of L_kk^-1 by forward substitution, kept for the dense substitution too),
// then X = A L_kk^-T for every block below it, one block row per thread: seven
// independent dot products with the inverse instead of a chain of seven
// dependent steps.  The column was written by other CTAs of the same launch:
// its loads bypass L1.
constexpr int SN_UPD_THREADS = 256;
__device__ void sn_panel_cta(int k, int sn0, int nf, const int* __restrict__ col_ptr,
                             const int* __restrict__ off_blk, double* L, double* idiag,
                             double* linv, unsigned* flags, int* fail, double* D, double* inv,
                             double* Li) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* Lkk = L + (size_t)k * NB;
  if (warp == 0) {
    for (int idx = lane; idx < NB; idx += 32) D[idx] = __ldcg(Lkk + idx);
    __syncwarp();
    bool bad = false;
    for (int c = 0; c < 7; ++c) {
      const double d = D[8 * c];
      if (!(d > 0.0) || !isfinite(d)) bad = true;
      const double ip = rsqrt(fmax(d, 1e-300));
      __syncwarp();
      if (lane == 0) {
        D[8 * c] = d * ip;
        inv[c] = ip;
      }
      if (lane > c && lane < 7) D[7 * lane + c] *= ip;
      __syncwarp();
      for (int idx = lane; idx < NB; idx += 32) {
        const int r = idx / 7, cc = idx % 7;
        if (r > c && cc > c && cc <= r) D[idx] -= D[7 * r + c] * D[7 * cc + c];
      }
      __syncwarp();
    }
    if (bad && lane == 0) {
      atomicOr(flags, FLAG_NOT_SPD);
      atomicExch(fail, 1);
    }
    for (int idx = lane; idx < NB; idx += 32) Lkk[idx] = (idx % 7 <= idx / 7) ? D[idx] : 0.0;
    if (lane < 7) {
      idiag[7 * k + lane] = inv[lane];
      const int j = lane;  // column j of L^-1: L z = e_j
      double z[7];
#pragma unroll
      for (int r = 0; r < 7; ++r) {
        double v = r == j ? 1.0 : 0.0;
#pragma unroll
        for (int t = 0; t < r; ++t) v -= D[7 * r + t] * z[t];
        z[r] = r < j ? 0.0 : v * inv[r];
      }
      double* Lg = linv + (size_t)(k - sn0) * NB;
#pragma unroll
      for (int r = 0; r < 7; ++r) {
        Li[7 * r + j] = z[r];
        Lg[7 * r + j] = z[r];
      }
    }
  }
  __syncthreads();
  const int nrows = (nf - 1 - k) * 7;
  for (int q = threadIdx.x; q < nrows; q += SN_UPD_THREADS) {
    double* X = L + (size_t)off_blk[col_ptr[k] + q / 7] * NB + 7 * (q % 7);
    double v[7];
#pragma unroll
    for (int t = 0; t < 7; ++t) v[t] = __ldcg(X + t);
#pragma unroll
    for (int c = 0; c < 7; ++c) {
      double x = 0.0;
#pragma unroll
      for (int t = 0; t <= c; ++t) x = fma(Li[7 * c + t], v[t], x);
      X[c] = x;
    }
  }
}

// First panel of the supernode.
__global__ void __launch_bounds__(SN_UPD_THREADS) k_pg_sn_panel_first(
    int k, int nf, const int* __restrict__ col_ptr, const int* __restrict__ off_blk, double* L,
    double* idiag, double* linv, unsigned* flags, int* fail) {
  pdl_prologue();
  __shared__ double D[NB], inv[7], Li[NB];
  sn_panel_cta(k, k, nf, col_ptr, off_blk, L, idiag, linv, flags, fail, D, inv, Li);
}

// Trailing update after panel k, L_ij -= L_ik L_jk^T for k < j <= i < nf (one
// warp per block, blocks numbered column by column so that column k + 1 comes
// first), fused with panel k + 1: every CTA adds the number of its blocks in
// column k + 1 to cnt[k] after a fence; the CTA that completes the count (all
// of column k + 1 updated) factors column k + 1 while the later columns are
// still being updated.  No CTA waits on another.
__global__ void __launch_bounds__(SN_UPD_THREADS) k_pg_sn_update_panel(
    int k, int sn0, int nf, const int* __restrict__ col_ptr, const int* __restrict__ off_blk,
    double* L, double* idiag, double* linv, unsigned* flags, int* fail, int* cnt) {
  pdl_prologue();
  __shared__ double D[NB], inv[7], Li[NB];
  __shared__ int mine, last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mrem = nf - 1 - k;
  const int64_t nblk = (int64_t)mrem * (mrem + 1) / 2;
  const int64_t t = (int64_t)blockIdx.x * (SN_UPD_THREADS / 32) + warp;
  if (threadIdx.x == 0) mine = 0;
  __syncthreads();
  if (t < nblk) {
    // column jj holds mrem - jj blocks and starts at off(jj) = jj (2 mrem - jj + 1) / 2
    auto off = [mrem](int64_t c) { return c * (2 * (int64_t)mrem - c + 1) / 2; };
    const float b2 = 2.f * (float)mrem + 1.f;
    int jj = (int)((b2 - sqrtf(fmaxf(b2 * b2 - 8.f * (float)t, 0.f))) * 0.5f);
    jj = min(max(jj, 0), mrem - 1);
    while (jj + 1 < mrem && off(jj + 1) <= t) ++jj;
    while (jj > 0 && off(jj) > t) --jj;
    const int ii = jj + (int)(t - off(jj));
    const int i = k + 1 + ii, j = k + 1 + jj;
    double* Dst = L + (size_t)sn_block(col_ptr, off_blk, i, j) * NB;
    const double* A = L + (size_t)off_blk[col_ptr[k] + (i - k - 1)] * NB;
    const double* B = L + (size_t)off_blk[col_ptr[k] + (j - k - 1)] * NB;
    for (int idx = lane; idx < NB; idx += 32) {
      const int r = idx / 7, c = idx % 7;
      double s0 = 0.0, s1 = 0.0;
      s0 = fma(ldc(A + 7 * r + 0), ldc(B + 7 * c + 0), s0);
      s1 = fma(ldc(A + 7 * r + 1), ldc(B + 7 * c + 1), s1);
      s0 = fma(ldc(A + 7 * r + 2), ldc(B + 7 * c + 2), s0);
      s1 = fma(ldc(A + 7 * r + 3), ldc(B + 7 * c + 3), s1);
      s0 = fma(ldc(A + 7 * r + 4), ldc(B + 7 * c + 4), s0);
      s1 = fma(ldc(A + 7 * r + 5), ldc(B + 7 * c + 5), s1);
      s0 = fma(ldc(A + 7 * r + 6), ldc(B + 7 * c + 6), s0);
      Dst[idx] = ldc(Dst + idx) - (s0 + s1);
    }
    if (jj == 0 && lane == 0) atomicAdd(&mine, 1);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    last = 0;
    if (mine > 0) last = atomicAdd(cnt + k, mine) + mine == mrem;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  sn_panel_cta(k + 1, sn0, nf, col_ptr, off_blk, L, idiag, linv, flags, fail, D, inv, Li);
}

// Right-hand side of the supernode's forward substitution: b_k -= sum_j
// L_kj y_j over the sparse columns j < sn0 (final once the levels are done),
// one warp per supernode column k (lanes over terms, fixed shuffle tree).
__global__ void __launch_bounds__(32) k_pg_sn_rhs(int sn0, const int* __restrict__ row_ptr,
                                                  const int* __restrict__ row_it,
                                                  const double* __restrict__ L, double* bvec) {
  pdl_prologue();
  const int k = sn0 + blockIdx.x, lane = threadIdx.x;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int p = row_ptr[k] + lane; p < row_ptr[k + 1]; p += 32) {
    const int j = row_it[2 * p];
    if (j >= sn0) continue;  // supernode columns: right-looking in k_pg_sn_dense_forward
    const double* Lkj = L + (size_t)row_it[2 * p + 1] * NB;
    const double* yj = bvec + 7 * j;
    double yv[7];
    for (int t = 0; t < 7; ++t) yv[t] = ldc(yj + t);
    for (int r = 0; r < 7; ++r)
      for (int t = 0; t < 7; ++t) acc[r] = fma(ldc(Lkj + 7 * r + t), yv[t], acc[r]);
  }
  for (int r = 0; r < 7; ++r)
    for (int o = 16; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
  if (lane < 7) {
    double a = acc[0];
    for (int r = 1; r < 7; ++r) a = lane == r ? acc[r] : a;
    bvec[7 * k + lane] -= a;
  }
}

constexpr int SN_THREADS = 512;

// Dense forward and back substitution over the supernode (one CTA,
// right-looking, the supernode's right-hand side in shared memory):
//   forward, k ascending:  y_k = Lkk^-1 b_k, then b_i -= L_ik y_k for i > k;
//   backward, k descending: x_k = Lkk^-T y_k, then y_i -= L_ki^T x_k for i < k.
// The inverses of the diagonal blocks come from the factorisation, so each
// diagonal solve is seven independent dot products (lanes 0-6); one thread per
// row of each update; the next inverse is staged while the current update runs.
__device__ __forceinline__ void sn_stage_inv(int s, const double* linv, double* Li, int tid) {
  if (tid < NB) Li[tid] = ldc(linv + (size_t)s * NB + tid);
}

__global__ void __launch_bounds__(SN_THREADS) k_pg_sn_dense_solve(int sn0, int nf,
                                                                 const int* __restrict__ col_ptr,
                                                                 const int* __restrict__ off_blk,
                                                                 const double* __restrict__ L,
                                                                 const double* __restrict__ linv,
                                                                 double* bvec) {
  pdl_prologue();
  extern __shared__ double sn_b[];  // [ns * 7]
  __shared__ double Li[2][NB], v[7];
  const int ns = nf - sn0, tid = threadIdx.x;
  for (int i = tid; i < ns * 7; i += SN_THREADS) sn_b[i] = ldc(bvec + 7 * sn0 + i);
  sn_stage_inv(0, linv, Li[0], tid);
  __syncthreads();
  // forward
  for (int k = 0; k < ns; ++k) {
    const int cur = k & 1;
    if (tid < 7) {
      double y = 0.0;
#pragma unroll
      for (int t = 0; t < 7; ++t)
        if (t <= tid) y = fma(Li[cur][7 * tid + t], sn_b[7 * k + t], y);
      v[tid] = y;
    } else if (tid >= 32 && k + 1 < ns) {
      sn_stage_inv(k + 1, linv, Li[cur ^ 1], tid - 32);
    }
    __syncthreads();
    if (tid < 7) sn_b[7 * k + tid] = v[tid];
    const int kk = sn0 + k;
    for (int it = tid; it < (ns - 1 - k) * 7; it += SN_THREADS) {
      const int i = k + 1 + it / 7, r = it % 7;
      const double* Lik = L + (size_t)off_blk[col_ptr[kk] + (i - k - 1)] * NB + 7 * r;
      double s0 = ldc(Lik) * v[0], s1 = ldc(Lik + 1) * v[1], s2 = ldc(Lik + 2) * v[2];
      s0 = fma(ldc(Lik + 3), v[3], s0);
      s1 = fma(ldc(Lik + 4), v[4], s1);
      s2 = fma(ldc(Lik + 5), v[5], s2);
      s0 = fma(ldc(Lik + 6), v[6], s0);
      sn_b[7 * i + r] -= (s0 + s1) + s2;
    }
    __syncthreads();
  }
  // backward (the last inverse is staged: ns - 1 has parity (ns - 1) & 1)
  for (int k = ns - 1; k >= 0; --k) {
    const int cur = k & 1;
    if (tid < 7) {
      double x = 0.0;
#pragma unroll
      for (int t = 0; t < 7; ++t)
        if (t >= tid) x = fma(Li[cur][7 * t + tid], sn_b[7 * k + t], x);
      v[tid] = x;
    } else if (tid >= 32 && k > 0) {
      sn_stage_inv(k - 1, linv, Li[cur ^ 1], tid - 32);
    }
    __syncthreads();
    if (tid < 7) sn_b[7 * k + tid] = v[tid];
    for (int it = tid; it < k * 7; it += SN_THREADS) {
      const int i = it / 7, r = it % 7;  // block (k, i) of column i, its column r
      const double* Lki = L + (size_t)off_blk[col_ptr[sn0 + i] + (k - i - 1)] * NB + r;
      double s0 = ldc(Lki) * v[0], s1 = ldc(Lki + 7) * v[1], s2 = ldc(Lki + 14) * v[2];
      s0 = fma(ldc(Lki + 21), v[3], s0);
      s1 = fma(ldc(Lki + 28), v[4], s1);
      s2 = fma(ldc(Lki + 35), v[5], s2);
      s0 = fma(ldc(Lki + 42), v[6], s0);
      sn_b[7 * i + r] -= (s0 + s1) + s2;
    }
    __syncthreads();
  }
  for (int i = tid; i < ns * 7; i += SN_THREADS) bvec[7 * sn0 + i] = sn_b[i];
}

// Largest supernode: its right-hand side (7 doubles per column) stays in
// shared memory during the substitution.
constexpr int SN_DENSE_MAX = 3200;  // 3200 x 7 doubles = 175 KB


// --------------------------------------------------------------------------
// host: planning
// --------------------------------------------------------------------------
struct Plan : Extension {
  int n = 0, m = 0, fixed = 0, nf = 0, n_blocks = 0, rounds = 0;
  std::vector<int> level_ptr;   // columns of level l: level_cols[level_ptr[l] .. level_ptr[l+1])
  std::vector<void*> allocs;
  int *d_ei = nullptr, *d_ej = nullptr, *d_perm = nullptr;
  int *d_col_ptr = nullptr, *d_off_row = nullptr, *d_off_blk = nullptr;
  int *d_grp_ptr = nullptr, *d_grp = nullptr, *d_upd_ab = nullptr, *d_sn_grp = nullptr;
  int sn0 = 0, n_sn_groups = 0;  // columns >= sn0 form the dense trailing supernode
  int ordering = 0;              // 0 nested dissection, 1 minimum degree
  int *d_row_ptr = nullptr, *d_row = nullptr;
  int *d_level_cols = nullptr, *d_level_ptr = nullptr, *d_asm_ptr = nullptr, *d_asm = nullptr;
  int *d_col_meta = nullptr, *d_grp_slot = nullptr;
  int* d_sn_cnt = nullptr;       // per supernode column: its blocks updated so far
  double* d_sn_linv = nullptr;   // per supernode column: L_kk^-1 (7 x 7)
  int nlev = 0;
  int *d_g_ptr = nullptr, *d_g = nullptr;
  int *d_parent = nullptr, *d_tedge = nullptr, *d_tdir = nullptr;
  int *d_anc0 = nullptr, *d_anc1 = nullptr, *d_fail = nullptr;
  double *d_L = nullptr, *d_b = nullptr, *d_contrib = nullptr, *d_gvec = nullptr,
         *d_chi2e = nullptr, *d_idiag = nullptr;
  ec3r_sim3 *d_W0 = nullptr, *d_W1 = nullptr, *d_backup = nullptr;
  double* d_lm = nullptr;      // adaptive LM state
  unsigned* d_lm_flags = nullptr;  // absorbs non-SPD reports of rejected LM steps
  ~Plan() override {
    for (void* p : allocs) cudaFree(p);
  }
};

template <typename T>
static cudaError_t upload(Plan& P, T** dst, const std::vector<T>& v) {
  const size_t bytes = sizeof(T) * std::max<size_t>(v.size(), 1);
  cudaError_t e = cudaMalloc((void**)dst, bytes);
  if (e != cudaSuccess) return e;
  P.allocs.push_back(*dst);
  if (!v.empty()) e = cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
  return e;
}

template <typename T>
static cudaError_t alloc(Plan& P, T** dst, size_t count) {
  cudaError_t e = cudaMalloc((void**)dst, sizeof(T) * std::max<size_t>(count, 1));
  if (e == cudaSuccess) P.allocs.push_back(*dst);
  return e;
}

// Nested dissection on the node order: split a set at its median node and
// move one endpoint of every edge crossing the split into the separator.
static void nested_dissection(std::vector<int> S, const std::vector<std::set<int>>& adj,
                              std::vector<int>& order) {
  if (S.size() <= 3) {
    std::sort(S.begin(), S.end());
    for (int v : S) order.push_back(v);
    return;
  }
  std::sort(S.begin(), S.end());
  const int mid = S[S.size() / 2];
  std::set<int> inS(S.begin(), S.end()), sep;
  sep.insert(mid);
  for (int a : S) {
    if (a >= mid) break;
    for (int b : adj[a])
      if (b > mid && inS.count(b) && !sep.count(a) && !sep.count(b)) sep.insert(b);
  }
  std::vector<int> A, B;
  for (int v : S) {
    if (sep.count(v)) continue;
    (v < mid ? A : B).push_back(v);
  }
  nested_dissection(A, adj, order);
  nested_dissection(B, adj, order);
  for (int v : sep) order.push_back(v);
}

// Minimum degree on the exact elimination graph: repeatedly eliminate the node
// of fewest neighbours (ties by index), joining its neighbours into a clique.
// Fewer fill blocks than nested dissection on graphs with many long loops, but
// on a chain it eliminates from the ends inward (a deep elimination tree).
static void minimum_degree(const std::vector<int>& freev, const std::vector<std::set<int>>& adj,
                           std::vector<int>& order) {
  const int n = (int)adj.size();
  std::vector<std::set<int>> G(n);
  std::vector<char> gone(n, 1);
  using Item = std::pair<int, int>;
  std::priority_queue<Item, std::vector<Item>, std::greater<Item>> pq;
  for (int v : freev) {
    G[v] = adj[v];
    gone[v] = 0;
    pq.push({(int)G[v].size(), v});
  }
  while (!pq.empty()) {
    const auto [d, v] = pq.top();
    pq.pop();
    if (gone[v] || d != (int)G[v].size()) continue;  // stale entry
    gone[v] = 1;
    order.push_back(v);
    const std::vector<int> nb(G[v].begin(), G[v].end());
    for (int a : nb) {
      G[a].erase(v);
      for (int b : nb)
        if (b != a) G[a].insert(b);
      pq.push({(int)G[a].size(), a});
    }
    G[v].clear();
  }
}

// Symbolic factorisation of one elimination order: the block structure of
// every factor column, the elimination tree, the trailing dense supernode and
// an estimate of the numeric cost per Gauss-Newton iteration.
struct Symbolic {
  std::vector<int> perm, inew, parent;
  std::vector<std::vector<int>> children;
  std::vector<std::set<int>> st;
  int sn0 = 0, nlev = 0;
  double pairs = 0.0, cost = 0.0;
};

static void symbolic(const std::vector<std::set<int>>& adj, Symbolic& S) {
  const int nf = (int)S.perm.size();
  S.inew.assign(adj.size(), -1);
  for (int k = 0; k < nf; ++k) S.inew[S.perm[k]] = k;
  S.children.assign(nf, {});
  S.st.assign(nf, {});
  S.parent.assign(nf, -1);
  for (int k = 0; k < nf; ++k) {
    for (int u : adj[S.perm[k]]) {
      const int q = S.inew[u];
      if (q > k) S.st[k].insert(q);
    }
    for (int c : S.children[k])
      for (int q : S.st[c])
        if (q > k) S.st[k].insert(q);
    if (!S.st[k].empty()) {
      S.parent[k] = *S.st[k].begin();
      S.children[S.parent[k]].push_back(k);
    }
  }
}

// Cost model of one Gauss-Newton iteration (seconds), from measurements on
// this GPU: a sparse tree level costs a factor and a back-substitution launch
// (about 22 us together) plus its heaviest column's left-looking updates at
// one SM's FP64 rate; a supernode column costs about 25 us (its update and
// panel launch, its share of the two substitutions) plus the dense updates
// at the whole GPU's FP64 rate.  A 7x7 block product is 686 FLOP.
constexpr double LEVEL_S = 22e-6, SN_COL_S = 25e-6;
constexpr double SM_FP64 = 6.3e9, GPU_FP64 = 148 * 6.3e9, BLOCK_FLOP = 686.0;

// Per level l < n_levels (columns k < k_end at level lv[k]): LEVEL_S plus the
// block products that update its heaviest column (sum over the descendants j
// of column k of the entries of st[j] at or after k).
static std::vector<double> level_times(const Symbolic& S, const std::vector<int>& lv,
                                       int n_levels, int k_end = -1) {
  const int nf = (int)S.perm.size();
  if (k_end < 0) k_end = nf;
  std::vector<double> work(nf, 0.0);
  for (int j = 0; j < nf; ++j) {
    int idx = 0;
    const int len = (int)S.st[j].size();
    for (int k : S.st[j]) work[k] += (double)(len - idx++);  // entries of st[j] >= k
  }
  std::vector<double> worst(std::max(n_levels, 0), 0.0), t(std::max(n_levels, 0), 0.0);
  std::vector<char> any(std::max(n_levels, 0), 0);
  for (int k = 0; k < k_end; ++k) {
    worst[lv[k]] = std::max(worst[lv[k]], work[k]);
    any[lv[k]] = 1;
  }
  for (int l = 0; l < n_levels; ++l)
    t[l] = any[l] ? LEVEL_S + worst[l] * BLOCK_FLOP / SM_FP64 : 0.0;
  return t;
}

static double sn_time(int n) {
  const double d = (double)n;
  return n <= 0 ? 0.0 : SN_COL_S * d + d * d * d / 6.0 * BLOCK_FLOP / GPU_FP64;
}

static Symbolic analyse(const std::vector<int>& order, const std::vector<std::set<int>>& adj) {
  Symbolic S;
  S.perm = order;
  symbolic(adj, S);
  const int nf = (int)S.perm.size();
  // Columns at the top of the elimination tree that are alone in their level
  // form a chain that would be factored one launch at a time.  They are moved
  // to the end of the order (eliminating these separator-like nodes last adds
  // no fill elsewhere) and, with the root clique, become one dense supernode
  // (explicit zero fill) factored right-looking across many warps.
  {
    std::vector<int> lv(nf, 0), cnt(nf + 1, 0);
    for (int k = 0; k < nf; ++k)
      for (int c : S.children[k]) lv[k] = std::max(lv[k], lv[c] + 1);
    for (int k = 0; k < nf; ++k) cnt[lv[k]]++;
    std::vector<int> chain, rest;
    for (int k = 0; k < nf; ++k) (cnt[lv[k]] == 1 ? chain : rest).push_back(k);
    if ((int)chain.size() >= SN_MIN) {
      if (chain.front() != nf - (int)chain.size()) {
        std::vector<int> np;
        for (int k : rest) np.push_back(S.perm[k]);
        for (int k : chain) np.push_back(S.perm[k]);
        S.perm = np;
        symbolic(adj, S);
      }
      for (int k = nf - (int)chain.size(); k < nf; ++k) {
        S.st[k].clear();
        for (int q = k + 1; q < nf; ++q) S.st[k].insert(q);
      }
    }
  }
  // Likewise the top of the tree from a cut level on, when the cost model
  // below prefers it: a narrow level runs on a few CTAs, its (possibly large)
  // left-looking updates at one SM's FP64 rate, while as supernode columns
  // the updates spread over every SM.  The set is closed under parents, so
  // moving it last (in its own order) adds no fill: a column adjacent to one
  // of its columns later in the order is its ancestor.
  {
    std::vector<int> lv(nf, 0);
    int top = -1;
    for (int k = 0; k < nf; ++k) {
      for (int c : S.children[k]) lv[k] = std::max(lv[k], lv[c] + 1);
      top = std::max(top, lv[k]);
    }
    const std::vector<double> ltime = level_times(S, lv, top + 1);
    // the columns already dense at the end (from the rule above) stay there
    int s_old = nf;
    for (int k = nf - 1; k >= 0; --k) {
      if ((int)S.st[k].size() != nf - 1 - k) break;
      s_old = k;
    }
    std::vector<int> cnt_below(top + 2, 0);  // columns of level l below s_old
    for (int k = 0; k < s_old; ++k) cnt_below[lv[k]]++;
    double best = 1e300;
    int cut = top + 1;
    int n_up = nf - s_old;
    double sparse = 0.0;
    for (int l = 0; l <= top; ++l) sparse += cnt_below[l] > 0 ? ltime[l] : 0.0;
    for (int L = top + 1; L >= 0; --L) {
      if (L <= top) {  // level L joins the supernode
        sparse -= cnt_below[L] > 0 ? ltime[L] : 0.0;
        n_up += cnt_below[L];
      }
      const double c = sparse + sn_time(n_up);
      if (c < best - 1e-12) {
        best = c;
        cut = L;
      }
    }
    std::vector<int> upper, rest;
    for (int k = 0; k < nf; ++k) (k >= s_old || lv[k] >= cut ? upper : rest).push_back(k);
    if ((int)upper.size() >= SN_MIN && (int)upper.size() > nf - s_old) {
      std::vector<int> np;
      for (int k : rest) np.push_back(S.perm[k]);
      for (int k : upper) np.push_back(S.perm[k]);
      S.perm = np;
      symbolic(adj, S);
      for (int k = nf - (int)upper.size(); k < nf; ++k) {
        S.st[k].clear();
        for (int q = k + 1; q < nf; ++q) S.st[k].insert(q);
      }
    }
  }
  // trailing dense supernode: the longest suffix of columns whose structure is
  // every later column
  int s0 = nf;
  for (int k = nf - 1; k >= 0; --k) {
    if ((int)S.st[k].size() != nf - 1 - k) break;
    s0 = k;
  }
  S.sn0 = (nf - s0 >= SN_MIN) ? s0 : nf;
  std::vector<int> level(nf, 0);
  for (int k = 0; k < S.sn0; ++k) {
    for (int c : S.children[k]) level[k] = std::max(level[k], level[c] + 1);
    S.nlev = std::max(S.nlev, level[k] + 1);
  }
  for (int k = 0; k < nf; ++k) {
    const double c = (double)S.st[k].size() + 1.0;
    S.pairs += c * (c + 1.0) * 0.5;  // 7x7 block products of column k's updates
  }
  {
    std::vector<int> lv2(nf, 0);
    int top = -1;
    for (int k = 0; k < S.sn0; ++k) {
      for (int c : S.children[k]) lv2[k] = std::max(lv2[k], lv2[c] + 1);
      top = std::max(top, lv2[k]);
    }
    const std::vector<double> lt = level_times(S, lv2, top + 1, S.sn0);
    S.cost = sn_time(nf - S.sn0);
    for (double t : lt) S.cost += t;
  }
  return S;
}

static ec3r_status build_plan(ec3r_ctx* ctx, int n, int m, const int32_t* hi, const int32_t* hj,
                              int fixed, Plan& P) {
  P.n = n;
  P.m = m;
  P.fixed = fixed;
  // free nodes and their adjacency
  std::vector<std::set<int>> adj(n);
  for (int e = 0; e < m; ++e) {
    const int a = hi[e], b = hj[e];
    if (a != fixed && b != fixed) {
      adj[a].insert(b);
      adj[b].insert(a);
    }
  }
  std::vector<int> freev;
  for (int v = 0; v < n; ++v)
    if (v != fixed) freev.push_back(v);
  std::vector<int> nd_order, md_order;
  nested_dissection(freev, adj, nd_order);
  minimum_degree(freev, adj, md_order);
  Symbolic A = analyse(nd_order, adj), B = analyse(md_order, adj);
  Symbolic& S = B.cost < A.cost ? B : A;
  const int nf = (int)S.perm.size();
  P.nf = nf;
  P.ordering = &S == &B ? 1 : 0;
  std::vector<int>& perm = S.perm;
  std::vector<int>& inew = S.inew;
  std::vector<std::vector<int>>& children = S.children;
  std::vector<std::set<int>>& st = S.st;
  // blocks: diagonal k -> k; off-diagonal numbered column by column
  std::vector<int> col_ptr(nf + 1, 0), off_row, off_blk;
  std::map<std::pair<int, int>, int> bidx;  // (row, col) -> block
  int nb = nf;
  for (int k = 0; k < nf; ++k) {
    col_ptr[k] = (int)off_row.size();
    for (int r : st[k]) {
      off_row.push_back(r);
      off_blk.push_back(nb);
      bidx[{r, k}] = nb++;
    }
  }
  col_ptr[nf] = (int)off_row.size();
  P.n_blocks = nb;
  auto blk = [&](int r, int c) { return r == c ? c : bidx.at({r, c}); };
  // left-looking update lists and forward-substitution row lists
  std::vector<std::vector<int>> rowstruct(nf);
  for (int j = 0; j < nf; ++j)
    for (int k : st[j]) rowstruct[k].push_back(j);
  // trailing dense supernode: the longest suffix of columns whose structure is
  // every later column; it is factored right-looking across all SMs
  P.sn0 = S.sn0;
  if (nf - P.sn0 > SN_DENSE_MAX)
    return set_error(ctx, EC3R_ERR_INVALID_ARG,
                     "the factor's dense trailing block has %d nodes (at most %d)", nf - P.sn0,
                     SN_DENSE_MAX);
  // update groups: for every block (i, k) of column k, the products
  // L_ij L_kj^T of its descendants j, in descendant order (for supernode
  // columns only the descendants below the supernode, gathered in sn_grp)
  std::vector<int> grp_ptr(nf + 1, 0), grp, upd_ab, row_ptr(nf + 1, 0), row, sn_grp, grp_slot;
  for (int k = 0; k < nf; ++k) {
    grp_ptr[k] = (int)grp.size() / 3;
    row_ptr[k] = (int)row.size() / 2;
    std::sort(rowstruct[k].begin(), rowstruct[k].end());
    std::vector<int> targets;
    targets.push_back(k);
    for (int r : st[k]) targets.push_back(r);
    const bool in_sn = k >= P.sn0;
    for (size_t ti = 0; ti < targets.size(); ++ti) {
      const int i = targets[ti];
      const int first = (int)upd_ab.size() / 2;
      for (int j : rowstruct[k]) {
        if (in_sn && j >= P.sn0) continue;  // supernode columns update right-looking
        if (i != k && !st[j].count(i)) continue;
        upd_ab.push_back(blk(i, j));
        upd_ab.push_back(blk(k, j));
      }
      const int n_upd = (int)upd_ab.size() / 2 - first;
      if (n_upd > 0) {
        std::vector<int>& G = in_sn ? sn_grp : grp;
        G.push_back(blk(i, k));
        G.push_back(first);
        G.push_back(n_upd);
        if (!in_sn) grp_slot.push_back((int)ti);  // 0: diagonal, t: t-th block below it
      }
    }
    for (int j : rowstruct[k]) {
      row.push_back(j);
      row.push_back(blk(k, j));
    }
  }
  grp_ptr[nf] = (int)grp.size() / 3;
  row_ptr[nf] = (int)row.size() / 2;
  // levels (height in the elimination tree) of the columns below the supernode
  const int nsp = P.sn0;
  std::vector<int> level(nf, 0);
  int nlev = 0;
  for (int k = 0; k < nsp; ++k) {
    for (int c : children[k]) level[k] = std::max(level[k], level[c] + 1);
    nlev = std::max(nlev, level[k] + 1);
  }
  P.level_ptr.assign(nlev + 1, 0);
  for (int k = 0; k < nsp; ++k) P.level_ptr[level[k] + 1]++;
  for (int l = 0; l < nlev; ++l) P.level_ptr[l + 1] += P.level_ptr[l];
  std::vector<int> level_cols(std::max(nsp, 1)), fill = P.level_ptr;
  for (int k = 0; k < nsp; ++k) level_cols[fill[level[k]]++] = k;
  // per column in level order: ColMeta (k, groups, blocks below the diagonal,
  // forward-substitution terms, staged, slots filled by groups)
  std::vector<int> col_meta(META_INTS * (size_t)std::max(nsp, 1), 0);
  for (int pos = 0; pos < nsp; ++pos) {
    const int k = level_cols[pos];
    int* cm = &col_meta[META_INTS * (size_t)pos];
    cm[0] = k;
    cm[1] = grp_ptr[k];
    cm[2] = grp_ptr[k + 1];
    cm[3] = col_ptr[k];
    cm[4] = col_ptr[k + 1];
    cm[5] = row_ptr[k];
    cm[6] = row_ptr[k + 1];
    const bool fits = 1 + (col_ptr[k + 1] - col_ptr[k]) <= CB_MAX &&
                      row_ptr[k + 1] - row_ptr[k] <= FS_MAX;
    cm[7] = fits ? 1 : 0;
    if (fits)
      for (int g = grp_ptr[k]; g < grp_ptr[k + 1]; ++g)
        cm[8 + grp_slot[g] / 32] |= (int)(1u << (grp_slot[g] % 32));
  }
  P.n_sn_groups = (int)sn_grp.size() / 3;
  P.nlev = nlev;
  // assembly lists: kind 0 = Cii, 1 = Cjj, 2 = Cij, 3 = Cij^T
  std::vector<std::vector<int>> asmv(nb), gv(nf);
  for (int e = 0; e < m; ++e) {
    const int a = inew[hi[e]], b = inew[hj[e]];
    if (a >= 0) {
      asmv[a].push_back(e << 2 | 0);
      gv[a].push_back(e << 1 | 0);
    }
    if (b >= 0) {
      asmv[b].push_back(e << 2 | 1);
      gv[b].push_back(e << 1 | 1);
    }
    if (a >= 0 && b >= 0) {
      if (a > b) asmv[blk(a, b)].push_back(e << 2 | 2);
      else asmv[blk(b, a)].push_back(e << 2 | 3);
    }
  }
  std::vector<int> asm_ptr(nb + 1, 0), asm_it, g_ptr(nf + 1, 0), g_it;
  for (int b = 0; b < nb; ++b) {
    asm_ptr[b] = (int)asm_it.size();
    for (int x : asmv[b]) asm_it.push_back(x);
  }
  asm_ptr[nb] = (int)asm_it.size();
  for (int k = 0; k < nf; ++k) {
    g_ptr[k] = (int)g_it.size();
    for (int x : gv[k]) g_it.push_back(x);
  }
  g_ptr[nf] = (int)g_it.size();
  // chaining tree: edges in input order that join two components, walked from `fixed`
  std::vector<int> uf(n);
  for (int v = 0; v < n; ++v) uf[v] = v;
  std::function<int(int)> find = [&](int a) {
    while (uf[a] != a) a = uf[a] = uf[uf[a]];
    return a;
  };
  std::vector<std::vector<int>> tadj(n);
  for (int e = 0; e < m; ++e) {
    const int a = find(hi[e]), b = find(hj[e]);
    if (a != b) {
      uf[a] = b;
      tadj[hi[e]].push_back(e);
      tadj[hj[e]].push_back(e);
    }
  }
  std::vector<int> tpar(n, -1), tedge(n, -1), tdir(n, 0), depth(n, 0), q{fixed};
  std::vector<char> seen(n, 0);
  seen[fixed] = 1;
  int maxd = 0;
  for (size_t h = 0; h < q.size(); ++h) {
    const int a = q[h];
    for (int e : tadj[a]) {
      const int o = hi[e] == a ? hj[e] : hi[e];
      if (seen[o]) continue;
      seen[o] = 1;
      tpar[o] = a;
      tedge[o] = e;
      tdir[o] = hi[e] == a ? 1 : -1;
      depth[o] = depth[a] + 1;
      maxd = std::max(maxd, depth[o]);
      q.push_back(o);
    }
  }
  int rounds = 0;
  while ((1 << rounds) < maxd + 1) ++rounds;
  P.rounds = rounds;
  std::vector<int> vi(hi, hi + m), vj(hj, hj + m);
  cudaError_t err = cudaSuccess;
  auto chk = [&](cudaError_t e) {
    if (err == cudaSuccess) err = e;
  };
  chk(upload(P, &P.d_ei, vi));
  chk(upload(P, &P.d_ej, vj));
  chk(upload(P, &P.d_perm, perm));
  chk(upload(P, &P.d_col_ptr, col_ptr));
  chk(upload(P, &P.d_off_row, off_row));
  chk(upload(P, &P.d_off_blk, off_blk));
  chk(upload(P, &P.d_grp_ptr, grp_ptr));
  chk(upload(P, &P.d_grp, grp));
  chk(upload(P, &P.d_sn_grp, sn_grp));
  chk(upload(P, &P.d_upd_ab, upd_ab));
  chk(alloc(P, &P.d_idiag, (size_t)nf * 7));
  chk(upload(P, &P.d_row_ptr, row_ptr));
  chk(upload(P, &P.d_row, row));
  chk(upload(P, &P.d_level_cols, level_cols));
  chk(upload(P, &P.d_col_meta, col_meta));
  chk(upload(P, &P.d_grp_slot, grp_slot));
  chk(alloc(P, &P.d_sn_cnt, (size_t)nf));
  chk(alloc(P, &P.d_sn_linv, (size_t)std::max(nf - P.sn0, 1) * NB));
  chk(upload(P, &P.d_level_ptr, P.level_ptr));
  chk(upload(P, &P.d_asm_ptr, asm_ptr));
  chk(upload(P, &P.d_asm, asm_it));
  chk(upload(P, &P.d_g_ptr, g_ptr));
  chk(upload(P, &P.d_g, g_it));
  chk(upload(P, &P.d_parent, tpar));
  chk(upload(P, &P.d_tedge, tedge));
  chk(upload(P, &P.d_tdir, tdir));
  chk(alloc(P, &P.d_anc0, n));
  chk(alloc(P, &P.d_anc1, n));
  chk(alloc(P, &P.d_fail, 1));
  chk(alloc(P, &P.d_L, (size_t)nb * NB));
  chk(alloc(P, &P.d_b, (size_t)nf * 7));
  chk(alloc(P, &P.d_contrib, (size_t)m * 3 * NB));
  chk(alloc(P, &P.d_gvec, (size_t)m * 14));
  chk(alloc(P, &P.d_chi2e, m));
  chk(alloc(P, &P.d_W0, n));
  chk(alloc(P, &P.d_W1, n));
  chk(alloc(P, &P.d_backup, n));
  chk(alloc(P, &P.d_lm, 4));
  chk(alloc(P, &P.d_lm_flags, 1));
  if (err != cudaSuccess) {
    cudaGetLastError();
    return set_error(ctx, EC3R_ERR_OOM, "pose-graph plan allocation failed: %s",
                     cudaGetErrorString(err));
  }
  return EC3R_OK;
}

// B_2k/(2k)! = (-1)^{k+1} 2 zeta(2k) / (2 pi)^{2k}; zeta by direct sum plus an
// Euler-Maclaurin tail.
static void bernoulli_table(double* c) {
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int k = 1; k <= NBERN; ++k) {
    const int s = 2 * k;
    const int N = 1000;
    long double z = 0.0L;
    for (int i = N - 1; i >= 1; --i) z += powl((long double)i, -s);
    const long double Nn = N;
    z += powl(Nn, 1 - s) / (s - 1) + 0.5L * powl(Nn, -s) +
         (long double)s / 12.0L * powl(Nn, -s - 1) -
         (long double)s * (s + 1) * (s + 2) / 720.0L * powl(Nn, -s - 3);
    const long double v = 2.0L * z / powl(2.0L * pi, s);
    c[k - 1] = (double)((k % 2 == 1) ? v : -v);
  }
}

static uint64_t fnv(const int32_t* a, int n, uint64_t h) {
  for (int i = 0; i < n; ++i) {
    h ^= (uint32_t)a[i];
    h *= 1099511628211ULL;
  }
  return h;
}

}  // namespace pg
}  // namespace ec3r

using namespace ec3r;
using namespace ec3r::pg;

extern "C" {

void ec3r_pg_opts_default(ec3r_pg_opts* o) {
  if (!o) return;
  o->iters = 10;
  o->fixed_node = 0;
  o->lm_lambda = 0.0;
  o->init_by_chaining = 1;
  o->lm_adaptive = 0;
}

ec3r_status ec3r_pose_graph_correct(ec3r_ctx* ctx, int n_nodes, ec3r_sim3* d_nodes, int n_edges,
                                    const int32_t* h_i, const int32_t* h_j,
                                    const ec3r_sim3* d_Tij, const double* d_info,
                                    const ec3r_pg_opts* opts, double* d_chi2, void* stream) {
  if (!ctx) return EC3R_ERR_INVALID_ARG;
  if (!opts || n_nodes < 1 || n_edges < 0 || !d_nodes || (n_edges > 0 && (!h_i || !h_j || !d_Tij)))
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "bad pose-graph arguments");
  if (opts->iters < 0 || opts->iters > 1000 || opts->fixed_node < 0 ||
      opts->fixed_node >= n_nodes || !(opts->lm_lambda >= 0.0) || n_nodes > (1 << 24) ||
      (opts->lm_adaptive != 0 && opts->lm_adaptive != 1) ||
      (opts->lm_adaptive && !(opts->lm_lambda > 0.0 && opts->lm_lambda <= 1e10)) ||
      n_edges > (1 << 28))
    return set_error(ctx, EC3R_ERR_INVALID_ARG, "bad ec3r_pg_opts");
  for (int e = 0; e < n_edges; ++e)
    if (h_i[e] < 0 || h_i[e] >= n_nodes || h_j[e] < 0 || h_j[e] >= n_nodes || h_i[e] == h_j[e])
      return set_error(ctx, EC3R_ERR_INVALID_ARG, "edge %d has invalid endpoints (%d, %d)", e,
                       h_i[e], h_j[e]);
  EC3R_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (!ctx->ext.count("pg.bernoulli")) {  // constant table, once per context (device)
    if (stream_capturing(s))
      return set_error(ctx, EC3R_ERR_CAPTURE, "first pose-graph call during stream capture");
    double c[NBERN];
    bernoulli_table(c);
    EC3R_CUDA_TRY(ctx, cudaMemcpyToSymbol(c_bern, c, sizeof(c)));
    ctx->ext["pg.bernoulli"] = new Extension();
  }
  // plan (host symbolic analysis), cached per graph structure
  uint64_t h = 1469598103934665603ULL;
  h = fnv(h_i, n_edges, h);
  h = fnv(h_j, n_edges, h);
  const std::string pkey = key_of("pgplan", {(uint64_t)n_nodes, (uint64_t)n_edges,
                                             (uint64_t)opts->fixed_node, h});
  Plan* P = nullptr;
  auto it = ctx->ext.find(pkey);
  if (it != ctx->ext.end()) {
    P = static_cast<Plan*>(it->second);
  } else {
    if (stream_capturing(s))
      return set_error(ctx, EC3R_ERR_CAPTURE, "new pose-graph structure during stream capture");
    // keep at most 4 plans
    int count = 0;
    for (auto& kv : ctx->ext)
      if (kv.first.rfind("pgplan", 0) == 0) ++count;
    if (count >= 4) {
      cudaDeviceSynchronize();
      drop_graphs(ctx);
      for (auto j = ctx->ext.begin(); j != ctx->ext.end();) {
        if (j->first.rfind("pgplan", 0) == 0) {
          delete j->second;
          j = ctx->ext.erase(j);
        } else {
          ++j;
        }
      }
    }
    P = new Plan();
    ec3r_status st = build_plan(ctx, n_nodes, n_edges, h_i, h_j, opts->fixed_node, *P);
    if (st != EC3R_OK) {
      delete P;
      return st;
    }
    ctx->ext[pkey] = P;
  }
  const ec3r_pg_opts o = *opts;
  PgDev dv{};
  dv.n = n_nodes;
  dv.m = n_edges;
  dv.nf = P->nf;
  dv.n_blocks = P->n_blocks;
  dv.sn0 = P->sn0;
  dv.nlev = P->nlev;
  dv.n_sn_groups = P->n_sn_groups;
  dv.iters = o.iters;
  dv.lambda = o.lm_lambda;
  dv.ei = P->d_ei;
  dv.ej = P->d_ej;
  dv.perm = P->d_perm;
  dv.col_ptr = P->d_col_ptr;
  dv.off_row = P->d_off_row;
  dv.off_blk = P->d_off_blk;
  dv.grp_ptr = P->d_grp_ptr;
  dv.grp = P->d_grp;
  dv.upd_ab = P->d_upd_ab;
  dv.sn_grp = P->d_sn_grp;
  dv.row_ptr = P->d_row_ptr;
  dv.row = P->d_row;
  dv.level_ptr = P->d_level_ptr;
  dv.level_cols = P->d_level_cols;
  dv.col_meta = reinterpret_cast<const int4*>(P->d_col_meta);
  dv.grp_slot = P->d_grp_slot;
  dv.asm_ptr = P->d_asm_ptr;
  dv.asm_it = P->d_asm;
  dv.g_ptr = P->d_g_ptr;
  dv.g_it = P->d_g;
  dv.L = P->d_L;
  dv.b = P->d_b;
  dv.contrib = P->d_contrib;
  dv.gvec = P->d_gvec;
  dv.chi2e = P->d_chi2e;
  dv.idiag = P->d_idiag;
  dv.chi2 = d_chi2;
  dv.fail = P->d_fail;
  const bool lm = o.lm_adaptive != 0;
  dv.flags = lm ? P->d_lm_flags : ctx->d_flags;  // a rejected LM step is not an error
  dv.lm = lm ? P->d_lm : nullptr;
  dv.backup = P->d_backup;
  dv.Tij = d_Tij;
  dv.info = d_info;
  dv.nodes = d_nodes;
  const std::string gkey =
      key_of("pg", {(uint64_t)P, (uint64_t)d_nodes, (uint64_t)d_Tij, (uint64_t)d_info,
                    (uint64_t)d_chi2, (uint64_t)o.iters, dbits(o.lm_lambda),
                    (uint64_t)o.init_by_chaining, (uint64_t)o.lm_adaptive});
  static bool attr_set[64] = {};
  if (ctx->device < 64 && !attr_set[ctx->device]) {
    EC3R_CUDA_TRY(ctx, cudaFuncSetAttribute(k_pg_sn_dense_solve,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)(sizeof(double) * 7 * SN_DENSE_MAX)));
    attr_set[ctx->device] = true;
  }
  return run_graph(ctx, gkey, s, [&](cudaStream_t cs) -> ec3r_status {
    if (o.init_by_chaining)
      traced(ctx, cs, "pg_init", [&] {
        launch_pdl(k_pg_init, 1, 1024, 0, cs, n_nodes, o.fixed_node, P->d_parent, P->d_tedge,
                   P->d_tdir, d_Tij, d_nodes, P->d_W0, P->d_W1, P->d_anc0, P->d_anc1,
                   P->rounds);
      });
    const int nlev = P->nlev;
    if (lm)
      traced(ctx, cs, "pg_lm", [&] { launch_pdl(k_pg_lm_start, 1, 1, 0, cs, dv, o.lm_lambda); });
    for (int itn = 0; itn <= o.iters; ++itn) {
      const bool last = itn == o.iters;  // last pass only evaluates chi^2
      if (n_edges > 0)
        traced(ctx, cs, "pg_linearize", [&] {
          launch_pdl(k_pg_linearize, n_edges, 64, 0, cs, dv, last ? 0 : 1);
        });
      if (last) {
        if (d_chi2)
          traced(ctx, cs, "pg_assemble", [&] {
            launch_pdl(k_pg_assemble, 1, 32, 0, cs, dv, 0, 0, d_chi2 + itn, 0);
          });
        break;
      }
      traced(ctx, cs, "pg_assemble", [&] {
        launch_pdl(k_pg_assemble, P->n_blocks + P->nf + 1, 32, 0, cs, dv, P->n_blocks, P->nf,
                   d_chi2 ? d_chi2 + itn : nullptr, 0);
      });
      if (P->nf == 0) continue;
      for (int l = 0; l < nlev; ++l)
        traced(ctx, cs, "pg_factor", [&] {
          launch_pdl(k_pg_factor, P->level_ptr[l + 1] - P->level_ptr[l], 32 * FWARPS, 0, cs, dv,
                     P->level_ptr[l]);
        });
      if (P->sn0 < P->nf) {
        const int nf = P->nf;
        if (P->n_sn_groups > 0)
          traced(ctx, cs, "pg_sn_assemble", [&] {
            launch_pdl(k_pg_sn_assemble, P->n_sn_groups, 32, 0, cs, P->d_sn_grp, P->d_upd_ab,
                       P->d_L);
          });
        // panel sn0, then per column k one launch: its trailing update and,
        // in the CTA that completes column k + 1, panel k + 1
        EC3R_CUDA_TRY(ctx, cudaMemsetAsync(P->d_sn_cnt, 0, sizeof(int) * (size_t)nf, cs));
        traced(ctx, cs, "pg_sn_panel", [&] {
          launch_pdl(k_pg_sn_panel_first, 1, SN_UPD_THREADS, 0, cs, P->sn0, nf, P->d_col_ptr,
                     P->d_off_blk, P->d_L, P->d_idiag, P->d_sn_linv, dv.flags, P->d_fail);
        });
        for (int k = P->sn0; k + 1 < nf; ++k) {
          const int64_t mrem = nf - 1 - k;
          const int64_t blocks = (mrem * (mrem + 1) / 2 + SN_UPD_THREADS / 32 - 1) /
                                 (SN_UPD_THREADS / 32);
          traced(ctx, cs, "pg_sn_update", [&] {
            launch_pdl(k_pg_sn_update_panel, (unsigned)blocks, SN_UPD_THREADS, 0, cs, k,
                       P->sn0, nf, P->d_col_ptr, P->d_off_blk, P->d_L, P->d_idiag,
                       P->d_sn_linv, dv.flags, P->d_fail, P->d_sn_cnt);
          });
        }
        traced(ctx, cs, "pg_sn_solve", [&] {
          const int ns = nf - P->sn0;
          launch_pdl(k_pg_sn_rhs, ns, 32, 0, cs, P->sn0, P->d_row_ptr, P->d_row, P->d_L,
                     P->d_b);
          launch_pdl(k_pg_sn_dense_solve, 1, SN_THREADS, sizeof(double) * 7 * ns, cs, P->sn0,
                     nf, P->d_col_ptr, P->d_off_blk, P->d_L, P->d_sn_linv, P->d_b);
        });
      }
      for (int l = nlev - 1; l >= 0; --l)
        traced(ctx, cs, "pg_backsolve", [&] {
          launch_pdl(k_pg_backsolve, P->level_ptr[l + 1] - P->level_ptr[l], 32, 0, cs, dv,
                     P->level_ptr[l]);
        });
      if (lm)
        traced(ctx, cs, "pg_lm", [&] {
          launch_pdl(k_pg_backup, (n_nodes + 127) / 128, 128, 0, cs, dv);
        });
      traced(ctx, cs, "pg_update", [&] {
        launch_pdl(k_pg_update, (P->nf + 63) / 64, 64, 0, cs, dv);
      });
      if (lm) {  // chi^2 of the tentative step, then keep it or restore
        if (n_edges > 0)
          traced(ctx, cs, "pg_linearize", [&] {
            launch_pdl(k_pg_linearize, n_edges, 64, 0, cs, dv, 0);
          });
        traced(ctx, cs, "pg_assemble", [&] {
          launch_pdl(k_pg_assemble, 1, 32, 0, cs, dv, 0, 0, nullptr, 1);
        });
        traced(ctx, cs, "pg_lm", [&] {
          launch_pdl(k_pg_decide, (n_nodes + 127) / 128, 128, 0, cs, dv);
        });
      }
    }
    EC3R_CUDA_TRY(ctx, cudaGetLastError());
    return EC3R_OK;
  });
}

}  // extern "C"
