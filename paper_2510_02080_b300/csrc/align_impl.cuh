// Internal definitions shared by the registration's forward and backward
// translation units (align.cu, align_bwd.cu).
#pragma once

#include <cfloat>

#include "common.cuh"

namespace ec3r {
namespace align {

constexpr int TILE = 8192;  // pixels per sweep CTA
constexpr int THREADS = 256;
constexpr int NMOM = 19;
// moment slots
enum { M_W = 0, M_SP = 1, M_SQ = 4, M_PP = 7, M_QP = 8, M_COST = 17, M_CNT = 18 };
// The grid schedule's cost sweep leaves slots 1..16 free and stores there,
// from CS_SLOT on, the 12 sums of the adjoint's cost term (sum g p'^T
// row-major, sum g); the final sweep forms the same 12 sums.  Per pair the
// context keeps those 12 sums and then the cost itself (CS_STRIDE doubles),
// so the backward never reads the caller's outputs.
constexpr int CS_SLOT = 1, NCS = 12, CS_COST = NCS, CS_STRIDE = NCS + 1;
constexpr double RANK_REL_TOL = 1e-4;

struct PairState {
  // FP32 view of the current and previous estimate, pivot-relative:
  // residual e = A p' + b - q',  p' = p - piv_p, q' = q - piv_q, A = s R.
  float A[9], b[3];
  float Ap[9], bp[3];
  float piv_p[3], piv_q[3];
  float cmin;
  int active;
  int status;
  int pad;
  double Ad[9], bd[3];
  double Adp[9], bdp[3];
};

__device__ __forceinline__ bool finitef(float x) { return fabsf(x) <= FLT_MAX; }

// A link pixel's weight as the first FP32 sweep leaves it for the later
// sweeps and the backward pass (4 B per link pixel instead of both 4-byte
// confidences): w = c_p c_q (rule 0) or c_p when the correspondence is valid
// (p, q, c_p, c_q finite and both confidences above cmin), NaN when it is not.
// (A valid weight can be <= 0 only under a negative threshold, so validity
// cannot be read from the sign.)
__device__ __forceinline__ float pixel_weight(float p0, float p1, float p2, float q0, float q1,
                                              float q2, float cp, float cq, float cmin,
                                              int rule) {
  const bool v = finitef(p0) && finitef(p1) && finitef(p2) && finitef(q0) && finitef(q1) &&
                 finitef(q2) && finitef(cp) && finitef(cq) && cp > cmin && cq > cmin;
  return v ? (rule == 0 ? cp * cq : cp) : __int_as_float(0x7fc00000);
}

// Per pair and iteration, the forward solve keeps (for the backward pass) the
// 19 moments, A = s R (9) and b (3) of its estimate, its status, s and R
// themselves, and the singular values d (3) and right singular vectors V (9)
// of its cross-covariance (the pieces of the polar factor's derivative).
constexpr int CKPT = 56;
enum {
  CK_MOM = 0, CK_A = 19, CK_B = 28, CK_STATUS = 31, CK_S = 32, CK_R = 33, CK_D = 42, CK_V = 45
};

// --------------------------------------------------------------------------
// solve
// --------------------------------------------------------------------------
// Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix (row-major), FP32.
// Eigenvalues descending, eigenvectors in the columns of V.
__device__ inline void jacobi_eig3f(float B[9], float V[9], float lam[3]) {
  for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.f : 0.f;
  for (int sweep = 0; sweep < 8; ++sweep) {
    const float off = fabsf(B[1]) + fabsf(B[2]) + fabsf(B[5]);
    const float dia = fabsf(B[0]) + fabsf(B[4]) + fabsf(B[8]);
    if (off <= 1e-9f * dia) break;
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0;
      const int q = pq == 0 ? 1 : 2;
      const float bpq = B[3 * p + q];
      if (fabsf(bpq) < 1e-30f) continue;
      const float theta = (B[3 * q + q] - B[3 * p + p]) / (2.f * bpq);
      const float tt = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
      const float cs = rsqrtf(tt * tt + 1.f), sn = tt * cs;
      for (int r = 0; r < 3; ++r) {
        const float brp = B[3 * r + p], brq = B[3 * r + q];
        B[3 * r + p] = cs * brp - sn * brq;
        B[3 * r + q] = sn * brp + cs * brq;
      }
      for (int r = 0; r < 3; ++r) {
        const float bpr = B[3 * p + r], bqr = B[3 * q + r];
        B[3 * p + r] = cs * bpr - sn * bqr;
        B[3 * q + r] = sn * bpr + cs * bqr;
      }
      for (int r = 0; r < 3; ++r) {
        const float vrp = V[3 * r + p], vrq = V[3 * r + q];
        V[3 * r + p] = cs * vrp - sn * vrq;
        V[3 * r + q] = sn * vrp + cs * vrq;
      }
    }
  }
  lam[0] = B[0]; lam[1] = B[4]; lam[2] = B[8];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2 - a; ++b)
      if (lam[b] < lam[b + 1]) {
        const float tl = lam[b]; lam[b] = lam[b + 1]; lam[b + 1] = tl;
        for (int r = 0; r < 3; ++r) {
          const float tv = V[3 * r + b]; V[3 * r + b] = V[3 * r + b + 1]; V[3 * r + b + 1] = tv;
        }
      }
}

// Rotation R (FP64) of the Umeyama solution, R = U diag(1,1,det(U)det(V)) V^T,
// i.e. the orthogonal polar factor of Sig with det +1, and the Rayleigh
// estimates d[0..2] of the signed singular values.  An FP32 Jacobi SVD seeds
// R; two FP64 Newton-polar steps R <- R cay(w), (tr(Hs) I - Hs) w =
// vee(H - H^T), H = R^T Sig, bring it to FP64 round-off.
__device__ inline void polar_rotation(const double Sig[9], double R[9], double d[3],
                                      double* Vout = nullptr) {
  double nrm = 0.0;
  for (int i = 0; i < 9; ++i) nrm += Sig[i] * Sig[i];
  nrm = sqrt(nrm);
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  float Sf[9], B[9], V[9], lam[3];
  for (int i = 0; i < 9; ++i) Sf[i] = (float)(Sig[i] * inv);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      B[3 * i + j] = Sf[i] * Sf[j] + Sf[3 + i] * Sf[3 + j] + Sf[6 + i] * Sf[6 + j];
  jacobi_eig3f(B, V, lam);
  float v[3][3];
  for (int c = 0; c < 3; ++c)
    for (int r = 0; r < 3; ++r) v[c][r] = V[3 * r + c];
  float u[3][3];
  for (int c = 0; c < 2; ++c)
    for (int r = 0; r < 3; ++r)
      u[c][r] = Sf[3 * r] * v[c][0] + Sf[3 * r + 1] * v[c][1] + Sf[3 * r + 2] * v[c][2];
  float n0 = sqrtf(u[0][0] * u[0][0] + u[0][1] * u[0][1] + u[0][2] * u[0][2]);
  if (n0 < 1e-30f) { u[0][0] = 1.f; u[0][1] = 0.f; u[0][2] = 0.f; n0 = 1.f; }
  for (int r = 0; r < 3; ++r) u[0][r] /= n0;
  const float dp = u[0][0] * u[1][0] + u[0][1] * u[1][1] + u[0][2] * u[1][2];
  for (int r = 0; r < 3; ++r) u[1][r] -= dp * u[0][r];
  float n1 = sqrtf(u[1][0] * u[1][0] + u[1][1] * u[1][1] + u[1][2] * u[1][2]);
  if (n1 < 1e-30f) {  // any unit vector orthogonal to u0
    float a[3] = {0.f, 0.f, 0.f};
    a[fabsf(u[0][0]) < 0.5f ? 0 : 1] = 1.f;
    const float da = a[0] * u[0][0] + a[1] * u[0][1] + a[2] * u[0][2];
    for (int r = 0; r < 3; ++r) u[1][r] = a[r] - da * u[0][r];
    n1 = sqrtf(u[1][0] * u[1][0] + u[1][1] * u[1][1] + u[1][2] * u[1][2]);
  }
  for (int r = 0; r < 3; ++r) u[1][r] /= n1;
  u[2][0] = u[0][1] * u[1][2] - u[0][2] * u[1][1];
  u[2][1] = u[0][2] * u[1][0] - u[0][0] * u[1][2];
  u[2][2] = u[0][0] * u[1][1] - u[0][1] * u[1][0];
  const float detV = v[0][0] * (v[1][1] * v[2][2] - v[1][2] * v[2][1]) -
                     v[0][1] * (v[1][0] * v[2][2] - v[1][2] * v[2][0]) +
                     v[0][2] * (v[1][0] * v[2][1] - v[1][1] * v[2][0]);
  const float e3 = detV < 0.f ? -1.f : 1.f;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      R[3 * i + j] = (double)(u[0][i] * v[0][j] + u[1][i] * v[1][j] + e3 * u[2][i] * v[2][j]);
  // The FP32 seed is orthonormal only to ~1e-7 and the Cayley steps below keep
  // that defect, so make it a rotation to FP64 round-off first (Gram-Schmidt
  // on the rows, third row as the cross product).
  {
    double n = rsqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
    R[0] *= n; R[1] *= n; R[2] *= n;
    const double d = R[3] * R[0] + R[4] * R[1] + R[5] * R[2];
    R[3] -= d * R[0]; R[4] -= d * R[1]; R[5] -= d * R[2];
    n = rsqrt(R[3] * R[3] + R[4] * R[4] + R[5] * R[5]);
    R[3] *= n; R[4] *= n; R[5] *= n;
    R[6] = R[1] * R[5] - R[2] * R[4];
    R[7] = R[2] * R[3] - R[0] * R[5];
    R[8] = R[0] * R[4] - R[1] * R[3];
  }
  for (int it = 0; it < 2; ++it) {
    double H[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        H[3 * i + j] = R[i] * Sig[j] + R[3 + i] * Sig[3 + j] + R[6 + i] * Sig[6 + j];
    const double a0 = H[7] - H[5], a1 = H[2] - H[6], a2 = H[3] - H[1];
    const double tr = H[0] + H[4] + H[8];
    double M[9];
    M[0] = tr - H[0]; M[4] = tr - H[4]; M[8] = tr - H[8];
    M[1] = M[3] = -0.5 * (H[1] + H[3]);
    M[2] = M[6] = -0.5 * (H[2] + H[6]);
    M[5] = M[7] = -0.5 * (H[5] + H[7]);
    const double c00 = M[4] * M[8] - M[5] * M[7], c01 = M[5] * M[6] - M[3] * M[8],
                 c02 = M[3] * M[7] - M[4] * M[6];
    const double det = M[0] * c00 + M[1] * c01 + M[2] * c02;
    if (!(fabs(det) > 1e-300)) break;
    const double c11 = M[0] * M[8] - M[2] * M[6], c12 = M[2] * M[3] - M[0] * M[5],
                 c22 = M[0] * M[4] - M[1] * M[3];
    const double id = 1.0 / det;  // M symmetric: inverse = cofactor matrix / det
    const double w0 = (c00 * a0 + c01 * a1 + c02 * a2) * id;
    const double w1 = (c01 * a0 + c11 * a1 + c12 * a2) * id;
    const double w2 = (c02 * a0 + c12 * a1 + c22 * a2) * id;
    // Cayley transform of w: C = I + 2/(1+|h|^2) (h^ + h^ h^), h = w/2
    const double h0 = 0.5 * w0, h1 = 0.5 * w1, h2 = 0.5 * w2;
    const double f = 2.0 / (1.0 + h0 * h0 + h1 * h1 + h2 * h2);
    double C[9];
    C[0] = 1.0 - f * (h1 * h1 + h2 * h2);
    C[4] = 1.0 - f * (h0 * h0 + h2 * h2);
    C[8] = 1.0 - f * (h0 * h0 + h1 * h1);
    C[1] = f * (-h2 + h0 * h1);
    C[2] = f * (h1 + h0 * h2);
    C[3] = f * (h2 + h0 * h1);
    C[5] = f * (-h0 + h1 * h2);
    C[6] = f * (-h1 + h0 * h2);
    C[7] = f * (h0 + h1 * h2);
    double Rn[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        Rn[3 * i + j] = R[3 * i] * C[j] + R[3 * i + 1] * C[3 + j] + R[3 * i + 2] * C[6 + j];
    for (int i = 0; i < 9; ++i) R[i] = Rn[i];
  }
  double H[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      H[3 * i + j] = R[i] * Sig[j] + R[3 + i] * Sig[3 + j] + R[6 + i] * Sig[6 + j];
  if (Vout)
    for (int c = 0; c < 3; ++c)
      for (int r = 0; r < 3; ++r) Vout[3 * r + c] = v[c][r];
  for (int c = 0; c < 3; ++c) {
    const double x0 = v[c][0], x1 = v[c][1], x2 = v[c][2];
    const double y0 = H[0] * x0 + H[1] * x1 + H[2] * x2;
    const double y1 = H[3] * x0 + H[4] * x1 + H[5] * x2;
    const double y2 = H[6] * x0 + H[7] * x1 + H[8] * x2;
    d[c] = (x0 * y0 + x1 * y1 + x2 * y2) / (x0 * x0 + x1 * x1 + x2 * x2);
  }
}


// --------------------------------------------------------------------------
// moment sweep: one point's contribution
// --------------------------------------------------------------------------
enum Kind { FIRST = 0, IRLS = 1, COST = 2 };

// One point's contribution.  T is float (FP32 moments) or double (FP64).
template <typename T, int KIND>
struct PointOp {
  T A[9], b[3], Ap[9], bp[3], pp[3], pq[3], delta;
  float cmin;
  int rule;

  // from both confidences
  __device__ __forceinline__ void operator()(float p0, float p1, float p2, float q0, float q1,
                                             float q2, float cp, float cq, T* acc) const {
    const bool v = finitef(p0) && finitef(p1) && finitef(p2) && finitef(q0) && finitef(q1) &&
                   finitef(q2) && finitef(cp) && finitef(cq) && cp > cmin && cq > cmin;
    const T w = rule == 0 ? (T)cp * (T)cq : (T)cp;
    point(p0, p1, p2, q0, q1, q2, v, v ? w : T(0), acc);
  }

  // from the pixel weight that the first FP32 sweep stored (NaN: invalid;
  // the same FP32 product as above)
  __device__ __forceinline__ void operator()(float p0, float p1, float p2, float q0, float q1,
                                             float q2, float wv, T* acc) const {
    const bool v = wv == wv;
    point(p0, p1, p2, q0, q1, q2, v, v ? (T)wv : T(0), acc);
  }

  __device__ __forceinline__ void point(float p0, float p1, float p2, float q0, float q1,
                                        float q2, bool v, T w, T* acc) const {
    const T x0 = v ? (T)p0 - pp[0] : T(0), x1 = v ? (T)p1 - pp[1] : T(0),
            x2 = v ? (T)p2 - pp[2] : T(0);
    const T y0 = v ? (T)q0 - pq[0] : T(0), y1 = v ? (T)q1 - pq[1] : T(0),
            y2 = v ? (T)q2 - pq[2] : T(0);
    T h = T(1), r2 = T(0), f0 = T(0), f1 = T(0), f2 = T(0);
    if (KIND != FIRST) {
      const T* a = (KIND == COST) ? Ap : A;
      const T* c = (KIND == COST) ? bp : b;
      const T e0 = a[0] * x0 + a[1] * x1 + a[2] * x2 + c[0] - y0;
      const T e1 = a[3] * x0 + a[4] * x1 + a[5] * x2 + c[1] - y1;
      const T e2 = a[6] * x0 + a[7] * x1 + a[8] * x2 + c[2] - y2;
      const T rr = e0 * e0 + e1 * e1 + e2 * e2;
      if constexpr (sizeof(T) == 4) {
        h = fminf(1.f, (float)delta * rsqrtf(rr));
      } else {
        h = rr <= delta * delta ? 1.0 : delta / sqrt(rr);
      }
      if (KIND == COST) {
        f0 = A[0] * x0 + A[1] * x1 + A[2] * x2 + b[0] - y0;
        f1 = A[3] * x0 + A[4] * x1 + A[5] * x2 + b[1] - y1;
        f2 = A[6] * x0 + A[7] * x1 + A[8] * x2 + b[2] - y2;
        r2 = f0 * f0 + f1 * f1 + f2 * f2;
      } else {
        r2 = rr;
      }
    }
    const T om = w * h;
    acc[M_W] += om;
    acc[M_COST] += om * r2;
    acc[M_CNT] += v ? T(1) : T(0);
    if (KIND == COST) {
      // for the adjoint's cost term: sum g p'^T and sum g with g = om e(S_K),
      // in moment slots the cost sweep does not otherwise use
      const T g0 = om * f0, g1 = om * f1, g2 = om * f2;
      acc[CS_SLOT + 0] += g0 * x0; acc[CS_SLOT + 1] += g0 * x1; acc[CS_SLOT + 2] += g0 * x2;
      acc[CS_SLOT + 3] += g1 * x0; acc[CS_SLOT + 4] += g1 * x1; acc[CS_SLOT + 5] += g1 * x2;
      acc[CS_SLOT + 6] += g2 * x0; acc[CS_SLOT + 7] += g2 * x1; acc[CS_SLOT + 8] += g2 * x2;
      acc[CS_SLOT + 9] += g0; acc[CS_SLOT + 10] += g1; acc[CS_SLOT + 11] += g2;
      return;
    }
    const T wx0 = om * x0, wx1 = om * x1, wx2 = om * x2;
    const T wy0 = om * y0, wy1 = om * y1, wy2 = om * y2;
    acc[M_SP + 0] += wx0; acc[M_SP + 1] += wx1; acc[M_SP + 2] += wx2;
    acc[M_SQ + 0] += wy0; acc[M_SQ + 1] += wy1; acc[M_SQ + 2] += wy2;
    acc[M_PP] += wx0 * x0 + wx1 * x1 + wx2 * x2;
    acc[M_QP + 0] += wy0 * x0; acc[M_QP + 1] += wy0 * x1; acc[M_QP + 2] += wy0 * x2;
    acc[M_QP + 3] += wy1 * x0; acc[M_QP + 4] += wy1 * x1; acc[M_QP + 5] += wy1 * x2;
    acc[M_QP + 6] += wy2 * x0; acc[M_QP + 7] += wy2 * x1; acc[M_QP + 8] += wy2 * x2;
  }
};

// FP64 sum of partials[t * NV + v] over the tiles t in [t0, t1) for one v:
// four accumulators over consecutive tiles, so that eight loads are in flight
// at once instead of one dependent load per tile; fixed order (it depends
// only on the tile count).
template <int NV>
__device__ __forceinline__ double tile_sum(const double* __restrict__ partials, int64_t t0,
                                           int64_t t1, int v) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int64_t t = t0;
#pragma unroll 2
  for (; t + 4 <= t1; t += 4) {
    s0 += partials[t * NV + v];
    s1 += partials[(t + 1) * NV + v];
    s2 += partials[(t + 2) * NV + v];
    s3 += partials[(t + 3) * NV + v];
  }
  for (; t < t1; ++t) s0 += partials[t * NV + v];
  return (s0 + s1) + (s2 + s3);
}

// --------------------------------------------------------------------------
// per-pair solve from the 19 moments (shared by the pointmap and depth paths)
// --------------------------------------------------------------------------
__device__ inline void write_identity(ec3r_sim3* o) {
  o->s = 1.0;
  for (int i = 0; i < 9; ++i) o->R[i] = (i % 4 == 0) ? 1.0 : 0.0;
  for (int i = 0; i < 3; ++i) o->t[i] = 0.0;
}

// Weighted Umeyama (Sec. III-C, Eq. (sim3)) from pivot-centred moments M:
// the new estimate (R, s, b) with b the pivot-relative translation, or a
// status bit (R = I, s = 1, b = 0) for a degenerate pair.
__device__ inline unsigned umeyama_from_moments(const double* M, double R[9], double& s,
                                                double b[3], double* dV = nullptr) {
  for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0) ? 1.0 : 0.0;
  s = 1.0;
  b[0] = b[1] = b[2] = 0.0;
  const double W = M[M_W], N = M[M_CNT];
  if (N < 3.0) return EC3R_PAIR_FEW_POINTS;
  if (!(W > 0.0) || !isfinite(W)) return EC3R_PAIR_ZERO_WEIGHT;
  const double iw = 1.0 / W;
  const double mp[3] = {M[M_SP] * iw, M[M_SP + 1] * iw, M[M_SP + 2] * iw};
  const double mq[3] = {M[M_SQ] * iw, M[M_SQ + 1] * iw, M[M_SQ + 2] * iw};
  double Sig[9];
  bool fin = true;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      Sig[3 * i + j] = M[M_QP + 3 * i + j] * iw - mq[i] * mp[j];
      fin &= isfinite(Sig[3 * i + j]);
    }
  const double var = M[M_PP] * iw - (mp[0] * mp[0] + mp[1] * mp[1] + mp[2] * mp[2]);
  if (!fin || !isfinite(var)) return EC3R_PAIR_NONFINITE;
  if (!(var > 0.0)) return EC3R_PAIR_RANK;
  double d[3], Rn[9], V[9];
  polar_rotation(Sig, Rn, d, V);
  if (!(d[0] > 0.0) || fabs(d[1]) <= RANK_REL_TOL * d[0]) return EC3R_PAIR_RANK;
  // tr(R^T Sig) = tr(D E): the Umeyama scale numerator
  double tr = 0.0;
  for (int i = 0; i < 9; ++i) tr += Rn[i] * Sig[i];
  const double sn = tr / var;
  double bn[3];
  for (int i = 0; i < 3; ++i)
    bn[i] = mq[i] - sn * (Rn[3 * i] * mp[0] + Rn[3 * i + 1] * mp[1] + Rn[3 * i + 2] * mp[2]);
  bool ok = isfinite(sn) && sn > 0.0;
  for (int i = 0; i < 3; ++i) ok &= isfinite(bn[i]);
  if (!ok) return EC3R_PAIR_NONFINITE;
  for (int i = 0; i < 9; ++i) R[i] = Rn[i];
  s = sn;
  for (int i = 0; i < 3; ++i) b[i] = bn[i];
  if (dV) {
    for (int i = 0; i < 3; ++i) dV[i] = d[i];
    for (int i = 0; i < 9; ++i) dV[3 + i] = V[i];
  }
  return 0;
}

// Stores a solve's result in the pair state (current -> previous, new ->
// current) and, on the last iteration, the Sim(3) in submap coordinates; a
// degenerate pair is deactivated and returns the identity.
__device__ inline void commit_estimate(PairState& S, unsigned status, const double R[9], double s,
                                       const double b[3], bool last, ec3r_sim3& out,
                                       int32_t& status_out) {
  if (status) {
    S.status = (int)status;
    S.active = 0;
    write_identity(&out);
    status_out = (int)status;
    return;
  }
  for (int i = 0; i < 9; ++i) {
    S.Ap[i] = S.A[i];
    S.Adp[i] = S.Ad[i];
    S.Ad[i] = s * R[i];
    S.A[i] = (float)S.Ad[i];
  }
  for (int i = 0; i < 3; ++i) {
    S.bp[i] = S.b[i];
    S.bdp[i] = S.bd[i];
    S.bd[i] = b[i];
    S.b[i] = (float)b[i];
  }
  if (last) {
    out.s = s;
    for (int i = 0; i < 9; ++i) out.R[i] = R[i];
    const double pp[3] = {S.piv_p[0], S.piv_p[1], S.piv_p[2]};
    for (int i = 0; i < 3; ++i)
      out.t[i] = b[i] + (double)S.piv_q[i] -
                 s * (R[3 * i] * pp[0] + R[3 * i + 1] * pp[1] + R[3 * i + 2] * pp[2]);
    status_out = 0;
  }
}

// cost = sum om r^2 / sum om from the cost sweep's partials.
// One warp per pair: the cost sum W^-1 sum om r^2 of the last estimate and,
// when cost_sums is given, the pair's 12 sums of the adjoint's cost term
// (fixed-order tile sums, lane m owns slot m).
static __global__ void __launch_bounds__(32) k_cost(int n_pairs,
                                                    const int32_t* __restrict__ link_off,
                                                    int tpl, const double* __restrict__ partials,
                                                    const PairState* __restrict__ st,
                                                    double* __restrict__ cost,
                                                    double* __restrict__ cost_sums) {
  const int k = blockIdx.x, lane = threadIdx.x;
  __shared__ double red[NMOM];
  if (!st[k].active) {
    if (lane == 0) cost[k] = 0.0;
    if (cost_sums && lane <= NCS) cost_sums[(size_t)k * CS_STRIDE + lane] = 0.0;
    return;
  }
  const int64_t t0 = (int64_t)link_off[k] * tpl, t1 = (int64_t)link_off[k + 1] * tpl;
  if (lane < NMOM) red[lane] = tile_sum<NMOM>(partials, t0, t1, lane);
  __syncwarp();
  if (lane == 0) {
    const double w = red[M_W], c = red[M_COST];
    const double v = w > 0.0 ? c / w : 0.0;
    cost[k] = v;
    if (cost_sums) cost_sums[(size_t)k * CS_STRIDE + CS_COST] = v;
  }
  if (cost_sums && lane < NCS) cost_sums[(size_t)k * CS_STRIDE + lane] = red[CS_SLOT + lane];
}

// Checks the link offsets as one CSR array (link_off[0] = 0, non-decreasing,
// link_off[n_pairs] = n_links) and writes 1 to *malformed if they are not, else
// 0.  One CTA reads every offset, so that the set-up of every pair sees the
// same answer: a malformed batch marks all its pairs, and no two pairs of an
// accepted batch can claim the same link.
static __global__ void __launch_bounds__(1024) k_check_offsets(
    const int32_t* __restrict__ link_off, int n_pairs, int64_t n_links, int32_t* malformed) {
  int bad = 0;
  for (int j = threadIdx.x; j < n_pairs; j += blockDim.x) {
    const int64_t a = link_off[j], b = link_off[j + 1];
    bad |= (a > b) | (a < 0) | (b > n_links);
  }
  if (threadIdx.x == 0) bad |= (link_off[0] != 0) | ((int64_t)link_off[n_pairs] != n_links);
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) *malformed = bad ? 1 : 0;
}

// --------------------------------------------------------------------------
// persistent launches: per-pair epochs (release / acquire) and bounded waits
// --------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Epoch of a pair that no later sweep works on (degenerate): every wait passes.
constexpr unsigned EPOCH_DONE = 0xffffffffu;

// Waits until *ep >= want.  Gives up after `limit` cycles or 2^22 polls,
// whichever comes first, or as soon as another CTA has given up (*abort):
// then raises FLAG_TIMEOUT, sets *abort so that every other CTA stops too, and
// returns false.
static __device__ __noinline__ bool wait_epoch(const unsigned* ep, unsigned want, unsigned* abort,
                                        unsigned* flags, long long limit) {
  if (ld_acquire_u32(ep) >= want) return true;
  const long long t0 = clock64();
  unsigned ns = 32;
  for (int poll = 0; poll < (1 << 22); ++poll) {
    __nanosleep(ns);
    if (ns < 1024) ns <<= 1;
    if (ld_acquire_u32(ep) >= want) return true;
    if (ld_acquire_u32(abort) || clock64() - t0 > limit) break;
  }
  atomicOr(flags, FLAG_TIMEOUT);
  atomicExch(abort, 1u);
  return false;
}

// FP64 tile sums from L2 (the partials were written by other CTAs during
// this launch): four accumulators, fixed order, as tile_sum.
template <int NV>
__device__ __forceinline__ double tile_sum_cg(const double* partials, int64_t t0, int64_t t1,
                                              int v) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int64_t t = t0;
#pragma unroll 2
  for (; t + 4 <= t1; t += 4) {
    s0 += __ldcg(&partials[t * NV + v]);
    s1 += __ldcg(&partials[(t + 1) * NV + v]);
    s2 += __ldcg(&partials[(t + 2) * NV + v]);
    s3 += __ldcg(&partials[(t + 3) * NV + v]);
  }
  for (; t < t1; ++t) s0 += __ldcg(&partials[t * NV + v]);
  return (s0 + s1) + (s2 + s3);
}

// The persistent registration with FP32 moments (align_persist.cu): the
// autotuner's variants and the launch.  Variant v < 0 or out of range means
// the first (8192-pixel tiles, four CTAs per SM); unaligned pointmaps have one
// fixed configuration.
int reg_variant_count();
int reg_grid_variant();  // the variant that runs separate grids per sweep and solve
bool reg_variant_info(int v, int* tile, int* ctas, int* persistent);
int reg_min_tile();
size_t reg_ctl_bytes(int n_pairs);
ec3r_status launch_register(ec3r_ctx* ctx, cudaStream_t s, int v, bool vec, bool first,
                            const float* xyz, const float* conf, int64_t hw, int n_pairs,
                            int64_t n_links, const int32_t* link_off, const int32_t* src,
                            const int32_t* tgt, const int32_t* link_pair, float* weights,
                            PairState* st, double* partials, float delta, int rule, int iters,
                            int n_sweeps, ec3r_sim3* out, int32_t* status_out, double* cost,
                            double* cost_sums, double* ckpt, void* ctl, size_t ctl_bytes);
// Values per final-sweep tile (the partials buffer of launch_final holds
// this many doubles per TILE-pixel tile).
constexpr int FINAL_VALUES = NMOM + 18;
ec3r_status launch_final(ec3r_ctx* ctx, cudaStream_t s, bool vec, bool after_register,
                         const float* xyz, const float* conf, int64_t hw, int n_pairs,
                         int64_t n_links, const int32_t* link_off, const int32_t* src,
                         const int32_t* tgt, const int32_t* link_pair, float* weights,
                         PairState* st, double* partials, float delta, int rule, int iters,
                         ec3r_sim3* out,
                         int32_t* status_out, double* cost, double* cost_sums, double* ckpt,
                         void* ctl);

}  // namespace align
}  // namespace ec3r
