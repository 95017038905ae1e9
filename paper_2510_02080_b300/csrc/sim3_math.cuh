// FP64 Sim(3) algebra on the device, for the pose graph (Sec. III-E).
//
// A similarity T = (s, R, t) acts as x -> s R x + t.  Its tangent vector is
// xi = (rho[3], phi[3], sigma) with generator [[phi^ + sigma I, rho], [0, 0]]
// (the paper only says "R^7"; this coordinate order is the library's choice),
// so Exp(xi) = (e^sigma, exp(phi^), V rho) with
//   V = integral_0^1 e^{sigma u} exp(u phi^) du = a I + b phi^ + c phi^2,
//   a = int e^{su} du,  b = int e^{su} sin(th u)/th du,
//   c = int e^{su} (1 - cos(th u))/th^2 du,  th = |phi|.
// Closed forms are used away from the origin; near it (sigma^2 + th^2 < 1/4)
// the integrands are expanded in powers of sigma and th^2 and integrated term
// by term, so there is no cancellation.
#pragma once

namespace ec3r {
namespace s3 {

struct Sim3d {
  double s, R[9], t[3];
};

__device__ __forceinline__ void mat3_mul(const double* A, const double* B, double* C) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

__device__ __forceinline__ void mat3_vec(const double* A, const double* x, double* y) {
  for (int i = 0; i < 3; ++i) y[i] = A[3 * i] * x[0] + A[3 * i + 1] * x[1] + A[3 * i + 2] * x[2];
}

__device__ __forceinline__ void mat3T_vec(const double* A, const double* x, double* y) {
  for (int i = 0; i < 3; ++i) y[i] = A[i] * x[0] + A[3 + i] * x[1] + A[6 + i] * x[2];
}

__device__ inline Sim3d compose(const Sim3d& a, const Sim3d& b) {
  Sim3d c;
  c.s = a.s * b.s;
  mat3_mul(a.R, b.R, c.R);
  double u[3];
  mat3_vec(a.R, b.t, u);
  for (int i = 0; i < 3; ++i) c.t[i] = a.s * u[i] + a.t[i];
  return c;
}

__device__ inline Sim3d inverse(const Sim3d& a) {
  Sim3d c;
  c.s = 1.0 / a.s;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) c.R[3 * i + j] = a.R[3 * j + i];
  double u[3];
  mat3T_vec(a.R, a.t, u);
  for (int i = 0; i < 3; ++i) c.t[i] = -u[i] * c.s;
  return c;
}

__device__ inline Sim3d load(const ec3r_sim3& x) {
  Sim3d c;
  c.s = x.s;
  for (int i = 0; i < 9; ++i) c.R[i] = x.R[i];
  for (int i = 0; i < 3; ++i) c.t[i] = x.t[i];
  return c;
}

__device__ inline void store(const Sim3d& c, ec3r_sim3& x) {
  x.s = c.s;
  for (int i = 0; i < 9; ++i) x.R[i] = c.R[i];
  for (int i = 0; i < 3; ++i) x.t[i] = c.t[i];
}

__device__ inline Sim3d identity() {
  Sim3d c;
  c.s = 1.0;
  for (int i = 0; i < 9; ++i) c.R[i] = (i % 4 == 0) ? 1.0 : 0.0;
  for (int i = 0; i < 3; ++i) c.t[i] = 0.0;
  return c;
}

// Coefficients of the small-argument series of (a, b, c) below, as
// polynomials in sigma (Horner) for each power of -th2:
//   a = sum_i s^i / (i+1)!,
//   b = sum_j (-th2)^j sum_i s^i / ((2j+1)! i! (i+2j+2)),
//   c = sum_j (-th2)^j sum_i s^i / ((2j+2)! i! (i+2j+3)).
// For s^2 + th2 < 1/4 (|s| < 1/2, th2 < 1/4) 18 powers of s and 9 of th2 leave
// a truncation below 1e-19.
constexpr int VS_I = 18, VS_J = 9;
struct VSeries {
  double a[VS_I], b[VS_J][VS_I], c[VS_J][VS_I];
};
__host__ __device__ constexpr double factorial(int n) {
  double f = 1.0;
  for (int k = 2; k <= n; ++k) f *= (double)k;
  return f;
}
__host__ __device__ constexpr VSeries make_vseries() {
  VSeries t{};
  for (int i = 0; i < VS_I; ++i) {
    t.a[i] = 1.0 / factorial(i + 1);
    for (int j = 0; j < VS_J; ++j) {
      t.b[j][i] = 1.0 / (factorial(2 * j + 1) * factorial(i) * (double)(i + 2 * j + 2));
      t.c[j][i] = 1.0 / (factorial(2 * j + 2) * factorial(i) * (double)(i + 2 * j + 3));
    }
  }
  return t;
}
__constant__ constexpr VSeries c_vseries = make_vseries();

// Coefficients (a, b, c) of V = a I + b phi^ + c phi^2.
__device__ inline void v_coeffs(double sigma, double th2, double* a, double* b, double* c) {
  if (sigma * sigma + th2 < 0.25) {
    // Horner in sigma for every power of -th2 at once (independent chains),
    // then Horner in -th2; fewer powers of sigma when |sigma| is small
    const double as = fabs(sigma);
    const int ni = as < 1e-9 ? 2 : as < 1e-4 ? 5 : as < 1e-2 ? 8 : as < 0.1 ? 12 : VS_I;
    const VSeries& V = c_vseries;
    double pa = 0.0, pb[VS_J], pc[VS_J];
#pragma unroll
    for (int j = 0; j < VS_J; ++j) pb[j] = pc[j] = 0.0;
    for (int i = ni - 1; i >= 0; --i) {
      pa = fma(pa, sigma, V.a[i]);
#pragma unroll
      for (int j = 0; j < VS_J; ++j) {
        pb[j] = fma(pb[j], sigma, V.b[j][i]);
        pc[j] = fma(pc[j], sigma, V.c[j][i]);
      }
    }
    const double u = -th2;
    double sb = pb[VS_J - 1], sc = pc[VS_J - 1];
#pragma unroll
    for (int j = VS_J - 2; j >= 0; --j) {
      sb = fma(sb, u, pb[j]);
      sc = fma(sc, u, pc[j]);
    }
    *a = pa;
    *b = sb;
    *c = sc;
    return;
  }
  const double th = sqrt(th2);
  const double es = ::exp(sigma);
  const double sn = sin(th), cs = cos(th);
  const double A = (sigma == 0.0) ? 1.0 : expm1(sigma) / sigma;
  if (th2 < 1e-24) {  // pure scale: b, c from the th -> 0 limits
    // b -> int e^{su} u du, c -> int e^{su} u^2/2 du
    const double s2 = sigma * sigma;
    *a = A;
    *b = (es * (sigma - 1.0) + 1.0) / s2;
    *c = (es * (s2 - 2.0 * sigma + 2.0) - 2.0) / (2.0 * s2 * sigma);
    return;
  }
  const double d = sigma * sigma + th2;
  const double isn = (es * (sigma * sn - th * cs) + th) / d;      // int e^{su} sin(th u)
  const double ics = (es * (sigma * cs + th * sn) - sigma) / d;   // int e^{su} cos(th u)
  *a = A;
  *b = isn / th;
  *c = (A - ics) / th2;
}

__device__ inline void so3_exp(const double w[3], double R[9]) {
  const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double A, B;
  if (th2 < 1e-8) {
    A = 1.0 - th2 / 6.0 * (1.0 - th2 / 20.0);
    B = 0.5 - th2 / 24.0 * (1.0 - th2 / 30.0);
  } else {
    const double ith = rsqrt(th2);  // one rsqrt instead of sqrt and two divisions
    const double th = th2 * ith;
    double sn, cs;
    sincos(th, &sn, &cs);
    A = sn * ith;
    B = (1.0 - cs) * ith * ith;
  }
  const double x = w[0], y = w[1], z = w[2];
  R[0] = 1.0 - B * (y * y + z * z);
  R[4] = 1.0 - B * (x * x + z * z);
  R[8] = 1.0 - B * (x * x + y * y);
  R[1] = -A * z + B * x * y;
  R[3] = A * z + B * x * y;
  R[2] = A * y + B * x * z;
  R[6] = -A * y + B * x * z;
  R[5] = -A * x + B * y * z;
  R[7] = A * x + B * y * z;
}

// Rotation vector of R through its unit quaternion (stable at 0 and pi).
__device__ inline void so3_log(const double R[9], double w[3]) {
  const double tr = R[0] + R[4] + R[8];
  double q0, q1, q2, q3;
  if (tr > R[0] && tr > R[4] && tr > R[8]) {
    const double ir = rsqrt(1.0 + tr);
    q0 = 0.5 * (1.0 + tr) * ir;
    const double f = 0.5 * ir;
    q1 = (R[7] - R[5]) * f;
    q2 = (R[2] - R[6]) * f;
    q3 = (R[3] - R[1]) * f;
  } else if (R[0] >= R[4] && R[0] >= R[8]) {
    const double r = sqrt(1.0 + R[0] - R[4] - R[8]);
    q1 = 0.5 * r;
    const double f = 0.5 / r;
    q0 = (R[7] - R[5]) * f;
    q2 = (R[1] + R[3]) * f;
    q3 = (R[2] + R[6]) * f;
  } else if (R[4] >= R[8]) {
    const double r = sqrt(1.0 - R[0] + R[4] - R[8]);
    q2 = 0.5 * r;
    const double f = 0.5 / r;
    q0 = (R[2] - R[6]) * f;
    q1 = (R[1] + R[3]) * f;
    q3 = (R[5] + R[7]) * f;
  } else {
    const double r = sqrt(1.0 - R[0] - R[4] + R[8]);
    q3 = 0.5 * r;
    const double f = 0.5 / r;
    q0 = (R[3] - R[1]) * f;
    q1 = (R[2] + R[6]) * f;
    q2 = (R[5] + R[7]) * f;
  }
  if (q0 < 0.0) {
    q0 = -q0; q1 = -q1; q2 = -q2; q3 = -q3;
  }
  const double n2 = q1 * q1 + q2 * q2 + q3 * q3;
  double f;
  if (n2 < 1e-16) {
    f = 2.0 / q0 * (1.0 - n2 / (3.0 * q0 * q0));
  } else {
    const double in = rsqrt(n2);
    f = 2.0 * atan2(n2 * in, q0) * in;
  }
  w[0] = f * q1;
  w[1] = f * q2;
  w[2] = f * q3;
}

__device__ inline void v_matrix(const double phi[3], double sigma, double V[9]) {
  const double th2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
  double a, b, c;
  v_coeffs(sigma, th2, &a, &b, &c);
  const double x = phi[0], y = phi[1], z = phi[2];
  // phi^2 = phi phi^T - th2 I
  V[0] = a + c * (x * x - th2);
  V[4] = a + c * (y * y - th2);
  V[8] = a + c * (z * z - th2);
  V[1] = -b * z + c * x * y;
  V[3] = b * z + c * x * y;
  V[2] = b * y + c * x * z;
  V[6] = -b * y + c * x * z;
  V[5] = -b * x + c * y * z;
  V[7] = b * x + c * y * z;
}

__device__ inline Sim3d exp(const double xi[7]) {
  Sim3d T;
  T.s = ::exp(xi[6]);
  so3_exp(xi + 3, T.R);
  double V[9];
  v_matrix(xi + 3, xi[6], V);
  mat3_vec(V, xi, T.t);
  return T;
}

__device__ inline void log(const Sim3d& T, double xi[7]) {
  xi[6] = ::log(T.s);
  so3_log(T.R, xi + 3);
  double V[9];
  v_matrix(xi + 3, xi[6], V);
  // rho = V^-1 t (cofactor inverse)
  const double c00 = V[4] * V[8] - V[5] * V[7], c01 = V[5] * V[6] - V[3] * V[8],
               c02 = V[3] * V[7] - V[4] * V[6];
  const double c10 = V[2] * V[7] - V[1] * V[8], c11 = V[0] * V[8] - V[2] * V[6],
               c12 = V[1] * V[6] - V[0] * V[7];
  const double c20 = V[1] * V[5] - V[2] * V[4], c21 = V[2] * V[3] - V[0] * V[5],
               c22 = V[0] * V[4] - V[1] * V[3];
  const double id = 1.0 / (V[0] * c00 + V[1] * c01 + V[2] * c02);
  const double* t = T.t;
  xi[0] = (c00 * t[0] + c10 * t[1] + c20 * t[2]) * id;
  xi[1] = (c01 * t[0] + c11 * t[1] + c21 * t[2]) * id;
  xi[2] = (c02 * t[0] + c12 * t[1] + c22 * t[2]) * id;
}

}  // namespace s3
}  // namespace ec3r
