// Residual R(U) of the implicit HGKS (paper Eq. (finite), Sec. 4.1), FP64.
//
// Four kernels per evaluation, all on the caller's stream:
//  1. k_coef    one thread per (cell, conservative component): polynomial
//               coefficients of Eq. (polys) = per-cell fit matrix x stencil data
//               (non-compact: Q_k - Q_i over the big stencil; compact: Q_k - Q_i
//               of the face neighbours and the cell-averaged gradients).
//  2. k_recon   one thread per (cell, local face): characteristic projection at
//               Q* (Sec. 5), smoothness indicators and nonlinear weights of
//               Eq. (weno), values and directional derivatives at the face's 3
//               Gauss points, written in characteristic variables.
//  3. k_flux    one thread per (face, Gauss point): back-projection with the
//               face's R* (shared by both sides), positivity fallback, boundary
//               state, the BGK flux of Eq. (flux) averaged over [0, dt] and, for
//               the compact scheme, the point value of Eq. (point).
//  4. k_gather  one thread per cell: R_i = -sum of its faces' fluxes (signed),
//               compact G_new_i = sum of point values * n * S / |Omega_i|
//               (Eq. (derivative)). Gather, not scatter: no atomics, and the
//               summation order is fixed (deterministic results).
// Arrays are component-major with the cell or face index fastest, so
// consecutive threads touch consecutive addresses.
#include <cmath>
#include "hgks_internal.h"

namespace hgks {

thread_local int64_t g_launches = 0;

namespace {

constexpr int kBlock = 128;

// primitive state of a Maxwellian: lam = rho / (2 p), il = 1 / (2 lam) = p / rho, ir = 1 / rho
struct Prim { double rho, U, V, W, lam, il, ir; };

__device__ __forceinline__ Prim to_prim(const double *Q, double gamma) {
  // rho p from the conservative variables without a division; one reciprocal
  // r = 1 / (rho^2 p) then gives both 1/rho = rho p r and lam = rho / (2p) = rho^3 r / 2
  Prim p;
  p.rho = Q[0];
  const double rp = (gamma - 1.0) * (Q[4] * Q[0] - 0.5 * (Q[1] * Q[1] + Q[2] * Q[2] + Q[3] * Q[3]));   // rho p
  const double r = 1.0 / (Q[0] * rp);
  p.ir = rp * r;
  p.U = Q[1] * p.ir; p.V = Q[2] * p.ir; p.W = Q[3] * p.ir;
  p.il = rp * p.ir * p.ir;
  p.lam = 0.5 * Q[0] * Q[0] * Q[0] * r;
  return p;
}

// rotate momentum into the face frame (rows of T: n, t1, t2) and back
__device__ __forceinline__ void rot_in(const double *T, const double *in, double *out) {
  out[0] = in[0]; out[4] = in[4];
#pragma unroll
  for (int r = 0; r < 3; r++) out[1 + r] = T[3 * r] * in[1] + T[3 * r + 1] * in[2] + T[3 * r + 2] * in[3];
}
__device__ __forceinline__ void rot_out(const double *T, const double *in, double *out) {
  out[0] = in[0]; out[4] = in[4];
#pragma unroll
  for (int d = 0; d < 3; d++) out[1 + d] = T[d] * in[1] + T[3 + d] * in[2] + T[6 + d] * in[3];
}

// Euler eigen-system along x of a face-frame state: scalars from which the
// rows of R^{-1} (left) and columns of R (right) are formed.
struct Eig { double u, v, w, a, H, q2, b1, b2, ia; };
__device__ __forceinline__ Eig eig_of(const double *Q, double gamma) {
  Eig e;
  double ir = 1.0 / Q[0];
  e.u = Q[1] * ir; e.v = Q[2] * ir; e.w = Q[3] * ir;
  e.q2 = e.u * e.u + e.v * e.v + e.w * e.w;
  double p = (gamma - 1.0) * (Q[4] - 0.5 * Q[0] * e.q2);
  const double a2 = gamma * p * ir;
  e.ia = rsqrt(a2);
  e.a = a2 * e.ia;
  e.H = (Q[4] + p) * ir;
  e.b1 = (gamma - 1.0) * e.ia * e.ia;
  e.b2 = 0.5 * e.b1 * e.q2;
  return e;
}
// row c of R^{-1}
__device__ __forceinline__ void left_row(const Eig &e, int c, double *l) {
  switch (c) {
    case 0: l[0] = 0.5 * (e.b2 + e.u * e.ia); l[1] = -0.5 * (e.b1 * e.u + e.ia); l[2] = -0.5 * e.b1 * e.v; l[3] = -0.5 * e.b1 * e.w; l[4] = 0.5 * e.b1; break;
    case 1: l[0] = 1.0 - e.b2; l[1] = e.b1 * e.u; l[2] = e.b1 * e.v; l[3] = e.b1 * e.w; l[4] = -e.b1; break;
    case 2: l[0] = -e.v; l[1] = 0.0; l[2] = 1.0; l[3] = 0.0; l[4] = 0.0; break;
    case 3: l[0] = -e.w; l[1] = 0.0; l[2] = 0.0; l[3] = 1.0; l[4] = 0.0; break;
    default: l[0] = 0.5 * (e.b2 - e.u * e.ia); l[1] = -0.5 * (e.b1 * e.u - e.ia); l[2] = -0.5 * e.b1 * e.v; l[3] = -0.5 * e.b1 * e.w; l[4] = 0.5 * e.b1;
  }
}
// out = R q (characteristic -> conservative, face frame)
__device__ __forceinline__ void right_apply(const Eig &e, const double *q, double *out) {
  double s = q[0] + q[1] + q[4];
  out[0] = s;
  out[1] = e.u * s + e.a * (q[4] - q[0]);
  out[2] = e.v * s + q[2];
  out[3] = e.w * s + q[3];
  out[4] = e.H * (q[0] + q[4]) + e.u * e.a * (q[4] - q[0]) + 0.5 * e.q2 * q[1] + e.v * q[2] + e.w * q[3];
}

// ------------------------------------------------------------------------
// 1. polynomial coefficients
// ------------------------------------------------------------------------
// a real cell of a batch whose mesh still iterates (padding cells have mesh -1)
__device__ __forceinline__ bool live(const DevMesh &m, int i) {
  const int k = m.cmesh[i];
  return k >= 0 && m.mact[k];
}

// One thread per (component, cell): P0's 9 coefficients over the big stencil, then
// the four sub-stencils' 3 each over their six cells, whose differences the thread
// keeps in shared memory (its own column) from the first pass.
template <bool BATCH, class S>
__global__ void __launch_bounds__(kBlock) k_coef_weno(DevMesh m, const double *__restrict__ Q, double *__restrict__ coef) {
  constexpr int BIG = S::BIG, SUBK = S::SUBK;
  constexpr unsigned SLOTMASK = (1u << S::SLOTBITS) - 1u;
  __shared__ double sdq[BIG][kBlock];
  const int N = m.N;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int NL = BATCH ? m.NL : N;
  if (t >= 5 * NL) return;
  const int c = t / NL, i = t - c * NL;
  if (BATCH && !live(m, i)) return;
  const double qi = Q[(size_t)c * N + i];
  double a[9];
#pragma unroll
  for (int d = 0; d < 9; d++) a[d] = 0.0;
#pragma unroll
  for (int k = 0; k < BIG; k++) {
    int j = m.sten[(size_t)k * N + i];
    if (j < 0) break;
    const double dq = Q[(size_t)c * N + j] - qi;
    sdq[k][threadIdx.x] = dq;
#pragma unroll
    for (int d = 0; d < 9; d++) a[d] = fma(m.X0[(size_t)(d * BIG + k) * N + i], dq, a[d]);
  }
#pragma unroll
  for (int d = 0; d < 9; d++) coef[(size_t)(d * 5 + c) * N + i] = a[d];
#pragma unroll
  for (int mm = 0; mm < S::NSUBW; mm++) {
    const unsigned sl = m.ssl[(size_t)mm * N + i];
    double b[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int s = 0; s < SUBK; s++) {
      const double dq = sdq[(sl >> (S::SLOTBITS * s)) & SLOTMASK][threadIdx.x];
#pragma unroll
      for (int j = 0; j < 3; j++) b[j] = fma(m.Xs[(size_t)((mm * 3 + j) * SUBK + s) * N + i], dq, b[j]);
    }
#pragma unroll
    for (int j = 0; j < 3; j++) coef[(size_t)(kCoefA + (mm * 3 + j) * 5 + c) * N + i] = b[j];
  }
}

template <bool BATCH, class S>
__global__ void __launch_bounds__(kBlock) k_coef_hweno(DevMesh m, const double *__restrict__ Q, const double *__restrict__ G,
                                                        double *__restrict__ coef) {
  constexpr int NF = S::NF, HC = ShapeOf<S>::HCOLS;
  const int N = m.N;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int NL = BATCH ? m.NL : N;
  if (t >= 5 * NL) return;
  const int c = t / NL, i = t - c * NL;
  if (BATCH && !live(m, i)) return;
  const double qi = Q[(size_t)c * N + i];
  double data[HC];
  int nb[NF];
#pragma unroll
  for (int p = 0; p < NF; p++) {
    nb[p] = m.cnb[(size_t)p * N + i];
    data[p] = nb[p] >= 0 ? Q[(size_t)c * N + nb[p]] - qi : 0.0;
  }
#pragma unroll
  for (int j = 0; j < 3; j++) data[NF + j] = G[(size_t)(3 * c + j) * N + i];
#pragma unroll
  for (int p = 0; p < NF; p++)
#pragma unroll
    for (int j = 0; j < 3; j++) data[NF + 3 + 3 * p + j] = nb[p] >= 0 ? G[(size_t)(3 * c + j) * N + nb[p]] : 0.0;
#pragma unroll
  for (int d = 0; d < 9; d++) {
    double s = 0.0;
#pragma unroll
    for (int col = 0; col < HC; col++) s = fma(m.H0[(size_t)(d * HC + col) * N + i], data[col], s);
    coef[(size_t)(d * 5 + c) * N + i] = s;
  }
#pragma unroll
  for (int mm = 0; mm < NF; mm++) {
    double dm[7] = {data[mm], data[NF], data[NF + 1], data[NF + 2], data[NF + 3 + 3 * mm], data[NF + 4 + 3 * mm],
                    data[NF + 5 + 3 * mm]};
#pragma unroll
    for (int j = 0; j < 3; j++) {
      double s = 0.0;
#pragma unroll
      for (int col = 0; col < 7; col++) s = fma(m.Hm[(size_t)((mm * 3 + j) * 7 + col) * N + i], dm[col], s);
      coef[(size_t)(kCoefA + (mm * 3 + j) * 5 + c) * N + i] = s;
    }
  }
}

// ------------------------------------------------------------------------
// 2. reconstruction at the Gauss points of one face, one side
// ------------------------------------------------------------------------
template <bool BATCH, class S>
__global__ void __launch_bounds__(256) k_recon(DevMesh m, hgks_params Pv, const double *__restrict__ Q,
                                               const double *__restrict__ coef, double *__restrict__ wface) {
  constexpr int NF = S::NF, NG = S::NG, NSUB = ShapeOf<S>::NSUB;
  const int N = m.N, F = m.F;
  const int NL = BATCH ? m.NL : N;
  // block b covers local face (b mod NF) of cell range b / NF: the blocks of a
  // range run together and read its coefficients from L2 after the first
  const int slot = blockIdx.x % NF, i = (blockIdx.x / NF) * blockDim.x + threadIdx.x;
  if (i >= NL) return;
  if (BATCH && !live(m, i)) return;                     // padding cell, or a mesh that has stopped
  const hgks_params &P = BATCH ? m.ptab[m.cmesh[i]] : Pv;
  const int cf = m.cface[(size_t)slot * N + i];
  const int f = cf >> 1, side = cf & 1;
  double T[9];
#pragma unroll
  for (int k = 0; k < 9; k++) T[k] = m.fT[(size_t)k * F + f];
  const int L = m.fl[f], R = m.fr[f];
  double Qi[5], Qs[5], Qsl[5];
#pragma unroll
  for (int c = 0; c < 5; c++) {
    Qi[c] = Q[(size_t)c * N + i];
    Qs[c] = R >= 0 ? 0.5 * (Q[(size_t)c * N + L] + Q[(size_t)c * N + R]) : Qi[c];
  }
  rot_in(T, Qs, Qsl);
  const Eig e = eig_of(Qsl, P.gamma);
  const double ih = 1.0 / m.h[i];
  double m2[6], xg[3 * NG];
#pragma unroll
  for (int k = 0; k < 6; k++) m2[k] = m.m2[(size_t)k * N + i];
#pragma unroll
  for (int k = 0; k < 3 * NG; k++) xg[k] = m.xg[(size_t)(slot * 3 * NG + k) * N + i];
  // weights of the sub-stencils (compact: one per face)
  unsigned valid = P.scheme == HGKS_WENO ? m.subvalid[i] : (1u << NF) - 1u;
  const int M = __popc(valid);
  const double gm = P.lin_weight, g0 = M ? 1.0 - gm * M : 1.0;
  const double ig0 = 1.0 / g0, iM = M ? 1.0 / M : 0.0;
  double Th[9];                                         // face frame rows / h: scaled derivatives
#pragma unroll
  for (int k = 0; k < 9; k++) Th[k] = ih * T[k];
  double *out = wface + (size_t)side * NG * kFaceState * F + f;
  for (int c = 0; c < 5; c++) {
    double mr[5];
    if (P.characteristic) {
      double l[5];
      left_row(e, c, l);
      mr[0] = l[0]; mr[4] = l[4];
#pragma unroll
      for (int j = 0; j < 3; j++) mr[1 + j] = l[1] * T[j] + l[2] * T[3 + j] + l[3] * T[6 + j];
    } else {
#pragma unroll
      for (int k = 0; k < 5; k++) mr[k] = k == c ? 1.0 : 0.0;
    }
    double q0 = 0.0;
#pragma unroll
    for (int k = 0; k < 5; k++) q0 = fma(mr[k], Qi[k], q0);
    // Sub-stencil coefficients in characteristic variables: tetrahedra (4 sub-
    // stencils) keep all of them in registers; with 8 the arrays would go to local
    // memory, so hexahedra form them where they are used (twice) from the
    // coefficients, which the thread has just read (L1).
    constexpr bool kHold = NSUB <= 4;
    double ac[9], bc[kHold ? 3 * NSUB : 1];
#pragma unroll
    for (int d = 0; d < 9; d++) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < 5; k++) s = fma(mr[k], coef[(size_t)(d * 5 + k) * N + i], s);
      ac[d] = s;
    }
    if constexpr (kHold) {
#pragma unroll
      for (int d = 0; d < 3 * NSUB; d++) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < 5; k++) s = fma(mr[k], coef[(size_t)(kCoefA + d * 5 + k) * N + i], s);
        bc[d] = s;
      }
    }
    auto sub_coef = [&](int mm, double *b3) {
      if constexpr (kHold) {
#pragma unroll
        for (int j = 0; j < 3; j++) b3[j] = bc[3 * mm + j];
      } else {
#pragma unroll
        for (int j = 0; j < 3; j++) {
          double s = 0.0;
#pragma unroll
          for (int k = 0; k < 5; k++) s = fma(mr[k], coef[(size_t)(kCoefA + (3 * mm + j) * 5 + k) * N + i], s);
          b3[j] = s;
        }
      }
    };
    // smoothness indicators in the scaled frame: beta_0 = avg |grad P0|^2 + sum of squared second derivatives
    const double H00 = 2.0 * ac[3], H11 = 2.0 * ac[4], H22 = 2.0 * ac[5], H01 = ac[6], H02 = ac[7], H12 = ac[8];
    // avg |grad P0|^2 = |a|^2 + tr(M2 H^2) (M2: second moments, H symmetric)
    const double s00 = H00 * H00, s11 = H11 * H11, s22 = H22 * H22, s01 = H01 * H01, s02 = H02 * H02, s12 = H12 * H12;
    const double S00 = s00 + s01 + s02, S11 = s01 + s11 + s12, S22 = s02 + s12 + s22;
    const double S01 = fma(H00, H01, fma(H01, H11, H02 * H12));
    const double S02 = fma(H00, H02, fma(H01, H12, H02 * H22));
    const double S12 = fma(H01, H02, fma(H11, H12, H12 * H22));
    const double trMH2 = fma(m2[0], S00, fma(m2[1], S11, m2[2] * S22)) +
                         2.0 * fma(m2[3], S01, fma(m2[4], S02, m2[5] * S12));
    const double beta0 = fma(ac[0], ac[0], fma(ac[1], ac[1], ac[2] * ac[2])) + trMH2 +
                         ((s00 + s11 + s22) + (s01 + s02 + s12));
    double kap0, kap[NSUB];
    if (P.weights == HGKS_LINEAR || M == 0) {
      kap0 = 1.0;
#pragma unroll
      for (int mm = 0; mm < NSUB; mm++) kap[mm] = 0.0;
    } else {
      double beta[NSUB], tz = 0.0;
#pragma unroll
      for (int mm = 0; mm < NSUB; mm++) {
        double b3[3];
        sub_coef(mm, b3);
        beta[mm] = b3[0] * b3[0] + b3[1] * b3[1] + b3[2] * b3[2];
        if (valid >> mm & 1) tz += fabs(beta0 - beta[mm]);
      }
      tz *= iM;
      // 1 / (beta + eps) of all stencils from one division (prefix products
      // pre[k] = d0 dm[0] ... dm[k-1], then back through them)
      const double d0 = beta0 + P.weno_eps;
      double dm[NSUB], pre[NSUB + 1];
#pragma unroll
      for (int mm = 0; mm < NSUB; mm++) dm[mm] = (valid >> mm & 1) ? beta[mm] + P.weno_eps : 1.0;
      pre[0] = d0;
#pragma unroll
      for (int mm = 0; mm < NSUB; mm++) pre[mm + 1] = pre[mm] * dm[mm];
      double inv = 1.0 / pre[NSUB], r[NSUB];
#pragma unroll
      for (int mm = NSUB - 1; mm >= 0; mm--) {
        r[mm] = inv * pre[mm];
        inv *= dm[mm];
      }
      const double r0 = inv;
      double w0 = g0 * fma(tz, r0, 1.0), w[NSUB], sum = w0;
#pragma unroll
      for (int mm = 0; mm < NSUB; mm++) {
        w[mm] = (valid >> mm & 1) ? gm * fma(tz, r[mm], 1.0) : 0.0;
        sum += w[mm];
      }
      double is = 1.0 / sum;
      double wb0 = w0 * is;
      kap0 = wb0 * ig0;
#pragma unroll
      for (int mm = 0; mm < NSUB; mm++) kap[mm] = (valid >> mm & 1) ? w[mm] * is - wb0 * gm * ig0 : 0.0;
    }
    // combined polynomial: Q = kap0 P0 + sum kap_m P_m (kap0 + sum kap_m = 1)
    double lin[3];
    if constexpr (kHold) {
#pragma unroll
      for (int j = 0; j < 3; j++) {
        double s = kap0 * ac[j];
#pragma unroll
        for (int mm = 0; mm < NSUB; mm++) s = fma(kap[mm], bc[3 * mm + j], s);
        lin[j] = s;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 3; j++) lin[j] = kap0 * ac[j];
      if (kap0 != 1.0 || P.weights != HGKS_LINEAR) {
#pragma unroll
        for (int mm = 0; mm < NSUB; mm++) {
          double b3[3];
          sub_coef(mm, b3);
#pragma unroll
          for (int j = 0; j < 3; j++) lin[j] = fma(kap[mm], b3[j], lin[j]);
        }
      }
    }
    double qd[6];
#pragma unroll
    for (int k = 0; k < 6; k++) qd[k] = kap0 * ac[3 + k];
    // P(x) = q0 + lin . x + sum_k qd_k (mono_k(x) - m2_k), nested so that the value
    // and the gradient share their partial sums
    const double q0m = q0 - (qd[0] * m2[0] + qd[1] * m2[1] + qd[2] * m2[2] + qd[3] * m2[3] + qd[4] * m2[4] + qd[5] * m2[5]);
#pragma unroll
    for (int g = 0; g < NG; g++) {
      const double x = xg[3 * g], y = xg[3 * g + 1], z = xg[3 * g + 2];
      const double ax = fma(qd[0], x, fma(qd[3], y, fma(qd[4], z, lin[0])));   // lin0 + qd0 x + qd3 y + qd4 z
      const double by = fma(qd[1], y, fma(qd[5], z, lin[1]));                  // lin1 + qd1 y + qd5 z
      const double cz = fma(qd[2], z, lin[2]);                                 // lin2 + qd2 z
      const double val = fma(x, ax, fma(y, by, fma(z, cz, q0m)));
      const double gx = fma(qd[0], x, ax);
      const double gy = fma(qd[3], x, fma(qd[1], y, by));
      const double gz = fma(qd[4], x, fma(qd[5], y, fma(qd[2], z, cz)));
      double *o = out + (size_t)g * kFaceState * F;
      o[(size_t)c * F] = val;
#pragma unroll
      for (int k = 0; k < 3; k++) o[(size_t)(5 + 5 * k + c) * F] = Th[3 * k] * gx + Th[3 * k + 1] * gy + Th[3 * k + 2] * gz;
    }
  }
}

// ------------------------------------------------------------------------
// 3. gas-kinetic flux
// ------------------------------------------------------------------------
// moments of the normalised Maxwellian in u (full or half range) up to u^6
__device__ __forceinline__ void mom_u_full(const Prim &p, double *u) {
  const double il = p.il;
  u[0] = 1.0; u[1] = p.U;
#pragma unroll
  for (int n = 0; n < 5; n++) u[n + 2] = p.U * u[n + 1] + (n + 1) * il * u[n];
}
// sgn = +1: u > 0, sgn = -1: u < 0
__device__ __forceinline__ void mom_u_half(const Prim &p, double sgn, double *u) {
  // erfc(x) = erfcx(|x|) exp(-x^2) for x >= 0 and 2 - erfcx(|x|) exp(-x^2) below,
  // with the exponential that u[1] needs as well
  const double il = p.il, rs = rsqrt(p.lam), sl = p.lam * rs;
  const double x = -sgn * sl * p.U, e = exp(-p.lam * p.U * p.U);
  const double t = erfcx(fabs(x)) * e;
  u[0] = 0.5 * (x >= 0.0 ? t : 2.0 - t);
  u[1] = p.U * u[0] + sgn * 0.5 * e * rs * 0.56418958354775628695;   // 1/sqrt(pi)
#pragma unroll
  for (int n = 0; n < 5; n++) u[n + 2] = p.U * u[n + 1] + (n + 1) * il * u[n];
}

// The v, w and xi moments are taken in the frame that moves with the tangential
// velocity (V, W) of the Maxwellian: v' = v - V, w' = w - W. There they are the
// central moments of a Gaussian of variance il = 1 / (2 lambda),
//   <v'^b> = (b - 1)!! il^(b/2) for even b, 0 for odd b,   <xi^2> = K il,
//   <xi^4> = (K^2 + 2K) il^2,
// so every product with an odd tangential power vanishes and is dropped at
// compile time. The moment vectors follow from the Galilean transform psi = L psi',
//   psi_2 = psi'_2 + V psi'_0,   psi_3 = psi'_3 + W psi'_0,
//   psi_4 = psi'_4 + V psi'_2 + W psi'_3 + (V^2 + W^2)/2 psi'_0,
// as <phi psi> = L <phi psi'>; a slope enters as a . psi = (L^T a) . psi'.
struct Frame { double il, il2, K; };

// (b - 1)!!: <v'^b> / il^(b/2) for even b
__host__ __device__ constexpr double cmom(int b) { return b <= 0 ? 1.0 : (b - 1) * cmom(b - 2); }
template <int n>
__device__ __forceinline__ double il_pow(const Frame &f) {
  static_assert(n >= 0 && n <= 3, "tangential degree");
  if constexpr (n == 0) return 1.0;
  else if constexpr (n == 1) return f.il;
  else if constexpr (n == 2) return f.il2;
  else return f.il2 * f.il;
}

// out += s <u^A v'^B w'^C xi^(2E) psi'>   (E = 0 or 1; mu: moments of u)
template <int A, int B, int C, int E>
__device__ __forceinline__ void acc_c(const double *mu, const Frame &f, double s, double *out) {
  constexpr bool eb = B % 2 == 0, ec = C % 2 == 0;
  // the moment products do not depend on s: written this way they are shared by
  // every call with the same (A, B, C, E)
  if constexpr (eb && ec) {
    double t = (cmom(B) * cmom(C)) * il_pow<(B + C) / 2>(f);   // <v'^B w'^C>
    if constexpr (E == 1) t *= f.K * f.il;                       // <xi^2>
    // <... psi'_4> = 1/2 <v'^B w'^C xi^2E> (mu[A+2] + (B + C + 2 + 2E + K) il mu[A])
    constexpr double k4 = B + C + 2 + 2 * E;
    out[0] = fma(s, t * mu[A], out[0]);
    out[1] = fma(s, t * mu[A + 1], out[1]);
    out[4] = fma(s, (0.5 * t) * fma((k4 + f.K) * f.il, mu[A], mu[A + 2]), out[4]);
  } else if constexpr (!eb && ec) {
    double t = (cmom(B + 1) * cmom(C)) * il_pow<(B + C + 1) / 2>(f);
    if constexpr (E == 1) t *= f.K * f.il;
    out[2] = fma(s, t * mu[A], out[2]);
  } else if constexpr (eb && !ec) {
    double t = (cmom(B) * cmom(C + 1)) * il_pow<(B + C + 1) / 2>(f);
    if constexpr (E == 1) t *= f.K * f.il;
    out[3] = fma(s, t * mu[A], out[3]);
  }
}
// out += s <u^A v'^B w'^C (a . psi') psi'>
template <int A, int B, int C>
__device__ __forceinline__ void acc_capsi(const double *mu, const Frame &f, const double *a, double s, double *out) {
  acc_c<A, B, C, 0>(mu, f, s * a[0], out);
  acc_c<A + 1, B, C, 0>(mu, f, s * a[1], out);
  acc_c<A, B + 1, C, 0>(mu, f, s * a[2], out);
  acc_c<A, B, C + 1, 0>(mu, f, s * a[3], out);
  const double h = 0.5 * s * a[4];
  acc_c<A + 2, B, C, 0>(mu, f, h, out);
  acc_c<A, B + 2, C, 0>(mu, f, h, out);
  acc_c<A, B, C + 2, 0>(mu, f, h, out);
  acc_c<A, B, C, 1>(mu, f, h, out);
}
// out += s L x (x in the tangential frame of p)
__device__ __forceinline__ void acc_from_frame(const Prim &p, const double *x, double s, double *out) {
  const double h = 0.5 * (p.V * p.V + p.W * p.W);
  out[0] = fma(s, x[0], out[0]);
  out[1] = fma(s, x[1], out[1]);
  out[2] = fma(s, fma(p.V, x[0], x[2]), out[2]);
  out[3] = fma(s, fma(p.W, x[0], x[3]), out[3]);
  out[4] = fma(s, x[4] + p.V * x[2] + p.W * x[3] + h * x[0], out[4]);
}

// Slope a' (tangential frame) with <a . psi> = dq (moments of the Maxwellian
// normalised by rho; a is linear in dq, so dq = dW gives rho a): L^{-1} dq, then
// the closed form of the 5x5 moment system at V = W = 0. K + 3 = 2 / (gamma - 1),
// so (K + 3) / (4 lam) = il / (gamma - 1) and 4 lam^2 / (K + 3) = 2 (gamma - 1) lam^2.
__device__ __forceinline__ void slope_c(const Prim &p, double g1, double ig1, const double *dq, double *a) {
  const double d2 = dq[2] - p.V * dq[0], d3 = dq[3] - p.W * dq[0];
  const double d4 = dq[4] - p.V * d2 - p.W * d3 - 0.5 * (p.V * p.V + p.W * p.W) * dq[0];
  const double e2 = p.U * p.U + 2.0 * p.il * ig1;
  const double R1 = dq[1] - p.U * dq[0];
  const double tl = 2.0 * p.lam;
  a[4] = 2.0 * g1 * p.lam * p.lam * (2.0 * d4 - e2 * dq[0] - 2.0 * p.U * R1);
  a[3] = tl * d3;
  a[2] = tl * d2;
  a[1] = tl * R1 - p.U * a[4];
  a[0] = dq[0] - p.U * a[1] - 0.5 * a[4] * e2;
}

// boundary state outside a boundary face (face frame, x = outward normal):
// walls mirror the inner state in (p, U, V, W, T = p/rho), an isothermal wall's
// image with the density of zero mass exchange; far field = free stream
__device__ void boundary_state(const hgks_params &P, int tag, const double *T, const double *Wl, const double *dWl,
                               double *Wr, double *dWr) {
  const double g = P.gamma;
  if (tag == HGKS_BC_FARFIELD) {
    double u[3];
#pragma unroll
    for (int r = 0; r < 3; r++) u[r] = T[3 * r] * P.u_inf[0] + T[3 * r + 1] * P.u_inf[1] + T[3 * r + 2] * P.u_inf[2];
    Wr[0] = P.rho_inf;
#pragma unroll
    for (int r = 0; r < 3; r++) Wr[1 + r] = P.rho_inf * u[r];
    Wr[4] = P.p_inf / (g - 1.0) + 0.5 * P.rho_inf * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#pragma unroll
    for (int k = 0; k < 15; k++) dWr[k] = 0.0;
    return;
  }
  const double rho = Wl[0], ir = 1.0 / rho;
  double u[3] = {Wl[1] * ir, Wl[2] * ir, Wl[3] * ir};
  const double q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const double pr = (g - 1.0) * (Wl[4] - 0.5 * rho * q2), Tl = pr * ir;
  const bool T_odd = tag == HGKS_BC_WALL_ISO || tag == HGKS_BC_WALL_LID;
  bool vodd[3] = {true, tag != HGKS_BC_SLIP, tag != HGKS_BC_SLIP};
  double uw[3] = {0.0, 0.0, 0.0};
  if (tag == HGKS_BC_WALL_LID)
#pragma unroll
    for (int r = 0; r < 3; r++) uw[r] = T[3 * r] * P.lid_speed;
  double ug[3];
#pragma unroll
  for (int r = 0; r < 3; r++) ug[r] = vodd[r] ? 2.0 * uw[r] - u[r] : u[r];
  // an image colder than T_w / 2 (a cell hotter than 1.5 T_w) is held at T_w / 2, uniform
  const bool T_held = T_odd && 2.0 * P.wall_T - Tl < 0.5 * P.wall_T;
  const double Tg = T_held ? 0.5 * P.wall_T : (T_odd ? 2.0 * P.wall_T - Tl : Tl);
  // isothermal wall: the image sends back as much mass as the cell sends into the
  // wall, rho_g M(U_n, T_g) = rho M(U_n, T) with M(U, T) = <u>_{u>0} of a unit-density
  // Maxwellian = U erfc(-U / sqrt(2T)) / 2 + sqrt(T / (2 pi)) exp(-U^2 / (2T));
  // p_g = rho_g T_g, and the image keeps the cell's relative pressure gradient
  double rg, pscale = 1.0;
  if (T_odd) {
    const double Un = u[0];
    const double sl = rsqrt(2.0 * Tl), sg = rsqrt(2.0 * Tg);   // sqrt(lambda)
    const double Ml = 0.5 * Un * erfc(-sl * Un) + 0.28209479177387814347 * exp(-sl * sl * Un * Un) / sl;
    const double Mg = 0.5 * Un * erfc(-sg * Un) + 0.28209479177387814347 * exp(-sg * sg * Un * Un) / sg;
    rg = rho * Ml / Mg;
    pscale = rg * Tg / pr;
  } else {
    rg = pr / Tg;
  }
  const double pg = rg * Tg, qg2 = ug[0] * ug[0] + ug[1] * ug[1] + ug[2] * ug[2];
  Wr[0] = rg;
#pragma unroll
  for (int r = 0; r < 3; r++) Wr[1 + r] = rg * ug[r];
  Wr[4] = pg / (g - 1.0) + 0.5 * rg * qg2;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    const double *dW = dWl + 5 * d;
    double du[3], udu = 0.0;
#pragma unroll
    for (int r = 0; r < 3; r++) { du[r] = (dW[1 + r] - u[r] * dW[0]) * ir; udu += u[r] * du[r]; }
    const double dp = (g - 1.0) * (dW[4] - 0.5 * dW[0] * q2 - rho * udu);
    const double dT = (dp - Tl * dW[0]) * ir;
    const double sn = d == 0 ? -1.0 : 1.0;   // even quantities flip their normal derivative
    double dug[3], udug = 0.0;
#pragma unroll
    for (int r = 0; r < 3; r++) { dug[r] = vodd[r] ? -sn * du[r] : sn * du[r]; udug += ug[r] * dug[r]; }
    const double dpg = sn * dp * pscale, dTg = T_held ? 0.0 : (T_odd ? -sn * dT : sn * dT);
    const double drho = dpg / Tg - pg * dTg / (Tg * Tg);
    dWr[5 * d] = drho;
#pragma unroll
    for (int r = 0; r < 3; r++) dWr[5 * d + 1 + r] = drho * ug[r] + rg * dug[r];
    dWr[5 * d + 4] = dpg / (g - 1.0) + 0.5 * drho * qg2 + rg * udug;
  }
}

// out += s * J_d(W) x: the Euler flux along face-frame axis d, linearised at W
// and applied to x. For the full-range moments of a Maxwellian,
// <u_d (a_d . psi) psi> = J_d(W) dW/dx_d whenever <a_d> = dW/dx_d (a_d . psi g is the
// derivative of g along dW), which replaces the moment sums of the time slopes.
__device__ __forceinline__ void acc_jvp(const double *W, double ir, double gamma, int d, const double *x, double s,
                                        double *out) {
  const double u[3] = {W[1] * ir, W[2] * ir, W[3] * ir};
  const double q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const double p = (gamma - 1.0) * (W[4] - 0.5 * W[0] * q2);
  const double ud = u[d];
  const double dud = (x[1 + d] - ud * x[0]) * ir;
  const double dp = (gamma - 1.0) * (x[4] - (u[0] * x[1] + u[1] * x[2] + u[2] * x[3]) + 0.5 * q2 * x[0]);
  out[0] = fma(s, x[1 + d], out[0]);
#pragma unroll
  for (int i = 0; i < 3; i++) out[1 + i] = fma(s, x[1 + i] * ud + u[i] * (x[1 + d] - ud * x[0]) + (i == d ? dp : 0.0), out[1 + i]);
  out[4] = fma(s, (x[4] + dp) * ud + (W[4] + p) * dud, out[4]);
}

// Flux (time average over [0, dt] of int u psi f dXi, Eq. (flux)) and, if Qp
// is not NULL, the point value int psi f dXi at t* (Eq. (point)). Face frame.
// The moment sums of each Maxwellian are taken in its own tangential frame.
__device__ void gks_flux(const hgks_params &P, const double *Wl, const double *dWl, const double *Wr, const double *dWr,
                         double dt, double *F, double *Qp) {
  const double gam = P.gamma, g1 = gam - 1.0, ig1 = 1.0 / g1, K = (5.0 - 3.0 * gam) * ig1;
  const Prim pl = to_prim(Wl, gam), pr = to_prim(Wr, gam);
  double uhl[7], uhr[7];
  mom_u_half(pl, 1.0, uhl);
  mom_u_half(pr, -1.0, uhr);
  const Frame fl{pl.il, pl.il * pl.il, K}, fr{pr.il, pr.il * pr.il, K};
  // compatibility condition: Q0 = int_{u>0} psi g_l + int_{u<0} psi g_r
  double Q0[5] = {0, 0, 0, 0, 0};
  {
    double m[5] = {0, 0, 0, 0, 0};
    acc_c<0, 0, 0, 0>(uhl, fl, 1.0, m);
    acc_from_frame(pl, m, pl.rho, Q0);
#pragma unroll
    for (int c = 0; c < 5; c++) m[c] = 0.0;
    acc_c<0, 0, 0, 0>(uhr, fr, 1.0, m);
    acc_from_frame(pr, m, pr.rho, Q0);
  }
  const Prim p0 = to_prim(Q0, gam);
  // collision time (Sec. 5)
  const double prl = pl.rho * pl.il, prr = pr.rho * pr.il, pp0 = p0.rho * p0.il;
  const double jump = fabs((prl - prr) / (prl + prr));
  const double tau = P.viscous ? P.mu / pp0 + P.tau_C * jump * dt : (P.tau_eps + P.tau_C * jump) * dt;
  const double itau = 1.0 / tau;
  const double eta = exp(-dt * itau);
  const double c1 = dt - tau * (1.0 - eta);
  const double c2 = 2.0 * tau * tau * (1.0 - eta) - tau * dt * (1.0 + eta);
  const double c3 = 0.5 * dt * dt - tau * dt + tau * tau * (1.0 - eta);
  const double c4 = tau * (1.0 - eta);
  const double c5 = 2.0 * tau * tau * (1.0 - eta) - tau * dt * eta;
  const bool want_pt = Qp != nullptr, prandtl = P.Pr != 1.0;
  const double ts = P.tstar_end ? dt : 0.0, es = want_pt || prandtl ? exp(-ts * itau) : 1.0;
  double Fl[5] = {0, 0, 0, 0, 0}, Wb[5] = {0, 0, 0, 0, 0}, Pt[5] = {0, 0, 0, 0, 0};
  double dWs[15];
#pragma unroll
  for (int k = 0; k < 15; k++) dWs[k] = 0.5 * (dWl[k] + dWr[k]);
  // the two initial distributions g_l (u > 0) and g_r (u < 0)
#pragma unroll
  for (int s = 0; s < 2; s++) {
    const Prim &pk = s == 0 ? pl : pr;
    const Frame &fk = s == 0 ? fl : fr;
    const double *uh = s == 0 ? uhl : uhr;
    const double *dW = s == 0 ? dWl : dWr;
    const double irho = pk.ir;
    // rho a_d and rho A in the tangential frame of g_k (the slope is linear in dW, so
    // every moment sum below comes out multiplied by rho)
    double a[3][5], A[5];
#pragma unroll
    for (int d = 0; d < 3; d++) slope_c(pk, g1, ig1, dW + 5 * d, a[d]);
    // <a_n u + a_t1 v + a_t2 w + A> = 0 with <u_d (a_d.psi) psi> = J_d dW_d
    double rhs[5] = {0, 0, 0, 0, 0};
    const double *Wk = s == 0 ? Wl : Wr;
#pragma unroll
    for (int d = 0; d < 3; d++) acc_jvp(Wk, irho, gam, d, dW + 5 * d, -1.0, rhs);
    slope_c(pk, g1, ig1, rhs, A);
    // flux terms of g_k: c4 <u psi> - c5 sum_d <u u_d (a_d.psi) psi> - tau c4 <u (A.psi) psi>,
    // with v = v' + V, w = w' + W folded into the coefficients of <u (b.psi') psi'>
    double b[5], fkp[5] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int c = 0; c < 5; c++) b[c] = -tau * c4 * A[c] - c5 * (pk.V * a[1][c] + pk.W * a[2][c]);
    b[0] += c4 * pk.rho;
    acc_capsi<1, 0, 0>(uh, fk, b, 1.0, fkp);
    acc_capsi<2, 0, 0>(uh, fk, a[0], -c5, fkp);
    acc_capsi<1, 1, 0>(uh, fk, a[1], -c5, fkp);
    acc_capsi<1, 0, 1>(uh, fk, a[2], -c5, fkp);
    acc_from_frame(pk, fkp, 1.0, Fl);
    if (want_pt || prandtl) {
      // m0 = <psi>, ma = sum_d <u_d (a_d.psi) psi>, mA = <(A.psi) psi> (all times rho)
      double m0[5] = {0, 0, 0, 0, 0}, ma[5] = {0, 0, 0, 0, 0}, mA[5] = {0, 0, 0, 0, 0}, vw[5];
      acc_c<0, 0, 0, 0>(uh, fk, pk.rho, m0);
#pragma unroll
      for (int c = 0; c < 5; c++) vw[c] = pk.V * a[1][c] + pk.W * a[2][c];
      acc_capsi<0, 0, 0>(uh, fk, vw, 1.0, ma);
      acc_capsi<1, 0, 0>(uh, fk, a[0], 1.0, ma);
      acc_capsi<0, 1, 0>(uh, fk, a[1], 1.0, ma);
      acc_capsi<0, 0, 1>(uh, fk, a[2], 1.0, ma);
      acc_capsi<0, 0, 0>(uh, fk, A, 1.0, mA);
      double pt[5], wb[5];
#pragma unroll
      for (int c = 0; c < 5; c++) {
        pt[c] = es * (m0[c] - (tau + ts) * ma[c] - tau * mA[c]);
        wb[c] = c4 * m0[c] - c5 * ma[c] - tau * c4 * mA[c];
      }
      acc_from_frame(pk, pt, 1.0, Pt);
      acc_from_frame(pk, wb, 1.0, Wb);
    }
  }
  // the equilibrium part g0 with slopes from the average of both sides' gradients
  {
    const Frame f0{p0.il, p0.il * p0.il, K};
    double uf[7];
    mom_u_full(p0, uf);
    const double irho = p0.ir;
    double a[3][5];                       // rho_0 abar_d, tangential frame of g0
#pragma unroll
    for (int d = 0; d < 3; d++) slope_c(p0, g1, ig1, dWs + 5 * d, a[d]);
    // rho_0 S0 = rho_0 <(abar . u_vec) psi> = sum_d J_d(Q0) dQ0_d; <Abar psi> = -S0;
    // <u Abar psi> = -J_x(Q0) S0
    double S0[5] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int d = 0; d < 3; d++) acc_jvp(Q0, irho, gam, d, dWs + 5 * d, 1.0, S0);
    // rho_0 (c1 <u psi> + c2 sum_d <u u_d (abar_d.psi) psi> - c3 J_x(Q0) S0)
    double b[5], f0p[5] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int c = 0; c < 5; c++) b[c] = c2 * (p0.V * a[1][c] + p0.W * a[2][c]);
    b[0] += c1 * p0.rho;
    acc_capsi<1, 0, 0>(uf, f0, b, 1.0, f0p);
    acc_capsi<2, 0, 0>(uf, f0, a[0], c2, f0p);
    acc_capsi<1, 1, 0>(uf, f0, a[1], c2, f0p);
    acc_capsi<1, 0, 1>(uf, f0, a[2], c2, f0p);
    double f0v[5] = {0, 0, 0, 0, 0};
    acc_from_frame(p0, f0p, 1.0, f0v);
    acc_jvp(Q0, irho, gam, 0, S0, -c3, f0v);
#pragma unroll
    for (int c = 0; c < 5; c++) Fl[c] += f0v[c];
    if (want_pt || prandtl) {
      double g0p[5] = {0, 0, 0, 0, 0}, g0m[5] = {0, 0, 0, 0, 0};     // rho_0 <psi>
      acc_c<0, 0, 0, 0>(uf, f0, p0.rho, g0p);
      acc_from_frame(p0, g0p, 1.0, g0m);
#pragma unroll
      for (int c = 0; c < 5; c++) {
        Pt[c] += (1.0 - es) * g0m[c] + ((ts + tau) * es - tau) * S0[c] - (ts - tau + tau * es) * S0[c];
        Wb[c] += c1 * g0m[c] + c2 * S0[c] - c3 * S0[c];
      }
    }
  }
  const double idt = 1.0 / dt;
#pragma unroll
  for (int c = 0; c < 5; c++) F[c] = Fl[c] * idt;
  if (prandtl) {
    double Wt[5];
#pragma unroll
    for (int c = 0; c < 5; c++) Wt[c] = Wb[c] * idt;
    const double U = p0.U, V = p0.V, W = p0.W, q2 = U * U + V * V + W * W;
    const double q = F[4] - (U * F[1] + V * F[2] + W * F[3]) + 0.5 * q2 * F[0] - U * Wt[4] +
                     U * (U * Wt[1] + V * Wt[2] + W * Wt[3]) - 0.5 * U * q2 * Wt[0];
    F[4] += (1.0 / P.Pr - 1.0) * q;
  }
  if (want_pt)
#pragma unroll
    for (int c = 0; c < 5; c++) Qp[c] = Pt[c];
}

// rho > 0 and p > 0, the latter as rho p > 0 (no division)
__device__ __forceinline__ bool physical(const double *W, double gamma) {
  const double rp = (gamma - 1.0) * (W[4] * W[0] - 0.5 * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]));
  return W[0] > 0.0 && rp > 0.0;
}

template <bool BATCH, class S>
__global__ void __launch_bounds__(256) k_flux(DevMesh m, hgks_params Pv, const double *__restrict__ Q,
                                                  const double *__restrict__ dt, const double *__restrict__ wface,
                                                  double *__restrict__ fflux, double *__restrict__ fpt, int *__restrict__ flags) {
  constexpr int NG = S::NG;
  const int N = m.N, F = m.F;
  const int FL = BATCH ? m.FL : F;
  // block b covers Gauss point (b mod NG) of face range b / NG: the blocks of a
  // range run together and share the face's frame and cell states in L2
  const int g = blockIdx.x % NG, f = (blockIdx.x / NG) * blockDim.x + threadIdx.x;
  if (f >= FL) return;
  if (BATCH && !m.mact[m.fmesh[f]]) return;             // a mesh of a batch that has stopped
  const hgks_params &P = BATCH ? m.ptab[m.fmesh[f]] : Pv;
  double T[9];
#pragma unroll
  for (int k = 0; k < 9; k++) T[k] = m.fT[(size_t)k * F + f];
  const int L = m.fl[f], R = m.fr[f];
  double QL[5], QR[5], Qs[5], Qsl[5];
#pragma unroll
  for (int c = 0; c < 5; c++) {
    QL[c] = Q[(size_t)c * N + L];
    QR[c] = R >= 0 ? Q[(size_t)c * N + R] : QL[c];
    Qs[c] = R >= 0 ? 0.5 * (QL[c] + QR[c]) : QL[c];
  }
  rot_in(T, Qs, Qsl);
  const Eig e = eig_of(Qsl, P.gamma);
  double W[2][5], dW[2][15];
  int bad = 0;
#pragma unroll 1
  for (int s = 0; s < (R >= 0 ? 2 : 1); s++) {
    const double *in = wface + ((size_t)(s * NG + g) * kFaceState) * F + f;
    double q[5];
#pragma unroll
    for (int c = 0; c < 5; c++) q[c] = in[(size_t)c * F];
    if (P.characteristic) right_apply(e, q, W[s]);
    else rot_in(T, q, W[s]);
#pragma unroll
    for (int k = 0; k < 3; k++) {
#pragma unroll
      for (int c = 0; c < 5; c++) q[c] = in[(size_t)(5 + 5 * k + c) * F];
      if (P.characteristic) right_apply(e, q, dW[s] + 5 * k);
      else rot_in(T, q, dW[s] + 5 * k);
    }
    if (!physical(W[s], P.gamma)) {
      rot_in(T, s == 0 ? QL : QR, W[s]);
#pragma unroll
      for (int k = 0; k < 15; k++) dW[s][k] = 0.0;
      bad++;
    }
  }
  if (R < 0) boundary_state(P, m.ftag[f], T, W[0], dW[0], W[1], dW[1]);
  double dtf;
  if (P.flux_dt > 0.0) dtf = P.flux_dt;
  else dtf = (R >= 0 ? fmin(dt[L], dt[R]) : dt[L]) * (P.flux_cfl / P.cfl);
  double Fl[5], Qp[5];
  const bool compact = P.scheme == HGKS_HWENO;
  gks_flux(P, W[0], dW[0], W[1], dW[1], dtf, Fl, compact ? Qp : nullptr);
  // walls are impermeable: their faces carry momentum and energy, no mass
  if (R < 0 && m.ftag[f] >= HGKS_BC_WALL_ISO && m.ftag[f] <= HGKS_BC_NOSLIP_ADIA) Fl[0] = 0.0;
  if (bad) atomicAdd(flags, bad);
  // Gauss weight times area: 1/3 on a triangle, the area-element weight on a quadrilateral
  const double w = NG == 3 ? m.fS[f] * (1.0 / 3.0) : m.fS[f] * m.fw[(size_t)g * F + f];
  double Fg[5];
  rot_out(T, Fl, Fg);
#pragma unroll
  for (int c = 0; c < 5; c++) fflux[(size_t)(g * 5 + c) * F + f] = w * Fg[c];
  if (compact) {
    rot_out(T, Qp, Fg);
#pragma unroll
    for (int c = 0; c < 5; c++) fpt[(size_t)(g * 5 + c) * F + f] = w * Fg[c];
  }
}

// ------------------------------------------------------------------------
// 4. face -> cell
// ------------------------------------------------------------------------
template <bool BATCH, class S>
__global__ void __launch_bounds__(kBlock) k_gather(DevMesh m, int compact, const double *__restrict__ fflux,
                                                    const double *__restrict__ fpt, double *__restrict__ R,
                                                    double *__restrict__ Gnew) {
  constexpr int NF = S::NF, NG = S::NG;
  const int N = m.N, F = m.F;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (BATCH && m.cmesh[i] < 0) {                         // padding cell of a batch
#pragma unroll
    for (int c = 0; c < 5; c++) R[(size_t)c * N + i] = 0.0;
    if (compact)
#pragma unroll
      for (int k = 0; k < 15; k++) Gnew[(size_t)k * N + i] = 0.0;
    return;
  }
  if (BATCH && !m.mact[m.cmesh[i]]) return;             // a mesh of a batch that has stopped
  double r[5] = {0, 0, 0, 0, 0}, gr[15];
#pragma unroll
  for (int k = 0; k < 15; k++) gr[k] = 0.0;
#pragma unroll
  for (int p = 0; p < NF; p++) {
    const int cf = m.cface[(size_t)p * N + i];
    const int f = cf >> 1;
    const double sg = (cf & 1) ? 1.0 : -1.0;   // the flux leaves the left cell
#pragma unroll
    for (int c = 0; c < 5; c++) {
      double s = fflux[(size_t)c * F + f];
#pragma unroll
      for (int g = 1; g < NG; g++) s += fflux[(size_t)(5 * g + c) * F + f];
      r[c] = fma(sg, s, r[c]);
    }
    if (compact) {
      double n[3];
#pragma unroll
      for (int d = 0; d < 3; d++) n[d] = -sg * m.fT[(size_t)d * F + f];   // outward normal of this cell
#pragma unroll
      for (int c = 0; c < 5; c++) {
        double s = fpt[(size_t)c * F + f];
#pragma unroll
        for (int g = 1; g < NG; g++) s += fpt[(size_t)(5 * g + c) * F + f];
#pragma unroll
        for (int d = 0; d < 3; d++) gr[3 * c + d] = fma(s, n[d], gr[3 * c + d]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 5; c++) R[(size_t)c * N + i] = r[c];
  if (compact) {
    const double iv = m.inv_vol[i];
#pragma unroll
    for (int k = 0; k < 15; k++) Gnew[(size_t)k * N + i] = gr[k] * iv;
  }
}

template <bool BATCH, class S>
__global__ void k_local_dt(DevMesh m, hgks_params Pv, const double *__restrict__ Q, double *__restrict__ dt) {
  const int N = m.N, F = m.F;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (BATCH && m.cmesh[i] < 0) { dt[i] = 1.0; return; }   // padding cell of a batch
  if (BATCH && !m.mact[m.cmesh[i]]) return;
  const hgks_params &P = BATCH ? m.ptab[m.cmesh[i]] : Pv;
  double q[5];
#pragma unroll
  for (int c = 0; c < 5; c++) q[c] = Q[(size_t)c * N + i];
  const double ir = 1.0 / q[0], u = q[1] * ir, v = q[2] * ir, w = q[3] * ir;
  const double p = (P.gamma - 1.0) * (q[4] - 0.5 * q[0] * (u * u + v * v + w * w));
  const double a = sqrt(P.gamma * p * ir);
  const double nu = P.viscous ? 2.0 * P.gamma * P.mu / (P.Pr * q[0] * m.h[i]) : 0.0;
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < S::NF; k++) {
    const int f = m.cface[(size_t)k * N + i] >> 1;
    const double un = u * m.fT[f] + v * m.fT[(size_t)F + f] + w * m.fT[(size_t)2 * F + f];
    s += m.fS[f] * (fabs(un) + a + nu);
  }
  dt[i] = P.cfl * m.vol[i] / s;
}

}  // namespace

// force[3] = sum over the faces tagged `tag` of the momentum part of fflux ([3][5][F],
// global frame, area included); one block, fixed summation order
__global__ void __launch_bounds__(1024) k_wall_force(DevMesh m, int tag, int ng, const double *__restrict__ fflux,
                                                     double *__restrict__ force) {
  __shared__ double sh[3][1024];
  const int F = m.F;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int f = threadIdx.x; f < F; f += blockDim.x) {
    if (m.fr[f] >= 0 || m.ftag[f] != tag) continue;
    for (int g = 0; g < ng; g++)
#pragma unroll
      for (int d = 0; d < 3; d++) acc[d] += fflux[(size_t)(5 * g + 1 + d) * F + f];
  }
#pragma unroll
  for (int d = 0; d < 3; d++) sh[d][threadIdx.x] = acc[d];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int d = 0; d < 3; d++) sh[d][threadIdx.x] += sh[d][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int d = 0; d < 3; d++) force[d] = sh[d][0];
}

void launch_wall_force(const DevMesh &m, const Scratch &s, int tag, double *force_dev, cudaStream_t st) {
  HGKS_PROF_BEGIN(K_NORM, st);
  k_wall_force<<<1, 1024, 0, st>>>(m, tag, m.hex ? HexShape::NG : TetShape::NG, s.fflux, force_dev);
  HGKS_PROF_END(K_NORM, st);
}

void launch_local_dt(const DevMesh &m, const hgks_params &p, const double *Q, double *dt, cudaStream_t st) {
  HGKS_PROF_BEGIN(K_DT, st);
  if (m.ptab && m.hex) k_local_dt<true, HexShape><<<grid_for(m.NL, kBlock), kBlock, 0, st>>>(m, p, Q, dt);
  else if (m.ptab) k_local_dt<true, TetShape><<<grid_for(m.NL, kBlock), kBlock, 0, st>>>(m, p, Q, dt);
  else if (m.hex) k_local_dt<false, HexShape><<<grid_for(m.N, kBlock), kBlock, 0, st>>>(m, p, Q, dt);
  else k_local_dt<false, TetShape><<<grid_for(m.N, kBlock), kBlock, 0, st>>>(m, p, Q, dt);
  HGKS_PROF_END(K_DT, st);
}

namespace {
// the four residual kernels of one cell kind
template <bool BATCH, class S>
void residual_kernels(const DevMesh &m, Scratch &s, const hgks_params &p, const double *Q, const double *G, double *R,
                      double *Gnew, cudaStream_t st) {
  const int64_t NL = BATCH ? m.NL : m.N, FL = BATCH ? m.FL : m.F;
  HGKS_PROF_BEGIN(K_COEF, st);
  const unsigned gc = grid_for(5 * NL, kBlock);
  if (p.scheme == HGKS_WENO) k_coef_weno<BATCH, S><<<gc, kBlock, 0, st>>>(m, Q, s.coef);
  else k_coef_hweno<BATCH, S><<<gc, kBlock, 0, st>>>(m, Q, G, s.coef);
  HGKS_PROF_END(K_COEF, st);
  HGKS_PROF_BEGIN(K_RECON, st);
  k_recon<BATCH, S><<<S::NF * grid_for(NL, s.blk_recon), s.blk_recon, 0, st>>>(m, p, Q, s.coef, s.wface);
  HGKS_PROF_END(K_RECON, st);
  HGKS_PROF_BEGIN(K_FLUX, st);
  k_flux<BATCH, S><<<S::NG * grid_for(FL, s.blk_flux), s.blk_flux, 0, st>>>(m, p, Q, s.dt, s.wface, s.fflux, s.fpt, s.flags);
  HGKS_PROF_END(K_FLUX, st);
  HGKS_PROF_BEGIN(K_GATHER, st);
  const int grad = p.scheme == HGKS_HWENO && Gnew != nullptr;   // gradients wanted
  k_gather<BATCH, S><<<grid_for(NL, kBlock), kBlock, 0, st>>>(m, grad, s.fflux, s.fpt, R, Gnew);
  HGKS_PROF_END(K_GATHER, st);
}
}  // namespace

void launch_residual(const DevMesh &m, Scratch &s, const hgks_params &p, const double *Q, const double *G, double *R,
                     double *Gnew, cudaStream_t st, bool batch, bool fresh_dt) {
  HGKS_RANGE("hgks residual");
  batch = batch || m.ptab != nullptr;
  if (fresh_dt) launch_local_dt(m, p, Q, s.dt, st);
  if (batch && m.hex) residual_kernels<true, HexShape>(m, s, p, Q, G, R, Gnew, st);
  else if (batch) residual_kernels<true, TetShape>(m, s, p, Q, G, R, Gnew, st);
  else if (m.hex) residual_kernels<false, HexShape>(m, s, p, Q, G, R, Gnew, st);
  else residual_kernels<false, TetShape>(m, s, p, Q, G, R, Gnew, st);
}

}  // namespace hgks
