// Implicit part of one HGKS step (paper Sec. 4.1 - 4.3, Algorithm 1), FP64.
//
//  * A of Eq. (A-system-2) with the split Jacobians of Eq. (deri-matrix):
//      A_ii  = |Omega_i|/dt_i I + sum_p (J(Q_i) n_p + |lambda_p| I) S_p / 2
//      A_ij  = (J(Q_j) n_p - |lambda_p| I) S_p / 2
//    The Euler-Jacobian part of A_ii is J(Q_i) applied to sum_p n_p S_p, the
//    sum of a closed cell's outward area vectors, which is zero: A_ii is a
//    multiple of the identity and is stored as one number per cell. The
//    off-diagonal blocks form the per-cell "structure array" of Sec. 4.3,
//    stored component-major off[(p*25 + k)][N] (p = local face of the row cell)
//    so that the thread of cell i reads consecutive addresses with its warp.
//  * Jacobi preconditioner of Eq. (precond), k_max sweeps. The first sweep reads
//    D^{-1} b of the neighbours on the fly (no separate x0 pass).
//  * Restarted GMRES with modified Gram-Schmidt (Algorithm 1). Every inner
//    product finishes inside its launch: blocks write partial sums, the last
//    block to finish adds them in a fixed order (deterministic, no host round
//    trip); the first product (w, v_0) is fused into the last Jacobi sweep. The
//    Hessenberg least-squares problem (Givens rotations) runs on the device, so a
//    whole GMRES cycle is enqueued without synchronising the host.
#include <cmath>
#include <type_traits>
#include "hgks_internal.h"
#include "givens.cuh"
#include "offdiag.cuh"

namespace hgks {
namespace {

constexpr int kBlock = 256;
constexpr int kCellBlock = 128;
constexpr int kRedBlocks = 152 * 4;   // blocks of the vector reductions: a multiple of the SM count

__device__ __forceinline__ void euler_jacobian(const double *Q, const double *n, double gamma, double *J) {
  const double ir = 1.0 / Q[0];
  const double u = Q[1] * ir, v = Q[2] * ir, w = Q[3] * ir, E = Q[4] * ir;
  const double g1 = gamma - 1.0, phi = 0.5 * g1 * (u * u + v * v + w * w);
  const double un = u * n[0] + v * n[1] + w * n[2], H = gamma * E - phi;
  const double vel[3] = {u, v, w};
  J[0] = 0.0; J[1] = n[0]; J[2] = n[1]; J[3] = n[2]; J[4] = 0.0;
#pragma unroll
  for (int r = 0; r < 3; r++) {
    J[5 * (r + 1)] = phi * n[r] - vel[r] * un;
#pragma unroll
    for (int c = 0; c < 3; c++) J[5 * (r + 1) + 1 + c] = vel[r] * n[c] - g1 * vel[c] * n[r] + (r == c ? un : 0.0);
    J[5 * (r + 1) + 4] = g1 * n[r];
  }
  J[20] = (phi - H) * un;
#pragma unroll
  for (int c = 0; c < 3; c++) J[21 + c] = H * n[c] - g1 * vel[c] * un;
  J[24] = gamma * un;
}

// jv32 (may be null): FP32 operands of the product form of the off-diagonal
// blocks (mixed precision), with dval32, dinv32
template <bool BATCH, int NF>
__global__ void __launch_bounds__(kCellBlock) k_assemble(DevMesh m, hgks_params Pv, const double *__restrict__ Q,
                                                         const double *__restrict__ dt, double *__restrict__ dval,
                                                         double *__restrict__ dinv, double *__restrict__ off,
                                                         double *__restrict__ diag_out, double *__restrict__ off_out,
                                                         float *__restrict__ dval32, float *__restrict__ dinv32,
                                                         float *__restrict__ jv32) {
  const int N = m.N, F = m.F;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (BATCH && m.cmesh[i] < 0) {                          // padding cell of a batch: identity row
    dval[i] = 1.0;
    dinv[i] = 1.0;
#pragma unroll 4
    for (int k = 0; k < 25 * NF; k++) off[(size_t)k * N + i] = 0.0;
    if (jv32) {
      dval32[i] = 1.0f;
      dinv32[i] = 1.0f;
#pragma unroll 2
      for (int k = 0; k < 6 + 4 * NF; k++) jv32[(size_t)k * N + i] = 0.0f;
    }
    return;
  }
  if (BATCH && !m.mact[m.cmesh[i]]) return;             // a mesh of a batch that has stopped
  const hgks_params &P = BATCH ? m.ptab[m.cmesh[i]] : Pv;
  double Qi[5];
#pragma unroll
  for (int c = 0; c < 5; c++) Qi[c] = Q[(size_t)c * N + i];
  if (jv32) {                                           // this cell's primitives, for the rows of its neighbours
    const double ir = 1.0 / Qi[0], g1 = P.gamma - 1.0;
    const double u = Qi[1] * ir, v = Qi[2] * ir, w = Qi[3] * ir, phi = 0.5 * g1 * (u * u + v * v + w * w);
    const double pk[6] = {u, v, w, P.gamma * Qi[4] * ir - phi, phi, g1};
#pragma unroll
    for (int k = 0; k < 6; k++) jv32[(size_t)k * N + i] = (float)pk[k];
  }
  double d = m.vol[i] / dt[i];
#pragma unroll 1
  for (int p = 0; p < NF; p++) {
    const int cf = m.cface[(size_t)p * N + i], f = cf >> 1, side = cf & 1;
    const int j = m.cnb[(size_t)p * N + i];
    const double sg = side ? -1.0 : 1.0;
    double n[3];
#pragma unroll
    for (int k = 0; k < 3; k++) n[k] = sg * m.fT[(size_t)k * F + f];
    const double S = m.fS[f];
    double Qj[5], Qf[5];
#pragma unroll
    for (int c = 0; c < 5; c++) {
      Qj[c] = j >= 0 ? Q[(size_t)c * N + j] : Qi[c];
      Qf[c] = 0.5 * (Qi[c] + Qj[c]);
    }
    const double ir = 1.0 / Qf[0];
    const double u = Qf[1] * ir, v = Qf[2] * ir, w = Qf[3] * ir;
    const double pr = (P.gamma - 1.0) * (Qf[4] - 0.5 * Qf[0] * (u * u + v * v + w * w));
    double lam = fabs(u * n[0] + v * n[1] + w * n[2]) + sqrt(P.gamma * pr * ir);
    if (P.viscous) lam += 2.0 * P.mu / (Qf[0] * m.fdist[f]);
    d += 0.5 * lam * S;
    if (jv32)
#pragma unroll
      for (int k = 0; k < 4; k++)
        jv32[(size_t)(6 + 4 * p + k) * N + i] = j >= 0 ? (float)(0.5 * S * (k < 3 ? n[k] : lam)) : 0.0f;
    double J[25];
    if (j >= 0) euler_jacobian(Qj, n, P.gamma, J);
#pragma unroll
    for (int k = 0; k < 25; k++) {
      const double o = j >= 0 ? 0.5 * (J[k] - (k % 6 == 0 ? lam : 0.0)) * S : 0.0;
      off[(size_t)(p * 25 + k) * N + i] = o;
      if (off_out) off_out[(size_t)(p * 25 + k) * N + i] = o;
    }
  }
  dval[i] = d;
  dinv[i] = 1.0 / d;
  if (jv32) {
    dval32[i] = (float)d;
    dinv32[i] = (float)(1.0 / d);
  }
  if (diag_out)
#pragma unroll
    for (int k = 0; k < 25; k++) diag_out[(size_t)k * N + i] = k % 6 == 0 ? d : 0.0;
}

// Deterministic reduction: per-block partial sums, the last block adds them in
// a fixed order (strided per thread, then a fixed tree). T is the accumulation type.
template <typename T>
__device__ __forceinline__ T block_sum(T v) {
  __shared__ T sh[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  T s = T(0);
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;   // valid in thread 0
}
// *out = sum of all blocks' v (mode 0) or its square root (mode 1), stored as double
template <typename T>
__device__ __forceinline__ void grid_sum(T v, T *partials, unsigned int *count, double *out, int mode) {
  __shared__ bool last;
  const T bs = block_sum(v);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = bs;
    __threadfence();
    const unsigned int prev = atomicAdd(count, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  T s = T(0);
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) s += ((volatile T *)partials)[b];
  s = block_sum(s);
  if (threadIdx.x == 0) {
    *out = mode == 1 ? (double)sqrt(s) : (double)s;
    *count = 0u;
  }
}

// One product with the off-diagonal part of A. Modes:
//   kSpmv   : y = [b -] (d x + sum_p A_ip x_p)
//   kJacobi : y = D^{-1} (b - sum_p A_ip x_p); FirstSweep: x_p = D^{-1} b at the neighbours
//   kNeumann: y = b + D^{-1} sum_p A_ip x_p
//   kE, kNegE: y = +- D^{-1} sum_p A_ip x_p
// and optionally the inner product (y, dotv) reduced into *dot_out.
// TM: type of the stored blocks, TV: type of b and x (and of the accumulation),
// TO: type of y.
enum { kSpmv = 0, kJacobi = 1, kNeumann = 2, kE = 3, kNegE = 4 };

// TM = float: the off-diagonal blocks come as products from jv (mixed precision);
// TM = double: stored 5x5 blocks in off.
template <typename TM, typename TV, typename TO, int Mode, bool FirstSweep, int NF>
__global__ void __launch_bounds__(kCellBlock) k_apply(DevMesh m, const TM *__restrict__ off, const TM *__restrict__ dval,
                                                      const TM *__restrict__ dinv, const TV *__restrict__ b,
                                                      const TV *__restrict__ x, TO *__restrict__ y,
                                                      const TO *__restrict__ dotv, TO *partials, unsigned int *count,
                                                      double *dot_out) {
  const int N = m.N;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  TO part = TO(0);
  if (i < N) {
    TV acc[5];
    const TV di = Mode == kSpmv ? (TV)dval[i] : TV(0);
#pragma unroll
    for (int r = 0; r < 5; r++) acc[r] = Mode == kSpmv ? di * x[(size_t)r * N + i] : TV(0);
#pragma unroll
    for (int p = 0; p < NF; p++) {
      const int j = m.cnb[(size_t)p * N + i];
      if (j < 0) continue;
      TV xj[5];
      const TV sj = FirstSweep ? (TV)dinv[j] : TV(1);
#pragma unroll
      for (int c = 0; c < 5; c++) xj[c] = FirstSweep ? sj * b[(size_t)c * N + j] : x[(size_t)c * N + j];
      if constexpr (std::is_same<TM, float>::value) {
        offdiag_product<TV>(reinterpret_cast<const float *>(off), N, i, p, j, xj, acc);
      } else {
        const TM *O = off + (size_t)p * 25 * N + i;
#pragma unroll
        for (int r = 0; r < 5; r++)
#pragma unroll
          for (int c = 0; c < 5; c++) {
            if (r == 0 && c == 4) continue;     // row 0 of J(Q)n is (0, n, 0): this entry is zero
            acc[r] = fma((TV)O[(size_t)(5 * r + c) * N], xj[c], acc[r]);
          }
      }
    }
    TV out[5];
    if (Mode == kJacobi) {
      const TV dd = (TV)dinv[i];
#pragma unroll
      for (int r = 0; r < 5; r++) out[r] = dd * (b[(size_t)r * N + i] - acc[r]);
    } else if (Mode == kE || Mode == kNegE) {
      const TV dd = Mode == kE ? (TV)dinv[i] : -(TV)dinv[i];
#pragma unroll
      for (int r = 0; r < 5; r++) out[r] = dd * acc[r];
    } else if (Mode == kNeumann) {
      const TV dd = (TV)dinv[i];
#pragma unroll
      for (int r = 0; r < 5; r++) out[r] = fma(dd, acc[r], b[(size_t)r * N + i]);
    } else if (b) {
#pragma unroll
      for (int r = 0; r < 5; r++) out[r] = b[(size_t)r * N + i] - acc[r];
    } else {
#pragma unroll
      for (int r = 0; r < 5; r++) out[r] = acc[r];
    }
#pragma unroll
    for (int r = 0; r < 5; r++) {
      const TO o = (TO)out[r];
      y[(size_t)r * N + i] = o;
      if (dotv) part = fma(o, dotv[(size_t)r * N + i], part);
    }
  }
  if (dotv) grid_sum(part, partials, count, dot_out, 0);
}

// k_apply for the mesh's cell kind (4 or 6 off-diagonal blocks per row)
template <typename TM, typename TV, typename TO, int Mode, bool FirstSweep>
void apply_launch(unsigned grid, cudaStream_t st, const DevMesh &m, const TM *off, const TM *dval, const TM *dinv,
                  const TV *b, const TV *x, TO *y, const TO *dotv, TO *partials, unsigned int *count, double *dot_out) {
  if (m.hex)
    k_apply<TM, TV, TO, Mode, FirstSweep, HexShape::NF><<<grid, kCellBlock, 0, st>>>(m, off, dval, dinv, b, x, y, dotv,
                                                                                      partials, count, dot_out);
  else
    k_apply<TM, TV, TO, Mode, FirstSweep, TetShape::NF><<<grid, kCellBlock, 0, st>>>(m, off, dval, dinv, b, x, y, dotv,
                                                                                      partials, count, dot_out);
}

template <typename T>
__global__ void k_diag_scale(int N, const T *__restrict__ dinv, const T *__restrict__ b, T *__restrict__ x) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 5 * N) return;
  x[t] = dinv[t % N] * b[t];
}

// 16-byte vectors of T: every Krylov vector starts on a 256-byte boundary
// (vectors are padded to a multiple of 64 elements) and so do the device arrays
// the reductions read.
template <typename T> struct Vec16;
template <> struct Vec16<double> { typedef double2 type; static constexpr int n = 2; };
template <> struct Vec16<float> { typedef float4 type; static constexpr int n = 4; };

// w -= h v (if v != nullptr); *out = (w, x) (mode 0) or ||w|| (x == w, mode 1).
// In mode 1 nothing is read through x, so callers may pass w itself for it
// without breaking the restrict qualifiers.
// 16 bytes per vector per thread and step, four steps in flight; n need not be
// a multiple of the vector width.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_axpy_dot(int64_t n, T *__restrict__ w, const T *__restrict__ v,
                                                     const double *__restrict__ h, const T *__restrict__ x,
                                                     int self, T *partials, unsigned int *count, double *out) {
  typedef typename Vec16<T>::type TV;
  constexpr int L = Vec16<T>::n;
  const T hv = v ? (T)(-*h) : T(0);
  T s = T(0);
  const int64_t nv = n / L, stride = (int64_t)gridDim.x * blockDim.x;
  TV *wv = reinterpret_cast<TV *>(w);
  const TV *vv = reinterpret_cast<const TV *>(v);
  const TV *xv = reinterpret_cast<const TV *>(x);
#pragma unroll 4
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nv; k += stride) {
    TV wk = wv[k];
    T *wa = reinterpret_cast<T *>(&wk);
    if (v) {
      const TV vk = vv[k];
      const T *va = reinterpret_cast<const T *>(&vk);
#pragma unroll
      for (int l = 0; l < L; l++) wa[l] = fma(hv, va[l], wa[l]);
      wv[k] = wk;
    }
    if (self) {
#pragma unroll
      for (int l = 0; l < L; l++) s = fma(wa[l], wa[l], s);
    } else {
      const TV xk = xv[k];
      const T *xa = reinterpret_cast<const T *>(&xk);
#pragma unroll
      for (int l = 0; l < L; l++) s = fma(wa[l], xa[l], s);
    }
  }
  for (int64_t k = nv * L + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += stride) {
    T wk = w[k];
    if (v) { wk = fma(hv, v[k], wk); w[k] = wk; }
    s = fma(wk, self ? wk : x[k], s);
  }
  grid_sum(s, partials, count, out, self);
}

// ---- modified Gram-Schmidt from one pass over the basis ----
// Algorithm 1 orthogonalises w against v_0..v_j one vector after the other:
// h_i = (w_i, v_i), w_{i+1} = w_i - h_i v_i. Since w_i = w - sum_{k<i} h_k v_k,
//   h_i = a_i - sum_{k<i} h_k G_ki,  a_i = (w, v_i),  G_ki = (v_k, v_i),
// so one pass over the basis (k_mdot: all a_i, and the new row of G, v_j against
// the older vectors) and a forward substitution (k_mgs_coef) give the same
// coefficients, and one more pass (k_mupdate) subtracts them in MGS order and
// takes ||w||: about 2 (j + 1) vector passes instead of 4 (j + 1) for step j
// (used with FP32 vectors, see gmres_t).
constexpr int kMdot = 8;              // basis vectors per k_mdot launch (register accumulators)

// a[k] = (w, v_k) for k in [k0, k0 + nk), and g[k] = (v_j, v_k) for those k < j
template <typename T>
__global__ void __launch_bounds__(kBlock) k_mdot(int64_t n, const T *__restrict__ w, const T *__restrict__ V, int64_t vs,
                                                 int k0, int nk, int j, T *partials, unsigned int *count,
                                                 double *__restrict__ a, double *__restrict__ g) {
  typedef typename Vec16<T>::type TV;
  constexpr int L = Vec16<T>::n;
  T sa[kMdot], sg[kMdot];
#pragma unroll
  for (int q = 0; q < kMdot; q++) { sa[q] = T(0); sg[q] = T(0); }
  const int64_t nv = n / L, stride = (int64_t)gridDim.x * blockDim.x;
  const TV *wv = reinterpret_cast<const TV *>(w);
  const TV *jv = reinterpret_cast<const TV *>(V + (size_t)j * vs);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nv; k += stride) {
    const TV wk = wv[k], vj = jv[k];
    const T *wa = reinterpret_cast<const T *>(&wk);
    const T *ja = reinterpret_cast<const T *>(&vj);
#pragma unroll
    for (int q = 0; q < kMdot; q++) {
      if (q < nk) {
        const TV vk = reinterpret_cast<const TV *>(V + (size_t)(k0 + q) * vs)[k];
        const T *va = reinterpret_cast<const T *>(&vk);
#pragma unroll
        for (int l = 0; l < L; l++) sa[q] = fma(wa[l], va[l], sa[q]);
        if (k0 + q < j)
#pragma unroll
          for (int l = 0; l < L; l++) sg[q] = fma(ja[l], va[l], sg[q]);
      }
    }
  }
  for (int64_t k = nv * L + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += stride) {
    const T wk = w[k], vj = V[(size_t)j * vs + k];
#pragma unroll
    for (int q = 0; q < kMdot; q++)
      if (q < nk) {
        const T vk = V[(size_t)(k0 + q) * vs + k];
        sa[q] = fma(wk, vk, sa[q]);
        if (k0 + q < j) sg[q] = fma(vj, vk, sg[q]);
      }
  }
  // per block: 2 kMdot partials; the last block adds every slot's partials in block order
  __shared__ bool last;
#pragma unroll
  for (int q = 0; q < 2 * kMdot; q++) {
    const T bs = block_sum(q < kMdot ? sa[q] : sg[q - kMdot]);
    if (threadIdx.x == 0) partials[(size_t)q * gridDim.x + blockIdx.x] = bs;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    last = (atomicAdd(count, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int q = 0; q < 2 * kMdot; q++) {
    const int kk = k0 + (q % kMdot);
    const bool want = (q % kMdot) < nk && (q < kMdot || kk < j);   // uniform over the block
    if (!want) continue;
    T sum = T(0);
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) sum += ((volatile T *)partials)[(size_t)q * gridDim.x + b];
    sum = block_sum(sum);
    if (threadIdx.x == 0) (q < kMdot ? a : g)[kk] = (double)sum;
  }
  if (threadIdx.x == 0) *count = 0u;
}

// the MGS coefficients of step j by forward substitution; column j of H and row
// j of the basis Gram matrix G (leading dimension kGramLd, G[k][i] = (v_k, v_i), k < i)
constexpr int kGramLd = 65;
__global__ void k_mgs_coef(int j, int mk, const double *__restrict__ a, const double *__restrict__ g,
                           double *__restrict__ G, double *__restrict__ H) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int k = 0; k < j; k++) G[k * kGramLd + j] = g[k];
  for (int i = 0; i <= j; i++) {
    double h = a[i];
    for (int k = 0; k < i; k++) h -= H[k * mk + j] * G[k * kGramLd + i];
    H[i * mk + j] = h;
  }
}

// w -= sum_{k <= j} h_kj v_k in the order of k (MGS order), then h_{j+1,j} = ||w||
template <typename T>
__global__ void __launch_bounds__(kBlock) k_mupdate(int64_t n, T *__restrict__ w, const T *__restrict__ V, int64_t vs,
                                                    int j, int mk, const double *__restrict__ H, T *partials,
                                                    unsigned int *count, double *norm_out) {
  typedef typename Vec16<T>::type TV;
  constexpr int L = Vec16<T>::n;
  __shared__ T nh[kGramLd];
  for (int k = threadIdx.x; k <= j; k += blockDim.x) nh[k] = (T)(-H[k * mk + j]);
  __syncthreads();
  T s = T(0);
  const int64_t nv = n / L, stride = (int64_t)gridDim.x * blockDim.x;
  TV *wv = reinterpret_cast<TV *>(w);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nv; k += stride) {
    TV wk = wv[k];
    T *wa = reinterpret_cast<T *>(&wk);
#pragma unroll 4
    for (int q = 0; q <= j; q++) {
      const TV vk = reinterpret_cast<const TV *>(V + (size_t)q * vs)[k];
      const T *va = reinterpret_cast<const T *>(&vk);
#pragma unroll
      for (int l = 0; l < L; l++) wa[l] = fma(nh[q], va[l], wa[l]);
    }
    wv[k] = wk;
#pragma unroll
    for (int l = 0; l < L; l++) s = fma(wa[l], wa[l], s);
  }
  for (int64_t k = nv * L + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += stride) {
    T wk = w[k];
    for (int q = 0; q <= j; q++) wk = fma(nh[q], V[(size_t)q * vs + k], wk);
    w[k] = wk;
    s = fma(wk, wk, s);
  }
  grid_sum(s, partials, count, norm_out, 1);
}

// ---- modified Gram-Schmidt two basis vectors per pass (FP64 vectors) ----
// For a pair (v_c, v_{c+1}) Algorithm 1 takes h_c = (w_c, v_c) and
//   h_{c+1} = (w_c - h_c v_c, v_{c+1}) = (w_c, v_{c+1}) - h_c g_c,  g_c = (v_c, v_{c+1}),
// so one pass over w, v_c and v_{c+1} gives both coefficients. The same pass first
// subtracts the previous pair (v_a, v_b) with its known coefficients, in MGS
// order. The last pass of step j (vc == nullptr) subtracts the last vectors and
// takes ||w|| and (w, v_j): then g_j = (v_j, w / ||w||) = (v_j, v_{j+1}) for the
// steps that follow. Per pair 48 bytes and 4 FMAs per element (24 bytes per basis
// vector against 32 for one vector per pass) keep the pass bound by HBM.
//   update: w -= ha va; if vb: w -= hb vb
//   vc:     *hc_out = (w, vc); if vd: *hd_out = (w, vd) - (w, vc) * *g_io
//   !vc:    *hc_out = ||w||; *g_io = (w, vlast) / ||w|| (0 if ||w|| == 0), vlast = vb ? vb : va
template <typename T, int NB, int ND>
__global__ void __launch_bounds__(kBlock) k_mgs2(int64_t n, T *__restrict__ w, const T *__restrict__ va,
                                                 const T *__restrict__ vb, const double *__restrict__ ha,
                                                 const double *__restrict__ hb, const T *__restrict__ vc,
                                                 const T *__restrict__ vd, T *partials, unsigned int *count,
                                                 double *hc_out, double *hd_out, double *g_io) {
  // NB: vectors subtracted (1: va, 2: va and vb); ND: vectors dotted (0: the last
  // pass, 1: vc, 2: vc and vd)
  typedef typename Vec16<T>::type TV;
  constexpr int L = Vec16<T>::n;
  constexpr bool fin = ND == 0;
  const T na = (T)(-*ha), nb = NB == 2 ? (T)(-*hb) : T(0);
  // the vectors of the two sums: (w, x0) and (w, x1); the last pass: x0 = w, x1 = vlast
  const T *x1 = fin ? (NB == 2 ? vb : va) : vd;
  T s0 = T(0), s1 = T(0);
  const int64_t nv = n / L, stride = (int64_t)gridDim.x * blockDim.x;
  const TV *VA = reinterpret_cast<const TV *>(va), *VB = reinterpret_cast<const TV *>(vb);
  const TV *VC = reinterpret_cast<const TV *>(vc), *X1 = reinterpret_cast<const TV *>(x1);
  TV *WV = reinterpret_cast<TV *>(w);
#pragma unroll 2
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nv; k += stride) {
    // every load of the step first (w is written only after them)
    TV wk = WV[k];
    const TV ak = VA[k];
    TV bk, ck, xk;
    if constexpr (NB == 2) bk = VB[k];
    if constexpr (!fin) ck = VC[k];
    if constexpr (fin || ND == 2) xk = X1[k];
    T *wa = reinterpret_cast<T *>(&wk);
    const T *aa = reinterpret_cast<const T *>(&ak);
#pragma unroll
    for (int l = 0; l < L; l++) wa[l] = fma(na, aa[l], wa[l]);
    if constexpr (NB == 2) {
      const T *ba = reinterpret_cast<const T *>(&bk);
#pragma unroll
      for (int l = 0; l < L; l++) wa[l] = fma(nb, ba[l], wa[l]);
    }
    if constexpr (fin) {
#pragma unroll
      for (int l = 0; l < L; l++) s0 = fma(wa[l], wa[l], s0);
    } else {
      const T *ca = reinterpret_cast<const T *>(&ck);
#pragma unroll
      for (int l = 0; l < L; l++) s0 = fma(wa[l], ca[l], s0);
    }
    if constexpr (fin || ND == 2) {
      const T *xa = reinterpret_cast<const T *>(&xk);
#pragma unroll
      for (int l = 0; l < L; l++) s1 = fma(wa[l], xa[l], s1);
    }
    WV[k] = wk;
  }
  for (int64_t k = nv * L + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += stride) {
    T wk = fma(na, va[k], w[k]);
    if constexpr (NB == 2) wk = fma(nb, vb[k], wk);
    w[k] = wk;
    s0 = fma(wk, fin ? wk : vc[k], s0);
    if constexpr (fin || ND == 2) s1 = fma(wk, x1[k], s1);
  }
  // deterministic reduction of both sums (as grid_sum)
  __shared__ bool last;
  const T b0 = block_sum(s0);
  const T b1 = block_sum(s1);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = b0;
    partials[gridDim.x + blockIdx.x] = b1;
    __threadfence();
    const unsigned int prev = atomicAdd(count, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  T t0 = T(0), t1 = T(0);
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    t0 += ((volatile T *)partials)[b];
    t1 += ((volatile T *)partials)[gridDim.x + b];
  }
  t0 = block_sum(t0);
  t1 = block_sum(t1);
  if (threadIdx.x == 0) {
    if (fin) {
      const double nrm = sqrt((double)t0);
      *hc_out = nrm;
      *g_io = nrm > 0.0 ? (double)t1 / nrm : 0.0;
    } else {
      *hc_out = (double)t0;
      if (ND == 2) *hd_out = (double)t1 - (double)t0 * *g_io;
    }
    *count = 0u;
  }
}

// one pass of the pair MGS with the instance for the number of vectors
template <typename T>
void launch_mgs2(cudaStream_t st, int64_t n, T *w, const T *va, const T *vb, const double *ha, const double *hb,
                 const T *vc, const T *vd, T *partials, unsigned int *count, double *hc_out, double *hd_out,
                 double *g_io) {
  const int nb = vb ? 2 : 1, nd = vc ? (vd ? 2 : 1) : 0;
#define HGKS_MGS2(NB, ND)                                                                                        \
  k_mgs2<T, NB, ND><<<kRedBlocks, kBlock, 0, st>>>(n, w, va, vb, ha, hb, vc, vd, partials, count, hc_out, hd_out, \
                                                   g_io)
  if (nb == 1 && nd == 0) HGKS_MGS2(1, 0);
  else if (nb == 1 && nd == 1) HGKS_MGS2(1, 1);
  else if (nb == 1) HGKS_MGS2(1, 2);
  else if (nd == 0) HGKS_MGS2(2, 0);
  else if (nd == 1) HGKS_MGS2(2, 1);
  else HGKS_MGS2(2, 2);
#undef HGKS_MGS2
}

// v = w / h (v = 0 after a breakdown h == 0), 16 bytes per thread and step
template <typename T>
__global__ void k_scale(int64_t n, const T *__restrict__ w, const double *__restrict__ h, T *__restrict__ v) {
  typedef typename Vec16<T>::type TV;
  constexpr int L = Vec16<T>::n;
  const double hv = *h;
  const T ih = hv != 0.0 ? (T)(1.0 / hv) : T(0);
  const int64_t nv = n / L, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nv; k += stride) {
    TV x = reinterpret_cast<const TV *>(w)[k];
    T *xa = reinterpret_cast<T *>(&x);
#pragma unroll
    for (int l = 0; l < L; l++) xa[l] *= ih;
    reinterpret_cast<TV *>(v)[k] = x;
  }
  for (int64_t k = nv * L + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += stride) v[k] = w[k] * ih;
}

// y minimises || beta e1 - H y || (Givens rotations in place on H, one thread, FP64)
__global__ void k_givens(int m, double *__restrict__ H, const double *__restrict__ beta, double *__restrict__ y,
                         double *__restrict__ res_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  *res_out = givens_lsq(m, H, *beta, y);
}

// dx += sum_j y_j V_j (FP64 accumulation in the order of j; V of either
// precision, stride vs, read 16 bytes per vector and step)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_combine(int64_t n, int64_t vs, int m, const T *__restrict__ V,
                                                    const double *__restrict__ y, double *__restrict__ dx) {
  typedef typename Vec16<T>::type TV;
  constexpr int L = Vec16<T>::n;
  __shared__ double ys[kGramLd];
  for (int j = threadIdx.x; j < m; j += blockDim.x) ys[j] = y[j];
  __syncthreads();
  const int64_t nv = n / L, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nv; k += stride) {
    double acc[L];
#pragma unroll
    for (int l = 0; l < L; l++) acc[l] = dx[k * L + l];
#pragma unroll 4
    for (int j = 0; j < m; j++) {
      const TV v = reinterpret_cast<const TV *>(V + (size_t)j * vs)[k];
      const T *va = reinterpret_cast<const T *>(&v);
#pragma unroll
      for (int l = 0; l < L; l++) acc[l] = fma(ys[j], (double)va[l], acc[l]);
    }
#pragma unroll
    for (int l = 0; l < L; l++) dx[k * L + l] = acc[l];
  }
  for (int64_t k = nv * L + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += stride) {
    double acc = dx[k];
    for (int j = 0; j < m; j++) acc = fma(ys[j], (double)V[(size_t)j * vs + k], acc);
    dx[k] = acc;
  }
}

__global__ void __launch_bounds__(kBlock) k_density_l1(int N, const double *__restrict__ R, const double *__restrict__ inv_vol,
                                                       double *partials, unsigned int *count, double *out) {
  double s = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) s += fabs(R[k]) * inv_vol[k];
  grid_sum<double>(s, partials, count, out, 0);
}

__global__ void k_update(int64_t n5, int64_t ng, double *__restrict__ Q, const double *__restrict__ dQ, double *__restrict__ G,
                         const double *__restrict__ Gnew, double relax) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n5 + ng; k += (int64_t)gridDim.x * blockDim.x) {
    if (k < n5) Q[k] += dQ[k];
    else if (relax == 1.0) G[k - n5] = Gnew[k - n5];
    else G[k - n5] = fma(relax, Gnew[k - n5] - G[k - n5], G[k - n5]);
  }
}

// ---- matrix-free products (jv_mode 1), Eq. (frechet) ----
// Qp = Q + sigma x, sigma = sqrt(eps_mach) (1 + ||Q||) / ||x|| (0 for x = 0); nrm = {||Q||, ||x||, sigma}
template <typename TV>
__global__ void k_fd_perturb(int64_t n, const double *__restrict__ Q, const TV *__restrict__ x, double *__restrict__ nrm,
                             double *__restrict__ Qp) {
  const double nx = nrm[1];
  const double sigma = nx > 0.0 ? 0x1p-26 * (1.0 + nrm[0]) / nx : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) nrm[2] = sigma;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    Qp[k] = Q[k] + sigma * (double)x[k];
}

// y = A x or b - A x, A x = |Omega_i|/dt_i x - (L(Qp) - L(Q)) / sigma (A x = 0 when sigma = 0)
template <typename TV, typename TO>
__global__ void k_fd_combine(int N, const double *__restrict__ vol, const double *__restrict__ dt, const TV *__restrict__ x,
                             const double *__restrict__ Rp, const double *__restrict__ R0, const double *__restrict__ sig,
                             const double *__restrict__ b, TO *__restrict__ y) {
  const double sigma = *sig;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < 5 * (int64_t)N; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = k % N;
    const double ax = sigma > 0.0 ? vol[i] / dt[i] * (double)x[k] - (Rp[k] - R0[k]) / sigma : 0.0;
    y[k] = (TO)(b ? b[k] - ax : ax);
  }
}

unsigned vec_grid(int64_t n) {
  int64_t g = (n + kBlock - 1) / kBlock;
  const int64_t cap = 152 * 8;
  return (unsigned)std::max<int64_t>(1, std::min(g, cap));
}

// Buffers of one precision for the Krylov part of a step.
template <typename T>
struct KBuf {
  const T *off, *dval, *dinv;
  T *V, *w, *t, *t2, *red;
};
KBuf<double> kbuf64(Scratch &s) { return {s.off, s.dval, s.dinv, s.V, s.w, s.t, s.t2, s.red}; }
KBuf<float> kbuf32(Scratch &s) { return {s.jv32, s.dval32, s.dinv32, s.V32, s.w32, s.t32, s.t232, s.red32}; }

template <typename T> T *partials(Scratch &s);
template <> double *partials<double>(Scratch &s) { return s.red; }
template <> float *partials<float>(Scratch &s) { return s.red32; }

// y = A x (b null) or b - A x with the matrix-free A of Eq. (frechet); s.R = L(Q), s.dt, ||Q|| in hs
template <typename TV, typename TO>
void fd_apply(const DevMesh &m, Scratch &s, const hgks_params &p, const double *Q, const double *G, const TV *x,
              const double *b, TO *y, cudaStream_t st) {
  const int64_t n = 5 * (int64_t)m.N;
  double *nrm = s.hs + kHsNormQ;
  HGKS_PROF_BEGIN(K_DOT, st);
  k_axpy_dot<TV><<<kRedBlocks, kBlock, 0, st>>>(n, const_cast<TV *>(x), nullptr, nullptr, x, 1, partials<TV>(s),
                                                 s.red_count, nrm + 1);
  HGKS_PROF_END(K_DOT, st);
  HGKS_PROF_BEGIN(K_SPMV, st);
  k_fd_perturb<TV><<<vec_grid(n), kBlock, 0, st>>>(n, Q, x, nrm, s.Qp);
  HGKS_PROF_END(K_SPMV, st);
  launch_residual(m, s, p, s.Qp, G, s.Rp, nullptr, st, false, false);
  HGKS_PROF_BEGIN(K_SPMV, st);
  k_fd_combine<TV, TO><<<vec_grid(n), kBlock, 0, st>>>(m.N, m.vol, s.dt, x, s.Rp, s.R, nrm + 2, b, y);
  HGKS_PROF_END(K_SPMV, st);
}

// x = P^{-1} b (Eq. (precond)); if dotv is given, also (x, dotv) into *dot_out.
template <typename T>
void precondition_t(const DevMesh &m, Scratch &s, const KBuf<T> &k, int sweeps, const T *b, T *x, const T *dotv,
                    double *dot_out, cudaStream_t st) {
  const unsigned cg = grid_for(m.N, kCellBlock);
  if (sweeps == 0) {
    HGKS_PROF_BEGIN(K_DIAG, st);
    k_diag_scale<T><<<grid_for(5 * (int64_t)m.N, kBlock), kBlock, 0, st>>>(m.N, k.dinv, b, x);
    HGKS_PROF_END(K_DIAG, st);
    if (dotv) {
      HGKS_PROF_BEGIN(K_DOT, st);
      k_axpy_dot<T><<<kRedBlocks, kBlock, 0, st>>>(5 * (int64_t)m.N, x, nullptr, nullptr, dotv, 0, k.red, s.red_count, dot_out);
      HGKS_PROF_END(K_DOT, st);
    }
    return;
  }
  // sweep k writes to x when (sweeps - k) is even, else to t2: the last lands in x
  const T *prev = nullptr;
  for (int q = 1; q <= sweeps; q++) {
    T *dst = ((sweeps - q) % 2 == 0) ? x : k.t2;
    const T *dv = (q == sweeps) ? dotv : nullptr;
    HGKS_PROF_BEGIN(K_JACOBI, st);
    if (q == 1)
      apply_launch<T, T, T, kJacobi, true>(cg, st, m, k.off, k.dval, k.dinv, b, nullptr, dst, dv, k.red,
                                                                  s.red_count, dot_out);
    else
      apply_launch<T, T, T, kJacobi, false>(cg, st, m, k.off, k.dval, k.dinv, b, prev, dst, dv, k.red,
                                                                   s.red_count, dot_out);
    HGKS_PROF_END(K_JACOBI, st);
    prev = dst;
  }
}

// w = P^{-1} A v for a Krylov vector v, with the operator of precondition_t after
// the product with A. Write A = D (I + E), E = D^{-1} O (O: the off-diagonal
// blocks); the Jacobi iteration started from D^{-1} (A v) gives after k sweeps
// P^{-1} A v = v - (-E)^(k+1) v, i.e. w = v + E z with z = (-E)^k v (formed as
// E^k v with the sign in its first product): k + 1
// products with O instead of the product with A followed by k sweeps: the same
// vector up to rounding, without the diagonal terms of A and the scaling of the
// neighbours' values by D^{-1}. The last launch also reduces (w, dotv) into *dot_out.
template <typename T>
void neumann_t(const DevMesh &m, Scratch &s, const KBuf<T> &k, int sweeps, const T *v, T *w, const T *dotv,
               double *dot_out, cudaStream_t st) {
  const unsigned cg = grid_for(m.N, kCellBlock);
  const T *z = v;
  for (int q = 0; q < sweeps; q++) {
    T *dst = (q % 2 == 0) ? k.t : k.t2;
    HGKS_PROF_BEGIN(K_JACOBI, st);
    if (q == 0 && sweeps % 2 == 1)
      apply_launch<T, T, T, kNegE, false>(cg, st, m, k.off, k.dval, k.dinv, nullptr, z, dst, nullptr,
                                                                 k.red, s.red_count, nullptr);
    else
      apply_launch<T, T, T, kE, false>(cg, st, m, k.off, k.dval, k.dinv, nullptr, z, dst, nullptr,
                                                              k.red, s.red_count, nullptr);
    HGKS_PROF_END(K_JACOBI, st);
    z = dst;
  }
  HGKS_PROF_BEGIN(K_SPMV, st);
  apply_launch<T, T, T, kNeumann, false>(cg, st, m, k.off, k.dval, k.dinv, v, z, w, dotv, k.red,
                                                                s.red_count, dot_out);
  HGKS_PROF_END(K_SPMV, st);
}

// One restarted GMRES solve in precision T; rhs and dx stay FP64.
template <typename T>
void gmres_t(const DevMesh &m, Scratch &s, const KBuf<T> &k, const hgks_params &p, const double *rhs, double *dx,
             cudaStream_t st, const double *Q, const double *G) {
  const bool fd = p.jv_mode == 1;
  const int mk = p.krylov_dim;
  const int64_t n = 5 * (int64_t)m.N, vs = s.vstride;
  double *H = s.hs, *beta = s.hs + (mk + 1) * mk, *y = beta + 1, *lres = y + mk;
  double *gram = s.gram, *ga = s.gram + kGramLd * kGramLd, *gg = ga + kGramLd;   // G, a, g of the MGS passes
  // The one-pass MGS does 3 FMAs per element and basis vector against 2 for the
  // step-by-step form, and reads about half the bytes: with FP32 vectors it is
  // bound by HBM and wins; with FP64 vectors both forms sit at GB300's FP64 rate
  // (one FP64 FMA per 8 bytes read already exceeds it), so FP64 keeps the steps.
  constexpr bool one_pass = std::is_same<T, float>::value;
  const unsigned vg = vec_grid(n), cg = grid_for(m.N, kCellBlock);
  for (int it = 0; it < p.restarts; it++) {
    cudaMemsetAsync(H, 0, sizeof(double) * (mk + 1) * mk, st);
    // r0 = rhs - A dx (FP64 vectors, blocks of precision T), v1 = P^{-1} r0 / ||P^{-1} r0||
    if (fd && it > 0) {
      fd_apply<double, T>(m, s, p, Q, G, dx, rhs, k.t, st);
    } else if (fd) {                       // dx = 0: r0 = rhs (the product of a zero vector is zero)
      HGKS_PROF_BEGIN(K_SPMV, st);
      k_fd_combine<double, T><<<vec_grid(n), kBlock, 0, st>>>(m.N, m.vol, s.dt, dx, s.Rp, s.R, s.hs + kHsNormQ + 3, rhs, k.t);
      HGKS_PROF_END(K_SPMV, st);
    } else {
      HGKS_PROF_BEGIN(K_SPMV, st);
      apply_launch<T, double, T, kSpmv, false>(cg, st, m, k.off, k.dval, k.dinv, rhs, dx, k.t, nullptr,
                                                                      nullptr, nullptr, nullptr);
      HGKS_PROF_END(K_SPMV, st);
    }
    precondition_t<T>(m, s, k, p.jacobi_sweeps, k.t, k.w, nullptr, nullptr, st);
    HGKS_PROF_BEGIN(K_DOT, st);
    k_axpy_dot<T><<<kRedBlocks, kBlock, 0, st>>>(n, k.w, nullptr, nullptr, k.w, 1, k.red, s.red_count, beta);
    HGKS_PROF_END(K_DOT, st);
    if (it == 0) cudaMemcpyAsync(lres, beta, sizeof(double), cudaMemcpyDeviceToDevice, st);
    HGKS_PROF_BEGIN(K_SCALE, st);
    k_scale<T><<<vg, kBlock, 0, st>>>(n, k.w, beta, k.V);
    HGKS_PROF_END(K_SCALE, st);
    for (int j = 0; j < mk; j++) {
      // w = P^{-1} A v_j (FP64: with h_0j = (w, v_0) from the last launch)
      const T *dv = one_pass ? nullptr : k.V;
      double *dout = one_pass ? nullptr : H + j;
      if (fd) {
        fd_apply<T, T>(m, s, p, Q, G, k.V + (size_t)j * vs, nullptr, k.t, st);
        precondition_t<T>(m, s, k, p.jacobi_sweeps, k.t, k.w, dv, dout, st);
      } else {
        neumann_t<T>(m, s, k, p.jacobi_sweeps, k.V + (size_t)j * vs, k.w, dv, dout, st);
      }
      if (one_pass) {
        // modified Gram-Schmidt: the coefficients h_ij from one pass over the basis,
        // then w -= sum h_ij v_i in MGS order and h_{j+1,j} = ||w||
        for (int k0 = 0; k0 <= j; k0 += kMdot) {
          HGKS_PROF_BEGIN(K_DOT, st);
          k_mdot<T><<<kRedBlocks, kBlock, 0, st>>>(n, k.w, k.V, vs, k0, std::min(kMdot, j + 1 - k0), j, k.red,
                                                    s.red_count, ga, gg);
          HGKS_PROF_END(K_DOT, st);
        }
        HGKS_PROF_BEGIN(K_DOT, st);
        k_mgs_coef<<<1, 32, 0, st>>>(j, mk, ga, gg, gram, H);
        HGKS_PROF_END(K_DOT, st);
        HGKS_PROF_BEGIN(K_DOT, st);
        k_mupdate<T><<<kRedBlocks, kBlock, 0, st>>>(n, k.w, k.V, vs, j, mk, H, k.red, s.red_count, H + (j + 1) * mk + j);
        HGKS_PROF_END(K_DOT, st);
      } else {
        // modified Gram-Schmidt two vectors per pass (h_0j came with the product):
        // subtract the pending vectors (ua, ub), take the inner products with the
        // next two (c, c + 1); the last pass takes ||w|| and g_j = (v_j, v_{j+1})
        // into gram[j]
        auto vec = [&](int q) { return k.V + (size_t)q * vs; };
        int ua = 0, ub = -1, c = 1;
        for (;;) {
          const bool fin = c > j;
          const int d = (!fin && c + 1 <= j) ? c + 1 : -1;
          HGKS_PROF_BEGIN(K_DOT, st);
          launch_mgs2<T>(st, n, k.w, vec(ua), ub >= 0 ? vec(ub) : nullptr, H + ua * mk + j,
                         ub >= 0 ? H + ub * mk + j : nullptr, fin ? nullptr : vec(c), d >= 0 ? vec(d) : nullptr, k.red,
                         s.red_count, fin ? H + (j + 1) * mk + j : H + c * mk + j, d >= 0 ? H + d * mk + j : nullptr,
                         fin ? gram + j : (d >= 0 ? gram + c : nullptr));
          HGKS_PROF_END(K_DOT, st);
          if (fin) break;
          ua = c;
          ub = d;
          c += d >= 0 ? 2 : 1;
        }
      }
      HGKS_PROF_BEGIN(K_SCALE, st);
      k_scale<T><<<vg, kBlock, 0, st>>>(n, k.w, H + (j + 1) * mk + j, k.V + (size_t)(j + 1) * vs);
      HGKS_PROF_END(K_SCALE, st);
    }
    HGKS_PROF_BEGIN(K_GIVENS, st);
    k_givens<<<1, 32, 0, st>>>(mk, H, beta, y, lres + 1);
    HGKS_PROF_END(K_GIVENS, st);
    HGKS_PROF_BEGIN(K_COMBINE, st);
    k_combine<T><<<vg, kBlock, 0, st>>>(n, vs, mk, k.V, y, dx);
    HGKS_PROF_END(K_COMBINE, st);
  }
}

}  // namespace

void launch_assemble(const DevMesh &m, Scratch &s, const hgks_params &p, const double *Q, const double *dt,
                     double *diag_out, double *off_out, cudaStream_t st, bool batch) {
  HGKS_RANGE("hgks assemble");
  // mixed precision: the FP32 operands of the product form come out of the same pass
  const bool mixed = p.precision == HGKS_MIXED && s.jv32;
  float *dv32 = mixed ? s.dval32 : nullptr, *di32 = mixed ? s.dinv32 : nullptr, *jv = mixed ? s.jv32 : nullptr;
  HGKS_PROF_BEGIN(K_ASSEMBLE, st);
  batch = batch || m.ptab;
  if (batch && m.hex)
    k_assemble<true, HexShape::NF><<<grid_for(m.NL, kCellBlock), kCellBlock, 0, st>>>(m, p, Q, dt, s.dval, s.dinv, s.off,
                                                                                       diag_out, off_out, dv32, di32, jv);
  else if (batch)
    k_assemble<true, TetShape::NF><<<grid_for(m.NL, kCellBlock), kCellBlock, 0, st>>>(m, p, Q, dt, s.dval, s.dinv, s.off,
                                                                                       diag_out, off_out, dv32, di32, jv);
  else if (m.hex)
    k_assemble<false, HexShape::NF><<<grid_for(m.N, kCellBlock), kCellBlock, 0, st>>>(m, p, Q, dt, s.dval, s.dinv, s.off,
                                                                                       diag_out, off_out, dv32, di32, jv);
  else
    k_assemble<false, TetShape::NF><<<grid_for(m.N, kCellBlock), kCellBlock, 0, st>>>(m, p, Q, dt, s.dval, s.dinv, s.off,
                                                                                       diag_out, off_out, dv32, di32, jv);
  HGKS_PROF_END(K_ASSEMBLE, st);
}

void launch_apply_A(const DevMesh &m, const Scratch &s, const double *x, double *y, cudaStream_t st) {
  HGKS_PROF_BEGIN(K_SPMV, st);
  apply_launch<double, double, double, kSpmv, false>(grid_for(m.N, kCellBlock), st, m, s.off, s.dval, s.dinv,
                                                     (const double *)nullptr, x, y, (const double *)nullptr,
                                                     (double *)nullptr, nullptr, nullptr);
  HGKS_PROF_END(K_SPMV, st);
}

void launch_precondition(const DevMesh &m, Scratch &s, int sweeps, const double *b, double *x, cudaStream_t st) {
  precondition_t<double>(m, s, kbuf64(s), sweeps, b, x, nullptr, nullptr, st);
}

void launch_norm(const DevMesh &m, Scratch &s, const double *x, double *out_dev, cudaStream_t st) {
  HGKS_PROF_BEGIN(K_DOT, st);
  k_axpy_dot<double><<<kRedBlocks, kBlock, 0, st>>>(5 * (int64_t)m.N, const_cast<double *>(x), nullptr, nullptr, x, 1,
                                                     s.red, s.red_count, out_dev);
  HGKS_PROF_END(K_DOT, st);
}

void launch_apply_fd(const DevMesh &m, Scratch &s, const hgks_params &p, const double *Q, const double *G,
                     const double *x, const double *b, double *y, cudaStream_t st) {
  fd_apply<double, double>(m, s, p, Q, G, x, b, y, st);
}

void launch_density_l1(const DevMesh &m, Scratch &s, const double *R, double *out_dev, cudaStream_t st) {
  HGKS_PROF_BEGIN(K_NORM, st);
  k_density_l1<<<kRedBlocks, kBlock, 0, st>>>(m.N, R, m.inv_vol, s.red, s.red_count, out_dev);
  HGKS_PROF_END(K_NORM, st);
}

void launch_update(const DevMesh &m, double *Q, const double *dQ, double *G, const double *Gnew, int ncomp_g,
                   double relax, cudaStream_t st) {
  const int64_t n5 = 5 * (int64_t)m.N, ng = (int64_t)ncomp_g * m.N;
  HGKS_PROF_BEGIN(K_UPDATE, st);
  k_update<<<vec_grid(n5 + ng), kBlock, 0, st>>>(n5, ng, Q, dQ, G, Gnew, relax > 0.0 ? relax : 1.0);
  HGKS_PROF_END(K_UPDATE, st);
}

// hs layout: H[(m+1) m] | beta | y[m] | lin residual estimates
hgks_status gmres_solve(const DevMesh &m, Scratch &s, const hgks_params &p, const double *rhs, double *dx,
                        hgks_step_info *info, cudaStream_t st, const double *Q, const double *G) {
  HGKS_RANGE("hgks gmres");
  cudaMemsetAsync(dx, 0, sizeof(double) * 5 * (size_t)m.N, st);
  if (p.jv_mode == 1) {
    if (!Q || !s.Qp) return HGKS_ERR_ARG;
    cudaMemsetAsync(s.hs + kHsNormQ + 3, 0, sizeof(double), st);
    launch_norm(m, s, Q, s.hs + kHsNormQ, st);
  }
  if (p.precision == HGKS_MIXED) gmres_t<float>(m, s, kbuf32(s), p, rhs, dx, st, Q, G);
  else gmres_t<double>(m, s, kbuf64(s), p, rhs, dx, st, Q, G);
  if (info) info->krylov_iters = p.restarts * p.krylov_dim;
  return HGKS_OK;
}

}  // namespace hgks
