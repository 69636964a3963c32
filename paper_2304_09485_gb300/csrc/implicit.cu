// Implicit part of one HGKS step (paper Sec. 4.1 - 4.3, Algorithm 1), FP64.
//
//  * A of Eq. (A-system-2) with the split Jacobians of Eq. (deri-matrix):
//      A_ii  = |Omega_i|/dt_i I + sum_p (J(Q_i) n_p + |lambda_p| I) S_p / 2
//      A_ij  = (J(Q_j) n_p - |lambda_p| I) S_p / 2
//    The Euler-Jacobian part of A_ii is J(Q_i) applied to sum_p n_p S_p, the
//    sum of a closed cell's outward area vectors, which is zero: A_ii is a
//    multiple of the identity and is stored as one number per cell. The
//    off-diagonal blocks are stored per (face, side): side s holds the block
//    of the row of the face's side-s cell ("structure array" of Sec. 4.3, laid
//    out face-major so that a warp reads consecutive faces).
//  * Jacobi preconditioner of Eq. (precond), k_max sweeps.
//  * Restarted GMRES with modified Gram-Schmidt (Algorithm 1). Every inner
//    product is one launch: blocks write partial sums, the last block to finish
//    adds them in a fixed order (deterministic, no host round trip). The small
//    least-squares problem (Givens rotations) runs in a single device thread,
//    so a whole GMRES cycle is enqueued without synchronising the host.
#include <cmath>
#include "hgks_internal.h"

namespace hgks {
namespace {

constexpr int kBlock = 256;
constexpr int kRedBlocks = 2 * 152;   // blocks of every reduction: a multiple of the SM count

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

__global__ void k_assemble(DevMesh m, hgks_params P, const double *__restrict__ Q, const double *__restrict__ dt,
                           double *__restrict__ dval, double *__restrict__ dinv, double *__restrict__ off,
                           double *__restrict__ diag_out, double *__restrict__ off_out) {
  const int N = m.N, F = m.F;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double Qi[5];
#pragma unroll
  for (int c = 0; c < 5; c++) Qi[c] = Q[(size_t)c * N + i];
  double d = m.vol[i] / dt[i];
#pragma unroll 1
  for (int p = 0; p < 4; p++) {
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
    double J[25];
    if (j >= 0) {
      euler_jacobian(Qj, n, P.gamma, J);
#pragma unroll
      for (int k = 0; k < 25; k++) {
        double o = 0.5 * (J[k] - (k % 6 == 0 ? lam : 0.0)) * S;
        off[(size_t)(side * 25 + k) * F + f] = o;
        if (off_out) off_out[(size_t)(p * 25 + k) * N + i] = o;
      }
    } else if (off_out) {
#pragma unroll
      for (int k = 0; k < 25; k++) off_out[(size_t)(p * 25 + k) * N + i] = 0.0;
    }
  }
  dval[i] = d;
  dinv[i] = 1.0 / d;
  if (diag_out)
#pragma unroll
    for (int k = 0; k < 25; k++) diag_out[(size_t)k * N + i] = k % 6 == 0 ? d : 0.0;
}

// y = b - (sum_p A_ip x_p) [+ diag x when with_diag]; (L+U) x when b = nullptr and with_diag = 0
template <bool WithDiag, bool Jacobi>
__global__ void k_offdiag(DevMesh m, const double *__restrict__ off, const double *__restrict__ dval,
                          const double *__restrict__ dinv, const double *__restrict__ b, const double *__restrict__ x,
                          double *__restrict__ y) {
  const int N = m.N, F = m.F;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double acc[5];
#pragma unroll
  for (int r = 0; r < 5; r++) acc[r] = WithDiag ? dval[i] * x[(size_t)r * N + i] : 0.0;
#pragma unroll
  for (int p = 0; p < 4; p++) {
    const int j = m.cnb[(size_t)p * N + i];
    if (j < 0) continue;
    const int cf = m.cface[(size_t)p * N + i], f = cf >> 1, side = cf & 1;
    double xj[5];
#pragma unroll
    for (int c = 0; c < 5; c++) xj[c] = x[(size_t)c * N + j];
    const double *O = off + (size_t)side * 25 * F + f;
#pragma unroll
    for (int r = 0; r < 5; r++)
#pragma unroll
      for (int c = 0; c < 5; c++) acc[r] = fma(O[(size_t)(5 * r + c) * F], xj[c], acc[r]);
  }
  if (Jacobi) {
    const double di = dinv[i];
#pragma unroll
    for (int r = 0; r < 5; r++) y[(size_t)r * N + i] = di * (b[(size_t)r * N + i] - acc[r]);
  } else if (b) {
#pragma unroll
    for (int r = 0; r < 5; r++) y[(size_t)r * N + i] = b[(size_t)r * N + i] - acc[r];
  } else {
#pragma unroll
    for (int r = 0; r < 5; r++) y[(size_t)r * N + i] = acc[r];
  }
}

__global__ void k_diag_scale(int N, const double *__restrict__ dinv, const double *__restrict__ b, double *__restrict__ x) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 5 * N) return;
  x[t] = dinv[t % N] * b[t];
}

// Deterministic reduction: per-block partial sums, the last block adds them in order.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[kBlock / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < kBlock / 32 ? sh[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;   // valid in thread 0
}
// finish: out = f(sum of partials); mode 0: sum, 1: sqrt(sum)
__device__ __forceinline__ void finish_reduction(double bsum, double *partials, unsigned int *count, double *out, int mode) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = bsum;
    __threadfence();
    unsigned int prev = atomicAdd(count, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double s = 0.0;
    for (unsigned b = 0; b < gridDim.x; b++) s += ((volatile double *)partials)[b];
    *out = mode == 1 ? sqrt(s) : s;
    *count = 0u;
  }
}

// w -= h * v (if v != nullptr); out = (w . x) or ||w|| (x == w, mode 1)
__global__ void __launch_bounds__(kBlock) k_axpy_dot(int64_t n, double *__restrict__ w, const double *__restrict__ v,
                                                     const double *__restrict__ h, const double *__restrict__ x,
                                                     int self, double *partials, unsigned int *count, double *out) {
  const double hv = v ? -*h : 0.0;
  double s = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double wk = w[k];
    if (v) { wk = fma(hv, v[k], wk); w[k] = wk; }
    s = fma(wk, self ? wk : x[k], s);
  }
  finish_reduction(block_sum(s), partials, count, out, self);
}

// v = w / h (v = 0 after a breakdown h == 0)
__global__ void k_scale(int64_t n, const double *__restrict__ w, const double *__restrict__ h, double *__restrict__ v) {
  const double hv = *h;
  const double ih = hv != 0.0 ? 1.0 / hv : 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) v[k] = w[k] * ih;
}

// Givens QR of the (used+1) x used Hessenberg matrix and back substitution:
// y minimises || beta e1 - H y ||. H[i*m + j] holds h_{i,j}. Single thread.
__global__ void k_givens(int m, const double *__restrict__ H, const double *__restrict__ beta, double *__restrict__ y,
                         double *__restrict__ res_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double R[65 * 64], gv[65];
  int used = m;
  for (int j = 0; j < m; j++)
    if (H[(j + 1) * m + j] == 0.0) { used = j + 1; break; }
  for (int i = 0; i <= used; i++)
    for (int j = 0; j < used; j++) R[i * 64 + j] = H[i * m + j];
  for (int i = 0; i <= m; i++) gv[i] = 0.0;
  gv[0] = *beta;
  for (int j = 0; j < m; j++) y[j] = 0.0;
  if (gv[0] == 0.0) { *res_out = 0.0; return; }
  for (int j = 0; j < used; j++) {
    const double a = R[j * 64 + j], b = R[(j + 1) * 64 + j], r = sqrt(a * a + b * b);
    const double c = a / r, s = b / r;
    for (int k = j; k < used; k++) {
      const double h1 = R[j * 64 + k], h2 = R[(j + 1) * 64 + k];
      R[j * 64 + k] = c * h1 + s * h2;
      R[(j + 1) * 64 + k] = -s * h1 + c * h2;
    }
    const double g1 = gv[j], g2 = gv[j + 1];
    gv[j] = c * g1 + s * g2;
    gv[j + 1] = -s * g1 + c * g2;
  }
  for (int j = used - 1; j >= 0; j--) {
    double s = gv[j];
    for (int k = j + 1; k < used; k++) s -= R[j * 64 + k] * y[k];
    y[j] = s / R[j * 64 + j];
  }
  *res_out = fabs(gv[used]);
}

// dx += sum_j y_j V_j
__global__ void k_combine(int64_t n, int m, const double *__restrict__ V, const double *__restrict__ y, double *__restrict__ dx) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double s = dx[k];
    for (int j = 0; j < m; j++) s = fma(y[j], V[(size_t)j * n + k], s);
    dx[k] = s;
  }
}

__global__ void __launch_bounds__(kBlock) k_density_l1(int N, const double *__restrict__ R, const double *__restrict__ inv_vol,
                                                       double *partials, unsigned int *count, double *out) {
  double s = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) s += fabs(R[k]) * inv_vol[k];
  finish_reduction(block_sum(s), partials, count, out, 0);
}

__global__ void k_update(int64_t n5, int64_t ng, double *__restrict__ Q, const double *__restrict__ dQ, double *__restrict__ G,
                         const double *__restrict__ Gnew) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n5 + ng; k += (int64_t)gridDim.x * blockDim.x) {
    if (k < n5) Q[k] += dQ[k];
    else G[k - n5] = Gnew[k - n5];
  }
}

unsigned vec_grid(int64_t n) {
  int64_t g = (n + kBlock - 1) / kBlock;
  const int64_t cap = 152 * 8;
  return (unsigned)std::max<int64_t>(1, std::min(g, cap));
}

}  // namespace

void launch_assemble(const DevMesh &m, Scratch &s, const hgks_params &p, const double *Q, const double *dt,
                     double *diag_out, double *off_out, cudaStream_t st) {
  HGKS_PROF_BEGIN(K_ASSEMBLE, st);
  k_assemble<<<grid_for(m.N, 128), 128, 0, st>>>(m, p, Q, dt, s.dval, s.dinv, s.off, diag_out, off_out);
  HGKS_PROF_END(K_ASSEMBLE, st);
}

void launch_apply_A(const DevMesh &m, const Scratch &s, const double *x, double *y, cudaStream_t st) {
  HGKS_PROF_BEGIN(K_SPMV, st);
  k_offdiag<true, false><<<grid_for(m.N, 128), 128, 0, st>>>(m, s.off, s.dval, s.dinv, nullptr, x, y);
  HGKS_PROF_END(K_SPMV, st);
}

// x = P^{-1} b: x0 = D^{-1} b, x_k = D^{-1} (b - (L+U) x_{k-1})
void launch_precondition(const DevMesh &m, Scratch &s, int sweeps, const double *b, double *x, cudaStream_t st) {
  double *bufs[2] = {s.t2, x};
  double *cur = (sweeps % 2 == 0) ? x : s.t2;
  HGKS_PROF_BEGIN(K_DIAG, st);
  k_diag_scale<<<grid_for(5 * (int64_t)m.N, kBlock), kBlock, 0, st>>>(m.N, s.dinv, b, cur);
  HGKS_PROF_END(K_DIAG, st);
  for (int k = 1; k <= sweeps; k++) {
    double *nxt = (cur == x) ? bufs[0] : bufs[1];
    HGKS_PROF_BEGIN(K_JACOBI, st);
    k_offdiag<false, true><<<grid_for(m.N, 128), 128, 0, st>>>(m, s.off, s.dval, s.dinv, b, cur, nxt);
    HGKS_PROF_END(K_JACOBI, st);
    cur = nxt;
  }
}

void launch_density_l1(const DevMesh &m, Scratch &s, const double *R, double *out_dev, cudaStream_t st) {
  HGKS_PROF_BEGIN(K_NORM, st);
  k_density_l1<<<kRedBlocks, kBlock, 0, st>>>(m.N, R, m.inv_vol, s.red, s.red_count, out_dev);
  HGKS_PROF_END(K_NORM, st);
}

void launch_update(const DevMesh &m, double *Q, const double *dQ, double *G, const double *Gnew, int ncomp_g, cudaStream_t st) {
  const int64_t n5 = 5 * (int64_t)m.N, ng = (int64_t)ncomp_g * m.N;
  HGKS_PROF_BEGIN(K_UPDATE, st);
  k_update<<<vec_grid(n5 + ng), kBlock, 0, st>>>(n5, ng, Q, dQ, G, Gnew);
  HGKS_PROF_END(K_UPDATE, st);
}

// hs layout: H[(m+1) m] | beta | y[m] | lin residual estimates
hgks_status gmres_solve(const DevMesh &m, Scratch &s, const hgks_params &p, const double *rhs, double *dx,
                        hgks_step_info *info, cudaStream_t st) {
  const int mk = p.krylov_dim;
  const int64_t n = 5 * (int64_t)m.N;
  double *H = s.hs, *beta = s.hs + (mk + 1) * mk, *y = beta + 1, *lres = y + mk;
  const unsigned vg = vec_grid(n);
  cudaMemsetAsync(dx, 0, sizeof(double) * n, st);
  double *V = s.V;
  for (int it = 0; it < p.restarts; it++) {
    cudaMemsetAsync(H, 0, sizeof(double) * (mk + 1) * mk, st);
    // r0 = rhs - A dx, v1 = P^{-1} r0 / ||P^{-1} r0||
    HGKS_PROF_BEGIN(K_SPMV, st);
    k_offdiag<true, false><<<grid_for(m.N, 128), 128, 0, st>>>(m, s.off, s.dval, s.dinv, rhs, dx, s.t);
    HGKS_PROF_END(K_SPMV, st);
    launch_precondition(m, s, p.jacobi_sweeps, s.t, s.w, st);
    HGKS_PROF_BEGIN(K_DOT, st);
    k_axpy_dot<<<kRedBlocks, kBlock, 0, st>>>(n, s.w, nullptr, nullptr, s.w, 1, s.red, s.red_count, beta);
    HGKS_PROF_END(K_DOT, st);
    if (it == 0) cudaMemcpyAsync(lres, beta, sizeof(double), cudaMemcpyDeviceToDevice, st);
    HGKS_PROF_BEGIN(K_SCALE, st);
    k_scale<<<vg, kBlock, 0, st>>>(n, s.w, beta, V);
    HGKS_PROF_END(K_SCALE, st);
    for (int j = 0; j < mk; j++) {
      // w = P^{-1} A v_j
      HGKS_PROF_BEGIN(K_SPMV, st);
      k_offdiag<true, false><<<grid_for(m.N, 128), 128, 0, st>>>(m, s.off, s.dval, s.dinv, nullptr, V + (size_t)j * n, s.t);
      HGKS_PROF_END(K_SPMV, st);
      launch_precondition(m, s, p.jacobi_sweeps, s.t, s.w, st);
      // modified Gram-Schmidt: h_ij = (w, v_i); w -= h_ij v_i; h_{j+1,j} = ||w||
      HGKS_PROF_BEGIN(K_DOT, st);
      k_axpy_dot<<<kRedBlocks, kBlock, 0, st>>>(n, s.w, nullptr, nullptr, V, 0, s.red, s.red_count, H + j);
      HGKS_PROF_END(K_DOT, st);
      for (int i = 0; i <= j; i++) {
        const bool last = (i == j);
        HGKS_PROF_BEGIN(K_DOT, st);
        k_axpy_dot<<<kRedBlocks, kBlock, 0, st>>>(n, s.w, V + (size_t)i * n, H + i * mk + j,
                                                    last ? s.w : V + (size_t)(i + 1) * n, last ? 1 : 0, s.red, s.red_count,
                                                    H + (i + 1) * mk + j);
        HGKS_PROF_END(K_DOT, st);
      }
      HGKS_PROF_BEGIN(K_SCALE, st);
      k_scale<<<vg, kBlock, 0, st>>>(n, s.w, H + (j + 1) * mk + j, V + (size_t)(j + 1) * n);
      HGKS_PROF_END(K_SCALE, st);
    }
    HGKS_PROF_BEGIN(K_GIVENS, st);
    k_givens<<<1, 32, 0, st>>>(mk, H, beta, y, lres + 1);
    HGKS_PROF_END(K_GIVENS, st);
    HGKS_PROF_BEGIN(K_COMBINE, st);
    k_combine<<<vg, kBlock, 0, st>>>(n, mk, V, y, dx);
    HGKS_PROF_END(K_COMBINE, st);
  }
  if (info) info->krylov_iters = p.restarts * mk;
  return HGKS_OK;
}

}  // namespace hgks
