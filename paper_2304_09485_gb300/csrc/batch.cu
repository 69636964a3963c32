// Batches of independent meshes: one launch per phase for all of them.
//
// A batch merges its meshes into one cell space. Each mesh's cells start on a
// multiple of 256 (kBatchBlock), padded with inert cells, so a block of 256
// cells always belongs to exactly one mesh. The residual kernels run once over
// the merged space, reading each cell's (or face's) parameters from a per-mesh
// table. The GMRES part keeps one Krylov space per mesh: every inner product is
// a segmented reduction (the blocks of one mesh write partial sums, the last of
// them to finish adds that mesh's partials in a fixed order), the Hessenberg
// least-squares problems are solved one device thread per mesh, and the vector
// updates read their mesh's coefficients. A mesh in a batch therefore follows
// the same algorithm as alone (Algorithm 1), with its own Krylov space.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include "hgks_internal.h"
#include "givens.cuh"
#include "offdiag.cuh"

namespace hgks {
namespace {

constexpr int kB = kBatchBlock;

template <typename T>
__device__ __forceinline__ T bsum(T v) {
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
  return s;
}

// per-mesh segmented sum: *out(mesh) = sum over the mesh's blocks (or its sqrt)
template <typename T>
__device__ __forceinline__ void mesh_sum(T v, const BatchDev &b, T *part, double *out, int stride, int mode) {
  __shared__ bool last;
  const int mesh = b.bmesh[blockIdx.x];
  const T s0 = bsum(v);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s0;
    __threadfence();
    const unsigned prev = atomicAdd(b.counters + mesh, 1u);
    last = (prev == (unsigned)(b.bcount[mesh] - 1));
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  T s = T(0);
  const int k0 = b.bstart[mesh], k1 = k0 + b.bcount[mesh];
  for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) s += ((volatile T *)part)[k];
  s = bsum(s);
  if (threadIdx.x == 0) {
    out[(size_t)mesh * stride] = mode == 1 ? (double)sqrt(s) : (double)s;
    b.counters[mesh] = 0u;
  }
}

enum { kSpmv = 0, kJacobi = 1, kNeumann = 2, kE = 3, kNegE = 4 };   // as k_apply of the single-mesh path
// SpMV / Jacobi sweep over the merged cells with an optional per-mesh (y, dotv)
template <typename TM, typename TV, typename TO, int Mode, bool First, int NF>
__global__ void __launch_bounds__(kB) k_bapply(DevMesh m, BatchDev bd, const TM *__restrict__ off,
                                               const TM *__restrict__ dval, const TM *__restrict__ dinv,
                                               const TV *__restrict__ b, const TV *__restrict__ x, TO *__restrict__ y,
                                               const TO *__restrict__ dotv, TO *part, double *dot_out, int stride) {
  const int N = m.N;
  const int i = blockIdx.x * kB + threadIdx.x;
  if (!bd.active[bd.bmesh[blockIdx.x]]) return;
  TV acc[5];
  const TV di = Mode == kSpmv ? (TV)dval[i] : TV(0);
#pragma unroll
  for (int r = 0; r < 5; r++) acc[r] = Mode == kSpmv ? di * x[(size_t)r * N + i] : TV(0);
#pragma unroll
  for (int p = 0; p < NF; p++) {
    const int j = m.cnb[(size_t)p * N + i];
    if (j < 0) continue;
    TV xj[5];
    const TV sj = First ? (TV)dinv[j] : TV(1);
#pragma unroll
    for (int c = 0; c < 5; c++) xj[c] = First ? sj * b[(size_t)c * N + j] : x[(size_t)c * N + j];
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
  TO part_v = TO(0);
#pragma unroll
  for (int r = 0; r < 5; r++) {
    TV o;
    if (Mode == kJacobi) o = (TV)dinv[i] * (b[(size_t)r * N + i] - acc[r]);
    else if (Mode == kE) o = (TV)dinv[i] * acc[r];
    else if (Mode == kNegE) o = -(TV)dinv[i] * acc[r];
    else if (Mode == kNeumann) o = fma((TV)dinv[i], acc[r], b[(size_t)r * N + i]);
    else o = b ? b[(size_t)r * N + i] - acc[r] : acc[r];
    const TO oo = (TO)o;
    y[(size_t)r * N + i] = oo;
    if (dotv) part_v = fma(oo, dotv[(size_t)r * N + i], part_v);
  }
  if (dotv) mesh_sum(part_v, bd, part, dot_out, stride, 0);
}

// k_bapply for the batch's cell kind (4 or 6 off-diagonal blocks per row)
template <typename TM, typename TV, typename TO, int Mode, bool First>
void bapply(unsigned g, cudaStream_t st, const DevMesh &m, const BatchDev &bd, const TM *off, const TM *dval,
            const TM *dinv, const TV *b, const TV *x, TO *y, const TO *dotv, TO *part, double *dot_out, int stride) {
  if (m.hex)
    k_bapply<TM, TV, TO, Mode, First, HexShape::NF><<<g, kB, 0, st>>>(m, bd, off, dval, dinv, b, x, y, dotv, part,
                                                                      dot_out, stride);
  else
    k_bapply<TM, TV, TO, Mode, First, TetShape::NF><<<g, kB, 0, st>>>(m, bd, off, dval, dinv, b, x, y, dotv, part,
                                                                      dot_out, stride);
}

// w -= h(mesh) v (if v); out(mesh) = (w, x) or ||w|| (self; x is not read then,
// so callers may pass w for it)
template <typename T>
__global__ void __launch_bounds__(kB) k_baxpy_dot(int N, BatchDev bd, T *__restrict__ w, const T *__restrict__ v,
                                                  const double *__restrict__ h, int hstride, const T *__restrict__ x,
                                                  int self, T *part, double *out, int stride) {
  const int i = blockIdx.x * kB + threadIdx.x;
  const int mesh = bd.bmesh[blockIdx.x];
  if (!bd.active[mesh]) return;
  const T hv = v ? (T)(-h[(size_t)mesh * hstride]) : T(0);
  T s = T(0);
#pragma unroll
  for (int c = 0; c < 5; c++) {
    const size_t k = (size_t)c * N + i;
    T wk = w[k];
    if (v) { wk = fma(hv, v[k], wk); w[k] = wk; }
    s = fma(wk, self ? wk : x[k], s);
  }
  mesh_sum(s, bd, part, out, stride, self);
}

// ---- modified Gram-Schmidt from one pass over the basis (FP32 vectors) ----
// As the single-mesh path: with a_k = (w, v_k) and the basis Gram matrix
// G_ki = (v_k, v_i), Algorithm 1's MGS coefficients are h_i = a_i - sum_{k<i} h_k G_ki,
// so per Arnoldi step the batch takes a and the new Gram row from one pass
// (kBatchMdot basis vectors per launch, per-mesh sums), solves for h per mesh
// and subtracts sum h_i v_i in MGS order in one more pass with ||w||.

// a(mesh)[k] = (w, v_k) for k in [k0, k0 + nk), g(mesh)[k] = (v_j, v_k) for those k < j
template <typename T>
__global__ void __launch_bounds__(kB) k_bmdot(int N, BatchDev bd, const T *__restrict__ w, const T *__restrict__ V,
                                              int64_t vs, int k0, int nk, int j, T *part, double *hs, int hz, int aoff,
                                              int goff) {
  const int i = blockIdx.x * kB + threadIdx.x;
  const int mesh = bd.bmesh[blockIdx.x];
  if (!bd.active[mesh]) return;
  T sa[kBatchMdot], sg[kBatchMdot];
#pragma unroll
  for (int q = 0; q < kBatchMdot; q++) { sa[q] = T(0); sg[q] = T(0); }
#pragma unroll
  for (int c = 0; c < 5; c++) {
    const size_t k = (size_t)c * N + i;
    const T wk = w[k], vj = V[(size_t)j * vs + k];
#pragma unroll
    for (int q = 0; q < kBatchMdot; q++)
      if (q < nk) {
        const T vk = V[(size_t)(k0 + q) * vs + k];
        sa[q] = fma(wk, vk, sa[q]);
        if (k0 + q < j) sg[q] = fma(vj, vk, sg[q]);
      }
  }
  // per block 2 kBatchMdot partials (each warp reduces all of its sums by shuffles,
  // then one thread per sum adds the warps' values in warp order); the mesh's last
  // block adds each slot's partials in block order
  const int nb = gridDim.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ T wsum[2 * kBatchMdot][kB / 32];
  __shared__ bool last;
#pragma unroll
  for (int q = 0; q < 2 * kBatchMdot; q++) {
    T v = q < kBatchMdot ? sa[q] : sg[q - kBatchMdot];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) wsum[q][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < 2 * kBatchMdot) {
    T v = T(0);
#pragma unroll
    for (int q = 0; q < kB / 32; q++) v += wsum[threadIdx.x][q];
    part[(size_t)threadIdx.x * nb + blockIdx.x] = v;
    __threadfence();                       // visible to the mesh's last block
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(bd.counters + mesh, 1u);
    last = (prev == (unsigned)(bd.bcount[mesh] - 1));
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double *rec = hs + (size_t)mesh * hz;
  const int b0 = bd.bstart[mesh], b1 = b0 + bd.bcount[mesh];
  for (int q = 0; q < 2 * kBatchMdot; q++) {
    const int kk = k0 + (q % kBatchMdot);
    const bool want = (q % kBatchMdot) < nk && (q < kBatchMdot || kk < j);   // uniform over the block
    if (!want) continue;
    T sum = T(0);
    for (int b = b0 + threadIdx.x; b < b1; b += blockDim.x) sum += ((volatile T *)part)[(size_t)q * nb + b];
    sum = bsum(sum);
    if (threadIdx.x == 0) rec[(q < kBatchMdot ? aoff : goff) + kk] = (double)sum;
  }
  if (threadIdx.x == 0) bd.counters[mesh] = 0u;
}

// one thread per mesh: row j of the Gram matrix from g, then h_ij by forward substitution
__global__ void k_bmgs_coef(BatchDev bd, int j, int mk, double *__restrict__ hs, int hz, int aoff, int goff,
                            int gram_off) {
  const int mesh = blockIdx.x * blockDim.x + threadIdx.x;
  if (mesh >= bd.nmesh || !bd.active[mesh]) return;
  double *rec = hs + (size_t)mesh * hz, *G = rec + gram_off;
  const double *a = rec + aoff, *g = rec + goff;
  const int ld = mk + 1;
  for (int k = 0; k < j; k++) G[k * ld + j] = g[k];
  for (int i = 0; i <= j; i++) {
    double h = a[i];
    for (int k = 0; k < i; k++) h -= rec[k * mk + j] * G[k * ld + i];
    rec[i * mk + j] = h;
  }
}

// w -= sum_{k <= j} h_kj(mesh) v_k in the order of k, then h_{j+1,j}(mesh) = ||w||
template <typename T>
__global__ void __launch_bounds__(kB) k_bmupdate(int N, BatchDev bd, T *__restrict__ w, const T *__restrict__ V,
                                                 int64_t vs, int j, int mk, double *hs, int hz, T *part) {
  const int i = blockIdx.x * kB + threadIdx.x;
  const int mesh = bd.bmesh[blockIdx.x];
  if (!bd.active[mesh]) return;
  __shared__ T nh[65];
  const double *rec = hs + (size_t)mesh * hz;
  for (int k = threadIdx.x; k <= j; k += blockDim.x) nh[k] = (T)(-rec[k * mk + j]);
  __syncthreads();
  T s = T(0);
#pragma unroll
  for (int c = 0; c < 5; c++) {
    const size_t k = (size_t)c * N + i;
    T wk = w[k];
    for (int q = 0; q <= j; q++) wk = fma(nh[q], V[(size_t)q * vs + k], wk);
    w[k] = wk;
    s = fma(wk, wk, s);
  }
  mesh_sum(s, bd, part, hs + (size_t)(j + 1) * mk + j, hz, 1);
}

template <typename T>
__global__ void __launch_bounds__(kB) k_bscale(int N, BatchDev bd, const T *__restrict__ w, const double *__restrict__ h,
                                               int hstride, T *__restrict__ v) {
  const int i = blockIdx.x * kB + threadIdx.x;
  if (!bd.active[bd.bmesh[blockIdx.x]]) return;
  const double hv = h[(size_t)bd.bmesh[blockIdx.x] * hstride];
  const T ih = hv != 0.0 ? (T)(1.0 / hv) : T(0);
#pragma unroll
  for (int c = 0; c < 5; c++) v[(size_t)c * N + i] = w[(size_t)c * N + i] * ih;
}

// one thread per mesh: y(mesh) = argmin || beta e1 - H y ||
__global__ void k_bgivens(BatchDev bd, int m, double *__restrict__ hs, int stride) {
  const int mesh = blockIdx.x * blockDim.x + threadIdx.x;
  if (mesh >= bd.nmesh || !bd.active[mesh]) return;
  double *H = hs + (size_t)mesh * stride, *beta = H + (m + 1) * m, *y = beta + 1, *lres = y + m;
  lres[1] = givens_lsq(m, H, *beta, y);
}

template <typename T>
__global__ void __launch_bounds__(kB) k_bcombine(int N, BatchDev bd, int64_t vs, int m, const T *__restrict__ V,
                                                 const double *__restrict__ hs, int stride, double *__restrict__ dx) {
  const int i = blockIdx.x * kB + threadIdx.x;
  if (!bd.active[bd.bmesh[blockIdx.x]]) return;
  const double *y = hs + (size_t)bd.bmesh[blockIdx.x] * stride + (m + 1) * m + 1;
#pragma unroll
  for (int c = 0; c < 5; c++) {
    const size_t k = (size_t)c * N + i;
    double s = dx[k];
    for (int j = 0; j < m; j++) s = fma(y[j], (double)V[(size_t)j * vs + k], s);
    dx[k] = s;
  }
}

// per-mesh L1 norm of the density residual (padding cells hold R = 0)
__global__ void __launch_bounds__(kB) k_bdensity(int N, BatchDev bd, const double *__restrict__ R,
                                                 const double *__restrict__ inv_vol, double *part, double *out, int stride) {
  const int i = blockIdx.x * kB + threadIdx.x;
  if (!bd.active[bd.bmesh[blockIdx.x]]) return;
  mesh_sum(fabs(R[i]) * inv_vol[i], bd, part, out, stride, 0);
}

// Q += dQ and G = G_new for the meshes still iterating
__global__ void __launch_bounds__(kB) k_bupdate(int N, BatchDev bd, const hgks_params *__restrict__ ptab,
                                                double *__restrict__ Q, const double *__restrict__ dQ,
                                                double *__restrict__ G, const double *__restrict__ Gnew, int ng) {
  const int i = blockIdx.x * kB + threadIdx.x;
  const int mesh = bd.bmesh[blockIdx.x];
  if (!bd.active[mesh]) return;
#pragma unroll
  for (int c = 0; c < 5; c++) Q[(size_t)c * N + i] += dQ[(size_t)c * N + i];
  const double a = ptab[mesh].grad_relax > 0.0 ? ptab[mesh].grad_relax : 1.0;   // per-mesh relaxation of G
  for (int c = 0; c < ng; c++) {
    const size_t k = (size_t)c * N + i;
    G[k] = a == 1.0 ? Gnew[k] : fma(a, Gnew[k] - G[k], G[k]);
  }
}


// x = D^{-1} b (no Jacobi sweep), with an optional per-mesh (x, dotv)
template <typename T>
__global__ void __launch_bounds__(kB) k_bdiag(int N, BatchDev bd, const T *__restrict__ dinv, const T *__restrict__ b,
                                              T *__restrict__ x, const T *__restrict__ dotv, T *part, double *dot_out,
                                              int stride) {
  const int i = blockIdx.x * kB + threadIdx.x;
  if (!bd.active[bd.bmesh[blockIdx.x]]) return;
  const T di = dinv[i];
  T s = T(0);
#pragma unroll
  for (int c = 0; c < 5; c++) {
    const T v = di * b[(size_t)c * N + i];
    x[(size_t)c * N + i] = v;
    if (dotv) s = fma(v, dotv[(size_t)c * N + i], s);
  }
  if (dotv) mesh_sum(s, bd, part, dot_out, stride, 0);
}

// Convergence test of every active mesh on the mean density residual of its
// current state: history, running maximum (the reference), and the drop.
__global__ void k_bcheck(BatchState bs) {
  const int mesh = blockIdx.x * blockDim.x + threadIdx.x;
  const BatchDev &bd = bs.b;
  if (mesh >= bd.nmesh || !bd.active[mesh]) return;
  const double res = bs.hs[(size_t)mesh * bs.hsz + bs.l1_off] / (double)bs.ncell[mesh];
  const int k = bs.steps[mesh];
  bs.res[mesh] = res;
  if (bs.hist && k < bs.hist_len) bs.hist[(size_t)mesh * bs.hist_len + k] = res;
  if (!isfinite(res)) { bs.bad[mesh] = 1; bd.active[mesh] = 0; return; }
  if (res > bs.ref[mesh]) bs.ref[mesh] = res;
  if (bs.ref[mesh] > 0.0 && res <= bs.drop[mesh] * bs.ref[mesh]) { bs.conv[mesh] = 1; bd.active[mesh] = 0; return; }
  if (k >= bs.max_steps[mesh]) { bd.active[mesh] = 0; return; }
  bs.steps[mesh] = k + 1;
}

template <typename T>
__global__ void k_fill(T *a, int64_t n, T v) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) a[k] = v;
}

// a[r][c] += add where a[r][c] >= 0, for the n columns of rows r < rows (row pitch `pitch`)
__global__ void k_offset_index(int *a, int rows, int64_t n, int64_t pitch, int64_t add) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < (int64_t)rows * n; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = k / n, c = k - r * n;
    int *q = a + r * pitch + c;
    if (*q >= 0) *q = (int)(*q + add);
  }
}

template <typename T>
struct BBuf {
  const T *off, *dval, *dinv;
  T *V, *w, *t, *t2, *part;
};
BBuf<double> bbuf64(Scratch &s, BatchState &bs) { return {s.off, s.dval, s.dinv, s.V, s.w, s.t, s.t2, bs.part}; }
BBuf<float> bbuf32(Scratch &s, BatchState &bs) { return {s.jv32, s.dval32, s.dinv32, s.V32, s.w32, s.t32, s.t232, bs.part32}; }

// x = P^{-1} b for every mesh (Eq. (precond)); with dotv, also (x, dotv) per mesh
template <typename T>
void bprecondition(const DevMesh &m, BatchState &bs, const BBuf<T> &k, int sweeps, const T *b, T *x, const T *dotv,
                   double *dot_out, cudaStream_t st) {
  const unsigned g = std::max(1, bs.b.nblocks);
  const int hz = bs.hsz;
  if (sweeps == 0) {
    HGKS_PROF_BEGIN(K_DIAG, st);
    k_bdiag<T><<<g, kB, 0, st>>>(m.N, bs.b, k.dinv, b, x, dotv, k.part, dot_out, hz);
    HGKS_PROF_END(K_DIAG, st);
    return;
  }
  const T *prev = nullptr;
  for (int q = 1; q <= sweeps; q++) {
    T *dst = ((sweeps - q) % 2 == 0) ? x : k.t2;
    const T *dv = (q == sweeps) ? dotv : nullptr;
    HGKS_PROF_BEGIN(K_JACOBI, st);
    if (q == 1)
      bapply<T, T, T, kJacobi, true>(g, st, m, bs.b, k.off, k.dval, k.dinv, b, nullptr, dst, dv, k.part,
                                                          dot_out, hz);
    else
      bapply<T, T, T, kJacobi, false>(g, st, m, bs.b, k.off, k.dval, k.dinv, b, prev, dst, dv, k.part,
                                                           dot_out, hz);
    HGKS_PROF_END(K_JACOBI, st);
    prev = dst;
  }
}

// w = P^{-1} A v for a Krylov vector v of every mesh: w = v + E (-E)^k v with
// E = D^{-1} O (the sign in the first product), as neumann_t of the single-mesh
// path; (w, dotv) per mesh from the last launch
template <typename T>
void bneumann(const DevMesh &m, BatchState &bs, const BBuf<T> &k, int sweeps, const T *v, T *w, const T *dotv,
              double *dot_out, cudaStream_t st) {
  const unsigned g = std::max(1, bs.b.nblocks);
  const int hz = bs.hsz;
  const T *z = v;
  for (int q = 0; q < sweeps; q++) {
    T *dst = (q % 2 == 0) ? k.t : k.t2;
    HGKS_PROF_BEGIN(K_JACOBI, st);
    if (q == 0 && sweeps % 2 == 1)
      bapply<T, T, T, kNegE, false>(g, st, m, bs.b, k.off, k.dval, k.dinv, nullptr, z, dst, nullptr, k.part,
                                                         nullptr, hz);
    else
      bapply<T, T, T, kE, false>(g, st, m, bs.b, k.off, k.dval, k.dinv, nullptr, z, dst, nullptr, k.part,
                                                      nullptr, hz);
    HGKS_PROF_END(K_JACOBI, st);
    z = dst;
  }
  HGKS_PROF_BEGIN(K_SPMV, st);
  bapply<T, T, T, kNeumann, false>(g, st, m, bs.b, k.off, k.dval, k.dinv, v, z, w, dotv, k.part, dot_out,
                                                        hz);
  HGKS_PROF_END(K_SPMV, st);
}

// Restarted GMRES (Algorithm 1) for every mesh of the batch at once, each in
// its own Krylov space; the launch sequence does not depend on the data, so it
// can be captured in a CUDA graph.
template <typename T>
void bgmres_t(const DevMesh &m, Scratch &s, BatchState &bs, const BBuf<T> &k, const hgks_params &p, const double *rhs,
              double *dx, cudaStream_t st) {
  const int mk = p.krylov_dim, hz = bs.hsz, N = m.N, nm = bs.b.nmesh;
  const int64_t vs = s.vstride;
  double *H = bs.hs, *beta = H + (mk + 1) * mk, *lres = beta + 1 + mk;
  const unsigned g = std::max(1, bs.b.nblocks);
  for (int it = 0; it < p.restarts; it++) {
    cudaMemset2DAsync(H, sizeof(double) * hz, 0, sizeof(double) * (mk + 1) * mk, nm, st);
    HGKS_PROF_BEGIN(K_SPMV, st);
    bapply<T, double, T, kSpmv, false>(g, st, m, bs.b, k.off, k.dval, k.dinv, rhs, dx, k.t, nullptr, nullptr,
                                                            nullptr, hz);
    HGKS_PROF_END(K_SPMV, st);
    bprecondition<T>(m, bs, k, p.jacobi_sweeps, k.t, k.w, nullptr, nullptr, st);
    HGKS_PROF_BEGIN(K_DOT, st);
    k_baxpy_dot<T><<<g, kB, 0, st>>>(N, bs.b, k.w, nullptr, nullptr, hz, k.w, 1, k.part, beta, hz);
    HGKS_PROF_END(K_DOT, st);
    if (it == 0) cudaMemcpy2DAsync(lres, sizeof(double) * hz, beta, sizeof(double) * hz, sizeof(double), nm,
                                   cudaMemcpyDeviceToDevice, st);
    HGKS_PROF_BEGIN(K_SCALE, st);
    k_bscale<T><<<g, kB, 0, st>>>(N, bs.b, k.w, beta, hz, k.V);
    HGKS_PROF_END(K_SCALE, st);
    // FP32 vectors: MGS from one pass over the basis (HBM bound, about half the
    // bytes); FP64 vectors: one basis vector per pass (bound by the FP64 rate either way)
    constexpr bool one_pass = std::is_same<T, float>::value;
    for (int j = 0; j < mk; j++) {
      bneumann<T>(m, bs, k, p.jacobi_sweeps, k.V + (size_t)j * vs, k.w, one_pass ? nullptr : k.V,
                  one_pass ? nullptr : H + j, st);
      if constexpr (one_pass) {
        for (int k0 = 0; k0 <= j; k0 += kBatchMdot) {
          HGKS_PROF_BEGIN(K_DOT, st);
          k_bmdot<T><<<g, kB, 0, st>>>(N, bs.b, k.w, k.V, vs, k0, std::min(kBatchMdot, j + 1 - k0), j, k.part, bs.hs,
                                       hz, bs.a_off, bs.g_off);
          HGKS_PROF_END(K_DOT, st);
        }
        HGKS_PROF_BEGIN(K_DOT, st);
        k_bmgs_coef<<<(nm + 63) / 64, 64, 0, st>>>(bs.b, j, mk, bs.hs, hz, bs.a_off, bs.g_off, bs.gram_off);
        HGKS_PROF_END(K_DOT, st);
        HGKS_PROF_BEGIN(K_DOT, st);
        k_bmupdate<T><<<g, kB, 0, st>>>(N, bs.b, k.w, k.V, vs, j, mk, bs.hs, hz, k.part);
        HGKS_PROF_END(K_DOT, st);
      }
      for (int i = 0; !one_pass && i <= j; i++) {
        const bool last = (i == j);
        HGKS_PROF_BEGIN(K_DOT, st);
        k_baxpy_dot<T><<<g, kB, 0, st>>>(N, bs.b, k.w, k.V + (size_t)i * vs, H + i * mk + j, hz,
                                         last ? k.w : k.V + (size_t)(i + 1) * vs, last ? 1 : 0, k.part,
                                         H + (i + 1) * mk + j, hz);
        HGKS_PROF_END(K_DOT, st);
      }
      HGKS_PROF_BEGIN(K_SCALE, st);
      k_bscale<T><<<g, kB, 0, st>>>(N, bs.b, k.w, H + (j + 1) * mk + j, hz, k.V + (size_t)(j + 1) * vs);
      HGKS_PROF_END(K_SCALE, st);
    }
    HGKS_PROF_BEGIN(K_GIVENS, st);
    k_bgivens<<<(nm + 63) / 64, 64, 0, st>>>(bs.b, mk, bs.hs, hz);
    HGKS_PROF_END(K_GIVENS, st);
    HGKS_PROF_BEGIN(K_COMBINE, st);
    k_bcombine<T><<<g, kB, 0, st>>>(N, bs.b, vs, mk, k.V, bs.hs, hz, dx);
    HGKS_PROF_END(K_COMBINE, st);
  }
}

}  // namespace

void launch_batch_gmres(const DevMesh &m, Scratch &s, BatchState &bs, const hgks_params &p, const double *rhs,
                        double *dx, cudaStream_t st) {
  HGKS_RANGE("hgks batch gmres");
  cudaMemset2DAsync(dx, sizeof(double) * m.N, 0, sizeof(double) * m.NL, 5, st);
  if (p.precision == HGKS_MIXED) bgmres_t<float>(m, s, bs, bbuf32(s, bs), p, rhs, dx, st);
  else bgmres_t<double>(m, s, bs, bbuf64(s, bs), p, rhs, dx, st);
}

void launch_batch_density(const DevMesh &m, BatchState &bs, const double *R, cudaStream_t st) {
  HGKS_PROF_BEGIN(K_NORM, st);
  k_bdensity<<<std::max(1, bs.b.nblocks), kB, 0, st>>>(m.N, bs.b, R, m.inv_vol, bs.part, bs.hs + bs.l1_off, bs.hsz);
  HGKS_PROF_END(K_NORM, st);
}

void launch_batch_check(BatchState &bs, cudaStream_t st) {
  HGKS_PROF_BEGIN(K_NORM, st);
  k_bcheck<<<(bs.b.nmesh + 63) / 64, 64, 0, st>>>(bs);
  HGKS_PROF_END(K_NORM, st);
}

void launch_batch_update(const DevMesh &m, BatchState &bs, double *Q, const double *dQ, double *G, const double *Gnew,
                         int ncomp_g, cudaStream_t st) {
  HGKS_PROF_BEGIN(K_UPDATE, st);
  k_bupdate<<<std::max(1, bs.b.nblocks), kB, 0, st>>>(m.N, bs.b, m.ptab, Q, dQ, G, Gnew, ncomp_g);
  HGKS_PROF_END(K_UPDATE, st);
}

void launch_fill(double *a, int64_t n, double v, cudaStream_t st) {
  if (n <= 0) return;
  k_fill<double><<<grid_for(std::min<int64_t>(n, 152 * 2048), 256), 256, 0, st>>>(a, n, v);
  count_launch();
}

void launch_fill_short(short *a, int64_t n, short v, cudaStream_t st) {
  if (n <= 0) return;
  k_fill<short><<<grid_for(std::min<int64_t>(n, 152 * 2048), 256), 256, 0, st>>>(a, n, v);
  count_launch();
}

void launch_offset_index(int *a, int rows, int64_t n, int64_t pitch, int64_t add, cudaStream_t st) {
  if (n <= 0 || rows <= 0 || add == 0) return;
  k_offset_index<<<grid_for(std::min<int64_t>((int64_t)rows * n, 152 * 2048), 256), 256, 0, st>>>(a, rows, n, pitch, add);
  count_launch();
}

}  // namespace hgks
