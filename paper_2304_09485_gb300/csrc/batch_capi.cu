// C ABI of batches (hgks_batch_*): merging meshes into one cell space, state
// copies, and the per-step launch sequence (optionally a CUDA graph).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>
#include "hgks_internal.h"

using namespace hgks;

struct hgks_batch_s {
  Mesh m;                       // the merged cell space (its DevMesh carries ptab/cmesh/fmesh/mact)
  BatchState bs;
  int nmesh = 0;
  hgks_params p0{};             // the fields shared by every mesh (scheme, precision, Krylov sizes)
  std::vector<hgks_params> params;
  std::vector<int64_t> coff, ncell, foff, nface;
  double *Q = nullptr, *G = nullptr;
  int *ones = nullptr;          // [nmesh] 1s, copied into the active flags
  double *hist = nullptr;
  int hist_cap = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

namespace {

#define BCUDA(call)                                       \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_error(e_, #call);  \
  } while (0)

template <typename T>
hgks_status balloc(Mesh &m, T **p, size_t n) {
  void *q = nullptr;
  *p = nullptr;
  if (n == 0) return HGKS_OK;
  hgks_status st = mesh_alloc(m, &q, n * sizeof(T));
  *p = (T *)q;
  return st;
}

// rows x n_k block of a [rows][n_k] source array into columns [col, col + n_k) of a [rows][pitch] array
template <typename T>
hgks_status copy_rows(T *dst, int64_t pitch, int64_t col, const T *src, int64_t n_k, int rows, cudaStream_t st) {
  if (!src || !dst || n_k == 0 || rows == 0) return HGKS_OK;
  BCUDA(cudaMemcpy2DAsync(dst + col, sizeof(T) * pitch, src, sizeof(T) * n_k, sizeof(T) * n_k, rows,
                          cudaMemcpyDeviceToDevice, st));
  return HGKS_OK;
}

bool same_shared(const hgks_params &a, const hgks_params &b) {
  return a.scheme == b.scheme && a.precision == b.precision && a.jv_mode == b.jv_mode &&
         a.krylov_dim == b.krylov_dim && a.restarts == b.restarts && a.jacobi_sweeps == b.jacobi_sweeps;
}

// Allocate the merged arrays and copy every mesh's data into its range.
hgks_status merge(hgks_batch_s &B, const hgks_mesh *meshes, cudaStream_t st) {
  Mesh &M = B.m;
  DevMesh &d = M.d;
  const int64_t N = M.N, F = M.F;
  const bool weno = M.schemes & 1, hweno = M.schemes & 2;
  hgks_status s;
  if ((s = balloc(M, &d.vol, N)) || (s = balloc(M, &d.inv_vol, N)) || (s = balloc(M, &d.h, N)) ||
      (s = balloc(M, &d.m2, 6 * N)) || (s = balloc(M, &d.cnb, 4 * N)) || (s = balloc(M, &d.cface, 4 * N)) ||
      (s = balloc(M, &d.xg, 36 * N)) || (s = balloc(M, &d.subvalid, N)) || (s = balloc(M, &d.fl, F)) ||
      (s = balloc(M, &d.fr, F)) || (s = balloc(M, &d.ftag, F)) || (s = balloc(M, &d.fT, 9 * F)) ||
      (s = balloc(M, &d.fS, F)) || (s = balloc(M, &d.fdist, F)))
    return s;
  if (weno && ((s = balloc(M, &d.sten, (size_t)kBig * N)) || (s = balloc(M, &d.X0, (size_t)9 * kBig * N)) ||
               (s = balloc(M, &d.Xm, (size_t)12 * kBig * N))))
    return s;
  if (hweno && ((s = balloc(M, &d.H0, (size_t)9 * 19 * N)) || (s = balloc(M, &d.Hm, (size_t)12 * 7 * N)))) return s;
  // padding cells: unit volume and size, no neighbours, zero matrices
  launch_fill(d.vol, N, 1.0, st);
  launch_fill(d.inv_vol, N, 1.0, st);
  launch_fill(d.h, N, 1.0, st);
  BCUDA(cudaMemsetAsync(d.m2, 0, sizeof(double) * 6 * N, st));
  BCUDA(cudaMemsetAsync(d.xg, 0, sizeof(double) * 36 * N, st));
  BCUDA(cudaMemsetAsync(d.cnb, 0xff, sizeof(int) * 4 * N, st));
  BCUDA(cudaMemsetAsync(d.cface, 0xff, sizeof(int) * 4 * N, st));
  BCUDA(cudaMemsetAsync(d.subvalid, 0, N, st));
  if (weno) {
    BCUDA(cudaMemsetAsync(d.sten, 0xff, sizeof(int) * kBig * N, st));
    BCUDA(cudaMemsetAsync(d.X0, 0, sizeof(double) * 9 * kBig * N, st));
    BCUDA(cudaMemsetAsync(d.Xm, 0, sizeof(double) * 12 * kBig * N, st));
  }
  if (hweno) {
    BCUDA(cudaMemsetAsync(d.H0, 0, sizeof(double) * 9 * 19 * N, st));
    BCUDA(cudaMemsetAsync(d.Hm, 0, sizeof(double) * 12 * 7 * N, st));
  }
  for (int k = 0; k < B.nmesh; k++) {
    const DevMesh &a = mesh_of(meshes[k])->d;
    const int64_t c0 = B.coff[k], nk = B.ncell[k], f0 = B.foff[k], fk = B.nface[k];
    if ((s = copy_rows(d.vol, N, c0, a.vol, nk, 1, st)) || (s = copy_rows(d.inv_vol, N, c0, a.inv_vol, nk, 1, st)) ||
        (s = copy_rows(d.h, N, c0, a.h, nk, 1, st)) || (s = copy_rows(d.m2, N, c0, a.m2, nk, 6, st)) ||
        (s = copy_rows(d.cnb, N, c0, a.cnb, nk, 4, st)) || (s = copy_rows(d.cface, N, c0, a.cface, nk, 4, st)) ||
        (s = copy_rows(d.xg, N, c0, a.xg, nk, 36, st)) || (s = copy_rows(d.subvalid, N, c0, a.subvalid, nk, 1, st)) ||
        (s = copy_rows(d.fl, F, f0, a.fl, fk, 1, st)) || (s = copy_rows(d.fr, F, f0, a.fr, fk, 1, st)) ||
        (s = copy_rows(d.ftag, F, f0, a.ftag, fk, 1, st)) || (s = copy_rows(d.fT, F, f0, a.fT, fk, 9, st)) ||
        (s = copy_rows(d.fS, F, f0, a.fS, fk, 1, st)) || (s = copy_rows(d.fdist, F, f0, a.fdist, fk, 1, st)))
      return s;
    if (weno && ((s = copy_rows(d.sten, N, c0, a.sten, nk, kBig, st)) ||
                 (s = copy_rows(d.X0, N, c0, a.X0, nk, 9 * kBig, st)) ||
                 (s = copy_rows(d.Xm, N, c0, a.Xm, nk, 12 * kBig, st))))
      return s;
    if (hweno && ((s = copy_rows(d.H0, N, c0, a.H0, nk, 9 * 19, st)) || (s = copy_rows(d.Hm, N, c0, a.Hm, nk, 12 * 7, st))))
      return s;
    // cell indices move by the mesh's cell offset, face indices (2 f + side) by twice its face offset
    launch_offset_index(d.cnb + c0, 4, nk, N, c0, st);
    launch_offset_index(d.cface + c0, 4, nk, N, 2 * f0, st);
    if (weno) launch_offset_index(d.sten + c0, kBig, nk, N, c0, st);
    launch_offset_index(d.fl + f0, 1, fk, F, c0, st);
    launch_offset_index(d.fr + f0, 1, fk, F, c0, st);
  }
  return HGKS_OK;
}

hgks_status check_mesh(const hgks_batch_s *b, int32_t k) {
  if (!b) return fail_msg(HGKS_ERR_ARG, "batch is NULL");
  if (k < 0 || k >= b->nmesh) return fail_msg(HGKS_ERR_ARG, "mesh index out of range");
  return HGKS_OK;
}

// order the batch's own stream after the caller's
hgks_status enter(hgks_batch_s &B, cudaStream_t user) {
  BCUDA(cudaSetDevice(B.m.device));
  BCUDA(cudaEventRecord(B.ev_in, user));
  BCUDA(cudaStreamWaitEvent(B.stream, B.ev_in, 0));
  return HGKS_OK;
}
hgks_status leave(hgks_batch_s &B, cudaStream_t user) {
  BCUDA(cudaEventRecord(B.ev_out, B.stream));
  BCUDA(cudaStreamWaitEvent(user, B.ev_out, 0));
  return HGKS_OK;
}

}  // namespace

namespace {

template <typename T>
hgks_status copy_rows_out(T *dst, int64_t n_k, const T *src, int64_t pitch, int64_t col, int rows, cudaStream_t st) {
  if (!src || !dst || n_k == 0 || rows == 0) return HGKS_OK;
  BCUDA(cudaMemcpy2DAsync(dst, sizeof(T) * n_k, src + col, sizeof(T) * pitch, sizeof(T) * n_k, rows,
                          cudaMemcpyDeviceToDevice, st));
  return HGKS_OK;
}

template <typename T>
hgks_status upload_vec(Mesh &m, T **p, const std::vector<T> &v) {
  hgks_status s = balloc(m, p, v.size());
  if (s) return s;
  BCUDA(cudaMemcpy(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return HGKS_OK;
}

void destroy(hgks_batch_s *B) {
  if (!B) return;
  cudaSetDevice(B->m.device);
  if (B->stream) cudaStreamSynchronize(B->stream);
  mesh_free_all(B->m);
  if (B->hist) cudaFree(B->hist);
  if (B->ev_in) cudaEventDestroy(B->ev_in);
  if (B->ev_out) cudaEventDestroy(B->ev_out);
  if (B->stream) cudaStreamDestroy(B->stream);
  delete B;
}

hgks_status activate_all(hgks_batch_s &B) {
  BCUDA(cudaMemcpyAsync(B.bs.b.active, B.ones, sizeof(int) * B.nmesh, cudaMemcpyDeviceToDevice, B.stream));
  return HGKS_OK;
}

bool compact(const hgks_batch_s &B) { return B.p0.scheme == HGKS_HWENO; }

// One outer step of Algorithm 1 for every active mesh: R(Q), the density
// residual (and, in a solve, the convergence test that may stop a mesh), A,
// GMRES, Q += dQ. The sequence is data independent (graph capturable).
void enqueue_step(hgks_batch_s &B, bool check, double drop_tol, int max_steps) {
  DevMesh &d = B.m.d;
  Scratch &s = B.m.s;
  cudaStream_t st = B.stream;
  launch_residual(d, s, B.p0, B.Q, B.G, s.R, compact(B) ? s.Gnew : nullptr, st, true);
  launch_batch_density(d, B.bs, s.R, st);
  if (check) launch_batch_check(B.bs, drop_tol, max_steps, st);
  launch_assemble(d, s, B.p0, B.Q, s.dt, nullptr, nullptr, st, true);
  launch_batch_gmres(d, s, B.bs, B.p0, s.R, s.dQ, st);
  launch_batch_update(d, B.bs, B.Q, s.dQ, B.G, s.Gnew, compact(B) ? 15 : 0, st);
}

hgks_status launch_status() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "kernel launch");
  return HGKS_OK;
}

}  // namespace

extern "C" {

hgks_status hgks_batch_create(const hgks_mesh *meshes, const hgks_params *params, int32_t n_meshes, hgks_batch *out) {
  if (!out) return fail_msg(HGKS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!meshes || !params) return fail_msg(HGKS_ERR_ARG, "meshes or params is NULL");
  if (n_meshes < 1 || n_meshes > 32767) return fail_msg(HGKS_ERR_ARG, "n_meshes must be in 1..32767");
  for (int k = 0; k < n_meshes; k++)
    if (!meshes[k]) return fail_msg(HGKS_ERR_ARG, "a mesh handle is NULL");
  const int dev = mesh_of(meshes[0])->device;
  int schemes = 3;
  int64_t N = 0, F = 0, Fb = 0;
  hgks_status st;
  for (int k = 0; k < n_meshes; k++) {
    const Mesh &a = *mesh_of(meshes[k]);
    if (a.device != dev) return fail_msg(HGKS_ERR_ARG, "meshes of a batch must be on one device");
    if ((st = check_params(a, &params[k]))) return st;
    if (!same_shared(params[0], params[k]))
      return fail_msg(HGKS_ERR_ARG, "scheme, precision, jv_mode, krylov_dim, restarts, jacobi_sweeps must agree");
    schemes &= a.schemes;
    N += (a.N + kBatchBlock - 1) / kBatchBlock * kBatchBlock;
    F += a.F;
    Fb += a.Fb;
  }
  if (6 * std::max(N, F) >= (int64_t)INT32_MAX) return fail_msg(HGKS_ERR_ARG, "batch too large for 32-bit indexing");
  hgks_batch_s *B = new (std::nothrow) hgks_batch_s;
  if (!B) return fail_msg(HGKS_ERR_OOM, "host allocation");
  auto bail = [&](hgks_status s2) { destroy(B); return s2; };
  B->nmesh = n_meshes;
  B->params.assign(params, params + n_meshes);
  B->p0 = params[0];
  Mesh &M = B->m;
  M.device = dev; M.N = N; M.F = F; M.Fb = Fb; M.schemes = schemes;
  M.d.N = (int)N; M.d.F = (int)F;
  int64_t c = 0, f = 0;
  for (int k = 0; k < n_meshes; k++) {
    const Mesh &a = *mesh_of(meshes[k]);
    B->coff.push_back(c); B->ncell.push_back(a.N); B->foff.push_back(f); B->nface.push_back(a.F);
    c += (a.N + kBatchBlock - 1) / kBatchBlock * kBatchBlock;
    f += a.F;
  }
  if (cudaSetDevice(dev) != cudaSuccess) return bail(fail_msg(HGKS_ERR_CUDA, "cudaSetDevice"));
  if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&B->ev_out, cudaEventDisableTiming) != cudaSuccess)
    return bail(fail_msg(HGKS_ERR_CUDA, "stream or event creation"));
  if ((st = merge(*B, meshes, B->stream))) return bail(st);
  // per-cell, per-face and per-block mesh tables
  const int nblocks = (int)(N / kBatchBlock);
  std::vector<short> cmesh(N, (short)-1), fmesh(F), bmesh(nblocks);
  std::vector<int> bstart(n_meshes + 1), ncell(n_meshes), ones(n_meshes, 1);
  for (int k = 0; k < n_meshes; k++) {
    std::fill(cmesh.begin() + B->coff[k], cmesh.begin() + B->coff[k] + B->ncell[k], (short)k);
    std::fill(fmesh.begin() + B->foff[k], fmesh.begin() + B->foff[k] + B->nface[k], (short)k);
    const int b0 = (int)(B->coff[k] / kBatchBlock), b1 = (int)((B->coff[k] + (B->ncell[k] + kBatchBlock - 1) / kBatchBlock * kBatchBlock) / kBatchBlock);
    std::fill(bmesh.begin() + b0, bmesh.begin() + b1, (short)k);
    bstart[k] = b0;
    ncell[k] = (int)B->ncell[k];
  }
  bstart[n_meshes] = nblocks;
  BatchState &bs = B->bs;
  hgks_params *ptab = nullptr;
  short *cm = nullptr, *fm = nullptr, *bm = nullptr;
  int *bst = nullptr, *nc = nullptr;
  const int mk = B->p0.krylov_dim;
  bs.kdim = mk;
  bs.l1_off = (mk + 1) * mk + 1 + mk + 2;
  bs.hsz = (bs.l1_off + 1 + 7) / 8 * 8;
  const bool mixed = B->p0.precision == HGKS_MIXED;
  if ((st = upload_vec(M, &ptab, B->params)) || (st = upload_vec(M, &cm, cmesh)) || (st = upload_vec(M, &fm, fmesh)) ||
      (st = upload_vec(M, &bm, bmesh)) || (st = upload_vec(M, &bst, bstart)) || (st = upload_vec(M, &nc, ncell)) ||
      (st = upload_vec(M, &B->ones, ones)) || (st = balloc(M, &bs.b.counters, n_meshes)) ||
      (st = balloc(M, &bs.b.active, n_meshes)) || (st = balloc(M, &bs.steps, n_meshes)) ||
      (st = balloc(M, &bs.conv, n_meshes)) || (st = balloc(M, &bs.bad, n_meshes)) || (st = balloc(M, &bs.ref, n_meshes)) ||
      (st = balloc(M, &bs.res, n_meshes)) || (st = balloc(M, &bs.hs, (size_t)n_meshes * bs.hsz)) ||
      (st = balloc(M, &bs.part, nblocks)) || (mixed && (st = balloc(M, &bs.part32, nblocks))) ||
      (st = balloc(M, &B->Q, 5 * N)) || (compact(*B) && (st = balloc(M, &B->G, 15 * N))))
    return bail(st);
  if (cudaMemset(bs.b.counters, 0, sizeof(unsigned) * n_meshes) != cudaSuccess ||
      cudaMemset(bs.hs, 0, sizeof(double) * n_meshes * bs.hsz) != cudaSuccess ||
      cudaMemcpy(bs.b.active, B->ones, sizeof(int) * n_meshes, cudaMemcpyDeviceToDevice) != cudaSuccess ||
      cudaMemset(B->Q, 0, sizeof(double) * 5 * N) != cudaSuccess ||
      (B->G && cudaMemset(B->G, 0, sizeof(double) * 15 * N) != cudaSuccess))
    return bail(fail_msg(HGKS_ERR_CUDA, "batch table initialisation"));
  bs.b.nmesh = n_meshes;
  bs.b.nblocks = nblocks;
  bs.b.bmesh = bm;
  bs.b.bstart = bst;
  bs.ncell = nc;
  M.d.ptab = ptab;
  M.d.cmesh = cm;
  M.d.fmesh = fm;
  M.d.mact = bs.b.active;
  if ((st = ensure_scratch(M, mk, true, mixed))) return bail(st);
  if (cudaStreamSynchronize(B->stream) != cudaSuccess || (st = launch_status())) return bail(st ? st : fail_msg(HGKS_ERR_CUDA, "merge"));
  *out = B;
  return HGKS_OK;
}

hgks_status hgks_batch_destroy(hgks_batch batch) {
  if (!batch) return fail_msg(HGKS_ERR_ARG, "batch is NULL");
  destroy(batch);
  return HGKS_OK;
}

hgks_status hgks_batch_info(hgks_batch batch, hgks_batch_info_t *info) {
  if (!batch || !info) return fail_msg(HGKS_ERR_ARG, "NULL argument");
  info->n_cells = batch->m.N;
  info->n_faces = batch->m.F;
  info->device_bytes = (int64_t)batch->m.bytes;
  info->n_meshes = batch->nmesh;
  info->blk_recon = batch->m.s.blk_recon;
  info->blk_flux = batch->m.s.blk_flux;
  return HGKS_OK;
}

hgks_status hgks_batch_set_state(hgks_batch batch, int32_t k, const double *Q, const double *G, void *cuda_stream) {
  hgks_status st = check_mesh(batch, k);
  if (st) return st;
  hgks_batch_s &B = *batch;
  if (!Q || (compact(B) && !G)) return fail_msg(HGKS_ERR_ARG, "Q (or G) is NULL");
  cudaStream_t user = (cudaStream_t)cuda_stream;
  if ((st = enter(B, user))) return st;
  if ((st = copy_rows(B.Q, B.m.N, B.coff[k], Q, B.ncell[k], 5, B.stream))) return st;
  if (compact(B) && (st = copy_rows(B.G, B.m.N, B.coff[k], G, B.ncell[k], 15, B.stream))) return st;
  return leave(B, user);
}

hgks_status hgks_batch_get_state(hgks_batch batch, int32_t k, double *Q, double *G, double *R, double *G_new,
                                 void *cuda_stream) {
  hgks_status st = check_mesh(batch, k);
  if (st) return st;
  hgks_batch_s &B = *batch;
  cudaStream_t user = (cudaStream_t)cuda_stream;
  const int64_t N = B.m.N, c0 = B.coff[k], nk = B.ncell[k];
  if ((st = enter(B, user))) return st;
  if ((st = copy_rows_out(Q, nk, B.Q, N, c0, 5, B.stream)) || (st = copy_rows_out(R, nk, B.m.s.R, N, c0, 5, B.stream)))
    return st;
  if (compact(B) && ((st = copy_rows_out(G, nk, B.G, N, c0, 15, B.stream)) ||
                     (st = copy_rows_out(G_new, nk, B.m.s.Gnew, N, c0, 15, B.stream))))
    return st;
  return leave(B, user);
}

}  // extern "C"

extern "C" {

hgks_status hgks_batch_residual(hgks_batch batch, void *cuda_stream) {
  if (!batch) return fail_msg(HGKS_ERR_ARG, "batch is NULL");
  hgks_batch_s &B = *batch;
  cudaStream_t user = (cudaStream_t)cuda_stream;
  hgks_status st;
  if ((st = enter(B, user)) || (st = activate_all(B))) return st;
  launch_residual(B.m.d, B.m.s, B.p0, B.Q, B.G, B.m.s.R, compact(B) ? B.m.s.Gnew : nullptr, B.stream, true);
  if ((st = launch_status())) return st;
  return leave(B, user);
}

hgks_status hgks_batch_gmres_step(hgks_batch batch, hgks_step_info *info, void *cuda_stream) {
  if (!batch) return fail_msg(HGKS_ERR_ARG, "batch is NULL");
  hgks_batch_s &B = *batch;
  cudaStream_t user = (cudaStream_t)cuda_stream;
  hgks_status st;
  if ((st = enter(B, user)) || (st = activate_all(B))) return st;
  enqueue_step(B, false, 0.0, 0);
  if ((st = launch_status())) return st;
  const int n = B.nmesh, hz = B.bs.hsz;
  std::vector<double> hs((size_t)n * hz);
  int nonphys = 0;
  BCUDA(cudaMemcpyAsync(hs.data(), B.bs.hs, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, B.stream));
  BCUDA(cudaMemcpyAsync(&nonphys, B.m.s.flags, sizeof(int), cudaMemcpyDeviceToHost, B.stream));
  BCUDA(cudaMemsetAsync(B.m.s.flags, 0, sizeof(int), B.stream));
  BCUDA(cudaStreamSynchronize(B.stream));
  if ((st = leave(B, user))) return st;
  const int mk = B.p0.krylov_dim, lres = (mk + 1) * mk + 1 + mk;
  bool finite = true;
  for (int k = 0; k < n; k++) {
    const double *r = hs.data() + (size_t)k * hz;
    const double res = r[B.bs.l1_off] / (double)B.ncell[k];
    finite = finite && std::isfinite(res);
    if (info) {
      info[k].res_l1 = res;
      info[k].lin_res[0] = r[lres];
      info[k].lin_res[1] = r[lres + 1];
      info[k].krylov_iters = B.p0.restarts * mk;
      info[k].nonphysical = nonphys;   // counted over the whole batch
    }
  }
  if (!finite) return fail_msg(HGKS_ERR_NONPHYSICAL, "non-finite residual");
  return HGKS_OK;
}

hgks_status hgks_batch_solve_steady(hgks_batch batch, double drop_tol, int32_t max_steps, int32_t use_graph,
                                    double *hist_host, hgks_solve_info *info, void *cuda_stream) {
  if (!batch) return fail_msg(HGKS_ERR_ARG, "batch is NULL");
  if (!(drop_tol > 0.0) || max_steps < 0) return fail_msg(HGKS_ERR_ARG, "drop_tol must be > 0 and max_steps >= 0");
  hgks_batch_s &B = *batch;
  BatchState &bs = B.bs;
  const int n = B.nmesh;
  cudaStream_t user = (cudaStream_t)cuda_stream;
  hgks_status st;
  if ((st = enter(B, user))) return st;
  const size_t hlen = (size_t)max_steps + 1;
  if (hist_host && (size_t)B.hist_cap < hlen * n) {
    if (B.hist) { BCUDA(cudaStreamSynchronize(B.stream)); cudaFree(B.hist); B.hist = nullptr; B.hist_cap = 0; }
    BCUDA(cudaMalloc(&B.hist, sizeof(double) * hlen * n));
    B.hist_cap = (int)(hlen * n);
  }
  bs.hist = hist_host ? B.hist : nullptr;
  bs.hist_len = (int)hlen;
  if (hist_host) BCUDA(cudaMemsetAsync(B.hist, 0, sizeof(double) * hlen * n, B.stream));
  if ((st = activate_all(B))) return st;
  BCUDA(cudaMemsetAsync(bs.steps, 0, sizeof(int) * n, B.stream));
  BCUDA(cudaMemsetAsync(bs.conv, 0, sizeof(int) * n, B.stream));
  BCUDA(cudaMemsetAsync(bs.bad, 0, sizeof(int) * n, B.stream));
  BCUDA(cudaMemsetAsync(bs.ref, 0, sizeof(double) * n, B.stream));
  BCUDA(cudaMemsetAsync(bs.res, 0, sizeof(double) * n, B.stream));
  // the step, captured once (profiling records events around launches: no graph then)
  cudaGraphExec_t exec = nullptr;
  int64_t per_step = 0;
  if (use_graph && !g_prof_on) {
    cudaGraph_t graph = nullptr;
    BCUDA(cudaStreamBeginCapture(B.stream, cudaStreamCaptureModeThreadLocal));
    const int64_t l0 = g_launches;
    enqueue_step(B, true, drop_tol, max_steps);
    per_step = g_launches - l0;
    g_launches = l0;
    cudaError_t e = cudaStreamEndCapture(B.stream, &graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) { cudaGetLastError(); return cuda_error(e, "CUDA graph capture of the batch step"); }
  }
  // each mesh takes at most max_steps steps and one last test; the host polls
  // the active flags every few steps (finished meshes cost no work meanwhile)
  std::vector<int> act(n);
  const int poll = 4;
  for (int it = 0; it <= max_steps;) {
    const int chunk = std::min(poll, max_steps + 1 - it);
    for (int c = 0; c < chunk; c++) {
      if (exec) {
        cudaError_t e = cudaGraphLaunch(exec, B.stream);
        if (e != cudaSuccess) { cudaGraphExecDestroy(exec); return cuda_error(e, "cudaGraphLaunch"); }
        g_launches += per_step;
      } else {
        enqueue_step(B, true, drop_tol, max_steps);
      }
    }
    it += chunk;
    cudaError_t e = cudaMemcpyAsync(act.data(), bs.b.active, sizeof(int) * n, cudaMemcpyDeviceToHost, B.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B.stream);
    if (e != cudaSuccess) { if (exec) cudaGraphExecDestroy(exec); return cuda_error(e, "batch solve"); }
    if (std::none_of(act.begin(), act.end(), [](int a) { return a != 0; })) break;
  }
  if (exec) cudaGraphExecDestroy(exec);
  if ((st = launch_status())) return st;
  std::vector<int> steps(n), conv(n), bad(n);
  std::vector<double> ref(n), res(n);
  BCUDA(cudaMemcpyAsync(steps.data(), bs.steps, sizeof(int) * n, cudaMemcpyDeviceToHost, B.stream));
  BCUDA(cudaMemcpyAsync(conv.data(), bs.conv, sizeof(int) * n, cudaMemcpyDeviceToHost, B.stream));
  BCUDA(cudaMemcpyAsync(bad.data(), bs.bad, sizeof(int) * n, cudaMemcpyDeviceToHost, B.stream));
  BCUDA(cudaMemcpyAsync(ref.data(), bs.ref, sizeof(double) * n, cudaMemcpyDeviceToHost, B.stream));
  BCUDA(cudaMemcpyAsync(res.data(), bs.res, sizeof(double) * n, cudaMemcpyDeviceToHost, B.stream));
  if (hist_host) BCUDA(cudaMemcpyAsync(hist_host, B.hist, sizeof(double) * hlen * n, cudaMemcpyDeviceToHost, B.stream));
  BCUDA(cudaStreamSynchronize(B.stream));
  bs.hist = nullptr;
  if ((st = leave(B, user))) return st;
  bool all_conv = true, any_bad = false;
  for (int k = 0; k < n; k++) {
    if (info) { info[k].steps = steps[k]; info[k].converged = conv[k]; info[k].res_ref = ref[k]; info[k].res_final = res[k]; }
    all_conv = all_conv && conv[k];
    any_bad = any_bad || bad[k];
  }
  if (any_bad) return fail_msg(HGKS_ERR_NONPHYSICAL, "non-finite residual in a mesh of the batch");
  if (!all_conv) return fail_msg(HGKS_ERR_NOT_CONVERGED, "max_steps reached by a mesh of the batch");
  return HGKS_OK;
}

hgks_status hgks_batch_autotune(hgks_batch batch, int32_t *blk_recon, int32_t *blk_flux, void *cuda_stream) {
  if (!batch) return fail_msg(HGKS_ERR_ARG, "batch is NULL");
  hgks_batch_s &B = *batch;
  Scratch &s = B.m.s;
  cudaStream_t user = (cudaStream_t)cuda_stream;
  hgks_status st;
  if ((st = enter(B, user)) || (st = activate_all(B))) return st;
  cudaEvent_t a = nullptr, b = nullptr;
  BCUDA(cudaEventCreate(&a));
  BCUDA(cudaEventCreate(&b));
  auto time_residual = [&](float &ms) -> hgks_status {
    BCUDA(cudaEventRecord(a, B.stream));
    for (int r = 0; r < 3; r++)
      launch_residual(B.m.d, s, B.p0, B.Q, B.G, s.R, compact(B) ? s.Gnew : nullptr, B.stream, true);
    BCUDA(cudaEventRecord(b, B.stream));
    BCUDA(cudaEventSynchronize(b));
    BCUDA(cudaEventElapsedTime(&ms, a, b));
    return launch_status();
  };
  const int cand[3] = {64, 128, 256};
  float ms = 0.f;
  launch_residual(B.m.d, s, B.p0, B.Q, B.G, s.R, compact(B) ? s.Gnew : nullptr, B.stream, true);   // warm-up
  for (int pass = 0; pass < 2 && !st; pass++) {
    int *blk = pass == 0 ? &s.blk_recon : &s.blk_flux;
    int best = *blk;
    float best_ms = 1e30f;
    for (int c : cand) {
      *blk = c;
      if ((st = time_residual(ms))) break;
      if (ms < best_ms) { best_ms = ms; best = c; }
    }
    *blk = best;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st) return st;
  if (blk_recon) *blk_recon = s.blk_recon;
  if (blk_flux) *blk_flux = s.blk_flux;
  return leave(B, user);
}

}  // extern "C"
