// Batches (hgks_batch_*): an arena of cells and faces in which meshes are
// placed in ranges (slots), copies of state, and the per-step launch sequence
// (optionally replayed from a CUDA graph).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>
#include "batch_impl.h"

using namespace hgks;

struct hgks_batch_s {
  Batch *B = nullptr;
};

namespace hgks {

#define BCUDA(call)                                       \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_error(e_, #call);  \
  } while (0)

// ---------------------------------------------------------------- ranges
void RangeAlloc::init(int64_t c) {
  cap = c;
  free.clear();
  if (c > 0) free.push_back({0, c});
}
int64_t RangeAlloc::take(int64_t len) {
  if (len <= 0) return 0;
  for (size_t k = 0; k < free.size(); k++) {
    if (free[k].len < len) continue;
    const int64_t s = free[k].start;
    free[k].start += len;
    free[k].len -= len;
    if (free[k].len == 0) free.erase(free.begin() + (long)k);
    return s;
  }
  return -1;
}
void RangeAlloc::give(int64_t start, int64_t len) {
  if (len <= 0) return;
  auto it = std::lower_bound(free.begin(), free.end(), start, [](const Range &r, int64_t s) { return r.start < s; });
  it = free.insert(it, {start, len});
  size_t k = (size_t)(it - free.begin());
  if (k + 1 < free.size() && free[k].start + free[k].len == free[k + 1].start) {
    free[k].len += free[k + 1].len;
    free.erase(free.begin() + (long)k + 1);
  }
  if (k > 0 && free[k - 1].start + free[k - 1].len == free[k].start) {
    free[k - 1].len += free[k].len;
    free.erase(free.begin() + (long)k);
  }
}
int64_t RangeAlloc::largest() const {
  int64_t m = 0;
  for (auto &r : free) m = std::max(m, r.len);
  return m;
}

// ---------------------------------------------------------------- sources
MeshSource source_of(const Mesh &a) {
  MeshSource s;
  const DevMesh &d = a.d;
  s.N = a.N; s.F = a.F; s.Fb = a.Fb; s.schemes = a.schemes;
  s.vol = d.vol; s.inv_vol = d.inv_vol; s.h = d.h; s.m2 = d.m2; s.xg = d.xg;
  s.cnb = d.cnb; s.cface = d.cface; s.sten = d.sten; s.fl = d.fl; s.fr = d.fr; s.subvalid = d.subvalid;
  s.X0 = d.X0; s.Xs = d.Xs; s.ssl = d.ssl; s.H0 = d.H0; s.Hm = d.Hm; s.ftag = d.ftag; s.fT = d.fT; s.fS = d.fS; s.fdist = d.fdist;
  s.fw = d.fw; s.hex = d.hex;
  return s;
}
MeshSource source_of(const HostMesh &hm, std::vector<double> &inv) {
  MeshSource s;
  s.N = hm.N; s.F = hm.F; s.Fb = hm.Fb;
  s.schemes = (hm.X0.empty() ? 0 : 1) | (hm.H0.empty() ? 0 : 2);
  inv.resize(hm.N);
  for (int64_t i = 0; i < hm.N; i++) inv[i] = 1.0 / hm.vol[i];
  auto P = [](const auto &v) { return v.empty() ? nullptr : v.data(); };
  s.vol = P(hm.vol); s.inv_vol = inv.data(); s.h = P(hm.h); s.m2 = P(hm.m2); s.xg = P(hm.xg);
  s.cnb = P(hm.cnb); s.cface = P(hm.cface); s.sten = P(hm.sten); s.fl = P(hm.fl); s.fr = P(hm.fr);
  s.subvalid = P(hm.subvalid); s.X0 = P(hm.X0); s.Xs = P(hm.Xs); s.ssl = P(hm.ssl); s.H0 = P(hm.H0); s.Hm = P(hm.Hm);
  s.ftag = P(hm.ftag); s.fT = P(hm.fT); s.fS = P(hm.fS); s.fdist = P(hm.fdist);
  s.fw = P(hm.fw); s.hex = hm.hex;
  return s;
}

// ---------------------------------------------------------------- helpers
namespace {

template <typename T>
hgks_status balloc(Mesh &m, T **p, size_t n) {
  void *q = nullptr;
  *p = nullptr;
  if (n == 0) return HGKS_OK;
  hgks_status st = mesh_alloc(m, &q, n * sizeof(T));
  *p = (T *)q;
  return st;
}

// a [rows][n_k] source (host or device) into columns [col, col + n_k) of a [rows][pitch] array
template <typename T>
hgks_status copy_in(T *dst, int64_t pitch, int64_t col, const T *src, int64_t n_k, int rows, cudaStream_t st) {
  if (!src || !dst || n_k == 0 || rows == 0) return HGKS_OK;
  BCUDA(cudaMemcpy2DAsync(dst + col, sizeof(T) * pitch, src, sizeof(T) * n_k, sizeof(T) * n_k, rows,
                          cudaMemcpyDefault, st));
  return HGKS_OK;
}
template <typename T>
hgks_status copy_out(T *dst, int64_t n_k, const T *src, int64_t pitch, int64_t col, int rows, cudaStream_t st) {
  if (!src || !dst || n_k == 0 || rows == 0) return HGKS_OK;
  BCUDA(cudaMemcpy2DAsync(dst, sizeof(T) * n_k, src + col, sizeof(T) * pitch, sizeof(T) * n_k, rows,
                          cudaMemcpyDefault, st));
  return HGKS_OK;
}
template <typename T>
hgks_status upload(T *dst, const T *src, size_t n, cudaStream_t st) {
  BCUDA(cudaMemcpyAsync(dst, src, sizeof(T) * n, cudaMemcpyHostToDevice, st));
  return HGKS_OK;
}

hgks_status launch_status() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "kernel launch");
  return HGKS_OK;
}

}  // namespace

// rows of the per-cell and per-face arrays of a cell kind
struct Rows {
  int NF, NG, BIG, NSUBW, SUBK, HCOLS;
  explicit Rows(bool hex)
      : NF(hex ? HexShape::NF : TetShape::NF), NG(hex ? HexShape::NG : TetShape::NG),
        BIG(hex ? HexShape::BIG : TetShape::BIG), NSUBW(hex ? HexShape::NSUBW : TetShape::NSUBW),
        SUBK(hex ? HexShape::SUBK : TetShape::SUBK),
        HCOLS(hex ? ShapeOf<HexShape>::HCOLS : ShapeOf<TetShape>::HCOLS) {}
};

bool compact(const Batch &B) { return B.p0.scheme == HGKS_HWENO; }

// the cells and faces the kernels of a batch cover: up to the end of the last range in use
static void update_live(Batch &B) {
  int64_t nl = 0, fl = 0;
  for (auto &S : B.slots)
    if (S.used) { nl = std::max(nl, S.c0 + S.cpad); fl = std::max(fl, S.f0 + S.nface); }
  B.m.d.NL = (int)nl;
  B.m.d.FL = (int)fl;
  B.bs.b.nblocks = (int)(nl / kBatchBlock);
}

bool same_shared(const hgks_params &a, const hgks_params &b) {
  return a.scheme == b.scheme && a.precision == b.precision && a.jv_mode == b.jv_mode &&
         a.krylov_dim == b.krylov_dim && a.restarts == b.restarts && a.jacobi_sweeps == b.jacobi_sweeps;
}

// Device bytes of an arena (the allocations of batch_new and ensure_scratch).
int64_t arena_bytes(int64_t cells, int64_t faces, const hgks_params &p, int schemes, bool hex) {
  const int64_t N = cells, F = faces, nb = cells / kBatchBlock;
  const bool mixed = p.precision == HGKS_MIXED, hw = p.scheme == HGKS_HWENO;
  const Rows rw(hex);
  const int64_t ncoef = 45 + 15 * std::max(rw.NSUBW, rw.NF);
  int64_t c = 0;
  c += 8 * (3 + 6 + rw.NF * rw.NG * 3) + 4 * 2 * rw.NF + 1 + 2;   // geometry, neighbours, faces, mesh id
  if (schemes & 1) c += 4 * rw.BIG + 8 * 9 * rw.BIG + 8 * rw.NSUBW * 3 * rw.SUBK + 4 * rw.NSUBW;   // big stencil, matrices, slots
  if (schemes & 2) c += 8 * (9 * rw.HCOLS + rw.NF * 21);       // compact matrices
  c += 8 * (5 + (hw ? 15 : 0));                                 // Q, G
  c += 8 * (ncoef + 1 + 25 * rw.NF + 2 + 5 + 15 + 5 + 15);      // coef, dt, off, dval/dinv, R, Gnew, dQ, w/t/t2
  c += mixed ? (4 * (6 + 4 * rw.NF) + 4 * 2 + 4 * 15 + 4 * 5 * (p.krylov_dim + 1)) : 8 * 5 * (p.krylov_dim + 1);
  const int64_t f = 4 * 2 + 1 + 8 * (9 + 2 + (hex ? rw.NG : 0)) + 2 + 8 * (2 * rw.NG * kFaceState + 10 * rw.NG);
  return N * c + F * f + nb * (2 + 8 + 4 + (mixed ? 4 * 2 * kBatchMdot : 0)) + 8 * std::max<int64_t>(4096, N / 64 + 64) +
         (64 << 10);
}

void batch_delete(Batch *B) {
  if (!B) return;
  DeviceScope dev_scope(B->m.device);
  if (B->stream) cudaStreamSynchronize(B->stream);
  if (B->graph) cudaGraphExecDestroy(B->graph);
  mesh_free_all(B->m);
  if (B->hist) cudaFree(B->hist);
  if (B->ev_in) cudaEventDestroy(B->ev_in);
  if (B->ev_out) cudaEventDestroy(B->ev_out);
  if (B->stream) cudaStreamDestroy(B->stream);
  delete B;
}

// the caller has made the batch's device current (HGKS_ON_DEVICE)
hgks_status enter(Batch &B, cudaStream_t user) {
  BCUDA(cudaEventRecord(B.ev_in, user));
  BCUDA(cudaStreamWaitEvent(B.stream, B.ev_in, 0));
  return HGKS_OK;
}
hgks_status leave(Batch &B, cudaStream_t user) {
  BCUDA(cudaEventRecord(B.ev_out, B.stream));
  BCUDA(cudaStreamWaitEvent(user, B.ev_out, 0));
  return HGKS_OK;
}

}  // namespace hgks

namespace hgks {

// An empty arena of cell_cap cells (rounded up to kBatchBlock) and face_cap faces.
hgks_status batch_new(int device, int64_t cell_cap, int64_t face_cap, int nslot, const hgks_params &shared,
                      int schemes, Batch **out, bool hex) {
  *out = nullptr;
  const int64_t N = (cell_cap + kBatchBlock - 1) / kBatchBlock * kBatchBlock, F = std::max<int64_t>(face_cap, 1);
  if (N <= 0 || nslot < 1 || nslot > 32767) return fail_msg(HGKS_ERR_ARG, "batch capacity or slot count out of range");
  if (shared.jv_mode != 0) return fail_msg(HGKS_ERR_ARG, "batches use the assembled A (jv_mode 0)");
  if (6 * std::max(N, F) >= (int64_t)INT32_MAX) return fail_msg(HGKS_ERR_ARG, "batch too large for 32-bit indexing");
  if (!(schemes & (shared.scheme == HGKS_WENO ? 1 : 2))) return fail_msg(HGKS_ERR_ARG, "batch has no data for its scheme");
  Batch *B = new (std::nothrow) Batch;
  if (!B) return fail_msg(HGKS_ERR_OOM, "host allocation");
  auto bail = [&](hgks_status s) { batch_delete(B); return s; };
  B->nslot = nslot;
  B->p0 = shared;
  B->slots.resize(nslot);
  B->cells.init(N / kBatchBlock);
  B->faces.init(F);
  B->active_host.assign(nslot + 1, 0);
  Mesh &M = B->m;
  M.device = device; M.N = N; M.F = F; M.schemes = schemes;
  DevMesh &d = M.d;
  d.N = (int)N; d.F = (int)F; d.hex = hex ? 1 : 0;
  const Rows rw(hex);
  DeviceScope dev_scope(device);
  if (dev_scope.error() != cudaSuccess) return bail(fail_msg(HGKS_ERR_CUDA, "cudaSetDevice"));
  if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&B->ev_out, cudaEventDisableTiming) != cudaSuccess)
    return bail(fail_msg(HGKS_ERR_CUDA, "stream or event creation"));
  cudaStream_t st = B->stream;
  const bool weno = schemes & 1, hweno = schemes & 2, mixed = shared.precision == HGKS_MIXED;
  const int nb = (int)(N / kBatchBlock);
  hgks_status s;
  if ((s = balloc(M, &d.vol, N)) || (s = balloc(M, &d.inv_vol, N)) || (s = balloc(M, &d.h, N)) ||
      (s = balloc(M, &d.m2, 6 * N)) || (s = balloc(M, &d.cnb, (size_t)rw.NF * N)) ||
      (s = balloc(M, &d.cface, (size_t)rw.NF * N)) || (s = balloc(M, &d.xg, (size_t)rw.NF * rw.NG * 3 * N)) ||
      (s = balloc(M, &d.subvalid, N)) || (s = balloc(M, &d.fl, F)) ||
      (s = balloc(M, &d.fr, F)) || (s = balloc(M, &d.ftag, F)) || (s = balloc(M, &d.fT, 9 * F)) ||
      (s = balloc(M, &d.fS, F)) || (s = balloc(M, &d.fdist, F)) || (hex && (s = balloc(M, &d.fw, (size_t)rw.NG * F))) ||
      (weno && ((s = balloc(M, &d.sten, (size_t)rw.BIG * N)) || (s = balloc(M, &d.X0, (size_t)9 * rw.BIG * N)) ||
                (s = balloc(M, &d.Xs, (size_t)rw.NSUBW * 3 * rw.SUBK * N)) ||
                (s = balloc(M, &d.ssl, (size_t)rw.NSUBW * N)))) ||
      (hweno && ((s = balloc(M, &d.H0, (size_t)9 * rw.HCOLS * N)) || (s = balloc(M, &d.Hm, (size_t)rw.NF * 21 * N)))))
    return bail(s);
  BatchState &bs = B->bs;
  const int mk = shared.krylov_dim;
  bs.kdim = mk;
  bs.l1_off = (mk + 1) * mk + 1 + mk + 2;
  bs.a_off = bs.l1_off + 1;
  bs.g_off = bs.a_off + mk + 1;
  bs.gram_off = bs.g_off + mk + 1;
  bs.hsz = (bs.gram_off + (mk + 1) * (mk + 1) + 7) / 8 * 8;
  if ((s = balloc(M, &B->ptab, nslot)) || (s = balloc(M, &B->cmesh, N)) || (s = balloc(M, &B->fmesh, F)) ||
      (s = balloc(M, &B->bmesh, nb)) || (s = balloc(M, &B->bstart, nslot)) || (s = balloc(M, &B->bcount, nslot)) ||
      (s = balloc(M, &B->ncell, nslot)) || (s = balloc(M, &B->active_base, nslot + 1)) ||
      (s = balloc(M, &bs.b.counters, nslot)) || (s = balloc(M, &bs.steps, nslot)) || (s = balloc(M, &bs.conv, nslot)) ||
      (s = balloc(M, &bs.bad, nslot)) || (s = balloc(M, &bs.ref, nslot)) || (s = balloc(M, &bs.res, nslot)) ||
      (s = balloc(M, &bs.drop, nslot)) || (s = balloc(M, &bs.max_steps, nslot)) ||
      (s = balloc(M, &bs.hs, (size_t)nslot * bs.hsz)) || (s = balloc(M, &bs.part, nb)) ||
      (mixed && (s = balloc(M, &bs.part32, (size_t)kBatchMdot * 2 * nb))) || (s = balloc(M, &B->Q, 5 * N)) ||
      (compact(*B) && (s = balloc(M, &B->G, 15 * N))))
    return bail(s);
  // free cells: unit volume and size, no neighbours, zero matrices, mesh -1
  launch_fill(d.vol, N, 1.0, st);
  launch_fill(d.inv_vol, N, 1.0, st);
  launch_fill(d.h, N, 1.0, st);
  cudaMemsetAsync(d.m2, 0, sizeof(double) * 6 * N, st);
  cudaMemsetAsync(d.xg, 0, sizeof(double) * rw.NF * rw.NG * 3 * N, st);
  cudaMemsetAsync(d.cnb, 0xff, sizeof(int) * rw.NF * N, st);
  cudaMemsetAsync(d.cface, 0xff, sizeof(int) * rw.NF * N, st);
  if (hex) cudaMemsetAsync(d.fw, 0, sizeof(double) * rw.NG * F, st);
  cudaMemsetAsync(d.subvalid, 0, N, st);
  cudaMemsetAsync(d.fl, 0xff, sizeof(int) * F, st);
  cudaMemsetAsync(d.fr, 0xff, sizeof(int) * F, st);
  cudaMemsetAsync(d.ftag, 0, F, st);
  cudaMemsetAsync(d.fT, 0, sizeof(double) * 9 * F, st);
  cudaMemsetAsync(d.fS, 0, sizeof(double) * F, st);
  cudaMemsetAsync(d.fdist, 0, sizeof(double) * F, st);
  if (weno) {
    cudaMemsetAsync(d.sten, 0xff, sizeof(int) * rw.BIG * N, st);
    cudaMemsetAsync(d.X0, 0, sizeof(double) * 9 * rw.BIG * N, st);
    cudaMemsetAsync(d.Xs, 0, sizeof(double) * rw.NSUBW * 3 * rw.SUBK * N, st);
    cudaMemsetAsync(d.ssl, 0, sizeof(unsigned) * rw.NSUBW * N, st);
  }
  if (hweno) {
    cudaMemsetAsync(d.H0, 0, sizeof(double) * 9 * rw.HCOLS * N, st);
    cudaMemsetAsync(d.Hm, 0, sizeof(double) * rw.NF * 21 * N, st);
  }
  cudaMemsetAsync(B->ptab, 0, sizeof(hgks_params) * nslot, st);
  cudaMemsetAsync(B->cmesh, 0xff, sizeof(short) * N, st);
  cudaMemsetAsync(B->fmesh, 0xff, sizeof(short) * F, st);
  cudaMemsetAsync(B->bmesh, 0xff, sizeof(short) * nb, st);
  cudaMemsetAsync(B->bstart, 0, sizeof(int) * nslot, st);
  cudaMemsetAsync(B->bcount, 0, sizeof(int) * nslot, st);
  cudaMemsetAsync(B->active_base, 0, sizeof(int) * (nslot + 1), st);
  cudaMemsetAsync(bs.b.counters, 0, sizeof(unsigned) * nslot, st);
  cudaMemsetAsync(bs.hs, 0, sizeof(double) * nslot * bs.hsz, st);
  cudaMemsetAsync(B->Q, 0, sizeof(double) * 5 * N, st);
  if (B->G) cudaMemsetAsync(B->G, 0, sizeof(double) * 15 * N, st);
  std::vector<int> one(nslot, 1);
  if ((s = upload(B->ncell, one.data(), nslot, st))) return bail(s);
  if (cudaStreamSynchronize(st) != cudaSuccess || (s = launch_status()))
    return bail(s ? s : fail_msg(HGKS_ERR_CUDA, "batch initialisation"));
  bs.b.nmesh = nslot;
  bs.b.nblocks = 0;              // live blocks: none until a mesh is placed
  bs.b.bmesh = B->bmesh;
  bs.b.bstart = B->bstart;
  bs.b.bcount = B->bcount;
  bs.b.active = B->active_base + 1;
  bs.ncell = B->ncell;
  d.ptab = B->ptab;
  d.cmesh = B->cmesh;
  d.fmesh = B->fmesh;
  d.mact = B->active_base + 1;
  if ((s = ensure_scratch(M, mk, true, mixed))) return bail(s);
  *out = B;
  return HGKS_OK;
}

hgks_status batch_place(Batch &B, const MeshSource &src, const hgks_params &p, int *slot) {
  *slot = -1;
  if (!same_shared(B.p0, p)) return fail_msg(HGKS_ERR_ARG, "scheme, precision, jv_mode, krylov_dim, restarts, jacobi_sweeps must agree");
  if ((src.schemes & B.m.schemes) != B.m.schemes) return fail_msg(HGKS_ERR_ARG, "mesh lacks data for the batch's scheme");
  if (src.hex != B.m.d.hex) return fail_msg(HGKS_ERR_ARG, "the meshes of a batch are all tetrahedra or all hexahedra");
  const Rows rw(B.m.d.hex != 0);
  int k = 0;
  while (k < B.nslot && B.slots[k].used) k++;
  if (k == B.nslot) return HGKS_OK;
  const int64_t cpad = (src.N + kBatchBlock - 1) / kBatchBlock * kBatchBlock;
  const int64_t b0 = B.cells.take(cpad / kBatchBlock);
  if (b0 < 0) return HGKS_OK;
  const int64_t f0 = B.faces.take(src.F);
  if (f0 < 0) { B.cells.give(b0, cpad / kBatchBlock); return HGKS_OK; }
  const int64_t c0 = b0 * kBatchBlock, N = B.m.N, F = B.m.F, nk = src.N, fk = src.F;
  Slot &S = B.slots[k];
  S.used = true; S.c0 = c0; S.ncell = nk; S.cpad = cpad; S.f0 = f0; S.nface = fk; S.nbface = src.Fb; S.p = p;
  DevMesh &d = B.m.d;
  cudaStream_t st = B.stream;
  const bool weno = B.m.schemes & 1, hweno = B.m.schemes & 2;
  hgks_status s;
  if ((s = copy_in(d.vol, N, c0, src.vol, nk, 1, st)) || (s = copy_in(d.inv_vol, N, c0, src.inv_vol, nk, 1, st)) ||
      (s = copy_in(d.h, N, c0, src.h, nk, 1, st)) || (s = copy_in(d.m2, N, c0, src.m2, nk, 6, st)) ||
      (s = copy_in(d.cnb, N, c0, src.cnb, nk, rw.NF, st)) || (s = copy_in(d.cface, N, c0, src.cface, nk, rw.NF, st)) ||
      (s = copy_in(d.xg, N, c0, src.xg, nk, rw.NF * rw.NG * 3, st)) ||
      (s = copy_in(d.subvalid, N, c0, src.subvalid, nk, 1, st)) ||
      (d.fw && (s = copy_in(d.fw, F, f0, src.fw, fk, rw.NG, st))) ||
      (s = copy_in(d.fl, F, f0, src.fl, fk, 1, st)) || (s = copy_in(d.fr, F, f0, src.fr, fk, 1, st)) ||
      (s = copy_in(d.ftag, F, f0, src.ftag, fk, 1, st)) || (s = copy_in(d.fT, F, f0, src.fT, fk, 9, st)) ||
      (s = copy_in(d.fS, F, f0, src.fS, fk, 1, st)) || (s = copy_in(d.fdist, F, f0, src.fdist, fk, 1, st)) ||
      (weno && ((s = copy_in(d.sten, N, c0, src.sten, nk, rw.BIG, st)) ||
                (s = copy_in(d.X0, N, c0, src.X0, nk, 9 * rw.BIG, st)) ||
                (s = copy_in(d.Xs, N, c0, src.Xs, nk, rw.NSUBW * 3 * rw.SUBK, st)) ||
                (s = copy_in(d.ssl, N, c0, src.ssl, nk, rw.NSUBW, st)))) ||
      (hweno && ((s = copy_in(d.H0, N, c0, src.H0, nk, 9 * rw.HCOLS, st)) ||
                 (s = copy_in(d.Hm, N, c0, src.Hm, nk, rw.NF * 21, st)))))
    return s;
  // padding cells of the range: no neighbours
  if (cpad > nk) {
    BCUDA(cudaMemset2DAsync(d.cnb + c0 + nk, sizeof(int) * N, 0xff, sizeof(int) * (cpad - nk), rw.NF, st));
    BCUDA(cudaMemset2DAsync(d.cface + c0 + nk, sizeof(int) * N, 0xff, sizeof(int) * (cpad - nk), rw.NF, st));
    if (weno) BCUDA(cudaMemset2DAsync(d.sten + c0 + nk, sizeof(int) * N, 0xff, sizeof(int) * (cpad - nk), rw.BIG, st));
  }
  // cell indices move by the range's first cell, face indices (2 f + side) by twice its first face
  launch_offset_index(d.cnb + c0, rw.NF, nk, N, c0, st);
  launch_offset_index(d.cface + c0, rw.NF, nk, N, 2 * f0, st);
  if (weno) launch_offset_index(d.sten + c0, rw.BIG, nk, N, c0, st);
  launch_offset_index(d.fl + f0, 1, fk, F, c0, st);
  launch_offset_index(d.fr + f0, 1, fk, F, c0, st);
  launch_fill_short(B.cmesh + c0, nk, (short)k, st);
  launch_fill_short(B.fmesh + f0, fk, (short)k, st);
  launch_fill_short(B.bmesh + b0, cpad / kBatchBlock, (short)k, st);
  const int bst = (int)b0, bcn = (int)(cpad / kBatchBlock), nc = (int)nk;
  if ((s = upload(B.ptab + k, &S.p, 1, st)) || (s = upload(B.bstart + k, &bst, 1, st)) ||
      (s = upload(B.bcount + k, &bcn, 1, st)) || (s = upload(B.ncell + k, &nc, 1, st)))
    return s;
  BCUDA(cudaMemsetAsync(B.bs.hs + (size_t)k * B.bs.hsz, 0, sizeof(double) * B.bs.hsz, st));
  BCUDA(cudaMemsetAsync(B.active_base + 1 + k, 0, sizeof(int), st));
  B.active_host[1 + k] = 0;
  // pageable sources above (the small records) must be consumed before they change
  BCUDA(cudaStreamSynchronize(st));
  if ((s = launch_status())) return s;
  B.epoch++;
  update_live(B);
  *slot = k;
  return HGKS_OK;
}

void batch_release(Batch &B, int k) {
  if (k < 0 || k >= B.nslot || !B.slots[k].used) return;
  Slot &S = B.slots[k];
  cudaStream_t st = B.stream;
  launch_fill_short(B.cmesh + S.c0, S.cpad, (short)-1, st);
  launch_fill_short(B.fmesh + S.f0, S.nface, (short)-1, st);
  launch_fill_short(B.bmesh + S.c0 / kBatchBlock, S.cpad / kBatchBlock, (short)-1, st);
  cudaMemsetAsync(B.active_base + 1 + k, 0, sizeof(int), st);
  B.active_host[1 + k] = 0;
  B.cells.give(S.c0 / kBatchBlock, S.cpad / kBatchBlock);
  B.faces.give(S.f0, S.nface);
  S = Slot{};
  B.epoch++;
  update_live(B);
}

hgks_status batch_set_state(Batch &B, int k, const double *Q, const double *G) {
  const Slot &S = B.slots[k];
  hgks_status s;
  if ((s = copy_in(B.Q, B.m.N, S.c0, Q, S.ncell, 5, B.stream))) return s;
  if (compact(B) && G && (s = copy_in(B.G, B.m.N, S.c0, G, S.ncell, 15, B.stream))) return s;
  return HGKS_OK;
}

hgks_status batch_get_state(Batch &B, int k, double *Q, double *G, double *R, double *G_new) {
  const Slot &S = B.slots[k];
  const int64_t N = B.m.N;
  hgks_status s;
  if ((s = copy_out(Q, S.ncell, B.Q, N, S.c0, 5, B.stream)) || (s = copy_out(R, S.ncell, B.m.s.R, N, S.c0, 5, B.stream)))
    return s;
  if (compact(B) && ((s = copy_out(G, S.ncell, B.G, N, S.c0, 15, B.stream)) ||
                     (s = copy_out(G_new, S.ncell, B.m.s.Gnew, N, S.c0, 15, B.stream))))
    return s;
  return HGKS_OK;
}

namespace {
__global__ void k_arm(BatchState bs, int k, double drop, int max_steps) {
  bs.steps[k] = 0; bs.conv[k] = 0; bs.bad[k] = 0; bs.ref[k] = 0.0; bs.res[k] = 0.0;
  bs.drop[k] = drop; bs.max_steps[k] = max_steps;
}
}  // namespace

hgks_status batch_arm(Batch &B, int k, double drop_tol, int max_steps) {
  k_arm<<<1, 1, 0, B.stream>>>(B.bs, k, drop_tol, max_steps);
  count_launch();
  return launch_status();
}

hgks_status batch_set_active(Batch &B, const std::vector<int> &active) {
  for (int k = 0; k < B.nslot; k++) B.active_host[1 + k] = (B.slots[k].used && active[k]) ? 1 : 0;
  B.active_host[0] = 0;
  BCUDA(cudaMemcpyAsync(B.active_base, B.active_host.data(), sizeof(int) * (B.nslot + 1), cudaMemcpyHostToDevice, B.stream));
  BCUDA(cudaStreamSynchronize(B.stream));    // the host vector may change right after
  return HGKS_OK;
}

namespace {
void enqueue_eager(Batch &B, bool check) {
  DevMesh &d = B.m.d;
  Scratch &s = B.m.s;
  cudaStream_t st = B.stream;
  launch_residual(d, s, B.p0, B.Q, B.G, s.R, compact(B) ? s.Gnew : nullptr, st, true);
  launch_batch_density(d, B.bs, s.R, st);
  if (check) launch_batch_check(B.bs, st);
  launch_assemble(d, s, B.p0, B.Q, s.dt, nullptr, nullptr, st, true);
  launch_batch_gmres(d, s, B.bs, B.p0, s.R, s.dQ, st);
  launch_batch_update(d, B.bs, B.Q, s.dQ, B.G, s.Gnew, compact(B) ? 15 : 0, st);
}
}  // namespace

// One outer step of Algorithm 1 for every active slot: R(Q), the density
// residual (and, with `check`, the convergence test that may stop a slot), A,
// GMRES, Q += dQ. The launch sequence depends only on the arena (its sizes and
// arrays), not on which slots are in use, so one captured graph serves every
// membership; it is captured again only when the launch shapes or the
// history buffer change.
hgks_status batch_enqueue_step(Batch &B, bool check, bool use_graph) {
  if (!use_graph || g_prof_on) {
    enqueue_eager(B, check);
    return launch_status();
  }
  // what the captured launches depend on besides the arena: grids, shapes, history buffer
  const uint64_t key[6] = {(uint64_t)(uintptr_t)B.bs.hist, (uint64_t)B.bs.hist_len, (uint64_t)B.m.d.NL,
                           (uint64_t)B.m.d.FL, ((uint64_t)B.m.s.blk_recon << 32) | (uint64_t)B.m.s.blk_flux,
                           check ? 1ull : 0ull};
  if (!B.graph || std::memcmp(key, B.graph_key, sizeof(key)) != 0) {
    if (B.graph) { cudaGraphExecDestroy(B.graph); B.graph = nullptr; }
    cudaGraph_t g = nullptr;
    BCUDA(cudaStreamBeginCapture(B.stream, cudaStreamCaptureModeThreadLocal));
    const int64_t l0 = g_launches;
    enqueue_eager(B, check);
    B.graph_launches = g_launches - l0;
    g_launches = l0;
    cudaError_t e = cudaStreamEndCapture(B.stream, &g);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&B.graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) { cudaGetLastError(); B.graph = nullptr; return cuda_error(e, "CUDA graph capture of the batch step"); }
    std::memcpy(B.graph_key, key, sizeof(key));
  }
  BCUDA(cudaGraphLaunch(B.graph, B.stream));
  g_launches += B.graph_launches;
  return HGKS_OK;
}

}  // namespace hgks

// ---------------------------------------------------------------- C ABI
namespace {

hgks_status check_slot(const hgks_batch_s *b, int32_t k) {
  if (!b || !b->B) return fail_msg(HGKS_ERR_ARG, "batch is NULL");
  if (k < 0 || k >= b->B->nslot || !b->B->slots[k].used) return fail_msg(HGKS_ERR_ARG, "mesh index is not in use");
  return HGKS_OK;
}

std::vector<int> used_mask(const Batch &B) {
  std::vector<int> a(B.nslot);
  for (int k = 0; k < B.nslot; k++) a[k] = B.slots[k].used ? 1 : 0;
  return a;
}

}  // namespace

extern "C" {

hgks_status hgks_batch_create(const hgks_mesh *meshes, const hgks_params *params, int32_t n_meshes, hgks_batch *out) {
  if (!out) return fail_msg(HGKS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!meshes || !params) return fail_msg(HGKS_ERR_ARG, "meshes or params is NULL");
  if (n_meshes < 1 || n_meshes > 32767) return fail_msg(HGKS_ERR_ARG, "n_meshes must be in 1..32767");
  int schemes = 3;
  int64_t N = 0, F = 0;
  hgks_status st;
  std::vector<hgks_params> P(n_meshes);
  for (int k = 0; k < n_meshes; k++) {
    if (!meshes[k]) return fail_msg(HGKS_ERR_ARG, "a mesh handle is NULL");
    const Mesh &a = *mesh_of(meshes[k]);
    if (a.device != mesh_of(meshes[0])->device) return fail_msg(HGKS_ERR_ARG, "meshes of a batch must be on one device");
    if (a.d.hex != mesh_of(meshes[0])->d.hex)
      return fail_msg(HGKS_ERR_ARG, "the meshes of a batch are all tetrahedra or all hexahedra");
    if ((st = take_params(a, &params[k], &P[k]))) return st;
    if (!same_shared(P[0], P[k]))
      return fail_msg(HGKS_ERR_ARG, "scheme, precision, jv_mode, krylov_dim, restarts, jacobi_sweeps must agree");
    schemes &= a.schemes;
    N += (a.N + kBatchBlock - 1) / kBatchBlock * kBatchBlock;
    F += a.F;
  }
  // the batch carries the data of its scheme only
  schemes &= P[0].scheme == HGKS_WENO ? 1 : 2;
  HGKS_ON_DEVICE(mesh_of(meshes[0])->device);
  Batch *B = nullptr;
  if ((st = batch_new(mesh_of(meshes[0])->device, N, F, n_meshes, P[0], schemes, &B, mesh_of(meshes[0])->d.hex != 0)))
    return st;
  for (int k = 0; k < n_meshes; k++) {
    int slot = -1;
    if ((st = batch_place(*B, source_of(*mesh_of(meshes[k])), P[k], &slot)) || slot != k) {
      batch_delete(B);
      return st ? st : fail_msg(HGKS_ERR_CUDA, "batch placement");
    }
  }
  hgks_batch_s *h = new (std::nothrow) hgks_batch_s;
  if (!h) { batch_delete(B); return fail_msg(HGKS_ERR_OOM, "host allocation"); }
  h->B = B;
  *out = h;
  return HGKS_OK;
}

}  // extern "C"

namespace {
hgks_status create_empty(int32_t device, int64_t cell_capacity, int64_t face_capacity, int32_t max_meshes,
                         const hgks_params *shared, bool hex, hgks_batch *out) {
  if (!out || !shared) return fail_msg(HGKS_ERR_ARG, "NULL argument");
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return fail_msg(HGKS_ERR_ARG, "no such device");
  HGKS_ON_DEVICE(device);
  Batch *B = nullptr;
  hgks_status st = batch_new(device, cell_capacity, face_capacity, max_meshes, *shared,
                             shared->scheme == HGKS_WENO ? 1 : 2, &B, hex);
  if (st) return st;
  hgks_batch_s *h = new (std::nothrow) hgks_batch_s;
  if (!h) { batch_delete(B); return fail_msg(HGKS_ERR_OOM, "host allocation"); }
  h->B = B;
  *out = h;
  return HGKS_OK;
}
}  // namespace

extern "C" {

hgks_status hgks_batch_create_empty(int32_t device, int64_t cell_capacity, int64_t face_capacity, int32_t max_meshes,
                                    const hgks_params *shared, hgks_batch *out) {
  return create_empty(device, cell_capacity, face_capacity, max_meshes, shared, false, out);
}

hgks_status hgks_batch_create_empty_hex(int32_t device, int64_t cell_capacity, int64_t face_capacity,
                                        int32_t max_meshes, const hgks_params *shared, hgks_batch *out) {
  return create_empty(device, cell_capacity, face_capacity, max_meshes, shared, true, out);
}

hgks_status hgks_batch_add(hgks_batch batch, hgks_mesh mesh, const hgks_params *p, int32_t *k_out) {
  if (!batch || !batch->B || !mesh || !p || !k_out) return fail_msg(HGKS_ERR_ARG, "NULL argument");
  Batch &B = *batch->B;
  *k_out = -1;
  const Mesh &a = *mesh_of(mesh);
  if (a.device != B.m.device) return fail_msg(HGKS_ERR_ARG, "mesh is on another device");
  if (a.d.hex != B.m.d.hex) return fail_msg(HGKS_ERR_ARG, "the meshes of a batch are all tetrahedra or all hexahedra");
  hgks_params P;
  hgks_status st = take_params(a, p, &P);
  if (st) return st;
  HGKS_ON_DEVICE(B.m.device);
  int slot = -1;
  if ((st = batch_place(B, source_of(a), P, &slot))) return st;
  if (slot < 0) return fail_msg(HGKS_ERR_OOM, "no free slot, cell range or face range in the batch");
  *k_out = slot;
  return HGKS_OK;
}

hgks_status hgks_batch_remove(hgks_batch batch, int32_t k) {
  hgks_status st = check_slot(batch, k);
  if (st) return st;
  HGKS_ON_DEVICE(batch->B->m.device);
  batch_release(*batch->B, k);
  return HGKS_OK;
}

hgks_status hgks_batch_destroy(hgks_batch batch) {
  if (!batch) return fail_msg(HGKS_ERR_ARG, "batch is NULL");
  batch_delete(batch->B);
  delete batch;
  return HGKS_OK;
}

hgks_status hgks_batch_info(hgks_batch batch, hgks_batch_info_t *info) {
  if (!batch || !batch->B || !info) return fail_msg(HGKS_ERR_ARG, "NULL argument");
  const Batch &B = *batch->B;
  info->n_cells = B.m.N;
  info->n_faces = B.m.F;
  info->device_bytes = (int64_t)B.m.bytes;
  info->n_meshes = 0;
  for (auto &s : B.slots) info->n_meshes += s.used ? 1 : 0;
  info->blk_recon = B.m.s.blk_recon;
  info->blk_flux = B.m.s.blk_flux;
  return HGKS_OK;
}

hgks_status hgks_batch_set_state(hgks_batch batch, int32_t k, const double *Q, const double *G, void *cuda_stream) {
  hgks_status st = check_slot(batch, k);
  if (st) return st;
  Batch &B = *batch->B;
  if (!Q || (compact(B) && !G)) return fail_msg(HGKS_ERR_ARG, "Q (or G) is NULL");
  cudaStream_t user = (cudaStream_t)cuda_stream;
  HGKS_ON_DEVICE(B.m.device);
  if ((st = enter(B, user)) || (st = batch_set_state(B, k, Q, G))) return st;
  return leave(B, user);
}

hgks_status hgks_batch_get_state(hgks_batch batch, int32_t k, double *Q, double *G, double *R, double *G_new,
                                 void *cuda_stream) {
  hgks_status st = check_slot(batch, k);
  if (st) return st;
  Batch &B = *batch->B;
  cudaStream_t user = (cudaStream_t)cuda_stream;
  HGKS_ON_DEVICE(B.m.device);
  if ((st = enter(B, user)) || (st = batch_get_state(B, k, Q, G, R, G_new))) return st;
  return leave(B, user);
}

hgks_status hgks_batch_residual(hgks_batch batch, void *cuda_stream) {
  if (!batch || !batch->B) return fail_msg(HGKS_ERR_ARG, "batch is NULL");
  Batch &B = *batch->B;
  cudaStream_t user = (cudaStream_t)cuda_stream;
  hgks_status st;
  HGKS_ON_DEVICE(B.m.device);
  if ((st = enter(B, user)) || (st = batch_set_active(B, used_mask(B)))) return st;
  launch_residual(B.m.d, B.m.s, B.p0, B.Q, B.G, B.m.s.R, compact(B) ? B.m.s.Gnew : nullptr, B.stream, true);
  if ((st = launch_status())) return st;
  return leave(B, user);
}

hgks_status hgks_batch_gmres_step(hgks_batch batch, hgks_step_info *info, int32_t use_graph, void *cuda_stream) {
  if (!batch || !batch->B) return fail_msg(HGKS_ERR_ARG, "batch is NULL");
  Batch &B = *batch->B;
  cudaStream_t user = (cudaStream_t)cuda_stream;
  hgks_status st;
  HGKS_ON_DEVICE(B.m.device);
  if ((st = enter(B, user)) || (st = batch_set_active(B, used_mask(B)))) return st;
  if ((st = batch_enqueue_step(B, false, use_graph != 0))) return st;
  const int n = B.nslot, hz = B.bs.hsz;
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
    const bool used = B.slots[k].used;
    const double res = used ? r[B.bs.l1_off] / (double)B.slots[k].ncell : 0.0;
    finite = finite && std::isfinite(res);
    if (info) {
      info[k].res_l1 = res;
      info[k].lin_res[0] = used ? r[lres] : 0.0;
      info[k].lin_res[1] = used ? r[lres + 1] : 0.0;
      info[k].krylov_iters = used ? B.p0.restarts * mk : 0;
      info[k].nonphysical = nonphys;   // counted over the whole batch
    }
  }
  if (!finite) return fail_msg(HGKS_ERR_NONPHYSICAL, "non-finite residual");
  return HGKS_OK;
}

hgks_status hgks_batch_solve_steady(hgks_batch batch, double drop_tol, int32_t max_steps, int32_t use_graph,
                                    double *hist_host, hgks_solve_info *info, void *cuda_stream) {
  if (!batch || !batch->B) return fail_msg(HGKS_ERR_ARG, "batch is NULL");
  if (!(drop_tol > 0.0) || max_steps < 0) return fail_msg(HGKS_ERR_ARG, "drop_tol must be > 0 and max_steps >= 0");
  Batch &B = *batch->B;
  BatchState &bs = B.bs;
  const int n = B.nslot;
  cudaStream_t user = (cudaStream_t)cuda_stream;
  hgks_status st;
  HGKS_ON_DEVICE(B.m.device);
  if ((st = enter(B, user))) return st;
  const int64_t hlen = (int64_t)max_steps + 1;
  if (hist_host && B.hist_cap < hlen * n) {
    BCUDA(cudaStreamSynchronize(B.stream));
    if (B.hist) { cudaFree(B.hist); B.hist = nullptr; B.hist_cap = 0; }
    BCUDA(cudaMalloc(&B.hist, sizeof(double) * hlen * n));
    B.hist_cap = hlen * n;
  }
  bs.hist = hist_host ? B.hist : nullptr;
  bs.hist_len = (int)hlen;
  if (hist_host) BCUDA(cudaMemsetAsync(B.hist, 0, sizeof(double) * hlen * n, B.stream));
  for (int k = 0; k < n; k++)
    if (B.slots[k].used && (st = batch_arm(B, k, drop_tol, max_steps))) return st;
  if ((st = batch_set_active(B, used_mask(B)))) return st;
  // every mesh takes at most max_steps steps and one last test; the host polls
  // the active flags every few steps (finished meshes cost no work meanwhile)
  std::vector<int> act(n + 1);
  const int poll = 4;
  for (int it = 0; it <= max_steps;) {
    const int chunk = std::min(poll, max_steps + 1 - it);
    for (int c = 0; c < chunk; c++)
      if ((st = batch_enqueue_step(B, true, use_graph != 0))) return st;
    it += chunk;
    BCUDA(cudaMemcpyAsync(act.data(), B.active_base, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, B.stream));
    BCUDA(cudaStreamSynchronize(B.stream));
    if (std::none_of(act.begin() + 1, act.end(), [](int a) { return a != 0; })) break;
  }
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
  if ((st = leave(B, user))) return st;
  bool all_conv = true, any_bad = false;
  for (int k = 0; k < n; k++) {
    const bool used = B.slots[k].used;
    if (info) {
      info[k].steps = used ? steps[k] : 0;
      info[k].converged = used ? conv[k] : 0;
      info[k].res_ref = used ? ref[k] : 0.0;
      info[k].res_final = used ? res[k] : 0.0;
    }
    if (!used) continue;
    all_conv = all_conv && conv[k];
    any_bad = any_bad || bad[k];
  }
  if (any_bad) return fail_msg(HGKS_ERR_NONPHYSICAL, "non-finite residual in a mesh of the batch");
  if (!all_conv) return fail_msg(HGKS_ERR_NOT_CONVERGED, "max_steps reached by a mesh of the batch");
  return HGKS_OK;
}

hgks_status hgks_batch_autotune(hgks_batch batch, int32_t *blk_recon, int32_t *blk_flux, void *cuda_stream) {
  if (!batch || !batch->B) return fail_msg(HGKS_ERR_ARG, "batch is NULL");
  Batch &B = *batch->B;
  Scratch &s = B.m.s;
  cudaStream_t user = (cudaStream_t)cuda_stream;
  hgks_status st;
  HGKS_ON_DEVICE(B.m.device);
  if ((st = enter(B, user)) || (st = batch_set_active(B, used_mask(B)))) return st;
  cudaEvent_t a = nullptr, b = nullptr;
  BCUDA(cudaEventCreate(&a));
  BCUDA(cudaEventCreate(&b));
  auto residual = [&]() {
    launch_residual(B.m.d, s, B.p0, B.Q, B.G, s.R, compact(B) ? s.Gnew : nullptr, B.stream, true);
  };
  auto time_residual = [&](float &ms) -> hgks_status {
    BCUDA(cudaEventRecord(a, B.stream));
    for (int r = 0; r < 3; r++) residual();
    BCUDA(cudaEventRecord(b, B.stream));
    BCUDA(cudaEventSynchronize(b));
    BCUDA(cudaEventElapsedTime(&ms, a, b));
    return launch_status();
  };
  const int cand[3] = {64, 128, 256};
  residual();   // warm-up
  for (int pass = 0; pass < 2 && !st; pass++) {
    int *blk = pass == 0 ? &s.blk_recon : &s.blk_flux;
    int best = *blk;
    float best_ms = 1e30f, ms = 0.f;
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
