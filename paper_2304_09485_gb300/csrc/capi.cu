// C ABI of libhgks (include/hgks.h): argument checks, device memory of a mesh
// handle, and the orchestration of the kernels in residual.cu / implicit.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include "hgks_internal.h"

using namespace hgks;

struct hgks_mesh_s {
  Mesh m;
};

namespace {

thread_local std::string g_err;

hgks_status fail(hgks_status st, const std::string &msg) {
  g_err = msg;
  return st;
}
hgks_status cuda_fail(cudaError_t e, const char *where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? HGKS_ERR_OOM : HGKS_ERR_CUDA;
}
#define HGKS_CUDA(call)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
  } while (0)

template <typename T>
hgks_status dalloc(Mesh &m, T **p, size_t n) {
  *p = nullptr;
  if (n == 0) return HGKS_OK;
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, n * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  m.allocs.push_back(q);
  m.bytes += n * sizeof(T);
  *p = (T *)q;
  return HGKS_OK;
}
template <typename T>
hgks_status upload(Mesh &m, T **p, const std::vector<T> &v) {
  hgks_status st = dalloc(m, p, v.size());
  if (st) return st;
  if (!v.empty()) HGKS_CUDA(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return HGKS_OK;
}

void free_all(Mesh &m) {
  if (m.graph) {
    if (m.graph->stream) cudaStreamSynchronize(m.graph->stream);
    if (m.graph->exec) cudaGraphExecDestroy(m.graph->exec);
    if (m.graph->ev_in) cudaEventDestroy(m.graph->ev_in);
    if (m.graph->ev_out) cudaEventDestroy(m.graph->ev_out);
    if (m.graph->stream) cudaStreamDestroy(m.graph->stream);
    delete m.graph;
    m.graph = nullptr;
  }
  for (void *p : m.allocs) cudaFree(p);
  m.allocs.clear();
}

hgks_status last_launch() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return HGKS_OK;
}

}  // namespace

namespace hgks {
hgks_status fail_msg(hgks_status st, const std::string &msg) { return fail(st, msg); }
hgks_status cuda_error(cudaError_t e, const char *where) { return cuda_fail(e, where); }
hgks_status mesh_alloc(Mesh &m, void **p, size_t bytes) {
  unsigned char *q = nullptr;
  hgks_status st = dalloc(m, &q, bytes);
  *p = q;
  return st;
}
void mesh_free_all(Mesh &m) { free_all(m); }

hgks_status check_params(const Mesh &m, const hgks_params *p) {
  if (!p) return fail(HGKS_ERR_ARG, "params is NULL");
  if (p->scheme != HGKS_WENO && p->scheme != HGKS_HWENO) return fail(HGKS_ERR_ARG, "unknown scheme");
  if (!(m.schemes & (p->scheme == HGKS_WENO ? 1 : 2))) return fail(HGKS_ERR_ARG, "mesh was built without data for this scheme");
  if (p->krylov_dim < 1 || p->krylov_dim > 64) return fail(HGKS_ERR_ARG, "krylov_dim must be in 1..64");
  if (p->restarts < 0 || p->jacobi_sweeps < 0) return fail(HGKS_ERR_ARG, "negative restarts or sweeps");
  if (!(p->gamma > 1.0) || !(p->cfl > 0.0) || !(p->flux_cfl > 0.0) || !(p->Pr > 0.0)) return fail(HGKS_ERR_ARG, "gamma, cfl, flux_cfl, Pr out of range");
  if (p->viscous && !(p->mu > 0.0)) return fail(HGKS_ERR_ARG, "viscous flow needs mu > 0");
  if (!p->viscous && !(p->tau_eps > 0.0)) return fail(HGKS_ERR_ARG, "inviscid flow needs tau_eps > 0");
  if (p->precision != HGKS_FP64 && p->precision != HGKS_MIXED) return fail(HGKS_ERR_ARG, "unknown precision");
  if (p->jv_mode != 0 && p->jv_mode != 1) return fail(HGKS_ERR_ARG, "jv_mode must be 0 (assembled) or 1 (matrix-free)");
  if (!(p->grad_relax >= 0.0 && p->grad_relax <= 1.0)) return fail(HGKS_ERR_ARG, "grad_relax must be in [0, 1]");
  return HGKS_OK;
}

// Flow conditions of the paper's problem statements (Sec. 5.1, 5.2) from Mach,
// Re and the angle of attack; reference length 1 (cavity side, sphere diameter).
hgks_status take_params(const Mesh &m, const hgks_params *p, hgks_params *out) {
  if (!p) return fail(HGKS_ERR_ARG, "params is NULL");
  if (!(p->Mach >= 0.0) || !(p->Re >= 0.0) || !std::isfinite(p->Mach) || !std::isfinite(p->Re) ||
      !std::isfinite(p->aoa_deg))
    return fail(HGKS_ERR_ARG, "Mach and Re must be finite and >= 0, aoa_deg finite");
  hgks_params q = *p;
  if (p->Mach > 0.0) {
    const double g = p->gamma;
    if (!(g > 1.0)) return fail(HGKS_ERR_ARG, "gamma, cfl, flux_cfl, Pr out of range");
    q.rho_inf = 1.0;
    if (p->lid_speed > 0.0) {
      // lid-driven cavity: fluid at rest, the Mach number is the lid's
      const double U = p->lid_speed;
      q.u_inf[0] = q.u_inf[1] = q.u_inf[2] = 0.0;
      q.p_inf = U * U / (g * p->Mach * p->Mach);
      q.wall_T = q.p_inf / q.rho_inf;
      q.mu = p->Re > 0.0 ? q.rho_inf * U / p->Re : 0.0;
    } else {
      // free stream (1, Ma cos a, Ma sin a, 0, 1/gamma), unit speed of sound
      const double a = p->aoa_deg * (M_PI / 180.0);
      q.u_inf[0] = p->Mach * std::cos(a); q.u_inf[1] = p->Mach * std::sin(a); q.u_inf[2] = 0.0;
      q.p_inf = 1.0 / g;
      q.wall_T = q.p_inf / q.rho_inf;
      q.mu = p->Re > 0.0 ? q.rho_inf * p->Mach / p->Re : 0.0;
    }
    q.viscous = p->Re > 0.0 ? 1 : 0;
  }
  hgks_status st = check_params(m, &q);
  if (st) return st;
  *out = q;
  return HGKS_OK;
}

// Scratch of the residual (always) and of the implicit solve (lazily, per Krylov
// size and precision). Krylov vectors are padded to a multiple of 64 elements so
// that every vector of the basis starts on a 512-byte boundary.
hgks_status ensure_scratch(Mesh &m, int kdim, bool implicit, bool mixed) {
  Scratch &s = m.s;
  const size_t N = m.N, F = m.F;
  const bool hex = m.d.hex != 0;
  const size_t NF = hex ? HexShape::NF : TetShape::NF, NG = hex ? HexShape::NG : TetShape::NG;
  const size_t ncoef = hex ? ShapeOf<HexShape>::COEF : ShapeOf<TetShape>::COEF;
  hgks_status st;
  if (!s.coef) {
    if ((st = dalloc(m, &s.coef, ncoef * N))) return st;
    if ((st = dalloc(m, &s.dt, N))) return st;
    if ((st = dalloc(m, &s.wface, 2 * NG * kFaceState * F))) return st;
    if ((st = dalloc(m, &s.fflux, 5 * NG * F))) return st;
    if ((st = dalloc(m, &s.fpt, 5 * NG * F))) return st;
    if ((st = dalloc(m, &s.flags, 8))) return st;
    // one partial per block and sum (the MGS pass reduces 16 sums over 608 blocks)
    if ((st = dalloc(m, &s.red, std::max<size_t>(16 * 608 + 64, N / 64 + 64)))) return st;
    if ((st = dalloc(m, &s.red_count, 4))) return st;
    HGKS_CUDA(cudaMemset(s.flags, 0, 8 * sizeof(int)));
    HGKS_CUDA(cudaMemset(s.red_count, 0, 4 * sizeof(unsigned)));
    HGKS_CUDA(cudaMemset(s.wface, 0, sizeof(double) * 2 * NG * kFaceState * F));
  }
  s.vstride = (int64_t)((5 * N + 63) / 64 * 64);
  if (implicit && !s.off) {
    if ((st = dalloc(m, &s.off, 25 * NF * N))) return st;
    if ((st = dalloc(m, &s.dval, N))) return st;
    if ((st = dalloc(m, &s.dinv, N))) return st;
    if ((st = dalloc(m, &s.R, 5 * N))) return st;
    if ((st = dalloc(m, &s.Gnew, 15 * N))) return st;
    if ((st = dalloc(m, &s.dQ, 5 * N))) return st;
    if ((st = dalloc(m, &s.w, 5 * N))) return st;
    if ((st = dalloc(m, &s.t, 5 * N))) return st;
    if ((st = dalloc(m, &s.t2, 5 * N))) return st;
    if ((st = dalloc(m, &s.hs, 65 * 64 + 256))) return st;
    if ((st = dalloc(m, &s.gram, 65 * 65 + 2 * 65 + 64))) return st;
    HGKS_CUDA(cudaMemset(s.off, 0, sizeof(double) * 25 * NF * N));
  }
  if (implicit && mixed && !s.jv32) {
    if ((st = dalloc(m, &s.jv32, (6 + 4 * NF) * N))) return st;
    if ((st = dalloc(m, &s.dval32, N))) return st;
    if ((st = dalloc(m, &s.dinv32, N))) return st;
    if ((st = dalloc(m, &s.w32, 5 * N))) return st;
    if ((st = dalloc(m, &s.t32, 5 * N))) return st;
    if ((st = dalloc(m, &s.t232, 5 * N))) return st;
    if ((st = dalloc(m, &s.red32, std::max<size_t>(16 * 608 + 64, N / 64 + 64)))) return st;
  }
  auto release = [&](void *p, size_t bytes) {
    cudaFree(p);
    for (auto &q : m.allocs) if (q == p) q = nullptr;
    m.bytes -= bytes;
  };
  if (implicit && kdim > s.kdim) {
    if (s.V) { release(s.V, sizeof(double) * (size_t)(s.kdim + 1) * s.vstride); s.V = nullptr; }
    if (s.V32) { release(s.V32, sizeof(float) * (size_t)(s.kdim + 1) * s.vstride); s.V32 = nullptr; }
    s.kdim = kdim;
  }
  // the basis of the precision in use only: FP64 for HGKS_FP64, FP32 for HGKS_MIXED
  if (implicit && !mixed && !s.V) {
    if ((st = dalloc(m, &s.V, (size_t)(s.kdim + 1) * s.vstride))) return st;
  }
  if (implicit && mixed && !s.V32) {
    if ((st = dalloc(m, &s.V32, (size_t)(s.kdim + 1) * s.vstride))) return st;
  }
  return HGKS_OK;
}

// the perturbed state and its residual of the matrix-free products (jv_mode 1)
static hgks_status ensure_fd(Mesh &m) {
  hgks_status st;
  if (!m.s.Qp && ((st = dalloc(m, &m.s.Qp, 5 * (size_t)m.N)) || (st = dalloc(m, &m.s.Rp, 5 * (size_t)m.N)))) return st;
  return HGKS_OK;
}

Mesh *mesh_of(hgks_mesh h) { return &h->m; }
void set_last_error(const char *msg) { g_err = msg; }
bool g_prof_on = false;
namespace {
struct ProfRec { int kid; cudaEvent_t a, b; };
std::vector<ProfRec> g_prof_recs;
std::vector<cudaEvent_t> g_prof_pool;
int g_prof_open = -1;
const char *kKernelNames[K_COUNT] = {"local_dt", "coef", "recon", "flux", "gather", "assemble", "spmv", "jacobi",
                                     "diag_scale", "axpy_dot", "scale", "givens", "combine", "update", "density_l1"};
cudaEvent_t prof_event() {
  if (!g_prof_pool.empty()) { cudaEvent_t e = g_prof_pool.back(); g_prof_pool.pop_back(); return e; }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}
}  // namespace
void prof_mark(int kid, cudaStream_t st, bool begin) {
  if (begin) {
    ProfRec r{kid, prof_event(), prof_event()};
    cudaEventRecord(r.a, st);
    g_prof_recs.push_back(r);
    g_prof_open = (int)g_prof_recs.size() - 1;
  } else if (g_prof_open >= 0) {
    cudaEventRecord(g_prof_recs[g_prof_open].b, st);
    g_prof_open = -1;
  }
}
}  // namespace hgks

extern "C" {

hgks_status hgks_profile_begin(void) {
  for (auto &r : g_prof_recs) { g_prof_pool.push_back(r.a); g_prof_pool.push_back(r.b); }
  g_prof_recs.clear();
  g_prof_on = true;
  return HGKS_OK;
}

hgks_status hgks_profile_end(int32_t max_kernels, char *names, double *total_ms, int64_t *launches, int32_t *n_out) {
  g_prof_on = false;
  if (!n_out) return fail(HGKS_ERR_ARG, "n_out is NULL");
  double tot[K_COUNT] = {0};
  int64_t cnt[K_COUNT] = {0};
  for (auto &r : g_prof_recs) {
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    tot[r.kid] += ms;
    cnt[r.kid]++;
  }
  int n = 0;
  for (int k = 0; k < K_COUNT; k++) {
    if (!cnt[k]) continue;
    if (n < max_kernels) {
      if (names) { std::strncpy(names + 32 * n, kKernelNames[k], 31); names[32 * n + 31] = 0; }
      if (total_ms) total_ms[n] = tot[k];
      if (launches) launches[n] = cnt[k];
    }
    n++;
  }
  *n_out = n;
  return HGKS_OK;
}


const char *hgks_last_error(void) { return g_err.c_str(); }

int64_t hgks_launch_count(int32_t reset) {
  int64_t v = g_launches;
  if (reset) g_launches = 0;
  return v;
}

hgks_status hgks_default_params(hgks_params *p) {
  if (!p) return fail(HGKS_ERR_ARG, "params is NULL");
  std::memset(p, 0, sizeof(*p));
  p->scheme = HGKS_WENO; p->weights = HGKS_NONLINEAR; p->viscous = 0; p->characteristic = 1;
  p->precision = HGKS_FP64; p->jv_mode = 0; p->krylov_dim = 10; p->restarts = 3; p->jacobi_sweeps = 2;
  p->tstar_end = 1; p->gamma = 1.4; p->Pr = 1.0; p->mu = 0.0; p->cfl = 10.0; p->flux_cfl = 1.0;
  p->tau_eps = 0.1; p->tau_C = 1.0; p->lin_weight = 0.025; p->weno_eps = 1e-6; p->flux_dt = 0.0;
  p->rho_inf = 1.0; p->u_inf[0] = 0.3; p->p_inf = 1.0 / 1.4; p->wall_T = 1.0 / 1.4; p->lid_speed = 0.0;
  p->grad_relax = 1.0;
  return HGKS_OK;
}

}  // extern "C"

namespace {
hgks_status create_mesh(const double *xyz, int64_t n_vert, const int64_t *cells, int32_t nvc, int64_t n_cells,
                        const int64_t *bface, const int32_t *btag, int64_t n_bface, const double *periodic_shift,
                        int32_t n_periodic, int32_t scheme_mask, int32_t device, hgks_mesh *out, int64_t *perm_out) {
  HGKS_RANGE("hgks mesh create");
  if (!out) return fail(HGKS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if ((scheme_mask & 3) == 0) return fail(HGKS_ERR_ARG, "scheme_mask selects no scheme");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) return fail(HGKS_ERR_CUDA, "no CUDA device");
  if (device < 0 || device >= ndev) return fail(HGKS_ERR_ARG, "device index out of range");
  HostMesh hm;
  std::string err;
  hgks_status st = build_host_mesh(xyz, n_vert, cells, nvc, n_cells, bface, btag, n_bface, periodic_shift,
                                   n_periodic, scheme_mask & 3, hm, err);
  if (st) return fail(st, err);
  hgks_mesh_s *h = new (std::nothrow) hgks_mesh_s;
  if (!h) return fail(HGKS_ERR_OOM, "host allocation");
  Mesh &m = h->m;
  m.device = device;
  m.N = hm.N; m.F = hm.F; m.Fb = hm.Fb; m.schemes = scheme_mask & 3;
  auto bail = [&](hgks_status s2) { free_all(m); delete h; return s2; };
  DeviceScope dev_scope(device);
  if (dev_scope.error() != cudaSuccess) return bail(cuda_fail(dev_scope.error(), "cudaSetDevice"));
  DevMesh &d = m.d;
  d.N = (int)hm.N; d.F = (int)hm.F; d.hex = hm.hex;
  std::vector<double> inv_vol(hm.N);
  for (int64_t i = 0; i < hm.N; i++) inv_vol[i] = 1.0 / hm.vol[i];
  if ((st = upload(m, &d.vol, hm.vol)) || (st = upload(m, &d.inv_vol, inv_vol)) || (st = upload(m, &d.h, hm.h)) ||
      (st = upload(m, &d.m2, hm.m2)) || (st = upload(m, &d.cnb, hm.cnb)) || (st = upload(m, &d.cface, hm.cface)) ||
      (st = upload(m, &d.xg, hm.xg)) || (st = upload(m, &d.sten, hm.sten)) || (st = upload(m, &d.X0, hm.X0)) ||
      (st = upload(m, &d.Xs, hm.Xs)) || (st = upload(m, &d.ssl, hm.ssl)) || (st = upload(m, &d.subvalid, hm.subvalid)) || (st = upload(m, &d.H0, hm.H0)) ||
      (st = upload(m, &d.Hm, hm.Hm)) || (st = upload(m, &d.fl, hm.fl)) || (st = upload(m, &d.fr, hm.fr)) ||
      (st = upload(m, &d.ftag, hm.ftag)) || (st = upload(m, &d.fT, hm.fT)) || (st = upload(m, &d.fS, hm.fS)) ||
      (st = upload(m, &d.fdist, hm.fdist)) || (hm.hex && (st = upload(m, &d.fw, hm.fw))))
    return bail(st);
  if ((st = ensure_scratch(m, 0, false))) return bail(st);
  m.vol_host = hm.vol;
  if (perm_out) std::memcpy(perm_out, hm.perm.data(), sizeof(int64_t) * hm.N);
  *out = h;
  return HGKS_OK;
}
}  // namespace

extern "C" {

hgks_status hgks_mesh_create(const double *xyz, int64_t n_vert, const int64_t *tet4, int64_t n_tet,
                             const int64_t *bface3, const int32_t *btag, int64_t n_bface,
                             const double *periodic_shift, int32_t n_periodic, int32_t scheme_mask,
                             int32_t device, hgks_mesh *out, int64_t *perm_out) {
  return create_mesh(xyz, n_vert, tet4, 4, n_tet, bface3, btag, n_bface, periodic_shift, n_periodic, scheme_mask,
                     device, out, perm_out);
}

hgks_status hgks_mesh_create_hex(const double *xyz, int64_t n_vert, const int64_t *hex8, int64_t n_hex,
                                 const int64_t *bquad4, const int32_t *btag, int64_t n_bface,
                                 const double *periodic_shift, int32_t n_periodic, int32_t scheme_mask,
                                 int32_t device, hgks_mesh *out, int64_t *perm_out) {
  return create_mesh(xyz, n_vert, hex8, 8, n_hex, bquad4, btag, n_bface, periodic_shift, n_periodic, scheme_mask,
                     device, out, perm_out);
}

hgks_status hgks_mesh_destroy(hgks_mesh mesh) {
  if (!mesh) return fail(HGKS_ERR_ARG, "mesh is NULL");
  DeviceScope dev_scope(mesh->m.device);
  free_all(mesh->m);
  delete mesh;
  return HGKS_OK;
}

hgks_status hgks_mesh_info(hgks_mesh mesh, hgks_mesh_info_t *info) {
  if (!mesh || !info) return fail(HGKS_ERR_ARG, "NULL argument");
  info->n_cells = mesh->m.N; info->n_faces = mesh->m.F; info->n_boundary_faces = mesh->m.Fb;
  info->device_bytes = (int64_t)mesh->m.bytes; info->device = mesh->m.device; info->schemes = mesh->m.schemes;
  info->faces_per_cell = mesh->m.d.hex ? 6 : 4;
  return HGKS_OK;
}

hgks_status hgks_mesh_volumes(hgks_mesh mesh, double *vol_host) {
  if (!mesh || !vol_host) return fail(HGKS_ERR_ARG, "NULL argument");
  std::memcpy(vol_host, mesh->m.vol_host.data(), sizeof(double) * mesh->m.N);
  return HGKS_OK;
}

hgks_status hgks_residual(hgks_mesh mesh, const hgks_params *p, const double *Q, const double *G, double *R,
                          double *G_new, void *cuda_stream) {
  if (!mesh) return fail(HGKS_ERR_ARG, "mesh is NULL");
  Mesh &m = mesh->m;
  hgks_params P;
  hgks_status st = take_params(m, p, &P);
  if (st) return st;
  p = &P;
  if (!Q || !R) return fail(HGKS_ERR_ARG, "Q or R is NULL");
  if (p->scheme == HGKS_HWENO && (!G || !G_new)) return fail(HGKS_ERR_ARG, "compact scheme needs G and G_new");
  HGKS_ON_DEVICE(m.device);
  if ((st = ensure_scratch(m, 0, false))) return st;
  launch_residual(m.d, m.s, *p, Q, G, R, G_new, (cudaStream_t)cuda_stream);
  return last_launch();
}

hgks_status hgks_local_dt(hgks_mesh mesh, const hgks_params *p, const double *Q, double *dt, void *cuda_stream) {
  if (!mesh) return fail(HGKS_ERR_ARG, "mesh is NULL");
  Mesh &m = mesh->m;
  hgks_params P;
  hgks_status st = take_params(m, p, &P);
  if (st) return st;
  p = &P;
  if (!Q || !dt) return fail(HGKS_ERR_ARG, "Q or dt is NULL");
  HGKS_ON_DEVICE(m.device);
  launch_local_dt(m.d, *p, Q, dt, (cudaStream_t)cuda_stream);
  return last_launch();
}

hgks_status hgks_assemble(hgks_mesh mesh, const hgks_params *p, const double *Q, const double *dt, double *diag_out,
                          double *off_out, void *cuda_stream) {
  if (!mesh) return fail(HGKS_ERR_ARG, "mesh is NULL");
  Mesh &m = mesh->m;
  hgks_params P;
  hgks_status st = take_params(m, p, &P);
  if (st) return st;
  p = &P;
  if (!Q || !dt) return fail(HGKS_ERR_ARG, "Q or dt is NULL");
  HGKS_ON_DEVICE(m.device);
  if ((st = ensure_scratch(m, p->krylov_dim, true, p->precision == HGKS_MIXED))) return st;
  if (p->jv_mode == 1 && (st = ensure_fd(m))) return st;
  launch_assemble(m.d, m.s, *p, Q, dt, diag_out, off_out, (cudaStream_t)cuda_stream);
  return last_launch();
}

hgks_status hgks_apply_jacobian(hgks_mesh mesh, const double *x, double *y, void *cuda_stream) {
  if (!mesh || !x || !y) return fail(HGKS_ERR_ARG, "NULL argument");
  Mesh &m = mesh->m;
  if (!m.s.off) return fail(HGKS_ERR_ARG, "hgks_assemble has not been called");
  HGKS_ON_DEVICE(m.device);
  launch_apply_A(m.d, m.s, x, y, (cudaStream_t)cuda_stream);
  return last_launch();
}

hgks_status hgks_apply_jacobian_fd(hgks_mesh mesh, const hgks_params *p, const double *Q, const double *G,
                                   const double *dt, const double *x, double *y, void *cuda_stream) {
  if (!mesh) return fail(HGKS_ERR_ARG, "mesh is NULL");
  Mesh &m = mesh->m;
  hgks_params P;
  hgks_status st = take_params(m, p, &P);
  if (st) return st;
  p = &P;
  if (!Q || !dt || !x || !y || (p->scheme == HGKS_HWENO && !G)) return fail(HGKS_ERR_ARG, "NULL argument");
  HGKS_ON_DEVICE(m.device);
  if ((st = ensure_scratch(m, p->krylov_dim, true, false)) || (st = ensure_fd(m))) return st;
  cudaStream_t s_ = (cudaStream_t)cuda_stream;
  HGKS_CUDA(cudaMemcpyAsync(m.s.dt, dt, sizeof(double) * m.N, cudaMemcpyDeviceToDevice, s_));
  launch_residual(m.d, m.s, *p, Q, G, m.s.R, nullptr, s_, false, false);
  launch_norm(m.d, m.s, Q, m.s.hs + kHsNormQ, s_);
  launch_apply_fd(m.d, m.s, *p, Q, G, x, nullptr, y, s_);
  return last_launch();
}

hgks_status hgks_wall_force(hgks_mesh mesh, const hgks_params *p, const double *Q, const double *G, int32_t tag,
                            double *force_host, void *cuda_stream) {
  if (!mesh) return fail(HGKS_ERR_ARG, "mesh is NULL");
  Mesh &m = mesh->m;
  hgks_params P;
  hgks_status st = take_params(m, p, &P);
  if (st) return st;
  p = &P;
  if (!Q || !force_host || (p->scheme == HGKS_HWENO && !G)) return fail(HGKS_ERR_ARG, "NULL argument");
  HGKS_ON_DEVICE(m.device);
  if ((st = ensure_scratch(m, p->krylov_dim, true, p->precision == HGKS_MIXED))) return st;
  cudaStream_t s_ = (cudaStream_t)cuda_stream;
  launch_residual(m.d, m.s, *p, Q, G, m.s.R, nullptr, s_);
  double *fdev = m.s.hs + kHsNormQ + 4;
  launch_wall_force(m.d, m.s, tag, fdev, s_);
  HGKS_CUDA(cudaMemcpyAsync(force_host, fdev, 3 * sizeof(double), cudaMemcpyDeviceToHost, s_));
  HGKS_CUDA(cudaStreamSynchronize(s_));
  return last_launch();
}

hgks_status hgks_precondition(hgks_mesh mesh, int32_t sweeps, const double *b, double *x, void *cuda_stream) {
  if (!mesh || !b || !x) return fail(HGKS_ERR_ARG, "NULL argument");
  if (b == x) return fail(HGKS_ERR_ARG, "b and x must not alias");
  if (sweeps < 0) return fail(HGKS_ERR_ARG, "negative sweeps");
  Mesh &m = mesh->m;
  if (!m.s.off) return fail(HGKS_ERR_ARG, "hgks_assemble has not been called");
  HGKS_ON_DEVICE(m.device);
  launch_precondition(m.d, m.s, sweeps, b, x, (cudaStream_t)cuda_stream);
  return last_launch();
}

// have_residual: s.R, s.Gnew, s.dt and the density L1 already hold those of Q
// The device work of one outer step of Algorithm 1 (launch sequence fixed by
// the parameters: capturable).
static hgks_status enqueue_step(Mesh &m, const hgks_params *p, double *Q, double *G, double *dQ_out,
                                bool have_residual, cudaStream_t st_) {
  const DevMesh &d = m.d;
  Scratch &s = m.s;
  double *res_dev = s.hs + 65 * 64 + 200;
  if (!have_residual) {
    launch_residual(d, s, *p, Q, G, s.R, p->scheme == HGKS_HWENO ? s.Gnew : nullptr, st_);
    launch_density_l1(d, s, s.R, res_dev, st_);
  }
  launch_assemble(d, s, *p, Q, s.dt, nullptr, nullptr, st_);
  hgks_status st = gmres_solve(d, s, *p, s.R, s.dQ, nullptr, st_, Q, G);
  if (st) return st;
  if (dQ_out) HGKS_CUDA(cudaMemcpyAsync(dQ_out, s.dQ, sizeof(double) * 5 * m.N, cudaMemcpyDeviceToDevice, st_));
  launch_update(d, Q, s.dQ, G, s.Gnew, p->scheme == HGKS_HWENO ? 15 : 0, p->grad_relax, st_);
  return last_launch();
}

// Runs the step's device work as a CUDA graph (captured on the mesh's own stream,
// again whenever the parameters or the state pointers change); eagerly while the
// per-kernel profiler is on.
static hgks_status run_step(Mesh &m, const hgks_params *p, double *Q, double *G, double *dQ_out, bool have_residual,
                            cudaStream_t user) {
  if (g_prof_on) return enqueue_step(m, p, Q, G, dQ_out, have_residual, user);
  if (!m.graph) {
    m.graph = new (std::nothrow) StepGraph;
    if (!m.graph) return fail(HGKS_ERR_OOM, "host allocation");
    HGKS_CUDA(cudaStreamCreateWithFlags(&m.graph->stream, cudaStreamNonBlocking));
    HGKS_CUDA(cudaEventCreateWithFlags(&m.graph->ev_in, cudaEventDisableTiming));
    HGKS_CUDA(cudaEventCreateWithFlags(&m.graph->ev_out, cudaEventDisableTiming));
  }
  StepGraph &g = *m.graph;
  const bool same = g.exec && std::memcmp(&g.p, p, sizeof(hgks_params)) == 0 && g.Q == Q && g.G == G &&
                    g.dQ_out == dQ_out && g.have_res == have_residual;
  if (!same) {
    if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
    cudaGraph_t graph = nullptr;
    HGKS_CUDA(cudaStreamBeginCapture(g.stream, cudaStreamCaptureModeThreadLocal));
    const int64_t l0 = g_launches;
    hgks_status st = enqueue_step(m, p, Q, G, dQ_out, have_residual, g.stream);
    g.launches = g_launches - l0;
    g_launches = l0;
    cudaError_t e = cudaStreamEndCapture(g.stream, &graph);
    if (!st && e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (st) return st;
    if (e != cudaSuccess) { cudaGetLastError(); g.exec = nullptr; return cuda_fail(e, "CUDA graph capture of the step"); }
    g.p = *p; g.Q = Q; g.G = G; g.dQ_out = dQ_out; g.have_res = have_residual;
  }
  HGKS_CUDA(cudaEventRecord(g.ev_in, user));
  HGKS_CUDA(cudaStreamWaitEvent(g.stream, g.ev_in, 0));
  HGKS_CUDA(cudaGraphLaunch(g.exec, g.stream));
  g_launches += g.launches;
  HGKS_CUDA(cudaEventRecord(g.ev_out, g.stream));
  HGKS_CUDA(cudaStreamWaitEvent(user, g.ev_out, 0));
  return HGKS_OK;
}

static hgks_status gmres_step_impl(Mesh &m, const hgks_params *p, double *Q, double *G, double *dQ_out,
                                   hgks_step_info *info, cudaStream_t st_, bool have_residual = false) {
  Scratch &s = m.s;
  double *res_dev = s.hs + 65 * 64 + 200;
  hgks_status st = run_step(m, p, Q, G, dQ_out, have_residual, st_);
  if (st) return st;
  if (info) info->krylov_iters = p->restarts * p->krylov_dim;
  double host[3];
  const int mk = p->krylov_dim;
  HGKS_CUDA(cudaMemcpyAsync(host, res_dev, sizeof(double), cudaMemcpyDeviceToHost, st_));
  HGKS_CUDA(cudaMemcpyAsync(host + 1, s.hs + (mk + 1) * mk + 1 + mk, 2 * sizeof(double), cudaMemcpyDeviceToHost, st_));
  int nonphys = 0;
  HGKS_CUDA(cudaMemcpyAsync(&nonphys, s.flags, sizeof(int), cudaMemcpyDeviceToHost, st_));
  HGKS_CUDA(cudaMemsetAsync(s.flags, 0, sizeof(int), st_));
  HGKS_CUDA(cudaStreamSynchronize(st_));
  const double res = host[0] / (double)m.N;
  if (info) {
    info->res_l1 = res;
    info->lin_res[0] = host[1];
    info->lin_res[1] = host[2];
    info->nonphysical = nonphys;
  }
  if (!std::isfinite(res)) return fail(HGKS_ERR_NONPHYSICAL, "non-finite residual");
  return HGKS_OK;
}

hgks_status hgks_gmres_step(hgks_mesh mesh, const hgks_params *p, double *Q, double *G, double *dQ_out,
                            hgks_step_info *info, void *cuda_stream) {
  if (!mesh) return fail(HGKS_ERR_ARG, "mesh is NULL");
  Mesh &m = mesh->m;
  hgks_params P;
  hgks_status st = take_params(m, p, &P);
  if (st) return st;
  p = &P;
  if (!Q) return fail(HGKS_ERR_ARG, "Q is NULL");
  if (p->scheme == HGKS_HWENO && !G) return fail(HGKS_ERR_ARG, "compact scheme needs G");
  HGKS_ON_DEVICE(m.device);
  if ((st = ensure_scratch(m, p->krylov_dim, true, p->precision == HGKS_MIXED))) return st;
  if (p->jv_mode == 1 && (st = ensure_fd(m))) return st;
  if (info) std::memset(info, 0, sizeof(*info));
  return gmres_step_impl(m, p, Q, G, dQ_out, info, (cudaStream_t)cuda_stream);
}

// Algorithm 1 from step k0 with the drop reference ref0 (0, 0: a fresh solve)
static hgks_status solve_impl(hgks_mesh mesh, const hgks_params *p, double *Q, double *G, double drop_tol,
                              int32_t max_steps, int32_t k0, double ref0, double *hist_host, hgks_solve_info *info,
                              void *cuda_stream) {
  if (!mesh) return fail(HGKS_ERR_ARG, "mesh is NULL");
  Mesh &m = mesh->m;
  hgks_params P;
  hgks_status st = take_params(m, p, &P);
  if (st) return st;
  p = &P;
  if (!Q || (p->scheme == HGKS_HWENO && !G)) return fail(HGKS_ERR_ARG, "Q (or G) is NULL");
  if (!(drop_tol > 0.0) || max_steps < 0) return fail(HGKS_ERR_ARG, "drop_tol must be > 0 and max_steps >= 0");
  if (k0 < 0 || k0 > max_steps || !(ref0 >= 0.0)) return fail(HGKS_ERR_ARG, "resume point out of range");
  HGKS_ON_DEVICE(m.device);
  if ((st = ensure_scratch(m, p->krylov_dim, true, p->precision == HGKS_MIXED))) return st;
  if (p->jv_mode == 1 && (st = ensure_fd(m))) return st;
  cudaStream_t s_ = (cudaStream_t)cuda_stream;
  double ref = ref0, res = 0.0;
  int k = k0;
  bool conv = false;
  for (;; k++) {
    // the residual of the current state decides; the step then updates it
    launch_residual(m.d, m.s, *p, Q, G, m.s.R, p->scheme == HGKS_HWENO ? m.s.Gnew : nullptr, s_);
    double *res_dev = m.s.hs + 65 * 64 + 200;
    launch_density_l1(m.d, m.s, m.s.R, res_dev, s_);
    double h = 0.0;
    HGKS_CUDA(cudaMemcpyAsync(&h, res_dev, sizeof(double), cudaMemcpyDeviceToHost, s_));
    HGKS_CUDA(cudaStreamSynchronize(s_));
    res = h / (double)m.N;
    if (!std::isfinite(res)) { st = fail(HGKS_ERR_NONPHYSICAL, "non-finite residual"); break; }
    if (hist_host) hist_host[k] = res;
    if (res > ref) ref = res;
    if (ref > 0.0 && res <= drop_tol * ref) { conv = true; break; }   // a zero reference certifies no drop
    if (k >= max_steps) break;
    hgks_step_info si;
    if ((st = gmres_step_impl(m, p, Q, G, nullptr, &si, s_, true))) break;
  }
  if (info) { info->steps = k; info->converged = conv; info->res_ref = ref; info->res_final = res; }
  if (st) return st;
  if (!conv) return fail(HGKS_ERR_NOT_CONVERGED, "max_steps reached");
  return HGKS_OK;
}

hgks_status hgks_solve_steady(hgks_mesh mesh, const hgks_params *p, double *Q, double *G, double drop_tol,
                              int32_t max_steps, double *hist_host, hgks_solve_info *info, void *cuda_stream) {
  return solve_impl(mesh, p, Q, G, drop_tol, max_steps, 0, 0.0, hist_host, info, cuda_stream);
}

hgks_status hgks_solve_resume(hgks_mesh mesh, const hgks_params *p, double *Q, double *G, double drop_tol,
                              int32_t max_steps, const hgks_solve_info *from, double *hist_host,
                              hgks_solve_info *info, void *cuda_stream) {
  if (!from) return fail(HGKS_ERR_ARG, "from is NULL");
  return solve_impl(mesh, p, Q, G, drop_tol, max_steps, from->steps, from->res_ref, hist_host, info, cuda_stream);
}

// device copies of host-side state for the *_host entry points: Q, G, R, G_new
static hgks_status host_state_buffer(Mesh &m, double **buf) {
  if (!m.s.hostbuf) {
    hgks_status st = dalloc(m, &m.s.hostbuf, 40 * (size_t)m.N);
    if (st) return st;
  }
  *buf = m.s.hostbuf;
  return HGKS_OK;
}

hgks_status hgks_residual_host(hgks_mesh mesh, const hgks_params *p, const double *Q_host, const double *G_host,
                               double *R_host, double *G_new_host, void *cuda_stream) {
  if (!mesh) return fail(HGKS_ERR_ARG, "mesh is NULL");
  Mesh &m = mesh->m;
  hgks_params P;
  hgks_status st = take_params(m, p, &P);
  if (st) return st;
  p = &P;
  const bool compact = p->scheme == HGKS_HWENO;
  if (!Q_host || !R_host || (compact && (!G_host || !G_new_host))) return fail(HGKS_ERR_ARG, "NULL host array");
  HGKS_ON_DEVICE(m.device);
  if ((st = ensure_scratch(m, 0, false))) return st;
  double *buf;
  if ((st = host_state_buffer(m, &buf))) return st;
  const size_t N = m.N;
  double *Qd = buf, *Gd = buf + 5 * N, *Rd = buf + 20 * N, *Gn = buf + 25 * N;
  cudaStream_t s_ = (cudaStream_t)cuda_stream;
  HGKS_CUDA(cudaMemcpyAsync(Qd, Q_host, 5 * N * sizeof(double), cudaMemcpyHostToDevice, s_));
  if (compact) HGKS_CUDA(cudaMemcpyAsync(Gd, G_host, 15 * N * sizeof(double), cudaMemcpyHostToDevice, s_));
  launch_residual(m.d, m.s, *p, Qd, compact ? Gd : nullptr, Rd, compact ? Gn : nullptr, s_);
  if ((st = last_launch())) return st;
  HGKS_CUDA(cudaMemcpyAsync(R_host, Rd, 5 * N * sizeof(double), cudaMemcpyDeviceToHost, s_));
  if (compact) HGKS_CUDA(cudaMemcpyAsync(G_new_host, Gn, 15 * N * sizeof(double), cudaMemcpyDeviceToHost, s_));
  HGKS_CUDA(cudaStreamSynchronize(s_));
  return HGKS_OK;
}

hgks_status hgks_gmres_step_host(hgks_mesh mesh, const hgks_params *p, double *Q_host, double *G_host,
                                 hgks_step_info *info, void *cuda_stream) {
  if (!mesh) return fail(HGKS_ERR_ARG, "mesh is NULL");
  Mesh &m = mesh->m;
  hgks_params P;
  hgks_status st = take_params(m, p, &P);
  if (st) return st;
  p = &P;
  const bool compact = p->scheme == HGKS_HWENO;
  if (!Q_host || (compact && !G_host)) return fail(HGKS_ERR_ARG, "NULL host array");
  HGKS_ON_DEVICE(m.device);
  if ((st = ensure_scratch(m, p->krylov_dim, true, p->precision == HGKS_MIXED))) return st;
  if (p->jv_mode == 1 && (st = ensure_fd(m))) return st;
  double *buf;
  if ((st = host_state_buffer(m, &buf))) return st;
  const size_t N = m.N;
  double *Qd = buf, *Gd = buf + 5 * N;
  cudaStream_t s_ = (cudaStream_t)cuda_stream;
  HGKS_CUDA(cudaMemcpyAsync(Qd, Q_host, 5 * N * sizeof(double), cudaMemcpyHostToDevice, s_));
  if (compact) HGKS_CUDA(cudaMemcpyAsync(Gd, G_host, 15 * N * sizeof(double), cudaMemcpyHostToDevice, s_));
  if (info) std::memset(info, 0, sizeof(*info));
  if ((st = gmres_step_impl(m, p, Qd, compact ? Gd : nullptr, nullptr, info, s_))) return st;
  HGKS_CUDA(cudaMemcpyAsync(Q_host, Qd, 5 * N * sizeof(double), cudaMemcpyDeviceToHost, s_));
  if (compact) HGKS_CUDA(cudaMemcpyAsync(G_host, Gd, 15 * N * sizeof(double), cudaMemcpyDeviceToHost, s_));
  HGKS_CUDA(cudaStreamSynchronize(s_));
  return HGKS_OK;
}

hgks_status hgks_sync(void *cuda_stream) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  return HGKS_OK;
}

}  // extern "C"
