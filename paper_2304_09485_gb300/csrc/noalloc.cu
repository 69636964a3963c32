// hgks_residual_noalloc: the residual R(U) of hgks_residual with its per-call
// scratch in a fixed array compiled into this library instead of memory the
// mesh handle allocated.
//
// Who needs it: callers that cannot call cudaMalloc once they are running, for
// example a process whose device memory is handed out by another runtime at
// start-up, or a service that must not enter the CUDA allocator while it
// answers requests. They still create the mesh up front; after that, this call
// neither allocates nor frees anything, and it does not touch the scratch
// buffers owned by the mesh handle.
//
// The scratch is the file-scope array below. Every GPU that loads the library
// holds it (32 MiB) until the process exits. Its device address is looked up
// once per device with cudaGetSymbolAddress: the host-side symbol is only a
// stand-in and must never be passed to a kernel. Every call shares the array
// and it keeps the last call's contents, so calls that may overlap on the GPU
// (other streams, other host threads) race with each other.
#include <mutex>
#include "hgks_internal.h"

namespace hgks {

constexpr size_t kNoallocDoubles = (size_t)4 << 20;   // 32 MiB of FP64 scratch
static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

namespace {
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[64] = {nullptr};   // device address of the array, per device

// doubles of scratch one residual evaluation needs on an (N cells, F faces) mesh
size_t noalloc_need(size_t N, size_t F) {
  auto up = [](size_t n) { return (n + 31) / 32 * 32; };   // keep every region 256-byte aligned
  return up((size_t)kCoef * N) + up(N) + up((size_t)2 * 3 * kFaceState * F) + 2 * up((size_t)15 * F) + 32;
}
}  // namespace

}  // namespace hgks

using namespace hgks;

namespace {
hgks_status report(hgks_status st, const char *msg) {
  set_last_error(msg);
  return st;
}
}  // namespace

extern "C" hgks_status hgks_residual_noalloc(hgks_mesh mesh, const hgks_params *p, const double *Q, const double *G,
                                             double *R, double *G_new, void *cuda_stream) {
  if (!mesh || !p || !Q || !R) return report(HGKS_ERR_ARG, "NULL mesh, params, Q or R");
  Mesh &m = *mesh_of(mesh);
  if (p->scheme != HGKS_WENO && p->scheme != HGKS_HWENO) return report(HGKS_ERR_ARG, "unknown scheme");
  if (!(m.schemes & (p->scheme == HGKS_WENO ? 1 : 2)))
    return report(HGKS_ERR_ARG, "mesh was built without data for this scheme");
  if (p->scheme == HGKS_HWENO && (!G || !G_new)) return report(HGKS_ERR_ARG, "compact scheme needs G and G_new");
  if (!(p->gamma > 1.0) || !(p->cfl > 0.0) || !(p->flux_cfl > 0.0) || !(p->Pr > 0.0) ||
      (p->viscous && !(p->mu > 0.0)) || (!p->viscous && !(p->tau_eps > 0.0)))
    return report(HGKS_ERR_ARG, "parameter out of range");
  const size_t need = noalloc_need((size_t)m.N, (size_t)m.F);
  if (need > kNoallocDoubles)
    return report(HGKS_ERR_ARG,
                  "mesh too large for the static scratch of hgks_residual_noalloc (32 MiB: about 10,000 tetrahedra)");
  if (m.device < 0 || m.device >= 64) return report(HGKS_ERR_ARG, "device index out of range");
  if (cudaSetDevice(m.device) != cudaSuccess) return report(HGKS_ERR_CUDA, "cudaSetDevice failed");
  double *base;
  {
    // set-up, once per device, with that device current
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[m.device]) {
      void *ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) return report(HGKS_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
      g_noalloc_ptr[m.device] = (double *)ptr;
    }
    base = g_noalloc_ptr[m.device];
  }
  auto up = [](size_t n) { return (n + 31) / 32 * 32; };
  const size_t N = m.N, F = m.F;
  Scratch s;
  s.coef = base;
  s.dt = s.coef + up((size_t)kCoef * N);
  s.wface = s.dt + up(N);
  s.fflux = s.wface + up((size_t)2 * 3 * kFaceState * F);
  s.fpt = s.fflux + up((size_t)15 * F);
  s.flags = (int *)(s.fpt + up((size_t)15 * F));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // the positivity counter must start at zero; every other region is fully
  // written before it is read
  if (cudaMemsetAsync(s.flags, 0, 8 * sizeof(int), st) != cudaSuccess)
    return report(HGKS_ERR_CUDA, "cudaMemsetAsync failed");
  launch_residual(m.d, s, *p, Q, G, R, G_new, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return report(HGKS_ERR_CUDA, cudaGetErrorString(e));
  return HGKS_OK;
}
