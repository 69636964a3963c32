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
// The scratch is the file-scope array below (32 MiB). Under CUDA's lazy module
// loading (the default) the driver allocates it on a device when this file's
// module is first used there, which is the first call of this entry point on
// that device: that call also looks up the array's device address with
// cudaGetSymbolAddress (the host-side symbol is only a stand-in and must never
// be passed to a kernel). So the first call on each device belongs to the
// caller's start-up, before any stream capture and before its device memory is
// handed to another runtime; from then on the device holds the array until the
// process exits and no call allocates. Every call shares the array and it keeps
// the last call's contents, so calls that may overlap on the GPU (other
// streams, other host threads) race with each other.
#include <mutex>
#include "hgks_internal.h"

namespace hgks {

constexpr size_t kNoallocDoubles = (size_t)4 << 20;   // 32 MiB of FP64 scratch
static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

namespace {
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[64] = {nullptr};   // device address of the array, per device

// sizes of the regions, per cell and per face, of one cell kind
struct NoallocRows {
  size_t coef, face;      // coefficients per cell; Gauss points per face
  explicit NoallocRows(bool hex)
      : coef(hex ? ShapeOf<HexShape>::COEF : ShapeOf<TetShape>::COEF), face(hex ? HexShape::NG : TetShape::NG) {}
};
// doubles of scratch one residual evaluation needs on an (N cells, F faces) mesh
size_t noalloc_need(size_t N, size_t F, bool hex) {
  auto up = [](size_t n) { return (n + 31) / 32 * 32; };   // keep every region 256-byte aligned
  const NoallocRows r(hex);
  return up(r.coef * N) + up(N) + up(2 * r.face * kFaceState * F) + 2 * up(5 * r.face * F) + 32;
}
}  // namespace

}  // namespace hgks

using namespace hgks;

extern "C" hgks_status hgks_residual_noalloc(hgks_mesh mesh, const hgks_params *p, const double *Q, const double *G,
                                             double *R, double *G_new, void *cuda_stream) {
  if (!mesh) return fail_msg(HGKS_ERR_ARG, "mesh is NULL");
  Mesh &m = *mesh_of(mesh);
  hgks_params P;   // the same argument checks (and flow conditions) as hgks_residual
  hgks_status st0 = take_params(m, p, &P);
  if (st0) return st0;
  p = &P;
  if (!Q || !R) return fail_msg(HGKS_ERR_ARG, "Q or R is NULL");
  if (p->scheme == HGKS_HWENO && (!G || !G_new)) return fail_msg(HGKS_ERR_ARG, "compact scheme needs G and G_new");
  const bool hex = m.d.hex != 0;
  const size_t need = noalloc_need((size_t)m.N, (size_t)m.F, hex);
  if (need > kNoallocDoubles)
    return fail_msg(HGKS_ERR_ARG, "mesh too large for the static scratch of hgks_residual_noalloc "
                                  "(32 MiB: about 10,000 tetrahedra or 5,000 hexahedra)");
  if (m.device < 0 || m.device >= 64) return fail_msg(HGKS_ERR_ARG, "device index out of range");
  HGKS_ON_DEVICE(m.device);
  double *base;
  {
    // set-up, once per device, with that device current
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[m.device]) {
      void *ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) return fail_msg(HGKS_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
      g_noalloc_ptr[m.device] = (double *)ptr;
    }
    base = g_noalloc_ptr[m.device];
  }
  auto up = [](size_t n) { return (n + 31) / 32 * 32; };
  const size_t N = m.N, F = m.F;
  const NoallocRows r(hex);
  Scratch s;
  s.coef = base;
  s.dt = s.coef + up(r.coef * N);
  s.wface = s.dt + up(N);
  s.fflux = s.wface + up(2 * r.face * kFaceState * F);
  s.fpt = s.fflux + up(5 * r.face * F);
  s.flags = (int *)(s.fpt + up(5 * r.face * F));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // the positivity counter must start at zero; every other region is fully
  // written before it is read
  if (cudaMemsetAsync(s.flags, 0, 8 * sizeof(int), st) != cudaSuccess)
    return fail_msg(HGKS_ERR_CUDA, "cudaMemsetAsync failed");
  launch_residual(m.d, s, *p, Q, G, R, G_new, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "kernel launch");
  return HGKS_OK;
}
