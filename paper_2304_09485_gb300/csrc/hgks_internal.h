// Internal declarations of libhgks (not part of the C ABI).
//
// Device data of one mesh, in the library's internal (space-filling-curve)
// cell order, component-major ("structure of arrays") so that a warp of
// consecutive cells reads consecutive addresses:
//   per cell  (N): volume, 1/volume, h = vol^(1/3), second moments, neighbours,
//                  faces, Gauss points in the cell's scaled frame, fits
//   per face  (F): left/right cell, boundary tag, frame (n, t1, t2), area
#pragma once
#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include "../../include/hgks.h"

namespace hgks {

constexpr int kCoefA = 45;      // quadratic coefficients: 9 x 5 (then 15 per sub-polynomial, ShapeOf::COEF)
constexpr int kFaceState = 20;  // W[5] + dW[3][5] at one Gauss point, face frame

// Compile-time shape of a cell kind (Sec. 3.1). Tetrahedra: 4 triangular faces
// with 3 Gauss points, big stencil <= 16 cells, 4 sub-stencils of up to 6 cells
// (slots in 4 bits). Hexahedra: 6 quadrilateral faces with 2 x 2 Gauss points,
// big stencil <= 24 cells, 8 sub-stencils of 3 face neighbours (slots in 8 bits).
// The compact scheme has one sub-stencil per face.
struct TetShape {
  static constexpr int NF = 4, NG = 3, BIG = 16, NSUBW = 4, SUBK = 6, SLOTBITS = 4;
};
struct HexShape {
  static constexpr int NF = 6, NG = 4, BIG = 24, NSUBW = 8, SUBK = 3, SLOTBITS = 8;
};
template <class S> struct ShapeOf {
  static constexpr int NSUB = S::NSUBW > S::NF ? S::NSUBW : S::NF;   // sub-polynomials held per cell
  static constexpr int COEF = kCoefA + 15 * NSUB;                  // coefficients per cell
  static constexpr int HCOLS = S::NF + 3 * (1 + S::NF);            // data columns of the compact fit
};

struct DevMesh {
  int N = 0, F = 0;
  int hex = 0;                   // 0: tetrahedra (TetShape), 1: hexahedra (HexShape)
  // cells
  double *vol = nullptr, *inv_vol = nullptr, *h = nullptr;
  double *m2 = nullptr;          // [6][N] avg over the cell of xh_a xh_b: xx,yy,zz,xy,xz,yz
  // sizes below for tetrahedra; hexahedra: NF = 6 faces, NG = 4 Gauss points,
  // BIG = 24, 8 sub-stencils of SUBK = 3 cells with 8-bit slots, 27 compact columns
  int *cnb = nullptr;            // [NF][N] neighbour across local face p, -1 on a boundary
  int *cface = nullptr;          // [NF][N] 2*face + side (side 0: the cell is the face's left)
  double *xg = nullptr;          // [NF*NG*3][N] Gauss points of face slot p: (p*NG+g)*3+d, scaled frame
  // non-compact (WENO)
  int *sten = nullptr;           // [BIG][N] big stencil, -1 padded
  double *X0 = nullptr;          // [9*BIG][N] a_d = sum_k X0[d*BIG+k] (Q_k - Q_i)
  double *Xs = nullptr;          // [NSUBW*3*SUBK][N] b_j^m = sum_s Xs[(m*3+j)*SUBK+s] (Q_k(s) - Q_i)
  unsigned *ssl = nullptr;       // [NSUBW][N] k(s) of sub-stencil m: SLOTBITS-bit big-stencil slots, ascending
  unsigned char *subvalid = nullptr;  // [N] bit m: sub-stencil m used
  // compact (HWENO)
  double *H0 = nullptr;          // [9*HCOLS][N] a_d from (dQ of slots 0..NF-1, G_i, G of slots 0..NF-1)
  double *Hm = nullptr;          // [NF*3*7][N] b^m from (dQ_m, G_i, G_m)
  // faces
  int *fl = nullptr, *fr = nullptr;   // [F] left/right cell, fr = -1 on a boundary
  signed char *ftag = nullptr;        // [F] boundary tag, 0 inside
  double *fT = nullptr;          // [9][F] rows n, t1, t2 (n from left to right)
  double *fS = nullptr;          // [F] area
  double *fw = nullptr;          // [NG][F] Gauss weights of the quadrilateral faces (sum 1); null for tetrahedra
  double *fdist = nullptr;       // [F] |x_L - x_R| (or twice the wall distance on a boundary)
  // batches of meshes (hgks_batch_*): per-mesh parameters and the mesh of every
  // cell (-1 for the padding cells that align each mesh to a 256-cell block) and face
  const hgks_params *ptab = nullptr;
  const short *cmesh = nullptr, *fmesh = nullptr;
  const int *mact = nullptr;             // [meshes] 1 while the mesh iterates; its cells are skipped otherwise
  int NL = 0, FL = 0;                    // batches: cells [0, NL) and faces [0, FL) hold every mesh in use
};

// A batch is an arena of cells and faces shared by up to `nmesh` meshes (slots).
// Each mesh occupies a range of cells starting on a multiple of kBatchBlock, so
// that a block of the batched Krylov kernels (one thread per cell) lies in one
// mesh, and a range of faces. Cells and faces outside every range, and padding
// cells, have mesh -1; per-mesh arrays are indexed from -1 (entry -1 is a
// permanently inactive slot), so "mesh of x" can always be looked up.
constexpr int kBatchBlock = 256;
constexpr int kBatchMdot = 8;    // basis vectors per batched multi-dot launch (FP32 one-pass MGS)
struct BatchDev {
  int nmesh = 0, nblocks = 0;
  const short *bmesh = nullptr;    // [nblocks] mesh of each block of kBatchBlock cells (-1: free)
  const int *bstart = nullptr;     // [nmesh] first block of each mesh
  const int *bcount = nullptr;     // [nmesh] blocks of each mesh
  unsigned *counters = nullptr;    // [nmesh] arrival counters of the per-mesh reductions (0 between launches)
  int *active = nullptr;           // [-1 .. nmesh-1] 1 while the mesh iterates; active[-1] = 0
};
// Device scalars of a batch: per mesh hs[hsz] = H[(m+1) m] | beta | y[m] | lres[2] | density L1 |
// a[m+1] | g[m+1] | Gram[(m+1)(m+1)] (the one-pass MGS of FP32 vectors) | pad
struct BatchState {
  BatchDev b;
  int hsz = 0, kdim = 0;
  double *hs = nullptr;
  double *part = nullptr;          // [nblocks] partial sums
  float *part32 = nullptr;
  const int *ncell = nullptr;      // [nmesh] real cells of each mesh
  int *steps = nullptr, *conv = nullptr, *bad = nullptr;   // [nmesh]
  double *ref = nullptr, *res = nullptr;                   // [nmesh]
  double *drop = nullptr;          // [nmesh] drop tolerance of the convergence test
  int *max_steps = nullptr;        // [nmesh] step limit
  double *hist = nullptr;          // [nmesh][hist_len] density residual history (may be null)
  int hist_len = 0;
  int l1_off = 0;                  // offset of the density L1 in a mesh's hs record
  int a_off = 0, g_off = 0, gram_off = 0;   // offsets of a, g and the basis Gram matrix (leading dimension m + 1)
};

struct Scratch {
  double *coef = nullptr;        // [COEF][N] (105 tetrahedra, 165 hexahedra)
  double *dt = nullptr;          // [N]
  double *wface = nullptr;       // [2][NG][20][F] reconstructed states at Gauss points
  double *fflux = nullptr;       // [NG][5][F] global-frame flux * area * Gauss weight
  double *fpt = nullptr;         // [NG][5][F] global-frame point values * area * Gauss weight
  // implicit
  double *dinv = nullptr, *dval = nullptr;  // [N] the diagonal block is (|Omega|/dt + sum lambda S/2) I
  double *off = nullptr;         // [NF*25][N]: block of local face p of the row cell (0 on a boundary)
  float *jv32 = nullptr;         // [6 + 4 NF][N] mixed precision: the off-diagonal blocks as products,
                                 // rows 0-5 per cell (u, v, w, H, (gamma-1)|u|^2/2, gamma-1),
                                 // rows 6 + 4p + k per (cell, local face p): n S/2 (k < 3), lambda S/2
  float *dinv32 = nullptr, *dval32 = nullptr;
  float *red32 = nullptr;
  int64_t vstride = 0;           // elements between Krylov vectors (5N padded to a multiple of 64)
  double *R = nullptr, *Gnew = nullptr, *dQ = nullptr;   // [5][N], [15][N], [5][N]
  double *V = nullptr;           // [(m+1)][5N] Krylov basis (FP64)
  float *V32 = nullptr;          // [(m+1)][5N] Krylov basis (FP32)
  double *w = nullptr, *t = nullptr, *t2 = nullptr;      // [5N]
  float *w32 = nullptr, *t32 = nullptr, *t232 = nullptr;
  double *red = nullptr;         // reduction partials
  unsigned int *red_count = nullptr;
  double *hs = nullptr;          // small device scalars: H, beta, y, norms
  double *gram = nullptr;        // [65*65 + 2*65] Gram matrix of the Krylov basis and the MGS pass sums
  int *flags = nullptr;          // [8] device flags (nonphysical count, breakdown)
  double *hostbuf = nullptr;     // [40][N] device state of the *_host entry points
  double *Qp = nullptr, *Rp = nullptr;   // [5][N] perturbed state and its residual (matrix-free products)
  int kdim = 0;
  size_t bytes = 0;
  int blk_recon = 128, blk_flux = 128;   // launch shapes of the two FP64-bound kernels (autotuned for batches)
};

// A captured implicit step of one mesh (CUDA graph), replayed while the
// parameters and state pointers stay the same.
struct StepGraph {
  cudaStream_t stream = nullptr;   // capture and replay stream, ordered after the caller's by events
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t exec = nullptr;
  hgks_params p{};
  const double *Q = nullptr, *G = nullptr, *dQ_out = nullptr;
  bool have_res = false;
  int64_t launches = 0;
};

struct Mesh {
  int device = 0;
  int64_t N = 0, F = 0, Fb = 0;
  int schemes = 0;
  DevMesh d;
  Scratch s;
  std::vector<double> vol_host;
  size_t bytes = 0;
  std::vector<void *> allocs;
  StepGraph *graph = nullptr;
};

// ---- host mesh construction (mesh_setup.cpp) ----
struct HostMesh {
  int64_t N = 0, F = 0, Fb = 0;
  int hex = 0;                           // cell kind: 0 tetrahedra, 1 hexahedra
  std::vector<int64_t> perm;             // internal -> caller
  std::vector<double> vol, h, m2, xg;    // SoA-ready, internal order
  std::vector<int> cnb, cface, sten, fl, fr;
  std::vector<signed char> ftag;
  std::vector<unsigned char> subvalid;
  std::vector<double> X0, Xs, H0, Hm, fT, fS, fw, fdist;
  std::vector<unsigned> ssl;
};
// cells: [nt][nvc] vertex indices, nvc = 4 (tetrahedra) or 8 (hexahedra: 0-3 one
// quadrilateral in cyclic order, 4 + a above a); bface: [nb][3] triangles or
// [nb][4] quadrilaterals in cyclic order
hgks_status build_host_mesh(const double *xyz, int64_t nv, const int64_t *cells, int32_t nvc, int64_t nt,
                            const int64_t *bface, const int32_t *btag, int64_t nb,
                            const double *pshift, int32_t nps, int scheme_mask, HostMesh &hm,
                            std::string &err);

// ---- kernels (residual.cu, implicit.cu) ----
void launch_local_dt(const DevMesh &m, const hgks_params &p, const double *Q, double *dt, cudaStream_t st);
// fresh_dt = false keeps s.dt (the residual then uses the step's time step)
void launch_residual(const DevMesh &m, Scratch &s, const hgks_params &p, const double *Q, const double *G,
                     double *R, double *Gnew, cudaStream_t st, bool batch = false, bool fresh_dt = true);
void launch_assemble(const DevMesh &m, Scratch &s, const hgks_params &p, const double *Q, const double *dt,
                     double *diag_out, double *off_out, cudaStream_t st, bool batch = false);
void launch_apply_A(const DevMesh &m, const Scratch &s, const double *x, double *y, cudaStream_t st);
void launch_precondition(const DevMesh &m, Scratch &s, int sweeps, const double *b, double *x, cudaStream_t st);
// Q, G: the step's state, for the matrix-free products of jv_mode 1 (s.R = L(Q), s.dt its time step)
hgks_status gmres_solve(const DevMesh &m, Scratch &s, const hgks_params &p, const double *rhs, double *dx,
                        hgks_step_info *info, cudaStream_t st, const double *Q = nullptr, const double *G = nullptr);
// y = A x (b null) or b - A x with A x = |Omega|/dt x - (L(Q + sigma x) - L(Q)) / sigma, Eq. (frechet);
// needs s.R = L(Q) and s.dt, and ||Q|| in s.hs[kHsNormQ]
void launch_apply_fd(const DevMesh &m, Scratch &s, const hgks_params &p, const double *Q, const double *G,
                     const double *x, const double *b, double *y, cudaStream_t st);
void launch_norm(const DevMesh &m, Scratch &s, const double *x, double *out_dev, cudaStream_t st);
// force[3] on the boundary faces tagged `tag`, from the face fluxes of the last residual
void launch_wall_force(const DevMesh &m, const Scratch &s, int tag, double *force_dev, cudaStream_t st);
constexpr int kHsNormQ = 65 * 64 + 210;   // hs slots of the matrix-free products: ||Q||, ||x||, sigma, 0
void launch_density_l1(const DevMesh &m, Scratch &s, const double *R, double *out_dev, cudaStream_t st);
// G = G + relax (Gnew - G) (relax 0 or 1: G = Gnew)
void launch_update(const DevMesh &m, double *Q, const double *dQ, double *G, const double *Gnew, int ncomp_g,
                   double relax, cudaStream_t st);
// batches (batch.cu): one launch per phase for all meshes of the batch
void launch_batch_gmres(const DevMesh &m, Scratch &s, BatchState &bs, const hgks_params &p, const double *rhs,
                        double *dx, cudaStream_t st);
void launch_batch_density(const DevMesh &m, BatchState &bs, const double *R, cudaStream_t st);
void launch_batch_check(BatchState &bs, cudaStream_t st);
void launch_batch_update(const DevMesh &m, BatchState &bs, double *Q, const double *dQ, double *G, const double *Gnew,
                         int ncomp_g, cudaStream_t st);
void launch_fill(double *a, int64_t n, double v, cudaStream_t st);
void launch_fill_short(short *a, int64_t n, short v, cudaStream_t st);
void launch_offset_index(int *a, int rows, int64_t n, int64_t pitch, int64_t add, cudaStream_t st);

// shared by the entry points (capi.cu)
hgks_status ensure_scratch(Mesh &m, int kdim, bool implicit, bool mixed = false);
hgks_status mesh_alloc(Mesh &m, void **p, size_t bytes);   // tracked in m.allocs, freed with the mesh
void mesh_free_all(Mesh &m);
hgks_status check_params(const Mesh &m, const hgks_params *p);
// check_params of the parameters in effect: with p->Mach > 0 the flow conditions
// derived from Mach, Re and aoa_deg (Sec. 5.1, 5.2) replace the explicit ones
hgks_status take_params(const Mesh &m, const hgks_params *p, hgks_params *out);
hgks_status fail_msg(hgks_status st, const std::string &msg);
hgks_status cuda_error(cudaError_t e, const char *where);

// accessors for entry points defined outside capi.cu
Mesh *mesh_of(hgks_mesh h);
void set_last_error(const char *msg);

// The device of a mesh (batch, server) made current for the duration of one
// entry point; the caller's current device is made current again on return.
class DeviceScope {
 public:
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev_) != cudaSuccess) prev_ = -1;
    if (prev_ != dev) { err_ = cudaSetDevice(dev); changed_ = err_ == cudaSuccess && prev_ >= 0; }
  }
  ~DeviceScope() { if (changed_) cudaSetDevice(prev_); }
  cudaError_t error() const { return err_; }
  DeviceScope(const DeviceScope &) = delete;
  DeviceScope &operator=(const DeviceScope &) = delete;

 private:
  int prev_ = -1;
  bool changed_ = false;
  cudaError_t err_ = cudaSuccess;
};
#define HGKS_ON_DEVICE(dev)                                                                  \
  hgks::DeviceScope hgks_device_scope_(dev);                                                 \
  if (hgks_device_scope_.error() != cudaSuccess) return hgks::cuda_error(hgks_device_scope_.error(), "cudaSetDevice")

// NVTX range over one phase of Algorithm 1 (inert unless a profiler is attached)
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
#define HGKS_CAT2(a, b) a##b
#define HGKS_CAT(a, b) HGKS_CAT2(a, b)
#define HGKS_RANGE(name) hgks::NvtxRange HGKS_CAT(hgks_nvtx_, __LINE__)(name)

extern thread_local int64_t g_launches;
inline void count_launch() { ++g_launches; }

// Optional per-kernel timing with CUDA events on the launching stream
// (hgks_profile_begin / hgks_profile_end). Off by default: one branch per launch.
enum KernelId { K_DT, K_COEF, K_RECON, K_FLUX, K_GATHER, K_ASSEMBLE, K_SPMV, K_JACOBI, K_DIAG, K_DOT, K_SCALE,
                K_GIVENS, K_COMBINE, K_UPDATE, K_NORM, K_COUNT };
extern bool g_prof_on;
void prof_mark(int kid, cudaStream_t st, bool begin);
#define HGKS_PROF_BEGIN(kid, st) do { if (hgks::g_prof_on) hgks::prof_mark((kid), (st), true); } while (0)
#define HGKS_PROF_END(kid, st) do { if (hgks::g_prof_on) hgks::prof_mark((kid), (st), false); hgks::count_launch(); } while (0)
inline unsigned grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace hgks
