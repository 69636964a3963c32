// Internal interface of batches (batch_capi.cu) for the entry points and the
// request server (server.cpp): an arena of cells and faces holding up to
// `nslot` meshes, each placed in its own ranges and stepped together.
#pragma once
#include <cstdint>
#include <vector>
#include "hgks_internal.h"

namespace hgks {

// first-fit allocator of [start, start + len) ranges in [0, cap)
struct RangeAlloc {
  struct Range { int64_t start, len; };
  std::vector<Range> free;   // sorted by start, disjoint, never adjacent
  int64_t cap = 0;
  void init(int64_t c);
  int64_t take(int64_t len);           // start of the range, or -1
  void give(int64_t start, int64_t len);
  int64_t largest() const;
};

// where a mesh's arrays come from: a mesh handle (device) or a host build
struct MeshSource {
  int64_t N = 0, F = 0, Fb = 0;
  const double *vol = nullptr, *inv_vol = nullptr, *h = nullptr, *m2 = nullptr, *xg = nullptr;
  const int *cnb = nullptr, *cface = nullptr, *sten = nullptr, *fl = nullptr, *fr = nullptr;
  const unsigned char *subvalid = nullptr;
  const double *X0 = nullptr, *Xs = nullptr, *H0 = nullptr, *Hm = nullptr;
  const unsigned *ssl = nullptr;
  const signed char *ftag = nullptr;
  const double *fT = nullptr, *fS = nullptr, *fdist = nullptr;
  const double *fw = nullptr;            // hexahedra: Gauss weights [4][F]
  int schemes = 0;
  int hex = 0;                           // cell kind: 0 tetrahedra, 1 hexahedra
};
MeshSource source_of(const Mesh &m);
MeshSource source_of(const HostMesh &hm, std::vector<double> &inv_vol_scratch);

struct Slot {
  bool used = false;
  int64_t c0 = 0, ncell = 0, cpad = 0, f0 = 0, nface = 0, nbface = 0;
  hgks_params p{};
};

struct Batch {
  Mesh m;                                // the arena: m.N cells, m.F faces (capacities)
  BatchState bs;
  int nslot = 0;
  hgks_params p0{};                      // scheme, precision, jv_mode, krylov_dim, restarts, jacobi_sweeps
  std::vector<Slot> slots;
  RangeAlloc cells, faces;               // cells in units of kBatchBlock
  double *Q = nullptr, *G = nullptr;     // [5][N], [15][N] (compact scheme)
  hgks_params *ptab = nullptr;           // [nslot]
  short *cmesh = nullptr, *fmesh = nullptr, *bmesh = nullptr;
  int *bstart = nullptr, *bcount = nullptr, *ncell = nullptr;
  int *active_base = nullptr;            // [nslot + 1], entry 0 = slot -1
  std::vector<int> active_host;          // [nslot + 1]
  double *hist = nullptr;
  int64_t hist_cap = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // the captured step and the grids, shapes and buffers it was captured with
  cudaGraphExec_t graph = nullptr;
  int64_t graph_launches = 0;
  uint64_t graph_key[6] = {0, 0, 0, 0, 0, 0};
  uint64_t epoch = 0;                    // membership changes
};

bool compact(const Batch &B);
bool same_shared(const hgks_params &a, const hgks_params &b);
// device bytes of an arena of `cells` cells and `faces` faces
int64_t arena_bytes(int64_t cells, int64_t faces, const hgks_params &shared, int schemes, bool hex = false);
// hex: the arena holds hexahedral meshes (HexShape rows); a batch holds one cell kind
hgks_status batch_new(int device, int64_t cell_cap, int64_t face_cap, int nslot, const hgks_params &shared,
                      int schemes, Batch **out, bool hex = false);
void batch_delete(Batch *B);
// place a mesh into a free slot and free ranges: *slot = -1 if it does not fit
hgks_status batch_place(Batch &B, const MeshSource &src, const hgks_params &p, int *slot);
void batch_release(Batch &B, int slot);
// state copies of one slot, on the batch stream; Q, G device or host (cudaMemcpyDefault)
hgks_status batch_set_state(Batch &B, int slot, const double *Q, const double *G);
hgks_status batch_get_state(Batch &B, int slot, double *Q, double *G, double *R, double *G_new);
// reset the solve counters of a slot and set its test (drop tolerance, step limit)
hgks_status batch_arm(Batch &B, int slot, double drop_tol, int max_steps);
hgks_status batch_set_active(Batch &B, const std::vector<int> &active);   // [nslot]
// one step of every active slot (with the on-device convergence test when `check`)
hgks_status batch_enqueue_step(Batch &B, bool check, bool use_graph);
hgks_status enter(Batch &B, cudaStream_t user);
hgks_status leave(Batch &B, cudaStream_t user);

}  // namespace hgks
