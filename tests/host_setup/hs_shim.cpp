// Test-only shim: runs the library's host-side mesh construction
// (csrc/mesh_setup.cpp: cell order, face table, stencils, fits) without a GPU
// and hands its arrays out through plain pointers, for the CPU tests in
// tests/test_host_setup.py.
#include <cstring>
#include <string>
#include "../../paper_2304_09485_gb300/csrc/hgks_internal.h"

using namespace hgks;

namespace {
HostMesh g_hm;
std::string g_err;

template <typename T>
int copy_out(const std::vector<T> &v, void *out, int64_t bytes) {
  if ((int64_t)(v.size() * sizeof(T)) != bytes) return -1;
  if (bytes) std::memcpy(out, v.data(), (size_t)bytes);
  return 0;
}
}  // namespace

extern "C" int hs_build(const double *xyz, int64_t nv, const int64_t *tet, int64_t nt, const int64_t *bface,
                        const int32_t *btag, int64_t nb, const double *pshift, int32_t nps, int scheme_mask,
                        int64_t *sizes) {
  g_hm = HostMesh{};
  hgks_status st = build_host_mesh(xyz, nv, tet, 4, nt, bface, btag, nb, pshift, nps, scheme_mask, g_hm, g_err);
  sizes[0] = g_hm.N;
  sizes[1] = g_hm.F;
  sizes[2] = g_hm.Fb;
  return (int)st;
}

// cells of nvc = 4 or 8 vertices (hexahedra: boundary quadrilaterals [nb][4])
extern "C" int hs_build_cells(const double *xyz, int64_t nv, const int64_t *cells, int32_t nvc, int64_t nt,
                              const int64_t *bface, const int32_t *btag, int64_t nb, const double *pshift,
                              int32_t nps, int scheme_mask, int64_t *sizes) {
  g_hm = HostMesh{};
  hgks_status st = build_host_mesh(xyz, nv, cells, nvc, nt, bface, btag, nb, pshift, nps, scheme_mask, g_hm, g_err);
  sizes[0] = g_hm.N;
  sizes[1] = g_hm.F;
  sizes[2] = g_hm.Fb;
  return (int)st;
}

extern "C" const char *hs_error() { return g_err.c_str(); }

// copy array `name` into out (bytes must equal its size); -1 on a size mismatch, -2 unknown
extern "C" int hs_get(const char *name, void *out, int64_t bytes) {
  const std::string n(name);
  if (n == "perm") return copy_out(g_hm.perm, out, bytes);
  if (n == "vol") return copy_out(g_hm.vol, out, bytes);
  if (n == "h") return copy_out(g_hm.h, out, bytes);
  if (n == "xg") return copy_out(g_hm.xg, out, bytes);
  if (n == "X0") return copy_out(g_hm.X0, out, bytes);
  if (n == "Xs") return copy_out(g_hm.Xs, out, bytes);
  if (n == "H0") return copy_out(g_hm.H0, out, bytes);
  if (n == "Hm") return copy_out(g_hm.Hm, out, bytes);
  if (n == "fT") return copy_out(g_hm.fT, out, bytes);
  if (n == "fS") return copy_out(g_hm.fS, out, bytes);
  if (n == "fdist") return copy_out(g_hm.fdist, out, bytes);
  if (n == "cnb") return copy_out(g_hm.cnb, out, bytes);
  if (n == "cface") return copy_out(g_hm.cface, out, bytes);
  if (n == "sten") return copy_out(g_hm.sten, out, bytes);
  if (n == "fl") return copy_out(g_hm.fl, out, bytes);
  if (n == "fr") return copy_out(g_hm.fr, out, bytes);
  if (n == "ssl") return copy_out(g_hm.ssl, out, bytes);
  if (n == "subvalid") return copy_out(g_hm.subvalid, out, bytes);
  if (n == "fw") return copy_out(g_hm.fw, out, bytes);
  if (n == "m2") return copy_out(g_hm.m2, out, bytes);
  return -2;
}
