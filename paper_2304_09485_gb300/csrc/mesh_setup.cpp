// Host-side construction of a tetrahedral or hexahedral mesh for the HGKS
// residual (paper Sec. 3.1 - 3.3, Sec. 4.3).
//
//  * cells are renumbered along a Morton (Z-order) curve of their centroids, so
//    neighbours sit close in memory and a warp's gathers hit few cache lines;
//  * faces are matched by sorted vertex lists, then tagged boundary faces,
//    then periodic pairs (translation of the face centroid by a given shift);
//    faces are numbered by (left cell, local face) with left = lower cell;
//  * stencils: non-compact big stencil = face neighbours and their neighbours
//    (more rings only while fewer than 12 cells); sub-stencils (Sec. 3.1):
//    tetrahedron, sub-stencil m = three face neighbours plus the neighbours of
//    neighbour m; hexahedron, the three face neighbours across each of the eight
//    corners; kept when it has >= 3 cells whose centroids are not nearly
//    coplanar with the target's (sigma_min/sigma_max >= 1e-3); compact stencil =
//    face neighbours;
//  * fits: least squares for Eq. (polys) (modified Gram-Schmidt QR), and the
//    constrained least squares of Eq. (compact-big-1/2) (KKT system by LU),
//    in the target cell's scaled frame x_hat = (x - centroid)/h, h = vol^(1/3);
//    cell averages of monomials in closed form on a tetrahedron, by a 3 x 3 x 3
//    Gauss rule of the trilinear map on a hexahedron (exact: the integrands
//    are of degree <= 4 in each reference coordinate).
//  * hexahedron faces: the bilinear surface through the four vertices; area
//    and normal from its vector area (c - a) x (d - b) / 2, 2 x 2 Gauss points
//    of the bilinear map weighted by its area element there (sum 1). The
//    vertex order of a face is canonical (from its smallest vertex towards the
//    smaller neighbour of it), so both cells derive the same points.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>
#include <unordered_map>
#include "hgks_internal.h"

namespace hgks {
namespace {

constexpr int kFaceVerts[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
constexpr int kTriple[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {2, 0, 3}};
// hexahedron: corner (a, b, c) of each local vertex; faces (cyclic order): 0 and
// 5 the quadrilaterals 0123 and 4567, 1-4 the sides around them in order, so the
// faces at a corner are {0 or 5, k, k % 4 + 1}: Sec. 3.1's eight sub-stencils
constexpr int kHexCorner[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0}, {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
constexpr int kHexFace[6][4] = {{0, 1, 2, 3}, {0, 1, 5, 4}, {1, 2, 6, 5}, {2, 3, 7, 6}, {3, 0, 4, 7}, {4, 5, 6, 7}};
constexpr int kHexTriple[8][3] = {{0, 1, 2}, {0, 2, 3}, {0, 3, 4}, {0, 4, 1}, {5, 1, 2}, {5, 2, 3}, {5, 3, 4}, {5, 4, 1}};
constexpr int kHexQ = 27;   // points of the 3 x 3 x 3 Gauss rule

struct V3 { double x, y, z; };
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double comp(V3 a, int d) { return d == 0 ? a.x : (d == 1 ? a.y : a.z); }

struct Ref { int cell; V3 shift; };
inline bool same_shift(V3 a, V3 b) { return std::fabs(a.x - b.x) < 1e-9 && std::fabs(a.y - b.y) < 1e-9 && std::fabs(a.z - b.z) < 1e-9; }

uint64_t spread21(uint64_t v) {
  v &= 0x1fffff;
  v = (v | v << 32) & 0x1f00000000ffffULL;
  v = (v | v << 16) & 0x1f0000ff0000ffULL;
  v = (v | v << 8) & 0x100f00f00f00f00fULL;
  v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
  v = (v | v << 2) & 0x1249249249249249ULL;
  return v;
}

// modified Gram-Schmidt least-squares map: X (cols x rows), x = X b
bool lsq_map(int rows, int cols, const double *A, double *X) {
  if (rows < cols) return false;
  std::vector<double> Qm(A, A + rows * cols), R(cols * cols, 0.0);
  double rmax = 0.0;
  for (int j = 0; j < cols; j++) {
    for (int i = 0; i < j; i++) {
      double r = 0.0;
      for (int k = 0; k < rows; k++) r += Qm[k * cols + i] * Qm[k * cols + j];
      R[i * cols + j] = r;
      for (int k = 0; k < rows; k++) Qm[k * cols + j] -= r * Qm[k * cols + i];
    }
    double nn = 0.0;
    for (int k = 0; k < rows; k++) nn += Qm[k * cols + j] * Qm[k * cols + j];
    nn = std::sqrt(nn);
    R[j * cols + j] = nn;
    rmax = std::max(rmax, nn);
    if (nn == 0.0) return false;
    for (int k = 0; k < rows; k++) Qm[k * cols + j] /= nn;
  }
  for (int j = 0; j < cols; j++) if (R[j * cols + j] < 1e-12 * rmax) return false;
  for (int r = 0; r < rows; r++)
    for (int i = cols - 1; i >= 0; i--) {
      double s = Qm[r * cols + i];
      for (int l = i + 1; l < cols; l++) s -= R[i * cols + l] * X[l * rows + r];
      X[i * rows + r] = s / R[i * cols + i];
    }
  return true;
}

// Gaussian elimination with partial pivoting, n <= 16, several right-hand sides
bool lu_solve_multi(int n, std::vector<double> A, int nrhs, std::vector<double> &B) {
  for (int c = 0; c < n; c++) {
    int piv = c;
    for (int r = c + 1; r < n; r++) if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return false;
    if (piv != c) {
      for (int j = 0; j < n; j++) std::swap(A[c * n + j], A[piv * n + j]);
      for (int j = 0; j < nrhs; j++) std::swap(B[c * nrhs + j], B[piv * nrhs + j]);
    }
    for (int r = c + 1; r < n; r++) {
      double f = A[r * n + c] / A[c * n + c];
      if (f == 0.0) continue;
      for (int j = c; j < n; j++) A[r * n + j] -= f * A[c * n + j];
      for (int j = 0; j < nrhs; j++) B[r * nrhs + j] -= f * B[c * nrhs + j];
    }
  }
  for (int r = n - 1; r >= 0; r--)
    for (int j = 0; j < nrhs; j++) {
      double s = B[r * nrhs + j];
      for (int k = r + 1; k < n; k++) s -= A[r * n + k] * B[k * nrhs + j];
      B[r * nrhs + j] = s / A[r * n + r];
    }
  return true;
}

// sigma_min / sigma_max of an (rows x 3) matrix from the closed-form eigenvalues
// of the symmetric 3x3 matrix A^T A (trigonometric solution of the cubic)
double sv_ratio3(int rows, const double *A) {
  double S[3][3] = {};
  for (int r = 0; r < rows; r++)
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) S[a][b] += A[r * 3 + a] * A[r * 3 + b];
  double p1 = S[0][1] * S[0][1] + S[0][2] * S[0][2] + S[1][2] * S[1][2];
  double q = (S[0][0] + S[1][1] + S[2][2]) / 3.0;
  double p2 = (S[0][0] - q) * (S[0][0] - q) + (S[1][1] - q) * (S[1][1] - q) + (S[2][2] - q) * (S[2][2] - q) + 2.0 * p1;
  if (p2 <= 0.0) return q > 0.0 ? 1.0 : 0.0;
  double p = std::sqrt(p2 / 6.0);
  double B[3][3];
  for (int a = 0; a < 3; a++) for (int b = 0; b < 3; b++) B[a][b] = (S[a][b] - (a == b ? q : 0.0)) / p;
  double det = B[0][0] * (B[1][1] * B[2][2] - B[1][2] * B[2][1]) - B[0][1] * (B[1][0] * B[2][2] - B[1][2] * B[2][0]) +
               B[0][2] * (B[1][0] * B[2][1] - B[1][1] * B[2][0]);
  double r = std::min(1.0, std::max(-1.0, 0.5 * det));
  double phi = std::acos(r) / 3.0;
  double emax = q + 2.0 * p * std::cos(phi);
  double emin = q + 2.0 * p * std::cos(phi + 2.0 * M_PI / 3.0);
  if (emax <= 0.0) return 0.0;
  return std::sqrt(std::max(emin, 0.0) / emax);
}

struct Geo {
  const double *xyz;
  int nvc = 4;
  std::vector<int64_t> cv;       // internal order [N][nvc]
  std::vector<V3> cen;
  std::vector<double> vol, h;
  std::vector<V3> qx;            // hexahedra: [N][27] Gauss points (global frame)
  std::vector<double> qw;        // hexahedra: [N][27] weights w detJ / vol (sum 1)
  V3 vtx(int c, int a) const { const double *p = xyz + 3 * cv[(size_t)nvc * c + a]; return {p[0], p[1], p[2]}; }
  // averages over cell k (translated by s) of the 9 basis monomials, in cell i's scaled frame
  void avg_mono(int i, int k, V3 s, double *out) const {
    if (nvc == 8) {
      for (int d = 0; d < 9; d++) out[d] = 0.0;
      for (int q = 0; q < kHexQ; q++) {
        const V3 x = (1.0 / h[i]) * (qx[(size_t)kHexQ * k + q] + s - cen[i]);
        const double w = qw[(size_t)kHexQ * k + q];
        const double mo[9] = {x.x, x.y, x.z, x.x * x.x, x.y * x.y, x.z * x.z, x.x * x.y, x.x * x.z, x.y * x.z};
        for (int d = 0; d < 9; d++) out[d] += w * mo[d];
      }
      return;
    }
    V3 v[4];
    V3 sum{0, 0, 0};
    for (int a = 0; a < 4; a++) { v[a] = (1.0 / h[i]) * (vtx(k, a) + s - cen[i]); sum = sum + v[a]; }
    out[0] = 0.25 * sum.x; out[1] = 0.25 * sum.y; out[2] = 0.25 * sum.z;
    const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
    for (int t = 0; t < 6; t++) {
      double s2 = 0.0;
      for (int a = 0; a < 4; a++) s2 += comp(v[a], pa[t]) * comp(v[a], pb[t]);
      out[3 + t] = (s2 + comp(sum, pa[t]) * comp(sum, pb[t])) / 20.0;
    }
  }
};

// 3 x 3 x 3 Gauss rule of the trilinear map of hexahedron v[8]: points, weights
// w detJ (their sum is the volume); false if detJ <= 0 somewhere
bool hex_rule(const V3 *v, V3 *x, double *w) {
  const double g = std::sqrt(0.6);
  const double t[3] = {0.5 * (1.0 - g), 0.5, 0.5 * (1.0 + g)}, wt[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  int q = 0;
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++)
      for (int c = 0; c < 3; c++, q++) {
        const double r[3] = {t[a], t[b], t[c]};
        V3 p{0, 0, 0}, J[3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};   // J[e] = dx/dr_e
        for (int k = 0; k < 8; k++) {
          double f[3], df[3];
          for (int e = 0; e < 3; e++) { f[e] = kHexCorner[k][e] ? r[e] : 1.0 - r[e]; df[e] = kHexCorner[k][e] ? 1.0 : -1.0; }
          p = p + (f[0] * f[1] * f[2]) * v[k];
          J[0] = J[0] + (df[0] * f[1] * f[2]) * v[k];
          J[1] = J[1] + (f[0] * df[1] * f[2]) * v[k];
          J[2] = J[2] + (f[0] * f[1] * df[2]) * v[k];
        }
        const double det = dot(J[0], cross(J[1], J[2]));
        if (!(det > 0.0)) return false;
        x[q] = p;
        w[q] = wt[a] * wt[b] * wt[c] * det;
      }
  return true;
}

// the vertices of a quadrilateral in canonical cyclic order: from the smallest
// index towards the smaller of its two neighbours
void canonical_quad(const int64_t *cyc, int64_t *out) {
  int s = 0;
  for (int k = 1; k < 4; k++) if (cyc[k] < cyc[s]) s = k;
  const int dir = cyc[(s + 1) % 4] < cyc[(s + 3) % 4] ? 1 : 3;
  for (int k = 0; k < 4; k++) out[k] = cyc[(s + dir * k) % 4];
}

}  // namespace

hgks_status build_host_mesh(const double *xyz, int64_t nv, const int64_t *cells, int32_t nvc, int64_t nt,
                            const int64_t *bface, const int32_t *btag, int64_t nb,
                            const double *pshift, int32_t nps, int scheme_mask, HostMesh &hm,
                            std::string &err) {
  if (nt <= 0 || nv <= 0 || !xyz || !cells) { err = "empty mesh or NULL arrays"; return HGKS_ERR_ARG; }
  if (nvc != 4 && nvc != 8) { err = "cells must have 4 or 8 vertices"; return HGKS_ERR_ARG; }
  if (nt > (int64_t)0x3fffffff) { err = "too many cells for 32-bit indices"; return HGKS_ERR_ARG; }
  if (nb > 0 && (!bface || !btag)) { err = "NULL boundary arrays"; return HGKS_ERR_ARG; }
  if (nps > 0 && !pshift) { err = "NULL periodic shifts"; return HGKS_ERR_ARG; }
  const bool hex = nvc == 8;
  const int NF = hex ? HexShape::NF : TetShape::NF, NG = hex ? HexShape::NG : TetShape::NG;
  const int NFV = hex ? 4 : 3;                       // vertices of a face
  const int N = (int)nt;
  hm.hex = hex ? 1 : 0;
  // ---- per-cell geometry in caller order, then Morton order ----
  std::vector<V3> cen0(N);
  std::vector<double> vol0(N);
  std::vector<V3> qx0;
  std::vector<double> qw0;
  if (hex) { qx0.resize((size_t)kHexQ * N); qw0.resize((size_t)kHexQ * N); }
  for (int c = 0; c < N; c++) {
    V3 v[8];
    for (int a = 0; a < nvc; a++) {
      int64_t vi = cells[(size_t)nvc * c + a];
      if (vi < 0 || vi >= nv) { err = "vertex index out of range"; return HGKS_ERR_MESH; }
      v[a] = {xyz[3 * vi], xyz[3 * vi + 1], xyz[3 * vi + 2]};
    }
    if (!hex) {
      double det = dot(v[1] - v[0], cross(v[2] - v[0], v[3] - v[0]));
      vol0[c] = std::fabs(det) / 6.0;
      if (!(vol0[c] > 0.0) || !std::isfinite(vol0[c])) { err = "degenerate tetrahedron " + std::to_string(c); return HGKS_ERR_MESH; }
      cen0[c] = 0.25 * (v[0] + v[1] + v[2] + v[3]);
    } else {
      V3 *x = &qx0[(size_t)kHexQ * c];
      double *w = &qw0[(size_t)kHexQ * c];
      if (!hex_rule(v, x, w)) { err = "inverted or degenerate hexahedron " + std::to_string(c); return HGKS_ERR_MESH; }
      double vol = 0.0;
      V3 m1{0, 0, 0};
      for (int q = 0; q < kHexQ; q++) { vol += w[q]; m1 = m1 + w[q] * x[q]; }
      if (!std::isfinite(vol)) { err = "degenerate hexahedron " + std::to_string(c); return HGKS_ERR_MESH; }
      vol0[c] = vol;
      cen0[c] = (1.0 / vol) * m1;
      for (int q = 0; q < kHexQ; q++) w[q] /= vol;
    }
  }
  V3 lo = cen0[0], hi = cen0[0];
  for (auto &c : cen0) {
    lo = {std::min(lo.x, c.x), std::min(lo.y, c.y), std::min(lo.z, c.z)};
    hi = {std::max(hi.x, c.x), std::max(hi.y, c.y), std::max(hi.z, c.z)};
  }
  double ext = std::max({hi.x - lo.x, hi.y - lo.y, hi.z - lo.z, 1e-300});
  std::vector<std::pair<uint64_t, int>> key(N);
  for (int c = 0; c < N; c++) {
    auto q = [&](double x, double l) { return (uint64_t)std::min(2097151.0, std::floor((x - l) / ext * 2097151.0)); };
    key[c] = {spread21(q(cen0[c].x, lo.x)) | (spread21(q(cen0[c].y, lo.y)) << 1) | (spread21(q(cen0[c].z, lo.z)) << 2), c};
  }
  std::sort(key.begin(), key.end());
  hm.N = N;
  hm.perm.resize(N);
  std::vector<int> inv(N);
  Geo g;
  g.xyz = xyz;
  g.nvc = nvc;
  g.cv.resize((size_t)nvc * N);
  g.cen.resize(N); g.vol.resize(N); g.h.resize(N);
  if (hex) { g.qx.resize((size_t)kHexQ * N); g.qw.resize((size_t)kHexQ * N); }
  for (int i = 0; i < N; i++) {
    int c = key[i].second;
    hm.perm[i] = c; inv[c] = i;
    for (int a = 0; a < nvc; a++) g.cv[(size_t)nvc * i + a] = cells[(size_t)nvc * c + a];
    g.cen[i] = cen0[c]; g.vol[i] = vol0[c]; g.h[i] = std::cbrt(vol0[c]);
    if (hex)
      for (int q = 0; q < kHexQ; q++) { g.qx[(size_t)kHexQ * i + q] = qx0[(size_t)kHexQ * c + q]; g.qw[(size_t)kHexQ * i + q] = qw0[(size_t)kHexQ * c + q]; }
  }
  // ---- faces ----
  using Key = std::array<int64_t, 4>;                // sorted face vertices, -1 padded for triangles
  auto face_cycle = [&](int i, int p, int64_t *cyc) {
    for (int j = 0; j < NFV; j++) cyc[j] = g.cv[(size_t)nvc * i + (hex ? kHexFace[p][j] : kFaceVerts[p][j])];
  };
  struct FK { Key k; int cell; int slot; };
  std::vector<FK> fk((size_t)NF * N);
  for (int i = 0; i < N; i++)
    for (int p = 0; p < NF; p++) {
      FK &f = fk[(size_t)NF * i + p];
      int64_t cyc[4] = {-1, -1, -1, -1};
      face_cycle(i, p, cyc);
      for (int j = 0; j < 4; j++) f.k[j] = cyc[j];
      std::sort(f.k.begin(), f.k.begin() + NFV);
      f.cell = i; f.slot = p;
    }
  std::sort(fk.begin(), fk.end(), [](const FK &a, const FK &b) { return a.k != b.k ? a.k < b.k : a.cell < b.cell; });
  std::vector<std::pair<Key, int>> bkeys(nb);
  for (int64_t b = 0; b < nb; b++) {
    Key k = {-1, -1, -1, -1};
    for (int j = 0; j < NFV; j++) k[j] = bface[(size_t)NFV * b + j];
    std::sort(k.begin(), k.begin() + NFV);
    bkeys[b] = {k, btag[b]};
  }
  std::sort(bkeys.begin(), bkeys.end());
  struct Face { int L, Ls, R, Rs, tag; V3 shift; };
  std::vector<Face> faces;
  faces.reserve((size_t)NF * N / 2 + 16);
  std::vector<size_t> loose;
  for (size_t a = 0; a < fk.size();) {
    size_t b = a + 1;
    while (b < fk.size() && fk[b].k == fk[a].k) b++;
    if (b - a > 2) { err = "face shared by more than two cells"; return HGKS_ERR_MESH; }
    if (b - a == 2) faces.push_back({fk[a].cell, fk[a].slot, fk[a + 1].cell, fk[a + 1].slot, 0, {0, 0, 0}});
    else {
      auto it = std::lower_bound(bkeys.begin(), bkeys.end(), std::make_pair(fk[a].k, INT32_MIN));
      if (it != bkeys.end() && it->first == fk[a].k) {
        if (it->second < 1 || it->second > 5) { err = "unknown boundary tag"; return HGKS_ERR_ARG; }
        faces.push_back({fk[a].cell, fk[a].slot, -1, -1, it->second, {0, 0, 0}});
      } else loose.push_back(a);
    }
    a = b;
  }
  if (!loose.empty()) {
    if (nps <= 0) { err = std::to_string(loose.size()) + " faces are neither shared, tagged nor periodic"; return HGKS_ERR_MESH; }
    double scale = 0.0;
    for (int s = 0; s < nps; s++) scale = std::max(scale, std::sqrt(pshift[3 * s] * pshift[3 * s] + pshift[3 * s + 1] * pshift[3 * s + 1] + pshift[3 * s + 2] * pshift[3 * s + 2]));
    std::vector<V3> fc(loose.size());
    for (size_t u = 0; u < loose.size(); u++) {
      V3 s{0, 0, 0};
      for (int j = 0; j < NFV; j++) { const double *p = xyz + 3 * fk[loose[u]].k[j]; s = s + V3{p[0], p[1], p[2]}; }
      fc[u] = (1.0 / NFV) * s;
    }
    std::vector<char> used(loose.size(), 0);
    for (size_t u = 0; u < loose.size(); u++) {
      if (used[u]) continue;
      bool found = false;
      for (size_t w = u + 1; w < loose.size() && !found; w++) {
        if (used[w]) continue;
        for (int s = 0; s < nps && !found; s++)
          for (int sg = -1; sg <= 1 && !found; sg += 2) {
            V3 sh{sg * pshift[3 * s], sg * pshift[3 * s + 1], sg * pshift[3 * s + 2]};
            V3 d = fc[u] - (fc[w] + sh);
            if (std::sqrt(dot(d, d)) < 1e-9 * scale) {
              const FK &A = fk[loose[u]], &B = fk[loose[w]];
              // x_A = x_B + sh; the left cell is the lower index
              if (A.cell <= B.cell) faces.push_back({A.cell, A.slot, B.cell, B.slot, 0, sh});
              else faces.push_back({B.cell, B.slot, A.cell, A.slot, 0, -1.0 * sh});
              used[u] = used[w] = 1;
              found = true;
            }
          }
      }
      if (!found) { err = "unmatched face without a boundary tag"; return HGKS_ERR_MESH; }
    }
  }
  std::sort(faces.begin(), faces.end(), [](const Face &a, const Face &b) { return a.L != b.L ? a.L < b.L : a.Ls < b.Ls; });
  const int F = (int)faces.size();
  hm.F = F;
  hm.fl.resize(F); hm.fr.resize(F); hm.ftag.resize(F); hm.fT.resize(9 * (size_t)F); hm.fS.resize(F); hm.fdist.resize(F);
  if (hex) hm.fw.resize((size_t)NG * F);
  hm.cnb.assign((size_t)NF * N, -1); hm.cface.assign((size_t)NF * N, -1);
  std::vector<V3> nshift((size_t)NF * N, V3{0, 0, 0});   // neighbour + shift = this cell's frame
  std::vector<V3> fgp((size_t)NG * F);
  hm.Fb = 0;
  auto vert = [&](int64_t vi) { return V3{xyz[3 * vi], xyz[3 * vi + 1], xyz[3 * vi + 2]}; };
  for (int f = 0; f < F; f++) {
    const Face &fa = faces[f];
    hm.fl[f] = fa.L; hm.fr[f] = fa.R; hm.ftag[f] = (signed char)fa.tag;
    if (fa.R < 0) hm.Fb++;
    V3 n, fcen;
    if (!hex) {
      std::array<int64_t, 3> vk;
      for (int j = 0; j < 3; j++) vk[j] = g.cv[4 * (size_t)fa.L + kFaceVerts[fa.Ls][j]];
      std::sort(vk.begin(), vk.end());
      V3 a = vert(vk[0]), b = vert(vk[1]), c = vert(vk[2]);
      V3 opp = g.vtx(fa.L, fa.Ls);
      V3 nv3 = cross(b - a, c - a);
      double len = std::sqrt(dot(nv3, nv3));
      if (dot(nv3, a - opp) < 0) nv3 = -1.0 * nv3;
      n = (1.0 / len) * nv3;
      hm.fS[f] = 0.5 * len;
      V3 verts[3] = {a, b, c};
      for (int gp = 0; gp < 3; gp++)
        fgp[3 * (size_t)f + gp] = (2.0 / 3.0) * verts[gp] + (1.0 / 6.0) * (verts[(gp + 1) % 3] + verts[(gp + 2) % 3]);
      fcen = (1.0 / 3.0) * (a + b + c);
    } else {
      int64_t cyc[4], vk[4];
      face_cycle(fa.L, fa.Ls, cyc);
      canonical_quad(cyc, vk);
      V3 a = vert(vk[0]), b = vert(vk[1]), c = vert(vk[2]), d = vert(vk[3]);
      fcen = 0.25 * (a + b + c + d);
      V3 A = 0.5 * cross(c - a, d - b);                   // vector area of the bilinear face
      double len = std::sqrt(dot(A, A));
      if (dot(A, fcen - g.cen[fa.L]) < 0) A = -1.0 * A;   // out of the left cell
      n = (1.0 / len) * A;
      hm.fS[f] = len;
      const double gl = 0.5 - 0.5 / std::sqrt(3.0), gh = 0.5 + 0.5 / std::sqrt(3.0);
      const double st[4][2] = {{gl, gl}, {gh, gl}, {gh, gh}, {gl, gh}};
      double jac[4], jsum = 0.0;
      for (int gp = 0; gp < 4; gp++) {
        const double u = st[gp][0], v = st[gp][1];
        fgp[4 * (size_t)f + gp] = ((1 - u) * (1 - v)) * a + (u * (1 - v)) * b + (u * v) * c + ((1 - u) * v) * d;
        V3 xu = (1 - v) * (b - a) + v * (c - d), xv = (1 - u) * (d - a) + u * (c - b);
        V3 cr = cross(xu, xv);
        jac[gp] = std::sqrt(dot(cr, cr));
        jsum += jac[gp];
      }
      for (int gp = 0; gp < 4; gp++) hm.fw[(size_t)gp * F + f] = jac[gp] / jsum;
    }
    // frame: t1 = n x e_a / |.|, a = argmin |n_a| w_a with w = (1, 1.001, 1.002)
    const double wgt[3] = {1.0, 1.001, 1.002};
    int ax = 0;
    for (int k = 1; k < 3; k++) if (std::fabs(comp(n, k)) * wgt[k] < std::fabs(comp(n, ax)) * wgt[ax]) ax = k;
    V3 e{ax == 0 ? 1.0 : 0.0, ax == 1 ? 1.0 : 0.0, ax == 2 ? 1.0 : 0.0};
    V3 t1 = cross(n, e);
    t1 = (1.0 / std::sqrt(dot(t1, t1))) * t1;
    V3 t2 = cross(n, t1);
    V3 rows[3] = {n, t1, t2};
    for (int r = 0; r < 3; r++)
      for (int d = 0; d < 3; d++) hm.fT[(size_t)(3 * r + d) * F + f] = comp(rows[r], d);
    hm.cface[(size_t)fa.Ls * N + fa.L] = 2 * f;
    if (fa.R >= 0) {
      hm.cnb[(size_t)fa.Ls * N + fa.L] = fa.R;
      hm.cnb[(size_t)fa.Rs * N + fa.R] = fa.L;
      hm.cface[(size_t)fa.Rs * N + fa.R] = 2 * f + 1;
      nshift[(size_t)NF * fa.L + fa.Ls] = fa.shift;
      nshift[(size_t)NF * fa.R + fa.Rs] = -1.0 * fa.shift;
      V3 d = g.cen[fa.L] - (g.cen[fa.R] + fa.shift);
      hm.fdist[f] = std::sqrt(dot(d, d));
    } else {
      hm.fdist[f] = 2.0 * std::fabs(dot(fcen - g.cen[fa.L], n));
    }
  }
  std::vector<V3> fshift(F);
  for (int f = 0; f < F; f++) fshift[f] = faces[f].shift;
  // ---- per-cell data ----
  const int BIG = hex ? HexShape::BIG : TetShape::BIG, NSUBW = hex ? HexShape::NSUBW : TetShape::NSUBW;
  const int SUBK = hex ? HexShape::SUBK : TetShape::SUBK, SLOTBITS = hex ? HexShape::SLOTBITS : TetShape::SLOTBITS;
  const int HCOLS = hex ? ShapeOf<HexShape>::HCOLS : ShapeOf<TetShape>::HCOLS;
  hm.vol = g.vol; hm.h = g.h;
  hm.m2.assign(6 * (size_t)N, 0.0);
  hm.xg.assign((size_t)NF * NG * 3 * N, 0.0);
  const bool weno = scheme_mask & 1, hweno = scheme_mask & 2;
  if (weno) {
    hm.sten.assign((size_t)BIG * N, -1);
    hm.X0.assign((size_t)9 * BIG * N, 0.0);
    hm.Xs.assign((size_t)NSUBW * 3 * SUBK * N, 0.0);
    hm.ssl.assign((size_t)NSUBW * N, 0u);
    hm.subvalid.assign(N, 0);
  }
  if (hweno) {
    hm.H0.assign((size_t)9 * HCOLS * N, 0.0);
    hm.Hm.assign((size_t)NF * 3 * 7 * N, 0.0);
  }
  std::atomic<int> fail{0};
  std::atomic<int> next{0};
  auto work = [&]() {
    std::vector<double> A, X;
    for (;;) {
      int i0 = next.fetch_add(256);
      if (i0 >= N || fail.load()) return;
      for (int i = i0; i < std::min(N, i0 + 256); i++) {
        const V3 zero{0, 0, 0};
        double own[9];
        g.avg_mono(i, i, zero, own);
        for (int t = 0; t < 6; t++) hm.m2[(size_t)t * N + i] = own[3 + t];
        for (int p = 0; p < NF; p++) {
          int f = hm.cface[(size_t)p * N + i] >> 1, side = hm.cface[(size_t)p * N + i] & 1;
          for (int gp = 0; gp < NG; gp++) {
            V3 x = fgp[(size_t)NG * f + gp];
            if (side) x = x - fshift[f];
            V3 xh = (1.0 / g.h[i]) * (x - g.cen[i]);
            for (int d = 0; d < 3; d++) hm.xg[(size_t)((p * NG + gp) * 3 + d) * N + i] = comp(xh, d);
          }
        }
        auto nb_of = [&](const Ref &r, int q, Ref &out) {
          int j = hm.cnb[(size_t)q * N + r.cell];
          if (j < 0) return false;
          out.cell = j;
          out.shift = r.shift + nshift[(size_t)NF * r.cell + q];
          return true;
        };
        auto add = [&](std::vector<Ref> &list, const Ref &r, size_t cap) {
          if (r.cell == i && same_shift(r.shift, zero)) return false;
          for (auto &e : list) if (e.cell == r.cell && same_shift(e.shift, r.shift)) return false;
          if (list.size() >= cap) return false;
          list.push_back(r);
          return true;
        };
        Ref self{i, zero};
        if (weno) {
          std::vector<Ref> big;
          std::vector<Ref> l1;
          for (int p = 0; p < NF; p++) { Ref r; if (nb_of(self, p, r) && add(big, r, BIG)) l1.push_back(r); }
          size_t s2 = big.size();
          for (auto &r1 : l1) for (int q = 0; q < NF; q++) { Ref r; if (nb_of(r1, q, r)) add(big, r, BIG); }
          size_t fs = s2, fe = big.size();
          for (int level = 3; level <= 6 && big.size() < 12 && fe > fs; level++) {
            size_t ns = big.size();
            for (size_t a = fs; a < fe && big.size() < 12; a++)
              for (int q = 0; q < NF && big.size() < 12; q++) { Ref r; if (nb_of(big[a], q, r)) add(big, r, 12); }
            fs = ns; fe = big.size();
          }
          // the quadratic fit needs cells that determine it: while it is singular
          // over the cells found (on a regular grid the 12 cells of a boundary
          // cell are), add the neighbours of every stencil cell, in stencil and
          // local-face order, up to BIG cells
          int K = 0;
          double av[9];
          for (;;) {
            K = (int)big.size();
            bool ok = false;
            if (K >= 9) {
              A.assign(K * 9, 0.0); X.assign(9 * K, 0.0);
              for (int k = 0; k < K; k++) {
                g.avg_mono(i, big[k].cell, big[k].shift, av);
                for (int d = 0; d < 9; d++) A[k * 9 + d] = av[d] - own[d];
              }
              ok = lsq_map(K, 9, A.data(), X.data());
            }
            if (ok) break;
            const size_t before = big.size();
            for (size_t a = 0; a < before && big.size() < (size_t)BIG; a++)
              for (int q = 0; q < NF && big.size() < (size_t)BIG; q++) {
                Ref r;
                if (nb_of(big[a], q, r)) add(big, r, BIG);
              }
            if (big.size() == before) { fail = K < 9 ? 1 : 2; return; }
          }
          for (int k = 0; k < K; k++) hm.sten[(size_t)k * N + i] = big[k].cell;
          for (int d = 0; d < 9; d++)
            for (int k = 0; k < K; k++) hm.X0[(size_t)(d * BIG + k) * N + i] = X[d * K + k];
          unsigned char valid = 0;
          for (int m = 0; m < NSUBW; m++) {
            std::vector<Ref> sub;
            for (int t = 0; t < 3; t++) { Ref r; if (nb_of(self, hex ? kHexTriple[m][t] : kTriple[m][t], r)) add(sub, r, 8); }
            Ref rm;
            if (!hex && nb_of(self, m, rm))
              for (int q = 0; q < 4; q++) { Ref r; if (nb_of(rm, q, r)) add(sub, r, 8); }
            int Ks = (int)sub.size();
            if (Ks < 3) continue;
            std::vector<double> As(Ks * 3), Xs(3 * Ks);
            std::vector<int> slot(Ks);
            for (int k = 0; k < Ks; k++) {
              int s = -1;
              for (int b = 0; b < K; b++) if (big[b].cell == sub[k].cell && same_shift(big[b].shift, sub[k].shift)) { s = b; break; }
              if (s < 0) { fail = 3; return; }
              slot[k] = s;
              g.avg_mono(i, sub[k].cell, sub[k].shift, av);
              for (int d = 0; d < 3; d++) As[k * 3 + d] = av[d] - own[d];
            }
            if (sv_ratio3(Ks, As.data()) < 1e-3) continue;
            if (!lsq_map(Ks, 3, As.data(), Xs.data())) continue;
            if (Ks > SUBK) { fail = 5; return; }
            valid |= (unsigned char)(1u << m);
            // the sub-stencil's cells in the order of their big-stencil slots; unused
            // entries keep slot 0 and a zero weight
            std::vector<int> ord(Ks);
            for (int k = 0; k < Ks; k++) ord[k] = k;
            std::sort(ord.begin(), ord.end(), [&](int x, int y) { return slot[x] < slot[y]; });
            unsigned packed = 0;
            for (int s = 0; s < Ks; s++) {
              packed |= (unsigned)slot[ord[s]] << (SLOTBITS * s);
              for (int j = 0; j < 3; j++) hm.Xs[(size_t)((m * 3 + j) * SUBK + s) * N + i] = Xs[j * Ks + ord[s]];
            }
            hm.ssl[(size_t)m * N + i] = packed;
          }
          hm.subvalid[i] = valid;
        }
        if (hweno) {
          // KKT system of the constrained least squares: rows of cell averages
          // (equalities, slots with a neighbour) and h-scaled gradient averages
          Ref nbr[6]; bool has[6];
          for (int p = 0; p < NF; p++) has[p] = nb_of(self, p, nbr[p]);
          int ne = 0, slot_of_eq[6];
          for (int p = 0; p < NF; p++) if (has[p]) slot_of_eq[ne++] = p;
          double Cq[6][9], Bg[21][9], av[9];
          int nls = 0;
          for (int e = 0; e < ne; e++) {
            g.avg_mono(i, nbr[slot_of_eq[e]].cell, nbr[slot_of_eq[e]].shift, av);
            for (int d = 0; d < 9; d++) Cq[e][d] = av[d] - own[d];
          }
          // gradient rows: gradient of each basis monomial at the centroid of cell k
          auto grad_rows = [&](int k, V3 s, double hk, double rowsout[3][9]) {
            V3 c = (1.0 / g.h[i]) * (g.cen[k] + s - g.cen[i]);
            double f = hk / g.h[i];
            for (int j = 0; j < 3; j++) for (int d = 0; d < 9; d++) rowsout[j][d] = 0.0;
            for (int j = 0; j < 3; j++) { rowsout[j][j] = f; rowsout[j][3 + j] = f * 2.0 * comp(c, j); }
            rowsout[0][6] = f * c.y; rowsout[0][7] = f * c.z;
            rowsout[1][6] = f * c.x; rowsout[1][8] = f * c.z;
            rowsout[2][7] = f * c.x; rowsout[2][8] = f * c.y;
          };
          double rk[3][9];
          grad_rows(i, zero, g.h[i], rk);
          for (int j = 0; j < 3; j++) { for (int d = 0; d < 9; d++) Bg[nls][d] = rk[j][d]; nls++; }
          for (int p = 0; p < NF; p++) {
            if (!has[p]) continue;
            grad_rows(nbr[p].cell, nbr[p].shift, g.h[nbr[p].cell], rk);
            for (int j = 0; j < 3; j++) { for (int d = 0; d < 9; d++) Bg[nls][d] = rk[j][d]; nls++; }
          }
          // fewer than 3 face neighbours: the quadratic system is singular, P0 keeps its linear terms
          const int nu = ne >= 3 ? 9 : 3, n = nu + ne;
          std::vector<double> K(n * n, 0.0);
          for (int a = 0; a < nu; a++)
            for (int b = 0; b < nu; b++) { double s = 0.0; for (int r = 0; r < nls; r++) s += Bg[r][a] * Bg[r][b]; K[a * n + b] = s; }
          for (int e = 0; e < ne; e++) for (int d = 0; d < nu; d++) { K[d * n + nu + e] = Cq[e][d]; K[(nu + e) * n + d] = Cq[e][d]; }
          // right-hand sides: one per data column (dQ of slot p, then G of self and slots)
          const int ncol = HCOLS;
          std::vector<double> Rhs(n * ncol, 0.0);
          for (int e = 0; e < ne; e++) Rhs[(nu + e) * ncol + slot_of_eq[e]] = 1.0;
          int row = 0;
          for (int kk = 0; kk <= NF; kk++) {
            double hk;
            if (kk == 0) hk = g.h[i];
            else { if (!has[kk - 1]) continue; hk = g.h[nbr[kk - 1].cell]; }
            for (int j = 0; j < 3; j++, row++) {
              int col = NF + 3 * kk + j;   // data G_{k,j}; the equation's right side is h_k G_{k,j}
              for (int a = 0; a < nu; a++) Rhs[a * ncol + col] += Bg[row][a] * hk;
            }
          }
          if (!lu_solve_multi(n, K, ncol, Rhs)) { fail = 4; return; }
          for (int d = 0; d < nu; d++)
            for (int col = 0; col < ncol; col++) hm.H0[(size_t)(d * ncol + col) * N + i] = Rhs[d * ncol + col];
          // sub-stencils {i, i_m}: isotropic least squares plus at most one equality, in closed form
          for (int m = 0; m < NF; m++) {
            double Mx[3][7] = {};
            double hi_ = g.h[i];
            if (has[m]) {
              double hm_ = g.h[nbr[m].cell];
              V3 dl = (1.0 / hi_) * (g.cen[nbr[m].cell] + nbr[m].shift - g.cen[i]);
              double dd = dot(dl, dl);
              double wi = hi_ * hi_ / (hi_ * hi_ + hm_ * hm_), wm = hm_ * hm_ / (hi_ * hi_ + hm_ * hm_);
              // b = btilde + dl (e - dl.btilde)/|dl|^2, btilde = h_i (w_i G_i + w_m G_m)
              for (int j = 0; j < 3; j++) {
                Mx[j][0] = comp(dl, j) / dd;
                for (int k = 0; k < 3; k++) {
                  double proj = (j == k ? 1.0 : 0.0) - comp(dl, j) * comp(dl, k) / dd;
                  Mx[j][1 + k] = proj * hi_ * wi;
                  Mx[j][4 + k] = proj * hi_ * wm;
                }
              }
            } else {
              for (int j = 0; j < 3; j++) Mx[j][1 + j] = hi_;
            }
            for (int j = 0; j < 3; j++)
              for (int col = 0; col < 7; col++) hm.Hm[(size_t)((m * 3 + j) * 7 + col) * N + i] = Mx[j][col];
          }
        }
      }
    }
  };
  unsigned nth = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  for (unsigned t = 0; t < nth; t++) pool.emplace_back(work);
  for (auto &t : pool) t.join();
  if (fail.load()) {
    const char *why[] = {"", "non-compact stencil has fewer than 9 cells", "singular least-squares stencil",
                         "sub-stencil cell outside the big stencil", "singular constrained least-squares system",
                         "sub-stencil with more cells than its slots"};
    err = why[fail.load()];
    return HGKS_ERR_MESH;
  }
  return HGKS_OK;
}

}  // namespace hgks
