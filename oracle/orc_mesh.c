/* ORACLE (test infrastructure only): mesh, geometry, stencils and the
 * least-squares / constrained least-squares fits of Sec. 3.
 *
 * Cells are tetrahedra or hexahedra (Sec. 3.1).
 * Tetrahedron: volume and centroid; face p is the triangle opposite local
 * vertex p; 3-point Gauss rule on a face.
 * Hexahedron (vertices 0-3 one quadrilateral in cyclic order, 4-7 the opposite
 * one, 4 + a joined to a): the trilinear map of the reference cube; faces 0 and 5
 * are the quadrilaterals 0123 and 4567, faces 1-4 the side quadrilaterals in
 * cyclic order around them, so that the faces meeting at one corner are
 * {0 or 5, k, k+1}, Sec. 3.1's eight sub-stencils. A face is the bilinear
 * surface through its four vertices, its area the length of its vector area
 * (c - a) x (d - b) / 2 (the vector areas of a cell's faces add up to zero), n
 * that vector's direction, and the 2 x 2 Gauss points of the bilinear map are
 * weighted by its area element there (normalised to sum 1). Volume, centroid and
 * the cell averages come from a 4 x 4 x 4 Gauss rule of the trilinear map,
 * exact for those integrands (degree <= 4 in each reference coordinate).
 *
 * Faces are matched by their sorted vertex lists; unmatched faces are boundary
 * faces (tagged by the caller) or periodic images of each other under a
 * caller-given translation; n points out of the left cell.
 *
 * Cell averages over a tetrahedron are taken with a 4-point quadrature that is
 * exact for quadratics (all integrands here are of degree <= 2). Coordinates
 * inside a fit are those of the target cell: x_hat = (x - centroid)/h with
 * h = |Omega|^(1/3); this only changes the basis in which the same polynomial
 * is written (Eq. (polys)), for conditioning. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include "orc.h"

static const double QA = 0.5854101966249685, QB = 0.1381966011250105; /* degree-2 tet rule */

typedef struct { int64_t k[4]; int64_t cell; int p; } facekey;   /* k[3] = -1 on a triangle */

static int cmp_key(const void *a, const void *b) {
  const facekey *x = (const facekey *)a, *y = (const facekey *)b;
  for (int i = 0; i < 4; i++) {
    if (x->k[i] < y->k[i]) return -1;
    if (x->k[i] > y->k[i]) return 1;
  }
  if (x->cell < y->cell) return -1;
  if (x->cell > y->cell) return 1;
  return 0;
}
static int cmp3(const int64_t *a, const int64_t *b) {   /* four entries */
  for (int i = 0; i < 4; i++) {
    if (a[i] < b[i]) return -1;
    if (a[i] > b[i]) return 1;
  }
  return 0;
}
static void sortn(int64_t *v, int n) {
  for (int i = 0; i < n; i++)
    for (int j = i + 1; j < n; j++)
      if (v[j] < v[i]) { int64_t t = v[i]; v[i] = v[j]; v[j] = t; }
}
static void cross(const double *a, const double *b, double *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

void orc_mesh_destroy(orc_mesh *m) {
  if (!m) return;
  free(m->xyz); free(m->cv); free(m->vol); free(m->cen); free(m->h); free(m->fgw);
  free(m->cface); free(m->cnb); free(m->cshift); free(m->cside);
  free(m->fl); free(m->fr); free(m->flp); free(m->frp); free(m->ftag);
  free(m->farea); free(m->fnrm); free(m->fgp); free(m->fshift); free(m->fcen);
  free(m->fit);
  free(m);
}

static const int FACEV[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
/* hexahedron: corner (a, b, c) of each local vertex, and the faces (cyclic vertex order) */
static const int HCORNER[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0}, {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
static const int HFACEV[6][4] = {{0, 1, 2, 3}, {0, 1, 5, 4}, {1, 2, 6, 5}, {2, 3, 7, 6}, {3, 0, 4, 7}, {4, 5, 6, 7}};
/* 4-point Gauss-Legendre rule on [0, 1] */
static void gauss4(double *t, double *w) {
  const double a = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0)), b = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
  const double wa = (18.0 + sqrt(30.0)) / 36.0, wb = (18.0 - sqrt(30.0)) / 36.0;
  const double x[4] = {-b, -a, a, b}, ww[4] = {wb, wa, wa, wb};
  for (int k = 0; k < 4; k++) { t[k] = 0.5 * (1.0 + x[k]); w[k] = 0.5 * ww[k]; }
}
/* trilinear map of hexahedron c at reference point r: position and Jacobian determinant */
static void hex_map(const orc_mesh *m, int64_t c, const double *r, double *x, double *detJ) {
  double J[3][3] = {{0}};
  for (int d = 0; d < 3; d++) x[d] = 0.0;
  for (int a = 0; a < 8; a++) {
    double f[3], df[3];
    for (int e = 0; e < 3; e++) { f[e] = HCORNER[a][e] ? r[e] : 1.0 - r[e]; df[e] = HCORNER[a][e] ? 1.0 : -1.0; }
    const double *v = m->xyz + 3 * m->cv[8 * c + a];
    const double N = f[0] * f[1] * f[2];
    const double dN[3] = {df[0] * f[1] * f[2], f[0] * df[1] * f[2], f[0] * f[1] * df[2]};
    for (int d = 0; d < 3; d++) { x[d] += N * v[d]; for (int e = 0; e < 3; e++) J[d][e] += dN[e] * v[d]; }
  }
  *detJ = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
          J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}
/* raw 4 x 4 x 4 rule of a hexahedron: points and weights w detJ (their sum is the volume) */
static int hex_quad_raw(const orc_mesh *m, int64_t c, double (*xq)[3], double *wq) {
  double t[4], w[4];
  gauss4(t, w);
  int q = 0;
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++)
      for (int k = 0; k < 4; k++, q++) {
        const double r[3] = {t[i], t[j], t[k]};
        double dj;
        hex_map(m, c, r, xq[q], &dj);
        wq[q] = w[i] * w[j] * w[k] * dj;
      }
  return q;
}

int orc_cell_quad(const orc_mesh *m, int64_t k, double (*xq)[3], double *wq) {
  if (m->nvc == 4) {
    for (int q = 0; q < 4; q++) {
      for (int d = 0; d < 3; d++) {
        double x = 0.0;
        for (int a = 0; a < 4; a++) x += (a == q ? QA : QB) * m->xyz[3 * m->cv[4 * k + a] + d];
        xq[q][d] = x;
      }
      wq[q] = 0.25;
    }
    return 4;
  }
  int n = hex_quad_raw(m, k, xq, wq);
  for (int q = 0; q < n; q++) wq[q] /= m->vol[k];
  return n;
}

/* the face's vertices in a canonical cyclic order (from its smallest vertex,
 * towards the smaller of that vertex's two neighbours): both cells that share a
 * quadrilateral derive the same bilinear map and Gauss points from it */
static void canonical_quad(const int64_t *cyc, int64_t *out) {
  int s = 0;
  for (int k = 1; k < 4; k++) if (cyc[k] < cyc[s]) s = k;
  int dir = cyc[(s + 1) % 4] < cyc[(s + 3) % 4] ? 1 : 3;
  for (int k = 0; k < 4; k++) out[k] = cyc[(s + dir * k) % 4];
}

orc_mesh *orc_mesh_create(const double *xyz, int64_t nv, const int64_t *tet, int64_t nc,
                          const int64_t *bface, const int32_t *btag, int64_t nb,
                          const double *pshift, int32_t npshift, char *err, int errlen) {
  return orc_mesh_create_cells(xyz, nv, tet, 4, nc, bface, btag, nb, pshift, npshift, err, errlen);
}

orc_mesh *orc_mesh_create_cells(const double *xyz, int64_t nv, const int64_t *cells, int32_t nvc, int64_t nc,
                                const int64_t *bface, const int32_t *btag, int64_t nb,
                                const double *pshift, int32_t npshift, char *err, int errlen) {
  if (nvc != 4 && nvc != 8) { snprintf(err, errlen, "cells must have 4 or 8 vertices"); return NULL; }
  const int hex = nvc == 8, nfc = hex ? 6 : 4, nfv = hex ? 4 : 3, ngp = hex ? 4 : 3;
  orc_mesh *m = (orc_mesh *)calloc(1, sizeof(orc_mesh));
  m->nv = nv; m->nc = nc; m->nvc = nvc; m->nfc = nfc; m->ngp = ngp;
  m->xyz = (double *)malloc(sizeof(double) * 3 * (nv > 0 ? nv : 1));
  memcpy(m->xyz, xyz, sizeof(double) * 3 * nv);
  m->cv = (int64_t *)malloc(sizeof(int64_t) * nvc * (nc > 0 ? nc : 1));
  memcpy(m->cv, cells, sizeof(int64_t) * nvc * nc);
  m->vol = (double *)malloc(sizeof(double) * (nc + 1));
  m->cen = (double *)malloc(sizeof(double) * 3 * (nc + 1));
  m->h = (double *)malloc(sizeof(double) * (nc + 1));
  m->cface = (int64_t *)malloc(sizeof(int64_t) * nfc * (nc + 1));
  m->cnb = (int64_t *)malloc(sizeof(int64_t) * nfc * (nc + 1));
  m->cshift = (double *)calloc(3 * nfc * (nc + 1), sizeof(double));
  m->cside = (int32_t *)malloc(sizeof(int32_t) * nfc * (nc + 1));
  m->fit = (orc_fit *)calloc(nc + 1, sizeof(orc_fit));
  for (int64_t i = 0; i < nc; i++)
    for (int a = 0; a < nvc; a++)
      if (cells[nvc * i + a] < 0 || cells[nvc * i + a] >= nv) { snprintf(err, errlen, "vertex index out of range"); orc_mesh_destroy(m); return NULL; }
  for (int64_t i = 0; i < nc && !hex; i++) {
    const double *v[4];
    for (int a = 0; a < 4; a++) v[a] = xyz + 3 * cells[4 * i + a];
    double e1[3], e2[3], e3[3], c[3];
    for (int d = 0; d < 3; d++) { e1[d] = v[1][d] - v[0][d]; e2[d] = v[2][d] - v[0][d]; e3[d] = v[3][d] - v[0][d]; }
    cross(e2, e3, c);
    double vol = fabs(e1[0] * c[0] + e1[1] * c[1] + e1[2] * c[2]) / 6.0;
    if (!(vol > 0.0)) { snprintf(err, errlen, "degenerate tetrahedron %lld", (long long)i); orc_mesh_destroy(m); return NULL; }
    m->vol[i] = vol;
    m->h[i] = cbrt(vol);
    for (int d = 0; d < 3; d++) m->cen[3 * i + d] = 0.25 * (v[0][d] + v[1][d] + v[2][d] + v[3][d]);
  }
  for (int64_t i = 0; i < nc && hex; i++) {
    double xq[64][3], wq[64], vol = 0.0, cx[3] = {0, 0, 0};
    int n = hex_quad_raw(m, i, xq, wq);
    for (int q = 0; q < n; q++) {
      if (!(wq[q] > 0.0)) { snprintf(err, errlen, "inverted or degenerate hexahedron %lld", (long long)i); orc_mesh_destroy(m); return NULL; }
      vol += wq[q];
      for (int d = 0; d < 3; d++) cx[d] += wq[q] * xq[q][d];
    }
    m->vol[i] = vol;
    m->h[i] = cbrt(vol);
    for (int d = 0; d < 3; d++) m->cen[3 * i + d] = cx[d] / vol;
  }
  /* face table */
  facekey *fk = (facekey *)malloc(sizeof(facekey) * (nfc * nc + 1));
  for (int64_t i = 0; i < nc; i++)
    for (int p = 0; p < nfc; p++) {
      facekey *k = fk + nfc * i + p;
      for (int j = 0; j < nfv; j++) k->k[j] = cells[nvc * i + (hex ? HFACEV[p][j] : FACEV[p][j])];
      if (!hex) k->k[3] = -1;
      sortn(k->k, nfv);
      k->cell = i; k->p = p;
    }
  qsort(fk, nfc * nc, sizeof(facekey), cmp_key);
  int64_t *bkeys = (int64_t *)malloc(sizeof(int64_t) * 4 * (nb + 1));
  int64_t *border = (int64_t *)malloc(sizeof(int64_t) * (nb + 1));
  for (int64_t b = 0; b < nb; b++) {
    for (int j = 0; j < nfv; j++) bkeys[4 * b + j] = bface[nfv * b + j];
    if (!hex) bkeys[4 * b + 3] = -1;
    sortn(bkeys + 4 * b, nfv);
    border[b] = b;
  }
  /* insertion-free lookup: linear search list sorted by key (simple qsort on index) */
  for (int64_t a = 1; a < nb; a++) { /* insertion sort of border by key; nb is small in tests */
    int64_t x = border[a], b = a - 1;
    while (b >= 0 && cmp3(bkeys + 4 * border[b], bkeys + 4 * x) > 0) { border[b + 1] = border[b]; b--; }
    border[b + 1] = x;
  }
  int64_t maxf = nfc * nc + 1;
  m->fl = (int64_t *)malloc(sizeof(int64_t) * maxf); m->fr = (int64_t *)malloc(sizeof(int64_t) * maxf);
  m->flp = (int32_t *)malloc(sizeof(int32_t) * maxf); m->frp = (int32_t *)malloc(sizeof(int32_t) * maxf);
  m->ftag = (int32_t *)malloc(sizeof(int32_t) * maxf);
  m->fshift = (double *)calloc(3 * maxf, sizeof(double));
  int64_t nf = 0;
  int64_t *unm = (int64_t *)malloc(sizeof(int64_t) * maxf);  /* indices into fk of unmatched faces */
  int64_t nunm = 0;
  for (int64_t a = 0; a < nfc * nc;) {
    int64_t b = a + 1;
    while (b < nfc * nc && cmp3(fk[b].k, fk[a].k) == 0) b++;
    if (b - a > 2) { snprintf(err, errlen, "face shared by more than two cells"); goto fail; }
    if (b - a == 2) {
      m->fl[nf] = fk[a].cell; m->flp[nf] = fk[a].p; m->fr[nf] = fk[a + 1].cell; m->frp[nf] = fk[a + 1].p;
      m->ftag[nf] = 0; nf++;
    } else {
      /* boundary face? binary search in the tagged list */
      int64_t lo = 0, hi = nb - 1, found = -1;
      while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        int c = cmp3(bkeys + 4 * border[mid], fk[a].k);
        if (c == 0) { found = border[mid]; break; }
        if (c < 0) lo = mid + 1; else hi = mid - 1;
      }
      if (found >= 0) {
        if (btag[found] <= 0) { snprintf(err, errlen, "boundary tag must be positive"); goto fail; }
        m->fl[nf] = fk[a].cell; m->flp[nf] = fk[a].p; m->fr[nf] = -1; m->frp[nf] = -1;
        m->ftag[nf] = btag[found]; nf++;
      } else {
        unm[nunm++] = a;
      }
    }
    a = b;
  }
  /* periodic pairing of the remaining faces by translation of their centroids */
  if (nunm > 0) {
    if (npshift <= 0) { snprintf(err, errlen, "%lld faces are neither shared, tagged nor periodic", (long long)nunm); goto fail; }
    double *uc = (double *)malloc(sizeof(double) * 3 * nunm);
    char *used = (char *)calloc(nunm, 1);
    double scale = 0.0;
    for (int s = 0; s < npshift; s++) scale = fmax(scale, sqrt(pshift[3 * s] * pshift[3 * s] + pshift[3 * s + 1] * pshift[3 * s + 1] + pshift[3 * s + 2] * pshift[3 * s + 2]));
    for (int64_t u = 0; u < nunm; u++)
      for (int d = 0; d < 3; d++) {
        double sum = 0.0;
        for (int j = 0; j < nfv; j++) sum += xyz[3 * fk[unm[u]].k[j] + d];
        uc[3 * u + d] = sum / nfv;
      }
    for (int64_t u = 0; u < nunm; u++) {
      if (used[u]) continue;
      int64_t match = -1; double sh[3] = {0, 0, 0};
      for (int64_t w = u + 1; w < nunm && match < 0; w++) {
        if (used[w]) continue;
        for (int s = 0; s < npshift && match < 0; s++)
          for (int sg = -1; sg <= 1; sg += 2) {
            double dd = 0.0;
            for (int d = 0; d < 3; d++) { double t = uc[3 * u + d] - (uc[3 * w + d] + sg * pshift[3 * s + d]); dd += t * t; }
            if (sqrt(dd) < 1e-9 * scale) { match = w; for (int d = 0; d < 3; d++) sh[d] = sg * pshift[3 * s + d]; break; }
          }
      }
      if (match < 0) { free(uc); free(used); snprintf(err, errlen, "unmatched face without boundary tag"); goto fail; }
      used[u] = used[match] = 1;
      const facekey *A = fk + unm[u], *B = fk + unm[match];
      m->fl[nf] = A->cell; m->flp[nf] = A->p; m->fr[nf] = B->cell; m->frp[nf] = B->p; m->ftag[nf] = 0;
      for (int d = 0; d < 3; d++) m->fshift[3 * nf + d] = sh[d];   /* x_A = x_B + sh */
      nf++;
    }
    free(uc); free(used);
  }
  m->nf = nf;
  m->farea = (double *)malloc(sizeof(double) * (nf + 1));
  m->fnrm = (double *)malloc(sizeof(double) * 3 * (nf + 1));
  m->fgp = (double *)malloc(sizeof(double) * 3 * ngp * (nf + 1));
  m->fgw = (double *)malloc(sizeof(double) * ngp * (nf + 1));
  m->fcen = (double *)malloc(sizeof(double) * 3 * (nf + 1));
  for (int64_t i = 0; i < nfc * nc; i++) m->cnb[i] = -1;
  for (int64_t f = 0; f < nf; f++) {
    int64_t L = m->fl[f]; int p = m->flp[f];
    if (!hex) {
      int64_t vk[4];
      for (int j = 0; j < 3; j++) vk[j] = cells[4 * L + FACEV[p][j]];
      sortn(vk, 3);
      const double *a = xyz + 3 * vk[0], *b = xyz + 3 * vk[1], *c = xyz + 3 * vk[2], *o = xyz + 3 * cells[4 * L + p];
      double e1[3], e2[3], n[3];
      for (int d = 0; d < 3; d++) { e1[d] = b[d] - a[d]; e2[d] = c[d] - a[d]; }
      cross(e1, e2, n);
      double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      double out = (a[0] - o[0]) * n[0] + (a[1] - o[1]) * n[1] + (a[2] - o[2]) * n[2];
      double sg = out > 0 ? 1.0 : -1.0;
      m->farea[f] = 0.5 * nn;
      for (int d = 0; d < 3; d++) m->fnrm[3 * f + d] = sg * n[d] / nn;
      const double *vv[3] = {a, b, c};
      for (int g = 0; g < 3; g++) {          /* 3-point rule, barycentric (2/3,1/6,1/6), weights 1/3 */
        for (int d = 0; d < 3; d++)
          m->fgp[9 * f + 3 * g + d] = (2.0 / 3.0) * vv[g][d] + (1.0 / 6.0) * (vv[(g + 1) % 3][d] + vv[(g + 2) % 3][d]);
        m->fgw[3 * f + g] = 1.0 / 3.0;
      }
      for (int d = 0; d < 3; d++) m->fcen[3 * f + d] = (a[d] + b[d] + c[d]) / 3.0;
    } else {
      int64_t cyc[4], vk[4];
      for (int j = 0; j < 4; j++) cyc[j] = cells[8 * L + HFACEV[p][j]];
      canonical_quad(cyc, vk);
      const double *a = xyz + 3 * vk[0], *b = xyz + 3 * vk[1], *c = xyz + 3 * vk[2], *e = xyz + 3 * vk[3];
      double d1[3], d2[3], n[3], fc[3];
      for (int d = 0; d < 3; d++) { d1[d] = c[d] - a[d]; d2[d] = e[d] - b[d]; fc[d] = 0.25 * (a[d] + b[d] + c[d] + e[d]); }
      cross(d1, d2, n);
      double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      double out = 0.0;
      for (int d = 0; d < 3; d++) out += (fc[d] - m->cen[3 * L + d]) * n[d];
      double sg = out > 0 ? 1.0 : -1.0;
      m->farea[f] = 0.5 * nn;
      for (int d = 0; d < 3; d++) { m->fnrm[3 * f + d] = sg * n[d] / nn; m->fcen[3 * f + d] = fc[d]; }
      /* 2 x 2 Gauss points of x(s, t) = (1-s)(1-t) a + s(1-t) b + s t c + (1-s) t e */
      const double gl = 0.5 - 0.5 / sqrt(3.0), gh = 0.5 + 0.5 / sqrt(3.0);
      const double st[4][2] = {{gl, gl}, {gh, gl}, {gh, gh}, {gl, gh}};
      double jac[4], jsum = 0.0;
      for (int g = 0; g < 4; g++) {
        const double s_ = st[g][0], t_ = st[g][1];
        double xs[3], xt[3], cr[3];
        for (int d = 0; d < 3; d++) {
          m->fgp[12 * f + 3 * g + d] = (1 - s_) * (1 - t_) * a[d] + s_ * (1 - t_) * b[d] + s_ * t_ * c[d] + (1 - s_) * t_ * e[d];
          xs[d] = (1 - t_) * (b[d] - a[d]) + t_ * (c[d] - e[d]);
          xt[d] = (1 - s_) * (e[d] - a[d]) + s_ * (c[d] - b[d]);
        }
        cross(xs, xt, cr);
        jac[g] = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        jsum += jac[g];
      }
      for (int g = 0; g < 4; g++) m->fgw[4 * f + g] = jac[g] / jsum;
    }
    m->cface[nfc * L + p] = f; m->cnb[nfc * L + p] = m->fr[f]; m->cside[nfc * L + p] = 0;
    if (m->fr[f] >= 0) {
      int64_t R = m->fr[f]; int q = m->frp[f];
      m->cface[nfc * R + q] = f; m->cnb[nfc * R + q] = L; m->cside[nfc * R + q] = 1;
      for (int d = 0; d < 3; d++) {
        m->cshift[3 * nfc * L + 3 * p + d] = m->fshift[3 * f + d];   /* right cell + shift -> left frame */
        m->cshift[3 * nfc * R + 3 * q + d] = -m->fshift[3 * f + d];
      }
    }
  }
  free(fk); free(bkeys); free(border); free(unm);
  return m;
fail:
  free(fk); free(bkeys); free(border); free(unm);
  orc_mesh_destroy(m);
  return NULL;
}

/* ------------------------------------------------------------------------- */
/* cell averages in the scaled frame of a target cell                        */
/* ------------------------------------------------------------------------- */

/* quadrature points of cell k (translated by shift) in the scaled frame of cell i */
static int quad_points(const orc_mesh *m, int64_t i, int64_t k, const double *shift, double xq[64][3], double *wq) {
  int n = orc_cell_quad(m, k, xq, wq);
  for (int q = 0; q < n; q++)
    for (int d = 0; d < 3; d++) xq[q][d] = (xq[q][d] + shift[d] - m->cen[3 * i + d]) / m->h[i];
  return n;
}
/* monomials of the basis of Eq. (polys): x, y, z, x^2, y^2, z^2, xy, xz, yz */
static void monomials(const double *x, double *mo) {
  mo[0] = x[0]; mo[1] = x[1]; mo[2] = x[2];
  mo[3] = x[0] * x[0]; mo[4] = x[1] * x[1]; mo[5] = x[2] * x[2];
  mo[6] = x[0] * x[1]; mo[7] = x[0] * x[2]; mo[8] = x[1] * x[2];
}
/* derivative d/dx_hat_j of the monomials */
static void dmonomials(const double *x, int j, double *dm) {
  for (int d = 0; d < 9; d++) dm[d] = 0.0;
  dm[j] = 1.0;
  dm[3 + j] = 2.0 * x[j];
  if (j == 0) { dm[6] = x[1]; dm[7] = x[2]; }
  if (j == 1) { dm[6] = x[0]; dm[8] = x[2]; }
  if (j == 2) { dm[7] = x[0]; dm[8] = x[1]; }
}
/* average over cell k of the monomials, in cell i's frame */
static void avg_monomials(const orc_mesh *m, int64_t i, int64_t k, const double *shift, double *avg) {
  double xq[64][3], wq[64], mo[9];
  int n = quad_points(m, i, k, shift, xq, wq);
  for (int d = 0; d < 9; d++) avg[d] = 0.0;
  for (int q = 0; q < n; q++) { monomials(xq[q], mo); for (int d = 0; d < 9; d++) avg[d] += wq[q] * mo[d]; }
}
static void avg_dmonomials(const orc_mesh *m, int64_t i, int64_t k, const double *shift, int j, double *avg) {
  double xq[64][3], wq[64], dm[9];
  int n = quad_points(m, i, k, shift, xq, wq);
  for (int d = 0; d < 9; d++) avg[d] = 0.0;
  for (int q = 0; q < n; q++) { dmonomials(xq[q], j, dm); for (int d = 0; d < 9; d++) avg[d] += wq[q] * dm[d]; }
}

/* ------------------------------------------------------------------------- */
/* stencils (Sec. 3.1)                                                       */
/* ------------------------------------------------------------------------- */
static int same_ref(const orc_sref *a, int64_t cell, const double *s) {
  return a->cell == cell && fabs(a->shift[0] - s[0]) < 1e-9 && fabs(a->shift[1] - s[1]) < 1e-9 && fabs(a->shift[2] - s[2]) < 1e-9;
}
static int add_ref(orc_sref *list, int *n, int cap, int64_t target, int64_t cell, const double *s) {
  if (cell < 0) return 0;
  if (cell == target && fabs(s[0]) < 1e-9 && fabs(s[1]) < 1e-9 && fabs(s[2]) < 1e-9) return 0;
  for (int a = 0; a < *n; a++) if (same_ref(list + a, cell, s)) return 0;
  if (*n >= cap) return 0;
  list[*n].cell = cell; for (int d = 0; d < 3; d++) list[*n].shift[d] = s[d];
  (*n)++;
  return 1;
}
/* neighbour of stencil entry r across its local face q */
static int64_t nb_of(const orc_mesh *m, const orc_sref *r, int q, double *s) {
  int64_t j = m->cnb[m->nfc * r->cell + q];
  for (int d = 0; d < 3; d++) s[d] = r->shift[d] + m->cshift[3 * m->nfc * r->cell + 3 * q + d];
  return j;
}

/* sub-stencil triples of face neighbours, Sec. 3.1 (faces numbered from 0) */
static const int TRIPLE[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {2, 0, 3}};
/* hexahedron: the three faces that meet at each of the eight corners, one of the
 * opposite faces 0 and 5 with two consecutive side faces (Sec. 3.1's
 * S_{i_1} ... S_{i_8} with the faces numbered from 0) */
static const int HTRIPLE[8][3] = {{0, 1, 2}, {0, 2, 3}, {0, 3, 4}, {0, 4, 1}, {5, 1, 2}, {5, 2, 3}, {5, 3, 4}, {5, 4, 1}};

int orc_fit_cell(orc_mesh *m, int64_t i, int scheme) {
  orc_fit *F = m->fit + i;
  const int nfc = m->nfc, hex = m->nvc == 8;
  const double zero[3] = {0, 0, 0};
  orc_sref self; self.cell = i; self.shift[0] = self.shift[1] = self.shift[2] = 0.0;
  double avg_i[9];
  avg_monomials(m, i, i, zero, avg_i);
  if (scheme == 0 && !F->ready_weno) {
    /* big stencil: face neighbours, then their neighbours; a third level only
     * when fewer than 12 cells were found (boundary cells) */
    F->n_big = 0;
    orc_sref l1[ORC_MAXF]; int n1 = 0;
    for (int p = 0; p < nfc; p++) {
      double s[3]; int64_t j = nb_of(m, &self, p, s);
      if (add_ref(F->big, &F->n_big, ORC_MAXSTEN, i, j, s)) l1[n1++] = F->big[F->n_big - 1];
    }
    int start2 = F->n_big;
    for (int a = 0; a < n1; a++)
      for (int q = 0; q < nfc; q++) { double s[3]; int64_t k = nb_of(m, l1 + a, q, s); add_ref(F->big, &F->n_big, ORC_MAXSTEN, i, k, s); }
    /* further levels, ring by ring, only while fewer than 12 cells were found */
    int fs = start2, fe = F->n_big;
    for (int level = 3; level <= 6 && F->n_big < 12 && fe > fs; level++) {
      int ns = F->n_big;
      for (int a = fs; a < fe && F->n_big < 12; a++)
        for (int q = 0; q < nfc && F->n_big < 12; q++) { double s[3]; int64_t k = nb_of(m, F->big + a, q, s); add_ref(F->big, &F->n_big, 12, i, k, s); }
      fs = ns; fe = F->n_big;
    }
    /* the quadratic fit needs cells that determine it: while it is singular
     * over the cells found (on a regular grid the 12 cells of a boundary cell
     * are), add the neighbours of every stencil cell, in stencil and local-face
     * order, up to 16 cells around a tetrahedron or 24 around a hexahedron */
    const int cap = hex ? 24 : 16;
    double A[ORC_MAXSTEN * 9], av[9], X[9 * ORC_MAXSTEN];
    for (;;) {
      int ok = 0;
      if (F->n_big >= 9) {
        for (int r = 0; r < F->n_big; r++) {
          avg_monomials(m, i, F->big[r].cell, F->big[r].shift, av);
          for (int d = 0; d < 9; d++) A[r * 9 + d] = av[d] - avg_i[d];
        }
        ok = orc_lsq_pinv(F->n_big, 9, A, X) == 0;
      }
      if (ok) break;
      const int before = F->n_big;
      for (int a = 0; a < before && F->n_big < cap; a++)
        for (int q = 0; q < nfc && F->n_big < cap; q++) { double s[3]; int64_t k = nb_of(m, F->big + a, q, s); add_ref(F->big, &F->n_big, cap, i, k, s); }
      if (F->n_big == before) return before < 9 ? -1 : -2;
    }
    memset(F->X0, 0, sizeof(F->X0));
    for (int d = 0; d < 9; d++) for (int r = 0; r < F->n_big; r++) F->X0[d][r] = X[d * F->n_big + r];
    /* sub-stencils: tetrahedron, three face neighbours plus the neighbours of
     * one of them; hexahedron, the three face neighbours across one corner */
    const int nsub = hex ? 8 : 4;
    for (int mm = 0; mm < nsub; mm++) {
      F->n_sub[mm] = 0;
      for (int t = 0; t < 3; t++) {
        double s[3]; int64_t j = nb_of(m, &self, hex ? HTRIPLE[mm][t] : TRIPLE[mm][t], s);
        add_ref(F->sub[mm], &F->n_sub[mm], ORC_MAXSUB, i, j, s);
      }
      double s0[3]; int64_t jm = hex ? -1 : nb_of(m, &self, mm, s0);
      if (jm >= 0) {
        orc_sref rm; rm.cell = jm; for (int d = 0; d < 3; d++) rm.shift[d] = s0[d];
        for (int q = 0; q < 4; q++) { double s[3]; int64_t k = nb_of(m, &rm, q, s); add_ref(F->sub[mm], &F->n_sub[mm], ORC_MAXSUB, i, k, s); }
      }
      /* a sub-stencil is kept if it has at least 3 cells whose centroids are not
       * (nearly) coplanar with the target's: sigma_min/sigma_max >= 1e-3 */
      F->sub_valid[mm] = F->n_sub[mm] >= 3;
      memset(F->Xm[mm], 0, sizeof(F->Xm[mm]));
      if (F->sub_valid[mm]) {
        double As[ORC_MAXSUB * 3], Xs[3 * ORC_MAXSUB];
        for (int r = 0; r < F->n_sub[mm]; r++) {
          avg_monomials(m, i, F->sub[mm][r].cell, F->sub[mm][r].shift, av);
          for (int d = 0; d < 3; d++) As[r * 3 + d] = av[d] - avg_i[d];
        }
        if (orc_sv_ratio(F->n_sub[mm], 3, As) < 1e-3) F->sub_valid[mm] = 0;
        else if (orc_lsq_pinv(F->n_sub[mm], 3, As, Xs)) F->sub_valid[mm] = 0;
        else for (int d = 0; d < 3; d++) for (int r = 0; r < F->n_sub[mm]; r++) F->Xm[mm][d][r] = Xs[d * F->n_sub[mm] + r];
      }
    }
    for (int mm = nsub; mm < ORC_NSUB; mm++) { F->n_sub[mm] = 0; F->sub_valid[mm] = 0; }
    F->ready_weno = 1;
  }
  if (scheme == 1 && !F->ready_hweno) {
    /* compact: the target and its face neighbours, Eq. (compact-big-1) solved by
     * constrained least squares: cell averages exact, h-scaled gradients in the
     * least-squares sense */
    F->n_nb = 0;
    for (int p = 0; p < nfc; p++) {
      double s[3]; int64_t j = nb_of(m, &self, p, s);
      if (j >= 0) { F->nb[F->n_nb].cell = j; for (int d = 0; d < 3; d++) F->nb[F->n_nb].shift[d] = s[d]; F->nb_slot[F->n_nb] = p; F->n_nb++; }
    }
    /* with fewer than 3 face neighbours (an edge of the domain) the quadratic
     * system is singular: P0 keeps its linear terms only (nu = 3 unknowns) */
    int ne = F->n_nb, nls = 3 * (1 + F->n_nb), nu = ne >= 3 ? 9 : 3, n = nu + ne;
    double C[ORC_MAXF][9], B[3 * (1 + ORC_MAXF)][9], av[9];
    for (int r = 0; r < ne; r++) {
      avg_monomials(m, i, F->nb[r].cell, F->nb[r].shift, av);
      for (int d = 0; d < 9; d++) C[r][d] = av[d] - avg_i[d];
    }
    for (int k = 0; k <= ne; k++) {
      const orc_sref *rk = k == 0 ? &self : &F->nb[k - 1];
      double hk = m->h[rk->cell];
      for (int j = 0; j < 3; j++) {
        avg_dmonomials(m, i, rk->cell, rk->shift, j, av);
        for (int d = 0; d < 9; d++) B[3 * k + j][d] = (hk / m->h[i]) * av[d];
      }
    }
    double K[(9 + ORC_MAXF) * (9 + ORC_MAXF)];
    memset(K, 0, sizeof(K));
    for (int a = 0; a < nu; a++)
      for (int b = 0; b < nu; b++) { double s = 0; for (int r = 0; r < nls; r++) s += B[r][a] * B[r][b]; K[a * n + b] = s; }
    for (int r = 0; r < ne; r++) for (int d = 0; d < nu; d++) { K[d * n + nu + r] = C[r][d]; K[(nu + r) * n + d] = C[r][d]; }
    memset(F->H0, 0, sizeof(F->H0));
    /* the map from data to coefficients, one data unit vector at a time */
    for (int col = 0; col < nfc + 3 * (1 + nfc); col++) {
      double rhs[9 + ORC_MAXF] = {0}, sol[9 + ORC_MAXF];
      if (col < nfc) {
        if (col >= ne) continue;
        rhs[nu + col] = 1.0;
      } else {
        int k = (col - nfc) / 3, j = (col - nfc) % 3;
        if (k > ne) continue;
        const orc_sref *rk = k == 0 ? &self : &F->nb[k - 1];
        double dval = m->h[rk->cell];        /* d_row = h_k * G_kj */
        for (int a = 0; a < nu; a++) rhs[a] = B[3 * k + j][a] * dval;
      }
      if (orc_lu_solve(n, K, rhs, sol)) return -3;
      for (int d = 0; d < nu; d++) F->H0[d][col] = sol[d];
    }
    /* compact sub-stencils {target, one face neighbour}, Eq. (compact-big-2) */
    for (int mm = 0; mm < nfc; mm++) {
      memset(F->Hm[mm], 0, sizeof(F->Hm[mm]));
      double s[3]; int64_t jm = nb_of(m, &self, mm, s);
      F->hsub_has_nb[mm] = jm >= 0;
      int ne2 = jm >= 0 ? 1 : 0, n2 = 3 + ne2;
      double Cm[3] = {0, 0, 0};
      if (jm >= 0) { avg_monomials(m, i, jm, s, av); for (int d = 0; d < 3; d++) Cm[d] = av[d] - avg_i[d]; }
      double hk[2] = {m->h[i], jm >= 0 ? m->h[jm] : 0.0};
      double K2[16];
      memset(K2, 0, sizeof(K2));
      for (int a = 0; a < 3; a++) {
        double s2 = 0.0;
        for (int k = 0; k < 1 + ne2; k++) s2 += (hk[k] / m->h[i]) * (hk[k] / m->h[i]);
        K2[a * n2 + a] = s2;
      }
      if (ne2) for (int d = 0; d < 3; d++) { K2[d * n2 + 3] = Cm[d]; K2[3 * n2 + d] = Cm[d]; }
      for (int col = 0; col < 7; col++) {
        double rhs[4] = {0, 0, 0, 0}, sol[4];
        if (col == 0) { if (!ne2) continue; rhs[3] = 1.0; }
        else {
          int k = (col - 1) / 3, j = (col - 1) % 3;
          if (k >= 1 + ne2) continue;
          rhs[j] = (hk[k] / m->h[i]) * hk[k];
        }
        if (orc_lu_solve(n2, K2, rhs, sol)) return -4;
        for (int d = 0; d < 3; d++) F->Hm[mm][d][col] = sol[d];
      }
    }
    F->ready_hweno = 1;
  }
  return 0;
}

/* The stencils of cell i (for the tests): which = -1 the non-compact big
 * stencil, 0 .. 7 non-compact sub-stencil `which`; the cells go to out, *valid
 * gets the sub-stencil's flag; returns the number of cells, < 0 on error. */
int orc_stencil(orc_mesh *m, int64_t i, int which, int64_t *out, int *valid) {
  if (i < 0 || i >= m->nc || which < -1 || which >= ORC_NSUB) return -1;
  if (orc_fit_cell(m, i, 0)) return -2;
  const orc_fit *F = m->fit + i;
  if (which < 0) {
    for (int r = 0; r < F->n_big; r++) out[r] = F->big[r].cell;
    if (valid) *valid = 1;
    return F->n_big;
  }
  for (int r = 0; r < F->n_sub[which]; r++) out[r] = F->sub[which][r].cell;
  if (valid) *valid = F->sub_valid[which];
  return F->n_sub[which];
}
