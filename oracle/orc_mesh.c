/* ORACLE (test infrastructure only): mesh, geometry, stencils and the
 * least-squares / constrained least-squares fits of Sec. 3.
 *
 * Geometry: tetrahedron volume and centroid; face p is the triangle opposite
 * local vertex p, with its outward normal; faces are matched by their sorted
 * vertex triples; unmatched faces are boundary faces (tagged by the caller) or
 * periodic images of each other under a caller-given translation.
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

typedef struct { int64_t k[3]; int64_t cell; int p; } facekey;

static int cmp_key(const void *a, const void *b) {
  const facekey *x = (const facekey *)a, *y = (const facekey *)b;
  for (int i = 0; i < 3; i++) {
    if (x->k[i] < y->k[i]) return -1;
    if (x->k[i] > y->k[i]) return 1;
  }
  if (x->cell < y->cell) return -1;
  if (x->cell > y->cell) return 1;
  return 0;
}
static int cmp3(const int64_t *a, const int64_t *b) {
  for (int i = 0; i < 3; i++) {
    if (a[i] < b[i]) return -1;
    if (a[i] > b[i]) return 1;
  }
  return 0;
}
static void sort3(int64_t *v) {
  for (int i = 0; i < 3; i++)
    for (int j = i + 1; j < 3; j++)
      if (v[j] < v[i]) { int64_t t = v[i]; v[i] = v[j]; v[j] = t; }
}
static void cross(const double *a, const double *b, double *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

void orc_mesh_destroy(orc_mesh *m) {
  if (!m) return;
  free(m->xyz); free(m->tet); free(m->vol); free(m->cen); free(m->h);
  free(m->cface); free(m->cnb); free(m->cshift); free(m->cside);
  free(m->fl); free(m->fr); free(m->flp); free(m->frp); free(m->ftag);
  free(m->farea); free(m->fnrm); free(m->fgp); free(m->fshift); free(m->fcen);
  free(m->fit);
  free(m);
}

static const int FACEV[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

orc_mesh *orc_mesh_create(const double *xyz, int64_t nv, const int64_t *tet, int64_t nc,
                          const int64_t *bface, const int32_t *btag, int64_t nb,
                          const double *pshift, int32_t npshift, char *err, int errlen) {
  orc_mesh *m = (orc_mesh *)calloc(1, sizeof(orc_mesh));
  m->nv = nv; m->nc = nc;
  m->xyz = (double *)malloc(sizeof(double) * 3 * (nv > 0 ? nv : 1));
  memcpy(m->xyz, xyz, sizeof(double) * 3 * nv);
  m->tet = (int64_t *)malloc(sizeof(int64_t) * 4 * (nc > 0 ? nc : 1));
  memcpy(m->tet, tet, sizeof(int64_t) * 4 * nc);
  m->vol = (double *)malloc(sizeof(double) * (nc + 1));
  m->cen = (double *)malloc(sizeof(double) * 3 * (nc + 1));
  m->h = (double *)malloc(sizeof(double) * (nc + 1));
  m->cface = (int64_t *)malloc(sizeof(int64_t) * 4 * (nc + 1));
  m->cnb = (int64_t *)malloc(sizeof(int64_t) * 4 * (nc + 1));
  m->cshift = (double *)calloc(12 * (nc + 1), sizeof(double));
  m->cside = (int32_t *)malloc(sizeof(int32_t) * 4 * (nc + 1));
  m->fit = (orc_fit *)calloc(nc + 1, sizeof(orc_fit));
  for (int64_t i = 0; i < nc; i++) {
    const double *v[4];
    for (int a = 0; a < 4; a++) {
      if (tet[4 * i + a] < 0 || tet[4 * i + a] >= nv) { snprintf(err, errlen, "vertex index out of range"); orc_mesh_destroy(m); return NULL; }
      v[a] = xyz + 3 * tet[4 * i + a];
    }
    double e1[3], e2[3], e3[3], c[3];
    for (int d = 0; d < 3; d++) { e1[d] = v[1][d] - v[0][d]; e2[d] = v[2][d] - v[0][d]; e3[d] = v[3][d] - v[0][d]; }
    cross(e2, e3, c);
    double vol = fabs(e1[0] * c[0] + e1[1] * c[1] + e1[2] * c[2]) / 6.0;
    if (!(vol > 0.0)) { snprintf(err, errlen, "degenerate tetrahedron %lld", (long long)i); orc_mesh_destroy(m); return NULL; }
    m->vol[i] = vol;
    m->h[i] = cbrt(vol);
    for (int d = 0; d < 3; d++) m->cen[3 * i + d] = 0.25 * (v[0][d] + v[1][d] + v[2][d] + v[3][d]);
  }
  /* face table */
  facekey *fk = (facekey *)malloc(sizeof(facekey) * (4 * nc + 1));
  for (int64_t i = 0; i < nc; i++)
    for (int p = 0; p < 4; p++) {
      facekey *k = fk + 4 * i + p;
      for (int j = 0; j < 3; j++) k->k[j] = tet[4 * i + FACEV[p][j]];
      sort3(k->k);
      k->cell = i; k->p = p;
    }
  qsort(fk, 4 * nc, sizeof(facekey), cmp_key);
  int64_t *bkeys = (int64_t *)malloc(sizeof(int64_t) * 3 * (nb + 1));
  int64_t *border = (int64_t *)malloc(sizeof(int64_t) * (nb + 1));
  for (int64_t b = 0; b < nb; b++) { for (int j = 0; j < 3; j++) bkeys[3 * b + j] = bface[3 * b + j]; sort3(bkeys + 3 * b); border[b] = b; }
  /* insertion-free lookup: linear search list sorted by key (simple qsort on index) */
  for (int64_t a = 1; a < nb; a++) { /* insertion sort of border by key; nb is small in tests */
    int64_t x = border[a], b = a - 1;
    while (b >= 0 && cmp3(bkeys + 3 * border[b], bkeys + 3 * x) > 0) { border[b + 1] = border[b]; b--; }
    border[b + 1] = x;
  }
  int64_t maxf = 4 * nc + 1;
  m->fl = (int64_t *)malloc(sizeof(int64_t) * maxf); m->fr = (int64_t *)malloc(sizeof(int64_t) * maxf);
  m->flp = (int32_t *)malloc(sizeof(int32_t) * maxf); m->frp = (int32_t *)malloc(sizeof(int32_t) * maxf);
  m->ftag = (int32_t *)malloc(sizeof(int32_t) * maxf);
  m->fshift = (double *)calloc(3 * maxf, sizeof(double));
  int64_t nf = 0;
  int64_t *unm = (int64_t *)malloc(sizeof(int64_t) * maxf);  /* indices into fk of unmatched faces */
  int64_t nunm = 0;
  for (int64_t a = 0; a < 4 * nc;) {
    int64_t b = a + 1;
    while (b < 4 * nc && cmp3(fk[b].k, fk[a].k) == 0) b++;
    if (b - a > 2) { snprintf(err, errlen, "face shared by more than two cells"); goto fail; }
    if (b - a == 2) {
      m->fl[nf] = fk[a].cell; m->flp[nf] = fk[a].p; m->fr[nf] = fk[a + 1].cell; m->frp[nf] = fk[a + 1].p;
      m->ftag[nf] = 0; nf++;
    } else {
      /* boundary face? binary search in the tagged list */
      int64_t lo = 0, hi = nb - 1, found = -1;
      while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        int c = cmp3(bkeys + 3 * border[mid], fk[a].k);
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
      for (int d = 0; d < 3; d++)
        uc[3 * u + d] = (xyz[3 * fk[unm[u]].k[0] + d] + xyz[3 * fk[unm[u]].k[1] + d] + xyz[3 * fk[unm[u]].k[2] + d]) / 3.0;
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
  m->fgp = (double *)malloc(sizeof(double) * 9 * (nf + 1));
  m->fcen = (double *)malloc(sizeof(double) * 3 * (nf + 1));
  for (int64_t i = 0; i < 4 * nc; i++) m->cnb[i] = -1;
  for (int64_t f = 0; f < nf; f++) {
    int64_t L = m->fl[f]; int p = m->flp[f];
    int64_t vk[3];
    for (int j = 0; j < 3; j++) vk[j] = tet[4 * L + FACEV[p][j]];
    sort3(vk);
    const double *a = xyz + 3 * vk[0], *b = xyz + 3 * vk[1], *c = xyz + 3 * vk[2], *o = xyz + 3 * tet[4 * L + p];
    double e1[3], e2[3], n[3];
    for (int d = 0; d < 3; d++) { e1[d] = b[d] - a[d]; e2[d] = c[d] - a[d]; }
    cross(e1, e2, n);
    double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    double out = (a[0] - o[0]) * n[0] + (a[1] - o[1]) * n[1] + (a[2] - o[2]) * n[2];
    double sg = out > 0 ? 1.0 : -1.0;
    m->farea[f] = 0.5 * nn;
    for (int d = 0; d < 3; d++) m->fnrm[3 * f + d] = sg * n[d] / nn;
    const double *vv[3] = {a, b, c};
    for (int g = 0; g < 3; g++)            /* 3-point rule, barycentric (2/3,1/6,1/6), weights 1/3 */
      for (int d = 0; d < 3; d++)
        m->fgp[9 * f + 3 * g + d] = (2.0 / 3.0) * vv[g][d] + (1.0 / 6.0) * (vv[(g + 1) % 3][d] + vv[(g + 2) % 3][d]);
    for (int d = 0; d < 3; d++) m->fcen[3 * f + d] = (a[d] + b[d] + c[d]) / 3.0;
    m->cface[4 * L + p] = f; m->cnb[4 * L + p] = m->fr[f]; m->cside[4 * L + p] = 0;
    if (m->fr[f] >= 0) {
      int64_t R = m->fr[f]; int q = m->frp[f];
      m->cface[4 * R + q] = f; m->cnb[4 * R + q] = L; m->cside[4 * R + q] = 1;
      for (int d = 0; d < 3; d++) {
        m->cshift[12 * L + 3 * p + d] = m->fshift[3 * f + d];   /* right cell + shift -> left frame */
        m->cshift[12 * R + 3 * q + d] = -m->fshift[3 * f + d];
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
static void quad_points(const orc_mesh *m, int64_t i, int64_t k, const double *shift, double xq[4][3]) {
  for (int q = 0; q < 4; q++)
    for (int d = 0; d < 3; d++) {
      double x = 0.0;
      for (int a = 0; a < 4; a++) x += (a == q ? QA : QB) * m->xyz[3 * m->tet[4 * k + a] + d];
      xq[q][d] = (x + shift[d] - m->cen[3 * i + d]) / m->h[i];
    }
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
  double xq[4][3], mo[9];
  quad_points(m, i, k, shift, xq);
  for (int d = 0; d < 9; d++) avg[d] = 0.0;
  for (int q = 0; q < 4; q++) { monomials(xq[q], mo); for (int d = 0; d < 9; d++) avg[d] += 0.25 * mo[d]; }
}
static void avg_dmonomials(const orc_mesh *m, int64_t i, int64_t k, const double *shift, int j, double *avg) {
  double xq[4][3], dm[9];
  quad_points(m, i, k, shift, xq);
  for (int d = 0; d < 9; d++) avg[d] = 0.0;
  for (int q = 0; q < 4; q++) { dmonomials(xq[q], j, dm); for (int d = 0; d < 9; d++) avg[d] += 0.25 * dm[d]; }
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
  int64_t j = m->cnb[4 * r->cell + q];
  for (int d = 0; d < 3; d++) s[d] = r->shift[d] + m->cshift[12 * r->cell + 3 * q + d];
  return j;
}

/* sub-stencil triples of face neighbours, Sec. 3.1 (faces numbered from 0) */
static const int TRIPLE[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {2, 0, 3}};

int orc_fit_cell(orc_mesh *m, int64_t i, int scheme) {
  orc_fit *F = m->fit + i;
  const double zero[3] = {0, 0, 0};
  orc_sref self; self.cell = i; self.shift[0] = self.shift[1] = self.shift[2] = 0.0;
  double avg_i[9];
  avg_monomials(m, i, i, zero, avg_i);
  if (scheme == 0 && !F->ready_weno) {
    /* big stencil: face neighbours, then their neighbours; a third level only
     * when fewer than 12 cells were found (boundary cells) */
    F->n_big = 0;
    orc_sref l1[4]; int n1 = 0;
    for (int p = 0; p < 4; p++) {
      double s[3]; int64_t j = nb_of(m, &self, p, s);
      if (add_ref(F->big, &F->n_big, ORC_MAXSTEN, i, j, s)) l1[n1++] = F->big[F->n_big - 1];
    }
    int start2 = F->n_big;
    for (int a = 0; a < n1; a++)
      for (int q = 0; q < 4; q++) { double s[3]; int64_t k = nb_of(m, l1 + a, q, s); add_ref(F->big, &F->n_big, ORC_MAXSTEN, i, k, s); }
    /* further levels, ring by ring, only while fewer than 12 cells were found */
    int fs = start2, fe = F->n_big;
    for (int level = 3; level <= 6 && F->n_big < 12 && fe > fs; level++) {
      int ns = F->n_big;
      for (int a = fs; a < fe && F->n_big < 12; a++)
        for (int q = 0; q < 4 && F->n_big < 12; q++) { double s[3]; int64_t k = nb_of(m, F->big + a, q, s); add_ref(F->big, &F->n_big, 12, i, k, s); }
      fs = ns; fe = F->n_big;
    }
    if (F->n_big < 9) return -1;
    double A[ORC_MAXSTEN * 9], av[9];
    for (int r = 0; r < F->n_big; r++) {
      avg_monomials(m, i, F->big[r].cell, F->big[r].shift, av);
      for (int d = 0; d < 9; d++) A[r * 9 + d] = av[d] - avg_i[d];
    }
    double X[9 * ORC_MAXSTEN];
    if (orc_lsq_pinv(F->n_big, 9, A, X)) return -2;
    memset(F->X0, 0, sizeof(F->X0));
    for (int d = 0; d < 9; d++) for (int r = 0; r < F->n_big; r++) F->X0[d][r] = X[d * F->n_big + r];
    /* sub-stencils: three face neighbours plus the neighbours of one of them */
    for (int mm = 0; mm < 4; mm++) {
      F->n_sub[mm] = 0;
      for (int t = 0; t < 3; t++) { double s[3]; int64_t j = nb_of(m, &self, TRIPLE[mm][t], s); add_ref(F->sub[mm], &F->n_sub[mm], ORC_MAXSUB, i, j, s); }
      double s0[3]; int64_t jm = nb_of(m, &self, mm, s0);
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
    F->ready_weno = 1;
  }
  if (scheme == 1 && !F->ready_hweno) {
    /* compact: the target and its face neighbours, Eq. (compact-big-1) solved by
     * constrained least squares: cell averages exact, h-scaled gradients in the
     * least-squares sense */
    F->n_nb = 0;
    for (int p = 0; p < 4; p++) {
      double s[3]; int64_t j = nb_of(m, &self, p, s);
      if (j >= 0) { F->nb[F->n_nb].cell = j; for (int d = 0; d < 3; d++) F->nb[F->n_nb].shift[d] = s[d]; F->nb_slot[F->n_nb] = p; F->n_nb++; }
    }
    /* with fewer than 3 face neighbours (an edge of the domain) the quadratic
     * system is singular: P0 keeps its linear terms only (nu = 3 unknowns) */
    int ne = F->n_nb, nls = 3 * (1 + F->n_nb), nu = ne >= 3 ? 9 : 3, n = nu + ne;
    double C[4][9], B[15][9], av[9];
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
    double K[(9 + 4) * (9 + 4)];
    memset(K, 0, sizeof(K));
    for (int a = 0; a < nu; a++)
      for (int b = 0; b < nu; b++) { double s = 0; for (int r = 0; r < nls; r++) s += B[r][a] * B[r][b]; K[a * n + b] = s; }
    for (int r = 0; r < ne; r++) for (int d = 0; d < nu; d++) { K[d * n + nu + r] = C[r][d]; K[(nu + r) * n + d] = C[r][d]; }
    memset(F->H0, 0, sizeof(F->H0));
    /* the map from data to coefficients, one data unit vector at a time */
    for (int col = 0; col < 4 + 15; col++) {
      double rhs[13] = {0}, sol[13];
      if (col < 4) {
        if (col >= ne) continue;
        rhs[nu + col] = 1.0;
      } else {
        int k = (col - 4) / 3, j = (col - 4) % 3;
        if (k > ne) continue;
        const orc_sref *rk = k == 0 ? &self : &F->nb[k - 1];
        double dval = m->h[rk->cell];        /* d_row = h_k * G_kj */
        for (int a = 0; a < nu; a++) rhs[a] = B[3 * k + j][a] * dval;
      }
      if (orc_lu_solve(n, K, rhs, sol)) return -3;
      for (int d = 0; d < nu; d++) F->H0[d][col] = sol[d];
    }
    /* compact sub-stencils {target, one face neighbour}, Eq. (compact-big-2) */
    for (int mm = 0; mm < 4; mm++) {
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
