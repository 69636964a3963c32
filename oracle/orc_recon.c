/* ORACLE (test infrastructure only): reconstruction at the Gauss points of one
 * face, from one side (Sec. 3.2 - 3.4 and Sec. 5's characteristic variables).
 *
 * 1. Polynomials P0 (quadratic) and P_m (linear) of Eq. (polys) from the fits.
 * 2. Local frame of the face: n (left to right), t1 = n x e_a / |n x e_a| with
 *    a the axis minimising |n_a| * (1, 1 + 1e-3, 1 + 2e-3)_a (lowest index on an
 *    exact tie), t2 = n x t1.
 * 3. Characteristic projection with the right eigenvectors R* of the Euler
 *    Jacobian along n at Q* = (Q_left + Q_right)/2 (the cell's own average on a
 *    boundary face); R*^{-1} is taken by Gaussian elimination.
 * 4. Smoothness indicators and the nonlinear weights of Eq. (weno), per
 *    characteristic component.
 * 5. Values and gradients at the Gauss points, projected back with R*.
 * Cell averages over the target cell use the cell's quadrature (orc_cell_quad).
 * Sub-stencils: 4 (tetrahedron) or 8 (hexahedron) non-compact ones, one per
 * face for the compact scheme. */
#include <math.h>
#include <string.h>
#include "orc.h"

void orc_face_frame(const double *n, double *T) {
  const double wgt[3] = {1.0, 1.001, 1.002};
  int a = 0;
  for (int k = 1; k < 3; k++) if (fabs(n[k]) * wgt[k] < fabs(n[a]) * wgt[a]) a = k;
  double e[3] = {0, 0, 0}; e[a] = 1.0;
  double t1[3] = {n[1] * e[2] - n[2] * e[1], n[2] * e[0] - n[0] * e[2], n[0] * e[1] - n[1] * e[0]};
  double l = sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
  for (int d = 0; d < 3; d++) t1[d] /= l;
  double t2[3] = {n[1] * t1[2] - n[2] * t1[1], n[2] * t1[0] - n[0] * t1[2], n[0] * t1[1] - n[1] * t1[0]};
  for (int d = 0; d < 3; d++) { T[d] = n[d]; T[3 + d] = t1[d]; T[6 + d] = t2[d]; }
}

/* rotate the momentum of a conservative vector: out = blockdiag(1, T, 1) in */
static void rot5(const double *T, const double *in, double *out) {
  out[0] = in[0]; out[4] = in[4];
  for (int i = 0; i < 3; i++) out[1 + i] = T[3 * i] * in[1] + T[3 * i + 1] * in[2] + T[3 * i + 2] * in[3];
}
static void rot5t(const double *T, const double *in, double *out) {
  out[0] = in[0]; out[4] = in[4];
  for (int i = 0; i < 3; i++) out[1 + i] = T[i] * in[1] + T[3 + i] * in[2] + T[6 + i] * in[3];
}

/* Right eigenvectors (columns) of the Euler Jacobian along x at a local-frame
 * state; R^{-1} by elimination. */
void orc_char_eigen(const double *Q, double gamma, double *R, double *L) {
  double rho = Q[0], u = Q[1] / rho, v = Q[2] / rho, w = Q[3] / rho;
  double q2 = u * u + v * v + w * w, p = (gamma - 1.0) * (Q[4] - 0.5 * rho * q2);
  double a = sqrt(gamma * p / rho), H = (Q[4] + p) / rho;
  double cols[5][5] = {{1, u - a, v, w, H - u * a},
                       {1, u, v, w, 0.5 * q2},
                       {0, 0, 1, 0, v},
                       {0, 0, 0, 1, w},
                       {1, u + a, v, w, H + u * a}};
  for (int i = 0; i < 5; i++) for (int j = 0; j < 5; j++) R[i * 5 + j] = cols[j][i];
  orc_inverse(5, R, L);
}

int orc_recon_side(orc_mesh *m, const orc_params *p, const double *Q, const double *G,
                   int64_t cell, int slot, double *Wloc, double *dWloc, double *Wglob, double *gradglob) {
  const int64_t i = cell;
  if (orc_fit_cell(m, i, p->scheme)) return -1;
  const orc_fit *F = m->fit + i;
  const int nfc = m->nfc, ngp = m->ngp;
  const int64_t f = m->cface[nfc * i + slot];
  const int nsub = p->scheme == 0 ? (m->nvc == 8 ? 8 : 4) : nfc;
  /* 1. coefficients in conservative variables, per component: a[d][c], b[mm][j][c] */
  double a[9][5], b[ORC_NSUB][3][5];
  int valid[ORC_NSUB];
  memset(a, 0, sizeof(a)); memset(b, 0, sizeof(b));
  if (p->scheme == 0) {
    for (int c = 0; c < 5; c++) {
      for (int d = 0; d < 9; d++) {
        double s = 0.0;
        for (int r = 0; r < F->n_big; r++) s += F->X0[d][r] * (Q[5 * F->big[r].cell + c] - Q[5 * i + c]);
        a[d][c] = s;
      }
      for (int mm = 0; mm < nsub; mm++) {
        if (!F->sub_valid[mm]) continue;
        for (int j = 0; j < 3; j++) {
          double s = 0.0;
          for (int r = 0; r < F->n_sub[mm]; r++) s += F->Xm[mm][j][r] * (Q[5 * F->sub[mm][r].cell + c] - Q[5 * i + c]);
          b[mm][j][c] = s;
        }
      }
    }
    for (int mm = 0; mm < nsub; mm++) valid[mm] = F->sub_valid[mm];
  } else {
    for (int c = 0; c < 5; c++) {
      double data[ORC_HCOLS];
      memset(data, 0, sizeof(data));
      for (int r = 0; r < F->n_nb; r++) data[r] = Q[5 * F->nb[r].cell + c] - Q[5 * i + c];
      for (int k = 0; k <= F->n_nb; k++) {
        int64_t ck = k == 0 ? i : F->nb[k - 1].cell;
        for (int j = 0; j < 3; j++) data[nfc + 3 * k + j] = G[15 * ck + 3 * c + j];
      }
      for (int d = 0; d < 9; d++) { double s = 0.0; for (int col = 0; col < ORC_HCOLS; col++) s += F->H0[d][col] * data[col]; a[d][c] = s; }
      for (int mm = 0; mm < nfc; mm++) {
        double dm[7] = {0};
        int64_t jm = m->cnb[nfc * i + mm];
        if (jm >= 0) dm[0] = Q[5 * jm + c] - Q[5 * i + c];
        for (int j = 0; j < 3; j++) dm[1 + j] = G[15 * i + 3 * c + j];
        if (jm >= 0) for (int j = 0; j < 3; j++) dm[4 + j] = G[15 * jm + 3 * c + j];
        for (int j = 0; j < 3; j++) { double s = 0.0; for (int col = 0; col < 7; col++) s += F->Hm[mm][j][col] * dm[col]; b[mm][j][c] = s; }
      }
    }
    for (int mm = 0; mm < nfc; mm++) valid[mm] = 1;
  }
  /* 2. face frame, 3. projection */
  double T3[9];
  orc_face_frame(m->fnrm + 3 * f, T3);
  double Pm[25], Rb[25];
  if (p->characteristic) {
    double Qs[5], Qsl[5], L[25], Rt[25];
    int64_t L_ = m->fl[f], R_ = m->fr[f];
    for (int c = 0; c < 5; c++) Qs[c] = R_ >= 0 ? 0.5 * (Q[5 * L_ + c] + Q[5 * R_ + c]) : Q[5 * i + c];
    rot5(T3, Qs, Qsl);
    orc_char_eigen(Qsl, p->gamma, Rt, L);
    /* Pm = L * rot5 ; Rb = rot5^T * R (back to global conservative) */
    for (int c = 0; c < 5; c++)
      for (int k = 0; k < 5; k++) {
        double e[5] = {0, 0, 0, 0, 0}, re[5];
        e[k] = 1.0; rot5(T3, e, re);
        double s = 0.0; for (int l = 0; l < 5; l++) s += L[c * 5 + l] * re[l];
        Pm[c * 5 + k] = s;
      }
    for (int k = 0; k < 5; k++) {
      double col[5], gcol[5];
      for (int l = 0; l < 5; l++) col[l] = Rt[l * 5 + k];
      rot5t(T3, col, gcol);
      for (int l = 0; l < 5; l++) Rb[l * 5 + k] = gcol[l];
    }
  } else {
    for (int k = 0; k < 25; k++) Pm[k] = Rb[k] = (k % 6 == 0) ? 1.0 : 0.0;
  }
  double q0[5], ac[9][5], bc[ORC_NSUB][3][5];
  for (int c = 0; c < 5; c++) {
    double s = 0.0; for (int k = 0; k < 5; k++) s += Pm[c * 5 + k] * Q[5 * i + k]; q0[c] = s;
    for (int d = 0; d < 9; d++) { s = 0.0; for (int k = 0; k < 5; k++) s += Pm[c * 5 + k] * a[d][k]; ac[d][c] = s; }
    for (int mm = 0; mm < nsub; mm++)
      for (int j = 0; j < 3; j++) { s = 0.0; for (int k = 0; k < 5; k++) s += Pm[c * 5 + k] * b[mm][j][k]; bc[mm][j][c] = s; }
  }
  /* cell averages of the monomials over the target cell (basis offsets of Eq. (polys)) */
  double xq[64][3], wq[64], avg[9];
  const int nq = orc_cell_quad(m, i, xq, wq);
  for (int q = 0; q < nq; q++)
    for (int d = 0; d < 3; d++) xq[q][d] = (xq[q][d] - m->cen[3 * i + d]) / m->h[i];
  for (int d = 0; d < 9; d++) avg[d] = 0.0;
  for (int q = 0; q < nq; q++) {
    double x = xq[q][0], y = xq[q][1], z = xq[q][2];
    double mo[9] = {x, y, z, x * x, y * y, z * z, x * y, x * z, y * z};
    for (int d = 0; d < 9; d++) avg[d] += wq[q] * mo[d];
  }
  /* 4. smoothness indicators (scaled frame: the |Omega|^(2|l|/3 - 1) factors cancel the scaling) */
  int M = 0; for (int mm = 0; mm < nsub; mm++) M += valid[mm];
  double gam_m = p->lin_weight, gam0 = 1.0 - gam_m * M;
  double wbar[5][1 + ORC_NSUB];   /* [component][0..nsub], 0 = P0 */
  for (int c = 0; c < 5; c++) {
    double beta[1 + ORC_NSUB];
    /* beta_0: first derivatives (linear functions) averaged over the cell, second derivatives constant */
    double s = 0.0;
    for (int q = 0; q < nq; q++) {
      double x = xq[q][0], y = xq[q][1], z = xq[q][2];
      double dx = ac[0][c] + 2 * ac[3][c] * x + ac[6][c] * y + ac[7][c] * z;
      double dy = ac[1][c] + 2 * ac[4][c] * y + ac[6][c] * x + ac[8][c] * z;
      double dz = ac[2][c] + 2 * ac[5][c] * z + ac[7][c] * x + ac[8][c] * y;
      s += wq[q] * (dx * dx + dy * dy + dz * dz);
    }
    double hxx = 2 * ac[3][c], hyy = 2 * ac[4][c], hzz = 2 * ac[5][c];
    s += hxx * hxx + hyy * hyy + hzz * hzz + ac[6][c] * ac[6][c] + ac[7][c] * ac[7][c] + ac[8][c] * ac[8][c];
    beta[0] = s;
    for (int mm = 0; mm < nsub; mm++)
      beta[1 + mm] = bc[mm][0][c] * bc[mm][0][c] + bc[mm][1][c] * bc[mm][1][c] + bc[mm][2][c] * bc[mm][2][c];
    double om[1 + ORC_NSUB];
    if (p->weights == 1 || M == 0) {
      wbar[c][0] = M == 0 ? 1.0 : gam0;
      for (int mm = 0; mm < nsub; mm++) wbar[c][1 + mm] = valid[mm] ? gam_m : 0.0;
    } else {
      double tz = 0.0;
      for (int mm = 0; mm < nsub; mm++) if (valid[mm]) tz += fabs(beta[0] - beta[1 + mm]) / M;
      om[0] = gam0 * (1.0 + tz / (beta[0] + p->weno_eps));
      double sum = om[0];
      for (int mm = 0; mm < nsub; mm++) { om[1 + mm] = valid[mm] ? gam_m * (1.0 + tz / (beta[1 + mm] + p->weno_eps)) : 0.0; sum += om[1 + mm]; }
      for (int k = 0; k <= nsub; k++) wbar[c][k] = om[k] / sum;
    }
  }
  double g0eff = M == 0 ? 1.0 : gam0;
  /* 5. Gauss points */
  const double *sh = m->cside[nfc * i + slot] == 1 ? m->fshift + 3 * f : NULL;
  for (int gp = 0; gp < ngp; gp++) {
    double x[3];
    for (int d = 0; d < 3; d++) x[d] = (m->fgp[3 * ngp * f + 3 * gp + d] - (sh ? sh[d] : 0.0) - m->cen[3 * i + d]) / m->h[i];
    double pd[9] = {x[0], x[1], x[2], x[0] * x[0], x[1] * x[1], x[2] * x[2], x[0] * x[1], x[0] * x[2], x[1] * x[2]};
    for (int d = 0; d < 9; d++) pd[d] -= avg[d];
    double dpd[3][9];
    for (int j = 0; j < 3; j++) {
      for (int d = 0; d < 9; d++) dpd[j][d] = 0.0;
      dpd[j][j] = 1.0; dpd[j][3 + j] = 2 * x[j];
    }
    dpd[0][6] = x[1]; dpd[0][7] = x[2]; dpd[1][6] = x[0]; dpd[1][8] = x[2]; dpd[2][7] = x[0]; dpd[2][8] = x[1];
    double qv[5], qg[3][5];
    for (int c = 0; c < 5; c++) {
      double P0 = q0[c], dP0[3] = {0, 0, 0}, Pm_[ORC_NSUB], dPm[ORC_NSUB][3];
      for (int d = 0; d < 9; d++) { P0 += ac[d][c] * pd[d]; for (int j = 0; j < 3; j++) dP0[j] += ac[d][c] * dpd[j][d]; }
      for (int mm = 0; mm < nsub; mm++) {
        Pm_[mm] = q0[c];
        for (int j = 0; j < 3; j++) { Pm_[mm] += bc[mm][j][c] * pd[j]; dPm[mm][j] = bc[mm][j][c]; }
      }
      /* Eq. (weno) */
      double val = P0 / g0eff, grad[3] = {dP0[0] / g0eff, dP0[1] / g0eff, dP0[2] / g0eff};
      for (int mm = 0; mm < nsub; mm++) {
        if (!valid[mm]) continue;
        val -= gam_m / g0eff * Pm_[mm];
        for (int j = 0; j < 3; j++) grad[j] -= gam_m / g0eff * dPm[mm][j];
      }
      val *= wbar[c][0];
      for (int j = 0; j < 3; j++) grad[j] *= wbar[c][0];
      for (int mm = 0; mm < nsub; mm++) {
        if (!valid[mm]) continue;
        val += wbar[c][1 + mm] * Pm_[mm];
        for (int j = 0; j < 3; j++) grad[j] += wbar[c][1 + mm] * dPm[mm][j];
      }
      qv[c] = val;
      for (int j = 0; j < 3; j++) qg[j][c] = grad[j] / m->h[i];   /* d/dx = (1/h) d/dx_hat */
    }
    /* back to global conservative variables, then to the face frame */
    double Wg[5], dWg[3][5], Wl_[5], dWl_[3][5];
    for (int c = 0; c < 5; c++) {
      double s = 0.0; for (int k = 0; k < 5; k++) s += Rb[c * 5 + k] * qv[k]; Wg[c] = s;
      for (int j = 0; j < 3; j++) { s = 0.0; for (int k = 0; k < 5; k++) s += Rb[c * 5 + k] * qg[j][k]; dWg[j][c] = s; }
    }
    rot5(T3, Wg, Wl_);
    double dWc[3][5];   /* Cartesian derivatives of local-frame conservative variables */
    for (int j = 0; j < 3; j++) rot5(T3, dWg[j], dWc[j]);
    for (int k = 0; k < 3; k++)
      for (int c = 0; c < 5; c++) dWl_[k][c] = T3[3 * k] * dWc[0][c] + T3[3 * k + 1] * dWc[1][c] + T3[3 * k + 2] * dWc[2][c];
    /* positivity: fall back to the cell average with zero slopes */
    double rho = Wl_[0], pr = (p->gamma - 1.0) * (Wl_[4] - 0.5 * (Wl_[1] * Wl_[1] + Wl_[2] * Wl_[2] + Wl_[3] * Wl_[3]) / rho);
    if (!(rho > 0.0) || !(pr > 0.0)) {
      rot5(T3, Q + 5 * i, Wl_);
      memset(dWl_, 0, sizeof(dWl_));
      for (int c = 0; c < 5; c++) Wg[c] = Q[5 * i + c];
      memset(dWg, 0, sizeof(dWg));
    }
    for (int c = 0; c < 5; c++) {
      Wloc[5 * gp + c] = Wl_[c];
      for (int k = 0; k < 3; k++) dWloc[15 * gp + 5 * k + c] = dWl_[k][c];
      if (Wglob) Wglob[5 * gp + c] = Wg[c];
      if (gradglob) for (int j = 0; j < 3; j++) gradglob[15 * gp + 3 * c + j] = dWg[j][c];
    }
  }
  return 0;
}
