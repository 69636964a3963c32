/* ORACLE (test infrastructure only): residual, local time step, approximate
 * Jacobian, Jacobi preconditioner, restarted GMRES and the steady loop.
 *
 * Residual: Eq. (finite) with the time-averaged flux of Sec. 4.1, the face's
 * Gauss rule (3 points on a triangle, 2 x 2 on a quadrilateral); compact scheme: cell-averaged gradients from the point values
 * of Eq. (point) by Gauss's theorem, Eq. (derivative).
 * Implicit system: Eq. (A-system-2) with the Rusanov-type split Jacobians of
 * Eq. (deri-matrix); Jacobi preconditioner of Eq. (precond); Algorithm 1. */
#include <float.h>
#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>
#include "orc.h"

static void rot5t3(const double *T, const double *in, double *out) {
  out[0] = in[0]; out[4] = in[4];
  for (int i = 0; i < 3; i++) out[1 + i] = T[i] * in[1] + T[3 + i] * in[2] + T[6 + i] * in[3];
}

static void outward(const orc_mesh *m, int64_t i, int p, double *n) {
  int64_t f = m->cface[m->nfc * i + p];
  double s = m->cside[m->nfc * i + p] == 0 ? 1.0 : -1.0;
  for (int d = 0; d < 3; d++) n[d] = s * m->fnrm[3 * f + d];
}

/* Local time step (the paper gives no formula): CFL |Omega| / sum_p S_p (|U.n_p| + a + nu) */
int orc_local_dt(orc_mesh *m, const orc_params *p, const double *Q, double *dt) {
  for (int64_t i = 0; i < m->nc; i++) {
    double pr[5]; orc_primitive(Q + 5 * i, p->gamma, pr);
    double pres = pr[0] / (2.0 * pr[4]), a = sqrt(p->gamma * pres / pr[0]);
    double nu = p->viscous ? 2.0 * p->gamma * p->mu / (p->Pr * pr[0] * m->h[i]) : 0.0;
    double s = 0.0;
    for (int q = 0; q < m->nfc; q++) {
      double n[3]; outward(m, i, q, n);
      int64_t f = m->cface[m->nfc * i + q];
      s += m->farea[f] * (fabs(pr[1] * n[0] + pr[2] * n[1] + pr[3] * n[2]) + a + nu);
    }
    dt[i] = p->cfl * m->vol[i] / s;
  }
  return 0;
}

int orc_residual(orc_mesh *m, const orc_params *p, const double *Q, const double *G,
                 double *R, double *Gnew, const int64_t *cells, int64_t ncells) {
  return orc_residual_dt(m, p, Q, G, NULL, R, Gnew, cells, ncells);
}

static int residual_core(orc_mesh *m, const orc_params *p, const double *Q, const double *G, const double *dt_in,
                         double *R, double *Gnew, const int64_t *cells, int64_t ncells, double *Fface);

int orc_residual_dt(orc_mesh *m, const orc_params *p, const double *Q, const double *G, const double *dt_in,
                    double *R, double *Gnew, const int64_t *cells, int64_t ncells) {
  return residual_core(m, p, Q, G, dt_in, R, Gnew, cells, ncells, NULL);
}

/* Force of the flow on the boundary faces tagged `tag`: the sum over those faces
 * of the momentum part of the face flux of Eq. (flux) times the face area (the
 * flux leaving the fluid through the wall: pressure and viscous stress on it). */
int orc_wall_force(orc_mesh *m, const orc_params *p, const double *Q, const double *G, int tag, double *force) {
  const int64_t nc = m->nc, nf = m->nf;
  double *R = (double *)malloc(sizeof(double) * 5 * (nc + 1)), *Ff = (double *)calloc(5 * (nf + 1), sizeof(double));
  int rc = residual_core(m, p, Q, G, NULL, R, NULL, NULL, 0, Ff);
  force[0] = force[1] = force[2] = 0.0;
  if (!rc)
    for (int64_t f = 0; f < nf; f++)
      if (m->fr[f] < 0 && m->ftag[f] == tag)
        for (int d = 0; d < 3; d++) force[d] += Ff[5 * f + 1 + d];
  free(R); free(Ff);
  return rc;
}

static int residual_core(orc_mesh *m, const orc_params *p, const double *Q, const double *G, const double *dt_in,
                         double *R, double *Gnew, const int64_t *cells, int64_t ncells, double *Fface) {
  const int64_t nc = m->nc, nf = m->nf;
  char *fsel = (char *)calloc(nf + 1, 1), *csel = (char *)calloc(nc + 1, 1);
  if (cells) {
    for (int64_t a = 0; a < ncells; a++) {
      int64_t i = cells[a];
      for (int q = 0; q < m->nfc; q++) fsel[m->cface[m->nfc * i + q]] = 1;
    }
  } else memset(fsel, 1, nf);
  for (int64_t f = 0; f < nf; f++) if (fsel[f]) { csel[m->fl[f]] = 1; if (m->fr[f] >= 0) csel[m->fr[f]] = 1; }
  int err = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : err)
  for (int64_t i = 0; i < nc; i++) if (csel[i]) err |= orc_fit_cell(m, i, p->scheme) != 0;
  if (err) { free(fsel); free(csel); return -1; }
  double *dt = (double *)malloc(sizeof(double) * (nc + 1));
  if (dt_in) memcpy(dt, dt_in, sizeof(double) * nc);
  else orc_local_dt(m, p, Q, dt);
  double *Ff = (double *)calloc(5 * (nf + 1), sizeof(double)), *Pf = (double *)calloc(5 * (nf + 1), sizeof(double));
#pragma omp parallel for schedule(dynamic, 16) reduction(| : err)
  for (int64_t f = 0; f < nf; f++) {
    if (!fsel[f]) continue;
    int64_t L = m->fl[f], Rr = m->fr[f];
    const int ngp = m->ngp;
    double WL[5 * ORC_MAXG], dWL[15 * ORC_MAXG], WR[5 * ORC_MAXG], dWR[15 * ORC_MAXG], T3[9];
    orc_face_frame(m->fnrm + 3 * f, T3);
    err |= orc_recon_side(m, p, Q, G, L, m->flp[f], WL, dWL, NULL, NULL) != 0;
    if (Rr >= 0) err |= orc_recon_side(m, p, Q, G, Rr, m->frp[f], WR, dWR, NULL, NULL) != 0;
    else for (int g = 0; g < ngp; g++) orc_boundary_state(p, m->ftag[f], T3, WL + 5 * g, dWL + 15 * g, WR + 5 * g, dWR + 15 * g);
    /* time step inside the flux: the local step at CFL = flux_cfl, single-valued per face */
    double dtf = p->flux_dt > 0 ? p->flux_dt : (Rr >= 0 ? fmin(dt[L], dt[Rr]) : dt[L]) * (p->flux_cfl / p->cfl);
    for (int g = 0; g < ngp; g++) {
      double F[5], Qp[5], Fg[5], Qg[5];
      orc_gks_flux(p, WL + 5 * g, dWL + 15 * g, WR + 5 * g, dWR + 15 * g, dtf, F, Qp);
      rot5t3(T3, F, Fg); rot5t3(T3, Qp, Qg);
      /* walls (tags 1-4) are impermeable: their faces carry momentum and energy, no mass */
      if (Rr < 0 && m->ftag[f] >= 1 && m->ftag[f] <= 4) Fg[0] = 0.0;
      /* Gauss weights: 1/3 on a triangle, the area-element weights fgw on a quadrilateral */
      if (ngp == 3) for (int c = 0; c < 5; c++) { Ff[5 * f + c] += m->farea[f] * Fg[c] / 3.0; Pf[5 * f + c] += m->farea[f] * Qg[c] / 3.0; }
      else {
        const double wS = m->farea[f] * m->fgw[ngp * f + g];
        for (int c = 0; c < 5; c++) { Ff[5 * f + c] += wS * Fg[c]; Pf[5 * f + c] += wS * Qg[c]; }
      }
    }
  }
  if (err) { free(fsel); free(csel); free(dt); free(Ff); free(Pf); return -1; }
  for (int64_t i = 0; i < nc; i++) {
    for (int c = 0; c < 5; c++) R[5 * i + c] = 0.0;
    if (Gnew) for (int c = 0; c < 15; c++) Gnew[15 * i + c] = 0.0;
  }
  for (int64_t f = 0; f < nf; f++) {
    if (!fsel[f]) continue;
    int64_t L = m->fl[f], Rr = m->fr[f];
    const double *n = m->fnrm + 3 * f;
    for (int c = 0; c < 5; c++) {
      R[5 * L + c] -= Ff[5 * f + c];
      if (Rr >= 0) R[5 * Rr + c] += Ff[5 * f + c];
      if (Gnew)
        for (int d = 0; d < 3; d++) {
          Gnew[15 * L + 3 * c + d] += Pf[5 * f + c] * n[d];
          if (Rr >= 0) Gnew[15 * Rr + 3 * c + d] -= Pf[5 * f + c] * n[d];
        }
    }
  }
  if (Gnew) for (int64_t i = 0; i < nc; i++) for (int c = 0; c < 15; c++) Gnew[15 * i + c] /= m->vol[i];
  if (Fface) memcpy(Fface, Ff, sizeof(double) * 5 * nf);
  free(fsel); free(csel); free(dt); free(Ff); free(Pf);
  return 0;
}

/* Jacobian of the Euler flux F(Q).n along a unit vector n */
void orc_euler_jacobian(const double *Q, const double *n, double gamma, double *J) {
  double rho = Q[0], u = Q[1] / rho, v = Q[2] / rho, w = Q[3] / rho, E = Q[4] / rho;
  double g1 = gamma - 1.0, q2 = u * u + v * v + w * w, phi = 0.5 * g1 * q2;
  double un = u * n[0] + v * n[1] + w * n[2], H = gamma * E - phi;
  double vel[3] = {u, v, w};
  J[0] = 0; J[1] = n[0]; J[2] = n[1]; J[3] = n[2]; J[4] = 0;
  for (int r = 0; r < 3; r++) {
    J[5 * (r + 1) + 0] = phi * n[r] - vel[r] * un;
    for (int c = 0; c < 3; c++) J[5 * (r + 1) + 1 + c] = vel[r] * n[c] - g1 * vel[c] * n[r] + (r == c ? un : 0.0);
    J[5 * (r + 1) + 4] = g1 * n[r];
  }
  J[20] = (phi - H) * un;
  for (int c = 0; c < 3; c++) J[21 + c] = H * n[c] - g1 * vel[c] * un;
  J[24] = gamma * un;
}

/* Eq. (A-system-2) with Eq. (deri-matrix): |lambda| = |U_f.n| + a_f (+ 2 mu/(rho_f d_f))
 * at the face average Q_f = (Q_i + Q_ip)/2; boundary faces fold into the diagonal. */
int orc_jacobian(orc_mesh *m, const orc_params *p, const double *Q, const double *dt,
                 double *diag, double *off) {
  for (int64_t i = 0; i < m->nc; i++) {
    double *D = diag + 25 * i;
    for (int k = 0; k < 25; k++) D[k] = (k % 6 == 0) ? m->vol[i] / dt[i] : 0.0;
    for (int q = 0; q < m->nfc; q++) {
      double n[3], J[25], Qf[5], pf[5];
      outward(m, i, q, n);
      int64_t f = m->cface[m->nfc * i + q], j = m->cnb[m->nfc * i + q];
      double S = m->farea[f];
      for (int c = 0; c < 5; c++) Qf[c] = j >= 0 ? 0.5 * (Q[5 * i + c] + Q[5 * j + c]) : Q[5 * i + c];
      orc_primitive(Qf, p->gamma, pf);
      double pres = pf[0] / (2.0 * pf[4]), a = sqrt(p->gamma * pres / pf[0]);
      double lam = fabs(pf[1] * n[0] + pf[2] * n[1] + pf[3] * n[2]) + a;
      if (p->viscous) {
        double df;
        if (j >= 0) {
          double s2 = 0.0;
          for (int d = 0; d < 3; d++) { double t = m->cen[3 * i + d] - (m->cen[3 * j + d] + m->cshift[3 * m->nfc * i + 3 * q + d]); s2 += t * t; }
          df = sqrt(s2);
        } else {
          double s = 0.0;
          double fc[3];
          for (int d = 0; d < 3; d++) fc[d] = m->fcen[3 * f + d] - (m->cside[m->nfc * i + q] == 1 ? m->fshift[3 * f + d] : 0.0);
          for (int d = 0; d < 3; d++) s += (fc[d] - m->cen[3 * i + d]) * n[d];
          df = 2.0 * fabs(s);
        }
        lam += 2.0 * p->mu / (pf[0] * df);
      }
      orc_euler_jacobian(Q + 5 * i, n, p->gamma, J);
      for (int k = 0; k < 25; k++) D[k] += 0.5 * (J[k] + (k % 6 == 0 ? lam : 0.0)) * S;
      double *O = off + 25 * m->nfc * i + 25 * q;
      if (j >= 0) {
        orc_euler_jacobian(Q + 5 * j, n, p->gamma, J);
        for (int k = 0; k < 25; k++) O[k] = 0.5 * (J[k] - (k % 6 == 0 ? lam : 0.0)) * S;
      } else for (int k = 0; k < 25; k++) O[k] = 0.0;
    }
  }
  return 0;
}

void orc_apply_A(const orc_mesh *m, const double *diag, const double *off, const double *x, double *y) {
  for (int64_t i = 0; i < m->nc; i++)
    for (int r = 0; r < 5; r++) {
      double s = 0.0;
      for (int c = 0; c < 5; c++) s += diag[25 * i + 5 * r + c] * x[5 * i + c];
      for (int q = 0; q < m->nfc; q++) {
        int64_t j = m->cnb[m->nfc * i + q];
        if (j < 0) continue;
        for (int c = 0; c < 5; c++) s += off[25 * m->nfc * i + 25 * q + 5 * r + c] * x[5 * j + c];
      }
      y[5 * i + r] = s;
    }
}

/* Eq. (precond): b^0 = D^{-1} b, b^k = D^{-1}(b - (L+U) b^{k-1}), k = 1..sweeps */
int orc_precondition(const orc_mesh *m, const double *diag, const double *off, int sweeps,
                     const double *b, double *x) {
  const int64_t nc = m->nc;
  double *Dinv = (double *)malloc(sizeof(double) * 25 * (nc + 1)), *prev = (double *)malloc(sizeof(double) * 5 * (nc + 1));
  for (int64_t i = 0; i < nc; i++) if (orc_inverse(5, diag + 25 * i, Dinv + 25 * i)) { free(Dinv); free(prev); return -1; }
  for (int64_t i = 0; i < nc; i++)
    for (int r = 0; r < 5; r++) { double s = 0.0; for (int c = 0; c < 5; c++) s += Dinv[25 * i + 5 * r + c] * b[5 * i + c]; x[5 * i + r] = s; }
  for (int k = 1; k <= sweeps; k++) {
    memcpy(prev, x, sizeof(double) * 5 * nc);
    for (int64_t i = 0; i < nc; i++) {
      double t[5];
      for (int r = 0; r < 5; r++) {
        double s = b[5 * i + r];
        for (int q = 0; q < m->nfc; q++) {
          int64_t j = m->cnb[m->nfc * i + q];
          if (j < 0) continue;
          for (int c = 0; c < 5; c++) s -= off[25 * m->nfc * i + 25 * q + 5 * r + c] * prev[5 * j + c];
        }
        t[r] = s;
      }
      for (int r = 0; r < 5; r++) { double s = 0.0; for (int c = 0; c < 5; c++) s += Dinv[25 * i + 5 * r + c] * t[c]; x[5 * i + r] = s; }
    }
  }
  free(Dinv); free(prev);
  return 0;
}

static double dot(int64_t n, const double *a, const double *b) { double s = 0.0; for (int64_t i = 0; i < n; i++) s += a[i] * b[i]; return s; }

/* Matrix-free product with the implicit operator of Eq. (impEuler):
 * A = |Omega|/dt I - dL/dQ, where dL/dQ x is replaced by the Frechet difference
 * of Eq. (frechet), (L(Q + sigma x) - L(Q)) / sigma, with the step's dt and G
 * held fixed. The paper leaves sigma to the user; the reading taken is
 * sigma = sqrt(eps_mach) (1 + ||Q||_2) / ||x||_2. x = 0 gives y = 0. */
int orc_apply_fd(orc_mesh *m, const orc_params *p, const double *Q, const double *G, const double *dt,
                 const double *LQ, const double *x, double *y, double *sigma_out) {
  const int64_t nc = m->nc, n = 5 * nc;
  const double nx = sqrt(dot(n, x, x)), nq = sqrt(dot(n, Q, Q));
  if (nx == 0.0) {
    for (int64_t k = 0; k < n; k++) y[k] = 0.0;
    if (sigma_out) *sigma_out = 0.0;
    return 0;
  }
  const double sigma = sqrt(DBL_EPSILON) * (1.0 + nq) / nx;
  double *Qs = (double *)malloc(sizeof(double) * (n + 1)), *Ls = (double *)malloc(sizeof(double) * (n + 1));
  for (int64_t k = 0; k < n; k++) Qs[k] = Q[k] + sigma * x[k];
  int rc = orc_residual_dt(m, p, Qs, G, dt, Ls, NULL, NULL, 0);
  if (!rc)
    for (int64_t i = 0; i < nc; i++)
      for (int c = 0; c < 5; c++) {
        const int64_t k = 5 * i + c;
        y[k] = m->vol[i] / dt[i] * x[k] - (Ls[k] - LQ[k]) / sigma;
      }
  if (sigma_out) *sigma_out = sigma;
  free(Qs); free(Ls);
  return rc;
}

static int apply_op(const orc_mesh *m, const double *diag, const double *off, const orc_params *p,
                    const orc_fd_ctx *fd, const double *x, double *y) {
  if (fd && p->jv_mode == 1) return orc_apply_fd(fd->m, p, fd->Q, fd->G, fd->dt, fd->LQ, x, y, NULL);
  orc_apply_A(m, diag, off, x, y);
  return 0;
}

/* Restarted GMRES on P^{-1} A x = P^{-1} rhs from x = 0 with modified
 * Gram-Schmidt Arnoldi, Algorithm 1; hist[restart] = ||P^{-1} r0||. */
int orc_gmres(const orc_mesh *m, const double *diag, const double *off, const orc_params *p,
              const double *rhs, double *dx, double *hist) {
  return orc_gmres_fd(m, diag, off, p, NULL, rhs, dx, hist);
}

/* the same; with jv_mode 1 every product with A is the matrix-free one, while
 * the preconditioner keeps the assembled approximate A (Eq. (precond)) */
int orc_gmres_fd(const orc_mesh *m, const double *diag, const double *off, const orc_params *p,
                 const orc_fd_ctx *fd, const double *rhs, double *dx, double *hist) {
  const int64_t n = 5 * m->nc;
  const int mk = p->krylov_dim;
  double *V = (double *)malloc(sizeof(double) * n * (mk + 1)), *w = (double *)malloc(sizeof(double) * (n + 1)),
         *r = (double *)malloc(sizeof(double) * (n + 1)), *t = (double *)malloc(sizeof(double) * (n + 1));
  double *H = (double *)calloc((mk + 1) * mk, sizeof(double));
  memset(dx, 0, sizeof(double) * n);
  int rc = 0;
  for (int it = 0; it < p->restarts; it++) {
    if (apply_op(m, diag, off, p, fd, dx, t)) { rc = -1; break; }
    for (int64_t k = 0; k < n; k++) t[k] = rhs[k] - t[k];
    if (orc_precondition(m, diag, off, p->jacobi_sweeps, t, r)) { rc = -1; break; }
    double beta = sqrt(dot(n, r, r));
    if (hist) hist[it] = beta;
    if (beta == 0.0) break;
    for (int64_t k = 0; k < n; k++) V[k] = r[k] / beta;
    memset(H, 0, sizeof(double) * (mk + 1) * mk);
    int used = 0;
    for (int j = 0; j < mk; j++) {
      if (apply_op(m, diag, off, p, fd, V + n * j, t)) { rc = -1; break; }
      orc_precondition(m, diag, off, p->jacobi_sweeps, t, w);
      for (int i = 0; i <= j; i++) {
        double h = dot(n, w, V + n * i);
        H[i * mk + j] = h;
        for (int64_t k = 0; k < n; k++) w[k] -= h * V[n * i + k];
      }
      double hn = sqrt(dot(n, w, w));
      H[(j + 1) * mk + j] = hn;
      used = j + 1;
      if (hn == 0.0) break;
      for (int64_t k = 0; k < n; k++) V[n * (j + 1) + k] = w[k] / hn;
    }
    if (rc) break;
    /* minimise || beta e1 - H y || by Givens rotations, then back substitution */
    double *gvec = (double *)calloc(mk + 1, sizeof(double)), *y = (double *)calloc(mk + 1, sizeof(double));
    gvec[0] = beta;
    for (int j = 0; j < used; j++) {
      double a = H[j * mk + j], b = H[(j + 1) * mk + j], rr = sqrt(a * a + b * b);
      double c = a / rr, s = b / rr;
      for (int k = j; k < used; k++) {
        double h1 = H[j * mk + k], h2 = H[(j + 1) * mk + k];
        H[j * mk + k] = c * h1 + s * h2;
        H[(j + 1) * mk + k] = -s * h1 + c * h2;
      }
      double g1 = gvec[j], g2 = gvec[j + 1];
      gvec[j] = c * g1 + s * g2; gvec[j + 1] = -s * g1 + c * g2;
    }
    for (int j = used - 1; j >= 0; j--) {
      double s = gvec[j];
      for (int k = j + 1; k < used; k++) s -= H[j * mk + k] * y[k];
      y[j] = s / H[j * mk + j];
    }
    for (int j = 0; j < used; j++) for (int64_t k = 0; k < n; k++) dx[k] += y[j] * V[n * j + k];
    free(gvec); free(y);
  }
  free(V); free(w); free(r); free(t); free(H);
  return rc;
}

static double density_res(const orc_mesh *m, const double *R) {
  double s = 0.0;
  for (int64_t i = 0; i < m->nc; i++) s += fabs(R[5 * i]) / m->vol[i];
  return s / (double)m->nc;
}

/* One pass of Algorithm 1's outer loop: time step, residual (and f^n-driven
 * gradients), A, GMRES, update. res = L1 density residual of the input state. */
int orc_gmres_step(orc_mesh *m, const orc_params *p, double *Q, double *G, double *res, double *dQ_out) {
  const int64_t nc = m->nc;
  double *dt = (double *)malloc(sizeof(double) * (nc + 1)), *R = (double *)malloc(sizeof(double) * 5 * (nc + 1));
  double *Gn = p->scheme == 1 ? (double *)malloc(sizeof(double) * 15 * (nc + 1)) : NULL;
  double *diag = (double *)malloc(sizeof(double) * 25 * (nc + 1)), *off = (double *)malloc(sizeof(double) * 25 * m->nfc * (nc + 1));
  double *dQ = (double *)malloc(sizeof(double) * 5 * (nc + 1));
  int rc = orc_local_dt(m, p, Q, dt);
  if (!rc) rc = orc_residual(m, p, Q, G, R, Gn, NULL, 0);
  if (!rc) {
    if (res) *res = density_res(m, R);
    orc_jacobian(m, p, Q, dt, diag, off);
    orc_fd_ctx fd = {m, Q, G, dt, R};
    rc = orc_gmres_fd(m, diag, off, p, &fd, R, dQ, NULL);
  }
  if (!rc) {
    for (int64_t k = 0; k < 5 * nc; k++) Q[k] += dQ[k];
    if (Gn) {
      /* Algorithm 1: G^{n+1} = G_new; optionally under-relaxed, G += a (G_new - G) */
      const double a = p->grad_relax > 0.0 ? p->grad_relax : 1.0;
      if (a == 1.0) memcpy(G, Gn, sizeof(double) * 15 * nc);
      else for (int64_t k = 0; k < 15 * nc; k++) G[k] += a * (Gn[k] - G[k]);
    }
    if (dQ_out) memcpy(dQ_out, dQ, sizeof(double) * 5 * nc);
  }
  free(dt); free(R); free(Gn); free(diag); free(off); free(dQ);
  return rc;
}

/* Algorithm 1: iterate while res/res_ref > drop (the printed loop test is
 * inverted); res_ref is the largest residual seen so far (a flow started from
 * rest has a zero density residual at its first step, and while every residual
 * seen is zero there is no drop to measure). hist[k] = res of the
 * k-th state. Returns 0 if converged, 1 if the step limit was reached, < 0 on
 * error. */
int orc_solve_steady(orc_mesh *m, const orc_params *p, double *Q, double *G, double drop,
                     int max_steps, double *hist, int *steps_out) {
  const int64_t nc = m->nc;
  double *R = (double *)malloc(sizeof(double) * 5 * (nc + 1));
  double res0 = 0.0;
  int k = 0, rc = 1;
  for (;; k++) {
    if (orc_residual(m, p, Q, G, R, NULL, NULL, 0)) { rc = -1; break; }
    double res = density_res(m, R);
    if (hist) hist[k] = res;
    if (res > res0) res0 = res;
    if (res0 > 0.0 && res <= drop * res0) { rc = 0; break; }   /* a zero reference certifies no drop */
    if (k >= max_steps) { rc = 1; break; }
    double r2;
    if (orc_gmres_step(m, p, Q, G, &r2, NULL)) { rc = -1; break; }
  }
  if (steps_out) *steps_out = k;
  free(R);
  return rc;
}

/* Threads of the OpenMP loops (timing the oracle single-threaded and on all
 * cores); returns the previous maximum. */
int orc_set_threads(int n) {
  int prev = omp_get_max_threads();
  if (n > 0) omp_set_num_threads(n);
  return prev;
}
