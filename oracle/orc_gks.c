/* ORACLE (test infrastructure only): the gas-kinetic (BGK) flux of Sec. 2.
 *
 * Maxwellian g of Eq. (bgk) with N = (5 - 3 gamma)/(gamma - 1) internal degrees
 * of freedom; moments <...> = int g (...) dXi factorise into u, v, w and xi
 * parts. Every integrand is written as an explicit polynomial in
 * (u, v, w, xi^2) and integrated term by term; the 5x5 moment systems for the
 * slopes are solved by Gaussian elimination. The flux is the time average over
 * [0, dt] of int u psi f dXi with f from Eq. (flux), Sec. 4.1. */
#include <math.h>
#include <string.h>
#include "orc.h"

#define MAXT 512
typedef struct { int n; double c[MAXT]; unsigned char e[MAXT][4]; } poly;  /* e: powers of u, v, w, xi^2 */
typedef struct { double rho, mu[9], mv[9], mw[9], mxi[3]; } mtable;

static void p_zero(poly *p) { p->n = 0; }
static void p_term(poly *p, double c, int iu, int iv, int iw, int ix) {
  if (c == 0.0) return;
  p->c[p->n] = c; p->e[p->n][0] = iu; p->e[p->n][1] = iv; p->e[p->n][2] = iw; p->e[p->n][3] = ix; p->n++;
}
/* psi = (1, u, v, w, (u^2 + v^2 + w^2 + xi^2)/2) */
static void p_psi(poly *p, int a) {
  p_zero(p);
  switch (a) {
    case 0: p_term(p, 1.0, 0, 0, 0, 0); break;
    case 1: p_term(p, 1.0, 1, 0, 0, 0); break;
    case 2: p_term(p, 1.0, 0, 1, 0, 0); break;
    case 3: p_term(p, 1.0, 0, 0, 1, 0); break;
    default: p_term(p, 0.5, 2, 0, 0, 0); p_term(p, 0.5, 0, 2, 0, 0); p_term(p, 0.5, 0, 0, 2, 0); p_term(p, 0.5, 0, 0, 0, 1);
  }
}
/* a . psi for a coefficient vector a[5] */
static void p_dot_psi(poly *p, const double *a) {
  p_zero(p);
  p_term(p, a[0], 0, 0, 0, 0); p_term(p, a[1], 1, 0, 0, 0); p_term(p, a[2], 0, 1, 0, 0); p_term(p, a[3], 0, 0, 1, 0);
  p_term(p, 0.5 * a[4], 2, 0, 0, 0); p_term(p, 0.5 * a[4], 0, 2, 0, 0); p_term(p, 0.5 * a[4], 0, 0, 2, 0); p_term(p, 0.5 * a[4], 0, 0, 0, 1);
}
static void p_mul(const poly *a, const poly *b, poly *r) {
  p_zero(r);
  for (int i = 0; i < a->n; i++)
    for (int j = 0; j < b->n; j++)
      p_term(r, a->c[i] * b->c[j], a->e[i][0] + b->e[j][0], a->e[i][1] + b->e[j][1], a->e[i][2] + b->e[j][2], a->e[i][3] + b->e[j][3]);
}
static void p_add(poly *r, const poly *a, double s) {
  for (int i = 0; i < a->n; i++) p_term(r, s * a->c[i], a->e[i][0], a->e[i][1], a->e[i][2], a->e[i][3]);
}
/* (a . u_vec) = u (a_n . psi) + v (a_t1 . psi) + w (a_t2 . psi), for the three directional slopes */
static void p_slope_dot_u(poly *r, const double a[3][5]) {
  poly t, x, s;
  p_zero(r);
  for (int d = 0; d < 3; d++) {
    p_dot_psi(&t, a[d]);
    p_zero(&x); p_term(&x, 1.0, d == 0, d == 1, d == 2, 0);
    p_mul(&x, &t, &s);
    p_add(r, &s, 1.0);
  }
}
static double p_int(const poly *p, const mtable *T) {
  double s = 0.0;
  for (int i = 0; i < p->n; i++) s += p->c[i] * T->mu[p->e[i][0]] * T->mv[p->e[i][1]] * T->mw[p->e[i][2]] * T->mxi[p->e[i][3]];
  return T->rho * s;
}
/* int g (poly) psi dXi, as a 5-vector */
static void p_int_psi(const poly *p, const mtable *T, double *out) {
  poly ps, pr;
  for (int a = 0; a < 5; a++) { p_psi(&ps, a); p_mul(p, &ps, &pr); out[a] = p_int(&pr, T); }
}

void orc_primitive(const double *Q, double gamma, double *prim) {
  double rho = Q[0], U = Q[1] / rho, V = Q[2] / rho, W = Q[3] / rho;
  double p = (gamma - 1.0) * (Q[4] - 0.5 * rho * (U * U + V * V + W * W));
  prim[0] = rho; prim[1] = U; prim[2] = V; prim[3] = W; prim[4] = rho / (2.0 * p);
}

/* Moments of the normalised Maxwellian: full range (range 0), u > 0 (range +1)
 * or u < 0 (range -1) in u; v, w always full range. */
void orc_uvw_moments(double rho, double U, double V, double W, double lam, double K, int range,
                     double *mu, double *mv, double *mw, double *mxi) {
  (void)rho;
  if (range == 0) { mu[0] = 1.0; mu[1] = U; }
  else {
    double sl = sqrt(lam), ex = 0.5 * exp(-lam * U * U) / sqrt(M_PI * lam);
    if (range > 0) { mu[0] = 0.5 * erfc(-sl * U); mu[1] = U * mu[0] + ex; }
    else { mu[0] = 0.5 * erfc(sl * U); mu[1] = U * mu[0] - ex; }
  }
  mv[0] = 1.0; mv[1] = V; mw[0] = 1.0; mw[1] = W;
  for (int n = 0; n + 2 <= 8; n++) {
    mu[n + 2] = U * mu[n + 1] + (n + 1) / (2.0 * lam) * mu[n];
    mv[n + 2] = V * mv[n + 1] + (n + 1) / (2.0 * lam) * mv[n];
    mw[n + 2] = W * mw[n + 1] + (n + 1) / (2.0 * lam) * mw[n];
  }
  mxi[0] = 1.0; mxi[1] = K / (2.0 * lam); mxi[2] = (K * K + 2.0 * K) / (4.0 * lam * lam);
}
static void table(const double *prim, double K, int range, mtable *T) {
  T->rho = prim[0];
  orc_uvw_moments(prim[0], prim[1], prim[2], prim[3], prim[4], K, range, T->mu, T->mv, T->mw, T->mxi);
}
double orc_monomial_moment(const double *prim, double K, int range, int iu, int iv, int iw, int ixi) {
  mtable T; table(prim, K, range, &T);
  return T.rho * T.mu[iu] * T.mv[iv] * T.mw[iw] * T.mxi[ixi];
}

/* Solve <a> = int g (a . psi) psi dXi = dQ for the slope coefficients a. */
int orc_slope(const double *prim, double K, const double *dQ, double *a) {
  mtable T; table(prim, K, 0, &T);
  double M[25];
  poly pa, pb, pr;
  for (int i = 0; i < 5; i++)
    for (int j = 0; j < 5; j++) { p_psi(&pa, i); p_psi(&pb, j); p_mul(&pa, &pb, &pr); M[i * 5 + j] = p_int(&pr, &T); }
  return orc_lu_solve(5, M, dQ, a);
}
/* Time slope A from <a_n u + a_t1 v + a_t2 w + A> = 0 */
static void time_slope(const double *prim, double K, const double a[3][5], double *A) {
  mtable T; table(prim, K, 0, &T);
  poly pau; double rhs[5];
  p_slope_dot_u(&pau, a);
  p_int_psi(&pau, &T, rhs);
  for (int i = 0; i < 5; i++) rhs[i] = -rhs[i];
  orc_slope(prim, K, rhs, A);
}

void orc_gks_flux(const orc_params *p, const double *Wl, const double *dWl, const double *Wr,
                  const double *dWr, double dt, double *F, double *Qpt) {
  const double g = p->gamma, K = (5.0 - 3.0 * g) / (g - 1.0);
  double pl[5], pr[5], p0[5];
  orc_primitive(Wl, g, pl);
  orc_primitive(Wr, g, pr);
  mtable Tlp, Trm, Tl, Tr, T0;
  table(pl, K, +1, &Tlp); table(pr, K, -1, &Trm); table(pl, K, 0, &Tl); table(pr, K, 0, &Tr);
  /* compatibility: Q0 = int_{u>0} psi g_l + int_{u<0} psi g_r */
  double Q0[5];
  poly ps, one; p_zero(&one); p_term(&one, 1.0, 0, 0, 0, 0);
  for (int a = 0; a < 5; a++) { p_psi(&ps, a); Q0[a] = p_int(&ps, &Tlp) + p_int(&ps, &Trm); }
  orc_primitive(Q0, g, p0);
  table(p0, K, 0, &T0);
  /* spatial slopes (n, t1, t2) of g_l, g_r and of the equilibrium g0 */
  double al[3][5], ar[3][5], ab[3][5], Al[5], Ar[5], Ab[5];
  for (int d = 0; d < 3; d++) {
    double dQ0[5];
    orc_slope(pl, K, dWl + 5 * d, al[d]);
    orc_slope(pr, K, dWr + 5 * d, ar[d]);
    for (int c = 0; c < 5; c++) dQ0[c] = 0.5 * (dWl[5 * d + c] + dWr[5 * d + c]);
    orc_slope(p0, K, dQ0, ab[d]);
  }
  time_slope(pl, K, al, Al);
  time_slope(pr, K, ar, Ar);
  time_slope(p0, K, ab, Ab);
  /* collision time, Sec. 5 */
  double prl = pl[0] / (2.0 * pl[4]), prr = pr[0] / (2.0 * pr[4]), pp0 = p0[0] / (2.0 * p0[4]);
  double jump = fabs((prl - prr) / (prl + prr));
  double tau = p->viscous ? p->mu / pp0 + p->tau_C * jump * dt : p->tau_eps * dt + p->tau_C * jump * dt;
  double e = exp(-dt / tau);
  double c1 = dt - tau * (1.0 - e);
  double c2 = 2.0 * tau * tau * (1.0 - e) - tau * dt * (1.0 + e);
  double c3 = 0.5 * dt * dt - tau * dt + tau * tau * (1.0 - e);
  double c4 = tau * (1.0 - e);
  double c5 = 2.0 * tau * tau * (1.0 - e) - tau * dt * e;
  /* polynomials: u, (abar . u_vec), Abar . psi, and the same for l and r */
  poly pu, pabu, pAb, palu, pAl, paru, pAr, tmp;
  p_zero(&pu); p_term(&pu, 1.0, 1, 0, 0, 0);
  p_slope_dot_u(&pabu, ab); p_dot_psi(&pAb, Ab);
  p_slope_dot_u(&palu, al); p_dot_psi(&pAl, Al);
  p_slope_dot_u(&paru, ar); p_dot_psi(&pAr, Ar);
  /* moments without the u factor (point values, time averages) */
  double m0[5], mab[5], mAb[5], ml[5], mal[5], mAl[5], mr[5], mar[5], mAr[5];
  p_int_psi(&one, &T0, m0); p_int_psi(&pabu, &T0, mab); p_int_psi(&pAb, &T0, mAb);
  p_int_psi(&one, &Tlp, ml); p_int_psi(&palu, &Tlp, mal); p_int_psi(&pAl, &Tlp, mAl);
  p_int_psi(&one, &Trm, mr); p_int_psi(&paru, &Trm, mar); p_int_psi(&pAr, &Trm, mAr);
  /* moments with the u factor (fluxes) */
  double f0[5], fab[5], fAb[5], fl[5], fal[5], fAl[5], fr[5], far_[5], fAr[5];
  p_int_psi(&pu, &T0, f0);
  p_mul(&pu, &pabu, &tmp); p_int_psi(&tmp, &T0, fab);
  p_mul(&pu, &pAb, &tmp); p_int_psi(&tmp, &T0, fAb);
  p_int_psi(&pu, &Tlp, fl);
  p_mul(&pu, &palu, &tmp); p_int_psi(&tmp, &Tlp, fal);
  p_mul(&pu, &pAl, &tmp); p_int_psi(&tmp, &Tlp, fAl);
  p_int_psi(&pu, &Trm, fr);
  p_mul(&pu, &paru, &tmp); p_int_psi(&tmp, &Trm, far_);
  p_mul(&pu, &pAr, &tmp); p_int_psi(&tmp, &Trm, fAr);
  for (int a = 0; a < 5; a++)
    F[a] = (c1 * f0[a] + c2 * fab[a] + c3 * fAb[a]
            + c4 * fl[a] - c5 * fal[a] - tau * c4 * fAl[a]
            + c4 * fr[a] - c5 * far_[a] - tau * c4 * fAr[a]) / dt;
  if (p->Pr != 1.0) {
    /* Prandtl-number fix: energy flux += (1/Pr - 1) q, with q the heat flux of
     * the time-averaged distribution relative to the velocity of Q0 */
    double Wb[5];
    for (int a = 0; a < 5; a++)
      Wb[a] = (c1 * m0[a] + c2 * mab[a] + c3 * mAb[a] + c4 * ml[a] - c5 * mal[a] - tau * c4 * mAl[a]
               + c4 * mr[a] - c5 * mar[a] - tau * c4 * mAr[a]) / dt;
    double U = p0[1], V = p0[2], W = p0[3], q2 = U * U + V * V + W * W;
    double q = F[4] - (U * F[1] + V * F[2] + W * F[3]) + 0.5 * q2 * F[0] - U * Wb[4]
               + U * (U * Wb[1] + V * Wb[2] + W * Wb[3]) - 0.5 * U * q2 * Wb[0];
    F[4] += (1.0 / p->Pr - 1.0) * q;
  }
  if (Qpt) {
    /* Eq. (point) at t* = dt (or 0): macroscopic values of the evolved f */
    double ts = p->tstar_end ? dt : 0.0, es = exp(-ts / tau);
    for (int a = 0; a < 5; a++)
      Qpt[a] = (1.0 - es) * m0[a] + ((ts + tau) * es - tau) * mab[a] + (ts - tau + tau * es) * mAb[a]
               + es * (ml[a] - (tau + ts) * mal[a] - tau * mAl[a])
               + es * (mr[a] - (tau + ts) * mar[a] - tau * mAr[a]);
  }
}

/* Boundary state on the outer side of a boundary face, in the face frame
 * (x along the outward normal). Walls mirror the interior state through the
 * wall in primitive variables (p, U, V, W, T = p/rho): quantities even under
 * the reflection keep their value and flip their normal derivative; odd ones
 * (about the wall value) are reflected and keep their normal derivative. At an
 * isothermal wall the image's density is the one that sends back as much mass
 * as reaches the wall (its pressure follows from it); walls carry no mass
 * (orc_solver.c). The far field is the free stream with zero slopes. */
void orc_boundary_state(const orc_params *p, int tag, const double *T3, const double *Wl,
                        const double *dWl, double *Wr, double *dWr) {
  const double g = p->gamma;
  if (tag == 5) {
    double r = p->rho_inf, u[3];
    for (int i = 0; i < 3; i++) u[i] = T3[3 * i] * p->u_inf[0] + T3[3 * i + 1] * p->u_inf[1] + T3[3 * i + 2] * p->u_inf[2];
    Wr[0] = r; Wr[1] = r * u[0]; Wr[2] = r * u[1]; Wr[3] = r * u[2];
    Wr[4] = p->p_inf / (g - 1.0) + 0.5 * r * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (int i = 0; i < 15; i++) dWr[i] = 0.0;
    return;
  }
  /* interior primitive state and derivatives */
  double rho = Wl[0], u[3] = {Wl[1] / rho, Wl[2] / rho, Wl[3] / rho};
  double q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  double pr = (g - 1.0) * (Wl[4] - 0.5 * rho * q2), T = pr / rho;
  double du[3][3], dp[3], dT[3];
  for (int d = 0; d < 3; d++) {
    const double *dW = dWl + 5 * d;
    double udu = 0.0;
    for (int i = 0; i < 3; i++) { du[d][i] = (dW[1 + i] - u[i] * dW[0]) / rho; udu += u[i] * du[d][i]; }
    dp[d] = (g - 1.0) * (dW[4] - 0.5 * dW[0] * q2 - rho * udu);
    dT[d] = (dp[d] - T * dW[0]) / rho;
  }
  double uw[3] = {0, 0, 0};
  if (tag == 2) for (int i = 0; i < 3; i++) uw[i] = T3[3 * i] * p->lid_speed;
  int vel_odd[3], T_odd = (tag == 1 || tag == 2);
  double ug[3], Tg, pg = pr;
  if (tag == 3) { vel_odd[0] = 1; vel_odd[1] = 0; vel_odd[2] = 0; }
  else { vel_odd[0] = vel_odd[1] = vel_odd[2] = 1; }
  for (int i = 0; i < 3; i++) ug[i] = vel_odd[i] ? 2.0 * uw[i] - u[i] : u[i];
  Tg = T_odd ? 2.0 * p->wall_T - T : T;
  /* a cell hotter than 1.5 T_w would give an image colder than T_w / 2 (or
     negative): the image temperature is held at T_w / 2, uniform */
  int T_held = T_odd && Tg < 0.5 * p->wall_T;
  if (T_held) Tg = 0.5 * p->wall_T;
  double dug[3][3], dpg[3], dTg[3];
  for (int d = 0; d < 3; d++) {
    double sn = d == 0 ? -1.0 : 1.0;   /* even: flip the normal derivative */
    for (int i = 0; i < 3; i++) dug[d][i] = vel_odd[i] ? -sn * du[d][i] : sn * du[d][i];
    dpg[d] = sn * dp[d];
    dTg[d] = T_held ? 0.0 : (T_odd ? -sn * dT[d] : sn * dT[d]);
  }
  double rg = pg / Tg, qg2 = ug[0] * ug[0] + ug[1] * ug[1] + ug[2] * ug[2];
  if (T_odd) {
    /* an isothermal wall lets no mass through: the image emits toward the fluid as
       many particles as the cell sends into the wall (half-range Maxwellians, no
       slopes): rho_g <u>_{u>0}(U_n, T_g) = rho <u>_{u>0}(U_n, T) with the image's
       normal velocity -U_n; its pressure follows, p_g = rho_g T_g */
    double Un = u[0], Ml, Mg;
    double lam_l = 1.0 / (2.0 * T), lam_g = 1.0 / (2.0 * Tg);
    Ml = 0.5 * Un * erfc(-sqrt(lam_l) * Un) + 0.5 * exp(-lam_l * Un * Un) / sqrt(M_PI * lam_l);
    Mg = 0.5 * Un * erfc(-sqrt(lam_g) * Un) + 0.5 * exp(-lam_g * Un * Un) / sqrt(M_PI * lam_g);
    rg = rho * Ml / Mg;
    double ratio = rg * Tg / pr;   /* the image keeps the cell's relative pressure gradient */
    pg = rg * Tg;
    for (int d = 0; d < 3; d++) dpg[d] *= ratio;
  }
  Wr[0] = rg; Wr[1] = rg * ug[0]; Wr[2] = rg * ug[1]; Wr[3] = rg * ug[2];
  Wr[4] = pg / (g - 1.0) + 0.5 * rg * qg2;
  for (int d = 0; d < 3; d++) {
    double drho = dpg[d] / Tg - pg * dTg[d] / (Tg * Tg), udu = 0.0;
    for (int i = 0; i < 3; i++) udu += ug[i] * dug[d][i];
    dWr[5 * d] = drho;
    for (int i = 0; i < 3; i++) dWr[5 * d + 1 + i] = drho * ug[i] + rg * dug[d][i];
    dWr[5 * d + 4] = dpg[d] / (g - 1.0) + 0.5 * drho * qg2 + rg * udu;
  }
}
