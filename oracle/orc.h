/*
 * ORACLE for the implicit high-order gas-kinetic scheme (HGKS) on tetrahedra
 * and hexahedra.
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow, FP64 CPU restatement of the
 * paper's method, written to check the CUDA library against. Only tests/,
 * __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm may load
 * it. It shares no code with the CUDA library, and the library never calls it.
 *
 * Every routine names the passage it follows: Eq. (bgk), (semi), (finite),
 * (flux), (polys), (compact-big-1/2), (point), (derivative), (weno),
 * (impEuler), (impsystem), (A-system-1/2), (deri-matrix), (precond), the
 * algorithm "preconditioned GMRES" (Algorithm 1), and Sec. 5's collision time
 * and characteristic-variable reconstruction. Where the paper is silent the
 * oracle takes the same readings as the library, each stated where it is used.
 *
 * Data layout is the natural one for a reader: cell arrays are [cell][5] in the
 * caller's cell order, gradients [cell][5][3] (component, then direction).
 * Cells are tetrahedra or hexahedra (Sec. 3.1: four or six faces).
 *
 * Parity unpinned: the local time step (orc_local_dt) beyond its scaling
 * invariants, since the paper gives no formula for it, and the boundary states
 * (orc_boundary_state) beyond their involution, rest-state, wall-symmetry and
 * mass properties and the uniform flows they leave steady (far field, slip
 * walls, moving isothermal walls). Every other routine is pinned by the tests against closed
 * forms, library routines, invariants or brute force.
 */
#ifndef HGKS_ORACLE_H
#define HGKS_ORACLE_H
#include <stdint.h>

#define ORC_MAXF 6       /* faces of a cell: 4 (tetrahedron) or 6 (hexahedron) */
#define ORC_MAXG 4       /* Gauss points of a face: 3 (triangle) or 2 x 2 (quadrilateral) */
#define ORC_MAXSTEN 24   /* non-compact big stencil, excluding the target cell */
#define ORC_MAXSUB 8     /* cells of one sub-stencil, excluding the target cell */
#define ORC_NSUB 8       /* sub-stencils: 4 (tetrahedron) or 8 (hexahedron), Sec. 3.1 */
#define ORC_HCOLS (ORC_MAXF + 3 * (1 + ORC_MAXF))   /* data columns of the compact fit */

typedef struct {
  int32_t scheme;        /* 0: non-compact WENO, 1: compact HWENO           */
  int32_t weights;       /* 0: nonlinear weights, 1: linear weights (omega = gamma) */
  int32_t viscous;       /* 0: Euler collision time, 1: Navier-Stokes        */
  int32_t characteristic;/* 1: reconstruct characteristic variables (Sec. 5) */
  int32_t krylov_dim, restarts, jacobi_sweeps;
  int32_t tstar_end;     /* compact point value at t = dt (1) or t = 0 (0)  */
  int32_t jv_mode;       /* 0: assembled approximate A (Eq. (A-system-2)), 1: matrix-free A x
                            from the Frechet difference of Eq. (frechet)      */
  double gamma, Pr, mu, cfl, flux_cfl; /* flux_cfl: CFL of the time step used inside the flux */
  double tau_eps, tau_C, lin_weight, weno_eps;
  double flux_dt;        /* > 0: fixed time step inside the flux (tests)     */
  double rho_inf, u_inf[3], p_inf; /* far-field state                        */
  double wall_T, lid_speed;        /* isothermal wall temperature p/rho; lid speed along +x */
  double grad_relax;     /* compact: G += grad_relax (G_new - G); 0 or 1: G = G_new (Algorithm 1) */
} orc_params;

typedef struct { int64_t cell; double shift[3]; } orc_sref;

typedef struct {
  /* non-compact (WENO) */
  int n_big;                    orc_sref big[ORC_MAXSTEN];
  double X0[9][ORC_MAXSTEN];    /* a_d = sum_k X0[d][k] (Q_k - Q_0)           */
  int n_sub[ORC_NSUB];          orc_sref sub[ORC_NSUB][ORC_MAXSUB];
  double Xm[ORC_NSUB][3][ORC_MAXSUB];  /* b_j^m = sum_k Xm[m][j][k] (Q_k - Q_0) */
  int sub_valid[ORC_NSUB];
  /* compact (HWENO): data = (Q_k - Q_0 for the face neighbours k, in face order,
     then the gradients of the target and of those neighbours); columns
     [0, nfc) hold the differences, nfc + 3 k + j gradient j of entry k (0 = target) */
  int n_nb;                     orc_sref nb[ORC_MAXF]; int nb_slot[ORC_MAXF];
  double H0[9][ORC_HCOLS];      /* a_d = sum H0[d][col] data[col]              */
  double Hm[ORC_MAXF][3][1 + 6];/* b^m from (Q_m - Q_0, G_0 (3), G_m (3))      */
  int hsub_has_nb[ORC_MAXF];
  int ready_weno, ready_hweno;
} orc_fit;

/* Cells are tetrahedra (nvc 4, nfc 4 faces, ngp 3 Gauss points a face) or
 * hexahedra (nvc 8, nfc 6, ngp 4); every cell array is [nc][nfc]. */
typedef struct {
  int64_t nv, nc, nf;
  double *xyz;                 /* [nv][3] */
  int64_t *cv;                 /* [nc][nvc] cell vertices */
  double *vol, *cen, *h;       /* [nc], [nc][3] volume centroid, [nc] */
  int64_t *cface;              /* [nc][nfc] face across local face p */
  int64_t *cnb;                /* [nc][nfc] neighbour cell, -1 on a boundary */
  double *cshift;              /* [nc][nfc][3] add to the neighbour's coordinates to bring it next to this cell */
  int32_t *cside;              /* [nc][nfc] 0: this cell is the face's left cell, 1: right */
  int64_t *fl, *fr;            /* [nf] left/right cell (fr = -1 on a boundary) */
  int32_t *flp, *frp, *ftag;   /* local face index in left/right; boundary tag (0 interior) */
  double *farea, *fnrm;        /* [nf], [nf][3] unit normal from left to right */
  double *fgp;                 /* [nf][ngp][3] Gauss points, left cell's frame */
  double *fshift;              /* [nf][3] x(left frame) = x(right frame) + shift */
  double *fcen;                /* [nf][3] mean of the face's vertices, left frame */
  orc_fit *fit;                /* [nc], filled on demand */
  int32_t nvc, nfc, ngp, pad;
  double *fgw;                 /* [nf][ngp] Gauss weights of the face (sum 1) */
} orc_mesh;

/* ---- mesh (orc_mesh.c) ---- */
orc_mesh *orc_mesh_create(const double *xyz, int64_t nv, const int64_t *tet, int64_t nc,
                          const int64_t *bface, const int32_t *btag, int64_t nb,
                          const double *pshift, int32_t npshift, char *err, int errlen);
/* cells of nvc = 4 (tetrahedra) or 8 (hexahedra) vertices; boundary faces of
 * nvc == 4 ? 3 : 4 vertices (quadrilaterals in cyclic order) */
orc_mesh *orc_mesh_create_cells(const double *xyz, int64_t nv, const int64_t *cells, int32_t nvc, int64_t nc,
                                const int64_t *bface, const int32_t *btag, int64_t nb,
                                const double *pshift, int32_t npshift, char *err, int errlen);
/* quadrature of cell k exact for its degree-2 integrands: points (global frame)
 * and weights summing to 1; returns the number of points (<= 64) */
int orc_cell_quad(const orc_mesh *m, int64_t k, double (*xq)[3], double *wq);
void orc_mesh_destroy(orc_mesh *m);
int orc_fit_cell(orc_mesh *m, int64_t i, int scheme);   /* 0 ok, <0 error */
/* the non-compact stencils of cell i (which = -1: big stencil, 0..7: sub-stencil) */
int orc_stencil(orc_mesh *m, int64_t i, int which, int64_t *out, int *valid);

/* ---- small dense linear algebra (orc_linalg.c) ---- */
int orc_lu_solve(int n, const double *A, const double *b, double *x);  /* A row-major n x n */
int orc_inverse(int n, const double *A, double *Ainv);
int orc_lsq_pinv(int rows, int cols, const double *A, double *X);    /* X = (cols x rows) least-squares map */
double orc_sv_ratio(int rows, int cols, const double *A);            /* sigma_min / sigma_max of A */

/* ---- gas-kinetic flux (orc_gks.c) ---- */
void orc_uvw_moments(double rho, double U, double V, double W, double lam, double K, int range,
                     double *mu, double *mv, double *mw, double *mxi);
double orc_monomial_moment(const double *prim, double K, int range, int iu, int iv, int iw, int ixi);
int orc_slope(const double *prim, double K, const double *dQ, double *a);
void orc_gks_flux(const orc_params *p, const double *Wl, const double *dWl, const double *Wr,
                  const double *dWr, double dt, double *F, double *Qpt);
void orc_boundary_state(const orc_params *p, int tag, const double *nrm_frame /*3x3 rows n,t1,t2*/,
                        const double *Wl, const double *dWl, double *Wr, double *dWr);
void orc_primitive(const double *Q, double gamma, double *prim /*rho,U,V,W,lambda*/);

/* ---- reconstruction (orc_recon.c) ---- */
void orc_face_frame(const double *n, double *T /*3x3 rows*/);
void orc_char_eigen(const double *Qloc, double gamma, double *R, double *L);
int orc_recon_side(orc_mesh *m, const orc_params *p, const double *Q, const double *G,
                   int64_t cell, int slot, double *Wloc /*[ngp][5]*/, double *dWloc /*[ngp][3][5]*/,
                   double *Wglob /*[ngp][5] or NULL*/, double *gradglob /*[ngp][5][3] or NULL*/);

/* ---- residual and implicit solver (orc_solver.c) ---- */
void orc_euler_jacobian(const double *Q, const double *n, double gamma, double *J);
int orc_local_dt(orc_mesh *m, const orc_params *p, const double *Q, double *dt);
int orc_residual(orc_mesh *m, const orc_params *p, const double *Q, const double *G,
                 double *R, double *Gnew, const int64_t *cells, int64_t ncells);
/* the same with the local time step given (dt_in) instead of computed from Q */
int orc_residual_dt(orc_mesh *m, const orc_params *p, const double *Q, const double *G, const double *dt_in,
                    double *R, double *Gnew, const int64_t *cells, int64_t ncells);
/* force[3] of the flow on the boundary faces with tag `tag` (face fluxes x area) */
int orc_wall_force(orc_mesh *m, const orc_params *p, const double *Q, const double *G, int tag, double *force);
/* y = A x without A: |Omega|/dt x - (L(Q + sigma x) - L(Q)) / sigma (Eq. (frechet)) */
int orc_apply_fd(orc_mesh *m, const orc_params *p, const double *Q, const double *G, const double *dt,
                 const double *LQ, const double *x, double *y, double *sigma_out);
int orc_jacobian(orc_mesh *m, const orc_params *p, const double *Q, const double *dt,
                 double *diag /*[nc][25]*/, double *off /*[nc][nfc][25]*/);
void orc_apply_A(const orc_mesh *m, const double *diag, const double *off, const double *x, double *y);
int orc_precondition(const orc_mesh *m, const double *diag, const double *off, int sweeps,
                     const double *b, double *x);
/* the state a matrix-free product needs (jv_mode 1): Q, G, dt and L(Q) of the step */
typedef struct { orc_mesh *m; const double *Q, *G, *dt, *LQ; } orc_fd_ctx;
int orc_gmres(const orc_mesh *m, const double *diag, const double *off, const orc_params *p,
              const double *rhs, double *dx, double *hist);
int orc_gmres_fd(const orc_mesh *m, const double *diag, const double *off, const orc_params *p,
                 const orc_fd_ctx *fd, const double *rhs, double *dx, double *hist);
int orc_gmres_step(orc_mesh *m, const orc_params *p, double *Q, double *G, double *res,
                   double *dQ_out);
int orc_solve_steady(orc_mesh *m, const orc_params *p, double *Q, double *G, double drop,
                     int max_steps, double *hist, int *steps_out);
int orc_set_threads(int n);   /* OpenMP threads of the loops above; returns the previous maximum */
#endif
