/*
 * hgks.h -- C ABI of libhgks: the residual R(U) and the Jacobi-preconditioned
 * restarted GMRES step of the implicit high-order gas-kinetic scheme (HGKS)
 * on 3-D tetrahedral meshes (Yang, Pan, Xu, "Implicit high-order gas-kinetic
 * schemes for compressible flows on three-dimensional unstructured meshes I:
 * steady flows"), on one NVIDIA GB300 (sm_103a).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns an hgks_status; 0 (HGKS_OK) is success. No
 *    function throws, aborts or exits. hgks_last_error() returns a
 *    thread-local, NUL-terminated description of the last failure.
 *  - Argument errors are reported synchronously. Device-side failures are
 *    reported by the first later call that synchronises (hgks_gmres_step,
 *    hgks_solve_steady, the *_host variants, hgks_sync).
 *  - A mesh handle owns all device memory it needs (geometry, stencils,
 *    reconstruction matrices, Jacobian blocks, Krylov basis, scratch). The
 *    caller owns the state arrays Q, G, R, G_new: device pointers unless the
 *    name ends in _host.
 *  - Cells are held in the library's internal order (a space-filling curve on
 *    the cell centroids). hgks_mesh_create() returns perm_out[internal] =
 *    caller cell index; every device array passed to the library is in the
 *    internal order.
 *  - Device state layouts are component-major ("structure of arrays"):
 *      Q, R  : double[5][N]  conservative (rho, rho U, rho V, rho W, rho E)
 *      G     : double[15][N] cell-averaged Cartesian gradients,
 *              G[3*c + d][i] = d Q_c / d x_d  (compact scheme only)
 *  - R is L(Q) of Eq. (semi)/(finite): |Omega_i| dQ_i/dt, NOT divided by the
 *    cell volume; the face flux is the time average of Sec. 4.1.
 *  - Work is enqueued on the caller's CUDA stream (cudaStream_t passed as
 *    void*; NULL is the legacy default stream). Calls on one mesh handle must
 *    not overlap: the handle's scratch is shared.
 *  - Devices: a call makes the device of its mesh (batch, server) current
 *    while it runs and makes the caller's current device current again before
 *    it returns, so the calling thread's current device is unchanged. The
 *    stream passed must belong to that device.
 */
#ifndef HGKS_H
#define HGKS_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HGKS_OK = 0,
  HGKS_ERR_ARG = 1,          /* invalid argument (NULL, size, parameter)          */
  HGKS_ERR_MESH = 2,         /* degenerate tet, unmatched or over-shared face,
                                singular reconstruction stencil                  */
  HGKS_ERR_CUDA = 3,         /* a CUDA call failed                                 */
  HGKS_ERR_OOM = 4,          /* device allocation failed                           */
  HGKS_ERR_NONPHYSICAL = 5,  /* non-finite residual or non-positive cell state     */
  HGKS_ERR_BREAKDOWN = 6,    /* reserved                                           */
  HGKS_ERR_NOT_CONVERGED = 7,/* hgks_solve_steady reached max_steps                */
  HGKS_ERR_TIMEOUT = 8,      /* reserved                                           */
  HGKS_ERR_CANCELLED = 9     /* a server request cancelled with hgks_server_cancel */
} hgks_status;

/* boundary tags of hgks_mesh_create (paper Sec. 5.1, 5.2) */
enum {
  HGKS_BC_WALL_ISO = 1,       /* isothermal no-slip wall at rest                   */
  HGKS_BC_WALL_LID = 2,       /* isothermal no-slip wall moving with lid_speed +x   */
  HGKS_BC_SLIP = 3,           /* adiabatic slip wall                                */
  HGKS_BC_NOSLIP_ADIA = 4,    /* adiabatic no-slip wall                             */
  HGKS_BC_FARFIELD = 5        /* far field (free stream)                            */
};

enum { HGKS_WENO = 0, HGKS_HWENO = 1 };           /* non-compact / compact (Sec. 3.2, 3.3) */
enum { HGKS_NONLINEAR = 0, HGKS_LINEAR = 1 };     /* weights of Eq. (weno)                 */
enum { HGKS_FP64 = 0, HGKS_MIXED = 1 };           /* Krylov arithmetic                     */

typedef struct hgks_mesh_s *hgks_mesh;            /* opaque */

/* Plain-old-data parameters, copied by every call. Defaults (paper Sec. 3.4,
 * Sec. 4, Sec. 5): scheme WENO, nonlinear weights, characteristic variables,
 * Krylov 10, 3 restarts, 2 Jacobi sweeps, gamma 1.4, Pr 1, CFL 10,
 * tau_eps 0.1, tau_C 1, lin_weight 0.025, weno_eps 1e-6 (the paper leaves the
 * epsilon of Eq. (weno) open: Jiang and Shu's value); see hgks_default_params().
 *
 * Flow conditions. The paper states its problems by Mach number, Reynolds
 * number and angle of attack (Sec. 5.1, 5.2). With Mach > 0 the library derives
 * the free stream, the wall temperature and the viscosity from Mach, Re and
 * aoa_deg, and the explicit fields rho_inf, u_inf, p_inf, wall_T, mu and
 * viscous are ignored (reference length 1: the cavity's side, the sphere's
 * diameter):
 *   external flow (lid_speed == 0, Sec. 5.2): (rho, U, V, W, p) =
 *     (1, Mach cos a, Mach sin a, 0, 1/gamma) with a = aoa_deg in the x-y
 *     plane; wall_T = 1/gamma; mu = Mach / Re;
 *   lid-driven cavity (lid_speed > 0, Sec. 5.1): fluid at rest, rho = 1,
 *     p = lid_speed^2 / (gamma Mach^2) (Mach of the lid), wall_T = p;
 *     mu = lid_speed / Re;
 *   Re > 0 makes the flow viscous (tau = mu/p + ...), Re == 0 inviscid.
 * With Mach == 0 (the default) the explicit fields are used as given, which
 * serves states that no Mach number describes (tests, far-field states of
 * other problems). Mach, Re < 0 or a non-finite aoa_deg are HGKS_ERR_ARG. */
typedef struct {
  int32_t scheme;          /* HGKS_WENO | HGKS_HWENO                                  */
  int32_t weights;         /* HGKS_NONLINEAR | HGKS_LINEAR                            */
  int32_t viscous;         /* 0: tau = eps dt + C|dp|dt, 1: tau = mu/p + C|dp|dt (Sec. 5) */
  int32_t characteristic;  /* 1: reconstruct characteristic variables (Sec. 5), 0: conservative */
  int32_t precision;       /* HGKS_FP64 | HGKS_MIXED (FP32 Krylov basis, Arnoldi, Jacobi) */
  int32_t jv_mode;         /* 0: products with the assembled approximate A (Eq. (deri-matrix));
                              1: matrix-free products (Eq. (frechet), hgks_apply_jacobian_fd),
                              the Jacobi preconditioner still from the assembled A; single
                              meshes only (batches and servers take 0)                  */
  int32_t krylov_dim;      /* Arnoldi steps per restart, 1..64                        */
  int32_t restarts;        /* GMRES cycles per implicit step                          */
  int32_t jacobi_sweeps;   /* k_max of Eq. (precond)                                  */
  int32_t tstar_end;       /* compact gradients from f at t = dt_flux (1) or t = 0 (0) */
  double gamma;            /* specific heat ratio                                     */
  double Pr;               /* Prandtl number (energy-flux fix; 1 = plain BGK)         */
  double mu;               /* dynamic viscosity (constant)                            */
  double cfl;              /* CFL of the implicit pseudo-time step                    */
  double flux_cfl;         /* CFL of the time step used inside the gas-kinetic flux   */
  double tau_eps, tau_C;   /* collision time constants of Sec. 5                      */
  double lin_weight;       /* linear weight gamma_m of every sub-stencil              */
  double weno_eps;         /* epsilon of the nonlinear weights (default 1e-6)         */
  double flux_dt;          /* > 0: fixed time step inside the flux (overrides flux_cfl) */
  double rho_inf, u_inf[3], p_inf;  /* free stream (far field)                        */
  double wall_T;           /* isothermal wall temperature p/rho                       */
  double lid_speed;        /* speed of HGKS_BC_WALL_LID walls along +x                */
  double Mach;             /* > 0: derive the flow conditions (above); 0: explicit    */
  double Re;               /* Reynolds number (0: inviscid) when Mach > 0             */
  double aoa_deg;          /* angle of attack in degrees (x-y plane) when Mach > 0    */
  double grad_relax;       /* compact scheme: G^{n+1} = G^n + grad_relax (G_new - G^n);
                              1 (the default) or 0: Algorithm 1's G^{n+1} = G_new;
                              values in (0, 1) under-relax the update (an option the
                              paper does not have); outside [0, 1]: HGKS_ERR_ARG      */
} hgks_params;

typedef struct {
  int64_t n_cells, n_faces, n_boundary_faces;
  int64_t device_bytes;      /* device memory held by the handle */
  int32_t device;
  int32_t schemes;           /* bit 0: WENO data present, bit 1: HWENO data present */
  int32_t faces_per_cell;    /* 4: tetrahedra, 6: hexahedra */
  int32_t reserved;
} hgks_mesh_info_t;

typedef struct {
  double res_l1;             /* L1 norm of the density residual of the input state (Sec. 5) */
  double lin_res[2];         /* preconditioned linear residual before/after GMRES          */
  int32_t krylov_iters;      /* Arnoldi steps performed                                     */
  int32_t nonphysical;       /* count of Gauss-point states that fell back to cell averages */
} hgks_step_info;

typedef struct {
  int32_t steps;             /* implicit steps taken                                       */
  int32_t converged;         /* 1 if res/res_ref <= drop_tol                                */
  double res_ref;            /* largest density residual seen (the drop reference)         */
  double res_final;
} hgks_solve_info;

/* Fill *p with the defaults listed above. */
hgks_status hgks_default_params(hgks_params *p);

/* Build a mesh on `device` (paper Sec. 3.1, 4.3: cells, faces, stencils and the
 * per-cell reconstruction matrices of Eq. (polys), (compact-big-1/2)).
 *  xyz[n_vert][3]      vertex coordinates (host, copied)
 *  tet4[n_tet][4]      vertex indices of every tetrahedron (host, copied);
 *                      local face p is the triangle opposite local vertex p
 *  bface3[n_bface][3], btag[n_bface]  boundary triangles and their HGKS_BC_* tags
 *  periodic_shift[n_periodic][3]      translations pairing the remaining faces
 *                      (NULL / 0 if none)
 *  scheme_mask         bit 0: build WENO data, bit 1: build HWENO data
 *  perm_out[n_tet]     (host, may be NULL) internal index -> caller index
 * The non-compact big stencil is the face neighbours and their neighbours,
 * widened ring by ring to 12 cells near boundaries and then, while its
 * quadratic fit is singular (a regular grid's wall cells), by the neighbours
 * of its cells up to 16 (24 around a hexahedron).
 * Errors: HGKS_ERR_ARG (n_tet <= 0, NULL arrays), HGKS_ERR_MESH (degenerate or
 * non-conforming mesh, a stencil whose fit stays singular, or fewer than 9
 * other cells reachable for the non-compact fit, e.g. a mesh of under 10
 * cells), HGKS_ERR_CUDA/OOM. */
hgks_status hgks_mesh_create(const double *xyz, int64_t n_vert, const int64_t *tet4, int64_t n_tet,
                             const int64_t *bface3, const int32_t *btag, int64_t n_bface,
                             const double *periodic_shift, int32_t n_periodic, int32_t scheme_mask,
                             int32_t device, hgks_mesh *out, int64_t *perm_out);
/* The same for a hexahedral mesh (paper Sec. 3.1: six faces per cell, the
 * eight non-compact sub-stencils of three face neighbours across each corner,
 * one compact sub-stencil per face).
 *  hex8[n_hex][8]      vertex indices: 0-3 one quadrilateral in cyclic order,
 *                      4 + a the vertex joined to a; positively oriented
 *                      ((x1 - x0) x (x3 - x0)) . (x4 - x0) > 0; local faces
 *                      0 = 0123, 1 = 0154, 2 = 1265, 3 = 2376, 4 = 3047, 5 = 4567
 *  bquad4[n_bface][4]  boundary quadrilaterals (any cyclic vertex order)
 * A cell is the trilinear map of the unit cube; a face the bilinear surface
 * through its vertices, with area and normal from its vector area and 2 x 2
 * Gauss points weighted by the area element (exact for planar faces). Meshes
 * of hexahedra run through the single-mesh calls (residual, Jacobian, GMRES
 * step, solves, matrix-free products, hgks_residual_noalloc), through batches
 * of hexahedral meshes (hgks_batch_create, hgks_batch_create_empty_hex) and
 * through servers made by hgks_server_create_hex: a batch or a server holds one
 * cell kind (HGKS_ERR_ARG otherwise). Errors as hgks_mesh_create, and
 * HGKS_ERR_MESH for an inverted hexahedron (Jacobian determinant <= 0 at a
 * Gauss point). */
hgks_status hgks_mesh_create_hex(const double *xyz, int64_t n_vert, const int64_t *hex8, int64_t n_hex,
                                 const int64_t *bquad4, const int32_t *btag, int64_t n_bface,
                                 const double *periodic_shift, int32_t n_periodic, int32_t scheme_mask,
                                 int32_t device, hgks_mesh *out, int64_t *perm_out);
hgks_status hgks_mesh_destroy(hgks_mesh mesh);
hgks_status hgks_mesh_info(hgks_mesh mesh, hgks_mesh_info_t *info);
/* Cell volumes in internal order, into a host array of n_cells doubles. */
hgks_status hgks_mesh_volumes(hgks_mesh mesh, double *vol_host);

/* Residual R = L(Q) (Eq. (finite) with the time-averaged flux of Sec. 4.1):
 * reconstruction (Sec. 3.2/3.3 in characteristic variables, Sec. 5), the BGK
 * flux of Eq. (flux) at the Gauss points of every face (3 on a triangle, 2 x 2
 * on a quadrilateral), face-to-cell accumulation;
 * compact scheme: G_new = cell-averaged gradients from the point values of
 * Eq. (point) by Eq. (derivative). G and G_new are NULL for WENO.
 * All pointers are device pointers in internal order. */
hgks_status hgks_residual(hgks_mesh mesh, const hgks_params *p, const double *Q, const double *G,
                          double *R, double *G_new, void *cuda_stream);

/* Local time step dt[N] (device) at CFL p->cfl: dt_i = CFL |Omega_i| /
 * sum_p S_p (|U_i.n_p| + a_i + 2 gamma mu/(Pr rho_i h_i)) (the paper gives no
 * formula; this is the reading the library takes). */
hgks_status hgks_local_dt(hgks_mesh mesh, const hgks_params *p, const double *Q, double *dt,
                          void *cuda_stream);

/* Assemble A of Eq. (A-system-2) with Eq. (deri-matrix) at state Q and
 * time step dt (device arrays), into the handle. If diag_out / off_out are not
 * NULL they receive the blocks (device, double[25][N] and double[F][25][N] with
 * F = faces_per_cell of hgks_mesh_info (4 or 6), row-major 5x5, off block p
 * multiplies the neighbour across local face p; zero on boundary faces). */
hgks_status hgks_assemble(hgks_mesh mesh, const hgks_params *p, const double *Q, const double *dt,
                          double *diag_out, double *off_out, void *cuda_stream);
/* y = A x with the assembled A (device double[5][N]). */
hgks_status hgks_apply_jacobian(hgks_mesh mesh, const double *x, double *y, void *cuda_stream);
/* y = A x without A (Eq. (frechet)): y = |Omega|/dt x - (L(Q + sigma x) - L(Q)) / sigma
 * with sigma = sqrt(eps_mach) (1 + ||Q||_2) / ||x||_2 (y = 0 for x = 0), L evaluated
 * with the given time step dt and gradients G held fixed (G NULL for WENO). All
 * arrays device, internal order, [5][N] (dt [N]). Uses the handle's scratch. */
hgks_status hgks_apply_jacobian_fd(hgks_mesh mesh, const hgks_params *p, const double *Q, const double *G,
                                   const double *dt, const double *x, double *y, void *cuda_stream);
/* Force of the flow on the boundary faces tagged `tag` (HGKS_BC_*): the sum over
 * those faces of the momentum part of the face flux of Eq. (flux) times the face
 * area, i.e. pressure and viscous stress on the wall, in the global frame, into
 * force_host[3] (host). Evaluates R(Q) on the way (the handle's scratch);
 * synchronises the stream. Drag coefficient of a body: force . e_U / (rho U^2 A / 2). */
hgks_status hgks_wall_force(hgks_mesh mesh, const hgks_params *p, const double *Q, const double *G, int32_t tag,
                            double *force_host, void *cuda_stream);
/* x = P^{-1} b, Jacobi iteration of Eq. (precond) with `sweeps` sweeps. */
hgks_status hgks_precondition(hgks_mesh mesh, int32_t sweeps, const double *b, double *x,
                              void *cuda_stream);

/* One pass of Algorithm 1's outer loop: time step, R(Q) (and G_new), A,
 * `restarts` cycles of left-preconditioned GMRES(krylov_dim) with modified
 * Gram-Schmidt (Algorithm 1's coefficients up to rounding: an FP64 basis is
 * taken two vectors per pass, an FP32 basis from one pass with its Gram
 * matrix), Q += dQ, and G = G_new for the compact scheme. Q, G are device
 * arrays updated in place; dQ_out (device, may be NULL) receives the update.
 * Synchronises the stream (to return info->res_l1). */
hgks_status hgks_gmres_step(hgks_mesh mesh, const hgks_params *p, double *Q, double *G,
                            double *dQ_out, hgks_step_info *info, void *cuda_stream);

/* Algorithm 1 until res/res_ref <= drop_tol (res_ref = largest density
 * residual seen) or max_steps steps. hist_host (may be NULL) receives
 * max_steps + 1 residuals. Returns HGKS_ERR_NOT_CONVERGED if the limit was hit. */
hgks_status hgks_solve_steady(hgks_mesh mesh, const hgks_params *p, double *Q, double *G,
                              double drop_tol, int32_t max_steps, double *hist_host,
                              hgks_solve_info *info, void *cuda_stream);

/* Resume Algorithm 1 from a snapshot: Q, G the state a solve stopped with (for
 * example copied to the host and back) and *from its hgks_solve_info (steps
 * taken, res_ref). The solve continues counting steps from from->steps up to
 * max_steps with the same drop reference, so it reproduces the uninterrupted
 * solve's iterates bit for bit. hist_host (may be NULL) is indexed by the
 * absolute step (max_steps + 1 entries). */
hgks_status hgks_solve_resume(hgks_mesh mesh, const hgks_params *p, double *Q, double *G, double drop_tol,
                              int32_t max_steps, const hgks_solve_info *from, double *hist_host,
                              hgks_solve_info *info, void *cuda_stream);

/* Host-buffer variants: Q, G (and R, G_new) are host arrays in internal order
 * and layout above; the copies to and from the device happen inside the call
 * on the given stream, which is synchronised before return. */
hgks_status hgks_residual_host(hgks_mesh mesh, const hgks_params *p, const double *Q_host,
                               const double *G_host, double *R_host, double *G_new_host,
                               void *cuda_stream);
hgks_status hgks_gmres_step_host(hgks_mesh mesh, const hgks_params *p, double *Q_host,
                                 double *G_host, hgks_step_info *info, void *cuda_stream);

/* hgks_residual with no memory allocation of its own. The paper has no
 * counterpart: this serves callers that cannot call cudaMalloc once they are
 * running (for example a process whose device memory is handed out by another
 * runtime at start-up, or a service that must not enter the CUDA allocator while
 * it answers requests). The mesh is still created up front with
 * hgks_mesh_create; this call leaves the handle's own scratch untouched and uses
 * one fixed array of 32 MiB compiled into the library instead. Meshes larger
 * than that array allows (about 10,000 tetrahedra: 106 N + 150 F doubles; about
 * 5,000 hexahedra: 166 N + 200 F) are rejected with HGKS_ERR_ARG. Arguments, checks, layouts and results are those of
 * hgks_residual (the same kernels: the results are identical).
 * Set-up: under CUDA's lazy module loading (the default) the driver allocates
 * the array on a device when the first call of this entry point on that device
 * loads it, and that call also looks up the array's device address
 * (cudaGetSymbolAddress) with the device current. Make the first call on each
 * device at start-up, before any stream capture and before device memory is
 * handed to another runtime; from then on the device holds the array until the
 * process exits and no call allocates or frees anything. All calls share the one
 * array and it keeps the previous call's contents: calls that may overlap on the
 * GPU (several streams or host threads) race with each other. */
hgks_status hgks_residual_noalloc(hgks_mesh mesh, const hgks_params *p, const double *Q, const double *G,
                                  double *R, double *G_new, void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Batches: many independent steady problems advanced together, one kernel
 * launch per phase (reconstruction, flux, assembly, each Arnoldi step) for all
 * of them. Each mesh keeps its own parameters, state, Krylov space, Hessenberg
 * least-squares problem and convergence test, so a mesh follows Algorithm 1
 * exactly as it does alone (the only difference is the summation order inside
 * inner products). The paper solves one problem at a time; batching is this
 * library's way of filling one GPU with problems smaller than it.
 * ------------------------------------------------------------------------- */
typedef struct hgks_batch_s *hgks_batch;          /* opaque */

typedef struct {
  int64_t n_cells;           /* cells of the merged cell space, padding included      */
  int64_t n_faces;
  int64_t device_bytes;      /* device memory held by the batch                        */
  int32_t n_meshes;
  int32_t blk_recon, blk_flux;  /* launch shapes in use (hgks_batch_autotune)          */
} hgks_batch_info_t;

/* Merge n_meshes meshes (handles of one device) into a batch, with params[k]
 * for mesh k (copied). The batch holds its own copy of every mesh's device
 * data, so the handles may be destroyed afterwards. Mesh k's cells occupy a
 * range of the merged cell space that starts on a multiple of 256; the cells
 * between ranges are inert padding. scheme, precision, jv_mode, krylov_dim,
 * restarts and jacobi_sweeps must agree across params; the rest (gamma, Pr,
 * mu, viscous, cfl, free stream, walls, weights ...) may differ per mesh.
 * State starts at zero: set it with hgks_batch_set_state. Errors: HGKS_ERR_ARG
 * (n_meshes < 1 or > 32767, NULL, disagreeing parameters, a mesh built without
 * the scheme's data, meshes on different devices, tetrahedral and hexahedral
 * meshes mixed: a batch holds one cell kind), HGKS_ERR_OOM, HGKS_ERR_CUDA. */
hgks_status hgks_batch_create(const hgks_mesh *meshes, const hgks_params *params, int32_t n_meshes,
                              hgks_batch *out);
hgks_status hgks_batch_destroy(hgks_batch batch);
/* n_meshes counts the slots in use; n_cells and n_faces are the arena's capacities. */
hgks_status hgks_batch_info(hgks_batch batch, hgks_batch_info_t *info);

/* An empty batch: an arena of cell_capacity cells and face_capacity faces with
 * max_meshes slots, for meshes whose params agree with *shared in the fields
 * listed above (shared->scheme decides which reconstruction data it holds);
 * it holds tetrahedra (hgks_batch_create_empty_hex below: hexahedra).
 * Device memory: about 8 KB per cell and 1.3 KB per face (FP64, Krylov 10). */
hgks_status hgks_batch_create_empty(int32_t device, int64_t cell_capacity, int64_t face_capacity,
                                    int32_t max_meshes, const hgks_params *shared, hgks_batch *out);
/* The same arena for hexahedral meshes (add them with hgks_batch_add). */
hgks_status hgks_batch_create_empty_hex(int32_t device, int64_t cell_capacity, int64_t face_capacity,
                                        int32_t max_meshes, const hgks_params *shared, hgks_batch *out);
/* Place a mesh (copied; the handle stays the caller's) in a free slot and in
 * free cell and face ranges (first fit); *k_out receives the slot, the index
 * every other hgks_batch_* call takes. HGKS_ERR_OOM if no slot or range is
 * free (nothing changes then); HGKS_ERR_ARG for a mesh of the other cell kind. */
hgks_status hgks_batch_add(hgks_batch batch, hgks_mesh mesh, const hgks_params *p, int32_t *k_out);
/* Free slot k and its ranges; later launches skip them. */
hgks_status hgks_batch_remove(hgks_batch batch, int32_t k);

/* Copy the state of the mesh in slot k in (set) or out (get). Q, R: device double[5][N_k], G,
 * G_new: device double[15][N_k] (compact scheme; NULL otherwise), in mesh k's
 * internal order, N_k its cell count. Any pointer of get_state may be NULL;
 * R and G_new are those of the last hgks_batch_residual / step. */
hgks_status hgks_batch_set_state(hgks_batch batch, int32_t k, const double *Q, const double *G,
                                 void *cuda_stream);
hgks_status hgks_batch_get_state(hgks_batch batch, int32_t k, double *Q, double *G, double *R,
                                 double *G_new, void *cuda_stream);

/* R(Q) (and G_new) of every mesh of the batch, as hgks_residual does for one. */
hgks_status hgks_batch_residual(hgks_batch batch, void *cuda_stream);

/* One outer step of Algorithm 1 for every mesh (as hgks_gmres_step).
 * info (host, may be NULL) receives n_meshes records. With use_graph != 0 the
 * step's launches are replayed from a CUDA graph captured at the first such
 * call (and again when the arena's shapes change); the results are the same
 * bit for bit. Synchronises the stream. */
hgks_status hgks_batch_gmres_step(hgks_batch batch, hgks_step_info *info, int32_t use_graph, void *cuda_stream);

/* Algorithm 1 for every mesh until each has converged (res/res_ref <= drop_tol,
 * as hgks_solve_steady) or taken max_steps steps; a finished mesh is skipped
 * by every later launch and keeps its state. The convergence test runs on the
 * device, so the step's launch sequence is fixed: with use_graph != 0 it is
 * captured once in a CUDA graph (on a stream owned by the batch, ordered after
 * the caller's stream) and replayed. hist_host (may be NULL) receives
 * n_meshes x (max_steps + 1) residuals, row k for mesh k (0 past its last
 * step); info (host) n_meshes records. Returns HGKS_ERR_NOT_CONVERGED if any
 * mesh hit max_steps, HGKS_ERR_NONPHYSICAL if any residual was not finite. */
hgks_status hgks_batch_solve_steady(hgks_batch batch, double drop_tol, int32_t max_steps, int32_t use_graph,
                                    double *hist_host, hgks_solve_info *info, void *cuda_stream);

/* Time the reconstruction and flux kernels of this batch's current state at
 * block sizes 64, 128 and 256 (CUDA events, 3 runs each) and keep the fastest
 * for later calls; the chosen sizes are returned (may be NULL). */
hgks_status hgks_batch_autotune(hgks_batch batch, int32_t *blk_recon, int32_t *blk_flux, void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Request server: continuous batching of steady solves on one GPU. Requests
 * arrive at any time; a host thread builds each mesh (stencils, reconstruction
 * matrices) in arrival order; every hgks_server_step() admits built requests,
 * in arrival order, while the server's batch arena (sized from the HBM budget)
 * has a free slot and free ranges for them, advances every running solve by
 * one step of Algorithm 1 in one batched launch sequence (a replayed CUDA
 * graph), and retires the solves that converged or reached their step limit.
 * A solve gives the same result as alone (hgks_solve_steady with the same
 * parameters) up to the summation order of its inner products.
 * ------------------------------------------------------------------------- */
typedef struct hgks_server_s *hgks_server;          /* opaque */

typedef struct {
  int32_t state;             /* 0 waiting for its build, 1 built, 2 running, 3 finished, 4 failed */
  int32_t status;            /* HGKS_OK (converged), HGKS_ERR_NOT_CONVERGED, _NONPHYSICAL, or the build error */
  int64_t n_cells;
  hgks_solve_info solve;     /* steps, converged, res_ref, res_final (once finished)         */
  double t_submit, t_built, t_admit, t_done;   /* seconds since the server was created       */
} hgks_request_info;

/* A server on `device` whose arena takes at most hbm_budget_bytes of device
 * memory, with at most max_inflight solves running at once; every request's
 * params must agree with *shared in scheme, precision, jv_mode, krylov_dim,
 * restarts and jacobi_sweeps. use_graph != 0 replays the step from a CUDA graph. */
hgks_status hgks_server_create(int32_t device, int64_t hbm_budget_bytes, int32_t max_inflight,
                               const hgks_params *shared, int32_t use_graph, hgks_server *out);
/* The same for hexahedral meshes (a server takes one cell kind; submit them
 * with hgks_server_submit_hex). */
hgks_status hgks_server_create_hex(int32_t device, int64_t hbm_budget_bytes, int32_t max_inflight,
                                   const hgks_params *shared, int32_t use_graph, hgks_server *out);
/* Stops the build thread and frees everything, finished or not. */
hgks_status hgks_server_destroy(hgks_server server);
/* Queue a steady solve. Mesh arrays as hgks_mesh_create (host, copied); Q0
 * (host, caller cell order, double[n_tet][5]) the initial state, G0 (may be
 * NULL: zero) double[n_tet][15] the initial gradients of the compact scheme;
 * the solve stops at res/res_ref <= drop_tol or after max_steps steps.
 * *id_out receives the request's id. HGKS_ERR_ARG if the mesh cannot fit in
 * the arena at all. */
hgks_status hgks_server_submit(hgks_server server, const double *xyz, int64_t n_vert, const int64_t *tet4,
                               int64_t n_tet, const int64_t *bface3, const int32_t *btag, int64_t n_bface,
                               const double *periodic_shift, int32_t n_periodic, const hgks_params *p,
                               const double *Q0, const double *G0, double drop_tol, int32_t max_steps,
                               int64_t *id_out);
/* A hexahedral request (mesh arrays as hgks_mesh_create_hex) to a server made by
 * hgks_server_create_hex; HGKS_ERR_ARG on a tetrahedral server (and
 * hgks_server_submit on a hexahedral one). */
hgks_status hgks_server_submit_hex(hgks_server server, const double *xyz, int64_t n_vert, const int64_t *hex8,
                                   int64_t n_hex, const int64_t *bquad4, const int32_t *btag, int64_t n_bface,
                                   const double *periodic_shift, int32_t n_periodic, const hgks_params *p,
                                   const double *Q0, const double *G0, double drop_tol, int32_t max_steps,
                                   int64_t *id_out);
/* One scheduling round (admit, one batched step, retire). Outputs (may be
 * NULL): solves finished in this round, solves running, requests waiting
 * (for their build, in it, or for admission: zero running and zero waiting
 * means every request submitted so far has finished).
 * Drive the rounds from one thread; submit, status, cancel and collect may be
 * called from any thread meanwhile. */
hgks_status hgks_server_step(hgks_server server, int32_t *n_finished, int32_t *n_running, int32_t *n_waiting);
hgks_status hgks_server_status(hgks_server server, int64_t id, hgks_request_info *info);
/* Cancel a request: one waiting for its build or for admission is dropped at
 * once, one running leaves at the start of the next round with its current
 * state (collectable); either way it finishes with status HGKS_ERR_CANCELLED.
 * Cancelling a finished request does nothing. */
hgks_status hgks_server_cancel(hgks_server server, int64_t id);
/* Copy a finished request's state (host, caller order: Q double[n][5], G
 * double[n][15] or NULL) and forget the request. */
hgks_status hgks_server_collect(hgks_server server, int64_t id, double *Q, double *G);
/* The server's arena (n_meshes = solves running). */
hgks_status hgks_server_info(hgks_server server, hgks_batch_info_t *info);

/* Wait for the stream and report any deferred device-side error. */
hgks_status hgks_sync(void *cuda_stream);

/* Per-kernel timing with CUDA events recorded on the launching stream around
 * every kernel the library enqueues between hgks_profile_begin() and
 * hgks_profile_end(). end() waits for the events and fills, for up to
 * max_kernels kernels that ran: names (32 bytes each, NUL-terminated),
 * total_ms and launches; *n_out = number of distinct kernels. Host state is
 * per process; profile one stream at a time. */
hgks_status hgks_profile_begin(void);
hgks_status hgks_profile_end(int32_t max_kernels, char *names, double *total_ms, int64_t *launches,
                             int32_t *n_out);

/* Measured FP64 arithmetic rate of `device` in GFLOP/s (the roofline the
 * FP64-bound kernels are held against): independent double-precision FMA
 * chains (x <- x a + b, 2 flops each) in every thread of one full wave of
 * resident blocks, no memory traffic, timed with CUDA events on a stream of the
 * library's own; *gflops_out = the best of 10 launches of about seconds/10
 * each. Not part of the paper's method. Errors: HGKS_ERR_ARG (NULL, seconds
 * outside (0, 60], no such device), HGKS_ERR_CUDA/OOM. */
hgks_status hgks_fp64_peak(int32_t device, double seconds, double *gflops_out);

/* Kernel launches made by this thread since the last reset (profiling aid). */
int64_t hgks_launch_count(int32_t reset);

const char *hgks_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
