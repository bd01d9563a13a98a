/*
 * sps.h -- C ABI of the GB300 library for collision-resolving suspensions of
 * rigid spheres in Stokes flow (Yan, Corona, Malhotra, Veerapaneni, Shelley,
 * "A scalable computational platform for particulate Stokes suspensions",
 * arXiv 1909.06623).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Viscosity is 1 (Sec. 4.1).  Lengths, forces and times are in the caller's
 *    units.
 *  - Unless a name ends in _host, every array argument is a DEVICE pointer
 *    owned by the caller (for instance a torch CUDA tensor), must stay valid
 *    until the call returns, and is accessed in stream order on the stream
 *    given to sps_create.  Calls return after their work is complete (they read
 *    back convergence scalars), so outputs may be used right away.
 *  - Per-sphere arrays are row-major: pos[i*3 + d], FT[i*6 + k] (force then
 *    torque), UO[i*6 + k] (velocity then angular velocity).
 *  - Surface fields (densities, velocities, tractions) are stored as three
 *    component planes of length NP = N * P, P = (p+1)(2p+2) nodes per sphere:
 *    f[c*NP + i*P + k], node k = ring * (2p+2) + azimuth, rings in ascending
 *    cos(theta) (Gauss-Legendre nodes), azimuth phi_l = 2 pi l / (2p+2).
 *  - Every call returns an sps_status.  On an error nothing is guaranteed
 *    about the outputs except where stated; sps_last_error() describes it.
 *  - The context owns its scratch memory (device buffers sized by the last
 *    geometry) and the contact list.  A context is not thread safe.
 */
#ifndef SPS_H
#define SPS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SPS_OK = 0,
  SPS_ERR_INVALID_ARG = 1,   /* bad size, null pointer, p out of range ...   */
  SPS_ERR_CUDA = 2,          /* a CUDA call failed (message has the reason)  */
  SPS_ERR_OOM = 3,           /* device allocation failed                     */
  SPS_ERR_NOT_CONVERGED = 4, /* an iteration hit its cap; outputs hold the
                                last iterate                                  */
  SPS_ERR_BREAKDOWN = 5,     /* BBPGD step length undefined (s^T y <= 0)     */
  SPS_ERR_CAPACITY = 6,      /* output buffer too small (gamma_cap)          */
  SPS_ERR_NO_GEOMETRY = 7,   /* call needs sps_set_geometry first            */
  SPS_ERR_NONFINITE = 8      /* NaN or Inf met in an input or a residual     */
} sps_status;

/* Arithmetic of the layer operators.  SPS_FP64: FP64 throughout.  SPS_MIXED:
 * FP32 far-field pair sums with compensated totals, BF16-split tensor-core
 * VSH transforms, FP32 / double-float near field, FP64 Krylov and BBPGD.
 * SPS_FP64_DW: the FP64 path with the far-field pair terms in double-float
 * arithmetic on the FP32 pipe (about 2^-46 relative per operation, FP64
 * accumulation per source sphere), agreeing with SPS_FP64 to about 1e-13. */
typedef enum { SPS_FP64 = 0, SPS_MIXED = 1, SPS_FP64_DW = 2 } sps_precision;

/* Mobility used by the solves.  SPS_MOB_BIE is the boundary-integral mobility
 * of Sec. 4.  SPS_MOB_IDENTITY (U = F, Omega = T) is not in the paper: it
 * drops the fluid so that the collision machinery of Sec. 3 (contact search,
 * D, D^T, Algorithm 1) runs alone at sizes where no all-pairs layer sum can;
 * the LCP matrix is then D^T D. */
typedef enum { SPS_MOB_BIE = 0, SPS_MOB_IDENTITY = 1 } sps_mobility;

/* Contact search.  Both give the same list to the bit (the test of Sec. 3.2
 * is evaluated identically); the cell list is O(n) and needs finite positions. */
typedef enum {
  SPS_SEARCH_AUTO = 0,      /* cell list when n > 4096, else all pairs         */
  SPS_SEARCH_ALL_PAIRS = 1, /* every pair i < j                                */
  SPS_SEARCH_CELLS = 2      /* uniform grid of cells of side >= 2 max a_c + delta */
} sps_contact_search;

/* Layer operators of Sec. 4.1 evaluated on all surface nodes. */
typedef enum {
  SPS_OP_S = 0, /* single layer S[sigma](x) = int G(x-y) sigma(y) dS_y         */
  SPS_OP_K = 1, /* traction operator K[sigma](x) = int T(x-y) n(x) sigma(y) dS_y */
  SPS_OP_A = 2  /* (I/2 + K + L)[sigma], the operator of eq. rigidbodyrho      */
} sps_op;

typedef struct sps_params {
  int p;              /* spherical-harmonic order, 1 <= p <= 16 (Sec. 4.2)   */
  double beta;        /* near pair when |c_i-c_j| < beta (a_i+a_j) (Sec. 4.2)*/
  double delta;       /* contact set: Phi <= delta, absolute (Sec. 3.2)       */
  double a_c_scale;   /* collision radius a_c = a_c_scale * a (Sec. 6.1)      */
  double gmres_tol;   /* relative residual of the mobility solve (Sec. 4.1)   */
  int gmres_max;      /* GMRES iteration cap (Krylov basis size)              */
  double bbpgd_tol;   /* min-map residual tolerance eps_tol (eq. mmapnorm)    */
  int bbpgd_max;      /* j_max of Algorithm 1                                 */
  int precision;      /* sps_precision                                        */
  int bb_variant;     /* 1: alpha^BB1, 2: alpha^BB2, 3: BB1 on odd and BB2 on
                         even steps (Algorithm 1)                            */
  double ir_tol;      /* SPS_MIXED: refine against an FP64-accurate residual
                         until ||r||/||b|| < ir_tol (the velocity of a
                         refined solve is then evaluated FP64-accurate too);
                         0 disables refinement                                */
  int ir_max;         /* refinement sweep cap                                 */
  int warm_start;     /* 1: start GMRES from the previous solution where one
                         exists (BBPGD iterates 2.., U_nc of the next step,
                         consecutive sps_mobility_apply / _adjoint calls on
                         suspensions of the same size); 0: zero initial guess.
                         Only the Krylov path changes: every solve still meets
                         gmres_tol.                                           */
  int bb_safeguard;   /* Algorithm 1 defines no step when s^T y <= 0 (BB1) or
                         y^T y <= 0 (BB2): 0 stops with SPS_ERR_BREAKDOWN,
                         1 keeps the previous step length and continues       */
  int mobility;       /* sps_mobility (default SPS_MOB_BIE)                   */
  int contact_search; /* sps_contact_search (default SPS_SEARCH_AUTO)         */
  double delta_rel;   /* relative part of the contact threshold: a pair is in
                         the set when Phi <= delta + delta_rel (a_i + a_j)
                         (a: sphere radii, not collision radii).  Sec. 3.2
                         sets delta to 30% of the sum of the radii: delta = 0,
                         delta_rel = 0.3.  Default 0.                        */
  int bb_warm;        /* Algorithm 1 takes an initial guess gamma_0; the
                         paper's runs use 0.  1: sps_resolve_collisions on
                         the same number of spheres as the previous call
                         starts from the previous step's gamma on the pairs
                         both contact sets share (0 elsewhere); a nonzero
                         gamma_0 costs one more mobility solve (g_0 = M
                         gamma_0 + q) and is dropped for gamma_0 = 0 when its
                         min-map residual is not below that of gamma_0 = 0.
                         Every step still meets bbpgd_tol.  Boundary-integral
                         mobility only (the identity mobility always starts
                         from 0).  2: as 1, and alpha_0 is the last step
                         length of the previous step's converged Algorithm 1
                         instead of g_0^T g_0 / g_0^T M g_0 (one mobility
                         solve fewer; Algorithm 1's alpha_0 when there is
                         none).  Default 0.                                  */
  int ir_dw;          /* the FP64-accurate applications of the refinement
                         (ir_tol > 0): 1 evaluates their far field as
                         SPS_FP64_DW does (double-float on the FP32 pipe), 0
                         in native FP64.  Default 1.                         */
  int lcp_solver;     /* 0: BBPGD (Algorithm 1); 1: APGD, the accelerated
                         projected gradient method Sec. 3.3.1 compares with
                         (Nesterov momentum, an adaptive Lipschitz estimate
                         with a sufficient-decrease test, gradient restart; at
                         least two mobility solves per iteration); 2: the
                         minimum-map Newton method Sec. 3.3.1 names as the
                         second-order alternative (Newton on min(gamma, g)
                         with the step's free block solved by conjugate
                         gradients, one mobility solve per CG iteration, and
                         an Armijo line search; gamma may end with entries
                         down to -bbpgd_tol).  All stop on the min-map
                         residual bbpgd_tol and cap at bbpgd_max (Newton)
                         iterations.  Default 0.                             */
} sps_params;

typedef struct sps_stats {
  int status;           /* sps_status of the call                            */
  int mobility_solves;  /* mobility problems solved (MVOPs + the U_nc solve) */
  int gmres_iters;      /* GMRES iterations summed over solves               */
  int gmres_iters_max;  /* largest per solve                                 */
  int bbpgd_iters;      /* gradient steps of Algorithm 1                     */
  int mvops;            /* evaluations of M gamma (Sec. 6.2)                 */
  int n_contacts;       /* size of the contact set A                         */
  int n_active;         /* contacts with gamma > 0 (the active set A_c)      */
  int n_near_pairs;     /* directed near pairs (i, j), i != j                */
  int ir_sweeps;        /* refinement sweeps (SPS_MIXED with ir_tol > 0);
                           active-set iterations (sps_collision_adjoint)     */
  int bb_safeguards;    /* BBPGD steps that kept the previous step length    */
  long long kernel_launches; /* kernels launched by this call                */
  double final_phi;     /* min-map residual at exit                          */
  double gmres_res_max; /* largest final relative residual over the solves   */
  int layer_applies;    /* layer-operator applications (S, K or I/2 + K + L,
                           forward or transposed) made by this call          */
} sps_stats;

typedef struct sps_ctx sps_ctx;

/* Fills *out with the defaults: p 6, beta 1.75, delta 0.1, a_c_scale 1,
 * gmres 1e-10 / 200, bbpgd 1e-8 / 10000, FP64, BB1, no refinement, warm
 * starts on. */
int sps_default_params(sps_params* out);

/* Creates a context.  stream: a cudaStream_t (NULL = legacy default stream).
 * Errors: INVALID_ARG (p out of range, non-positive tolerances), CUDA, OOM. */
int sps_create(const sps_params* prm, void* stream, sps_ctx** out);
int sps_destroy(sps_ctx* ctx);

/* Human-readable description of the last error on ctx (never NULL). */
const char* sps_last_error(const sps_ctx* ctx);

/* Surface nodes for a geometry: the grid of Sec. 5.4 scaled and centred on
 * each sphere, and the near-pair lists of Sec. 4.2.  n >= 1; pos n x 3, radii n
 * (device).  Radii must be positive.  Keeps its own copy of the geometry. */
int sps_set_geometry(sps_ctx* ctx, int n, const double* pos, const double* radii);

/* Grid orientation (Sec. 5.4 orients every sphere's grid at random).  Q
 * (n x 9, device, row-major Q_i[3 r + c]) holds one rotation per sphere:
 * node k of sphere i then sits at c_i + a_i Q_i n_k with normal Q_i n_k,
 * and the sphere's VSH expansions live in its own frame (densities enter the
 * transforms as Q_i^T sigma, fields leave them as Q_i u).  The orientation
 * stays in force for every later call on n spheres (sps_set_geometry with
 * another count fails with INVALID_ARG) until Q = NULL restores identity
 * grids.  The geometry must be set again afterwards (the solving entry
 * points do that themselves); warm starts are dropped.  The adjoint entry
 * points (sps_layer_apply_transpose, sps_mobility_adjoint,
 * sps_collision_adjoint) return INVALID_ARG while an orientation is set.
 * Errors: INVALID_ARG (n < 1, a matrix not orthogonal to 1e-12 or with
 * determinant <= 0), NONFINITE. */
int sps_set_orientation(sps_ctx* ctx, int n, const double* Q);

/* Nodes of the current geometry: X, normals (3 planes of NP) and quadrature
 * weights (NP), device outputs; any pointer may be NULL.  *np_out = NP. */
int sps_nodes(sps_ctx* ctx, double* X, double* normals, double* weights, int* np_out);

/* Sizes of the current geometry's lists (host outputs, either may be NULL):
 * directed near pairs (i, j), i != j, |c_i - c_j| < beta (a_i + a_j)
 * (Sec. 4.2), and close near entries (target node, near source sphere) within
 * 1.5 source radii, which the mixed path evaluates in FP64.
 * Errors: NO_GEOMETRY before sps_set_geometry. */
int sps_geometry_counts(const sps_ctx* ctx, int* n_near_pairs, int* n_close_entries);

/* The near-pair lists of the current geometry (Sec. 4.2: sphere j is near
 * sphere i when j != i and |c_i - c_j| < beta (a_i + a_j), with
 * d^2 = (dx dx + dy dy) + dz dz and the product beta (a_j + a_i) each rounded
 * once), as CSR by target sphere: near_ptr (N + 1 int32, device output),
 * near_idx (the n_near_pairs of sps_geometry_counts, int32, device output),
 * the sources of sphere i in near_idx[near_ptr[i] .. near_ptr[i+1]), ascending.
 * These pairs take the VSH near evaluation; every other pair takes the far
 * quadrature.  Either pointer may be NULL.  Errors: NO_GEOMETRY. */
int sps_near_lists(sps_ctx* ctx, int* near_ptr, int* near_idx);

/* Layer operator (sps_op) applied to sigma (3 planes of NP, device) on the
 * current geometry; out (3 planes) is overwritten.  Self part: VSH multipliers
 * (Sec. 4.2); near pairs: VSH expansion of the source sphere (Sec. 4.2); all
 * other pairs: direct quadrature (Sec. 5.1).  Precision follows prm.precision
 * (SPS_MIXED: FP32 far field with compensated tile sums). */
int sps_layer_apply(sps_ctx* ctx, int op, const double* sigma, double* out);

/* Contact set of Sec. 3.2 for spheres (pos, radii): all i < j with
 * Phi = |c_i - c_j| - a_c,i - a_c,j <= delta, sorted by (i, j).  Kept in ctx;
 * the count is written to *n_contacts (host int).  Bit-exact definition:
 * d^2 = (dx*dx + dy*dy) + dz*dz rounded after every operation, d = sqrt(d^2),
 * Phi = (d - R_i) - R_j, n = (c_j - c_i) / d. */
int sps_build_contacts(sps_ctx* ctx, int n, const double* pos, const double* radii,
                       int* n_contacts);

/* Planar walls (Sec. 3.3.3: a particle-boundary collision adds a column of D
 * on that particle only; the boundary does not enter the mobility).  walls:
 * HOST array of n_walls rows (n_x, n_y, n_z, d), the plane n . x = d with unit
 * normal n pointing into the fluid; 0 <= n_walls <= 8, n_walls = 0 removes
 * them.  Sphere i and wall w are in the contact set when
 * Phi = (n . c_i - d) - a_c,i <= delta + delta_rel a_i, with
 * n . c = (n_x x + n_y y) + n_z z rounded after every operation; the column
 * carries +n on sphere i, so D^T U = n . U_i.  Every later contact build of
 * the context (sps_build_contacts, the collision steps, both mobilities)
 * includes them; sps_collision_adjoint returns INVALID_ARG while walls are
 * set, and sps_build_contacts_noalloc ignores them.  Errors: INVALID_ARG
 * (count, normal not unit to 1e-12), NONFINITE. */
int sps_set_walls(sps_ctx* ctx, int n_walls, const double* walls);

/* Copies the contact list out: ij (n_c x 2 int32), phi (n_c), normals
 * (n_c x 3); device pointers, any may be NULL.  With walls (sps_set_walls)
 * the sphere pairs come first, sorted by (i, j), then the wall contacts,
 * sorted by (sphere, wall), as rows (-1 - w, i) with the wall's normal. */
int sps_get_contacts(sps_ctx* ctx, int* ij, double* phi, double* normals);

/* D gamma (eq. Dmatdef): FT (n x 6) = force -gamma n on sphere i and
 * +gamma n on sphere j per contact; torques zero.  gamma: n_c (device). */
int sps_contact_force(sps_ctx* ctx, const double* gamma, double* FT);

/* D^T U (eq. Dtranspose): out_l = n_l . (U_j - U_i).  UO: n x 6 (device). */
int sps_contact_rate(sps_ctx* ctx, const double* UO, double* out);

/* Mobility problem of Sec. 4.1: U/Omega (n x 6) from force/torque FT (n x 6)
 * for spheres (pos, radii): rho from FT, GMRES on eq. rigidbodyrho, u = S[rho
 * + zeta] (eq. velS), averages over each sphere.  Sets the geometry.  stats
 * may be NULL.  NOT_CONVERGED leaves the last iterate's velocities in UO. */
int sps_mobility_apply(sps_ctx* ctx, int n, const double* pos, const double* radii,
                       const double* FT, double* UO, sps_stats* stats);

/* One collision-resolved Euler step (Sec. 3.2): U_nc = M F_ext; contact set
 * and D; BBPGD (Algorithm 1) for gamma with M = D^T M D and
 * q = Phi/dt + D^T U_nc; U = U_nc + M D gamma; pos_out = pos + U dt.
 * gamma: capacity gamma_cap (device), receives n_c values (CAPACITY if
 * n_c > gamma_cap, nothing else written); UO (n x 6) and pos_out (n x 3) may
 * alias nothing else; pos_out may be NULL. */
int sps_resolve_collisions(sps_ctx* ctx, int n, const double* pos, const double* radii,
                           const double* FT_ext, double dt, double* gamma, int gamma_cap,
                           double* UO, double* pos_out, sps_stats* stats);

/* `steps` collision-resolved steps of sps_resolve_collisions in a row, the
 * positions advanced in place: pos (n x 3, device) is read and overwritten
 * with the positions after each step; FT_ext (n x 6) acts at every step; UO
 * (n x 6) receives the velocities of the last step.  stats_per_step: HOST
 * array of `steps` sps_stats or NULL.  Stops at the first step whose status
 * is not SPS_OK and returns it (pos then holds that step's update, as
 * sps_resolve_collisions' pos_out would); *steps_done (host, may be NULL)
 * counts the steps completed with SPS_OK.  The multi-step workloads of Sec. 6 (for instance the
 * sedimenting cluster of Sec. 6.3) are this loop. */
int sps_simulate(sps_ctx* ctx, int n, double* pos, const double* radii, const double* FT_ext,
                 double dt, int steps, double* UO, sps_stats* stats_per_step, int* steps_done);

/* Same step with HOST arrays: copies the inputs to the device, runs the step
 * and copies gamma, UO and pos_out back (stream ordered, synchronised before
 * return).  *n_contacts_out receives n_c (host int, may be NULL). */
int sps_resolve_collisions_host(sps_ctx* ctx, int n, const double* pos, const double* radii,
                                const double* FT_ext, double dt, double* gamma, int gamma_cap,
                                double* UO, double* pos_out, int* n_contacts_out,
                                sps_stats* stats);

/* Transpose of a layer operator (sps_op) on the current geometry: out = Op^T v
 * with the Euclidean inner product on the node values (3 planes of NP).  The
 * exact transpose of the discrete operator of sps_layer_apply (same quadrature,
 * VSH maps and near lists), evaluated in FP64.  Used by the adjoint; exposed
 * for checks such as <w, Op v> = <Op^T w, v>.  The paper has no counterpart. */
int sps_layer_apply_transpose(sps_ctx* ctx, int op, const double* v, double* out);

/* Adjoint of sps_mobility_apply.  Given dL/dU (n x 6, device) for a loss L of
 * the velocities U = M F, computes dL/dF (n x 6: force and torque parts) and,
 * if dL_dpos is not NULL, dL/dc (n x 3) for the sphere centres c (radii and
 * the near-pair lists held fixed: the gradient of the discrete map on its
 * current piece).  The forward solve is repeated; its velocities go to UO if
 * UO is not NULL.  Method: lambda = A^{-T} S^T E^T dL/dU (adjoint GMRES on the
 * transpose of eq. rigidbodyrho), dL/dF = R^T (S^T E^T dL/dU - (I/2 + K)^T
 * lambda); dL/dc from the derivatives of the far and near sums (the self, L,
 * rho and averaging steps are translation invariant).  The paper has no
 * adjoint; this is the exact gradient of its discretised mobility map.
 * Errors as sps_mobility_apply; NOT_CONVERGED if either GMRES hit its cap. */
int sps_mobility_adjoint(sps_ctx* ctx, int n, const double* pos, const double* radii,
                         const double* FT, const double* dL_dU, double* UO, double* dL_dFT,
                         double* dL_dpos, sps_stats* stats);

/* Adjoint of one collision-resolved step (sps_resolve_collisions, Sec. 3.2)
 * in the external forces.  Runs the step (positions are not advanced; its
 * velocities U = U_nc + M D gamma go to UO, n x 6 device, required) and, for
 * dL/dU (n x 6 device), writes dL/dF_ext (n x 6 device).  On the active set
 * A = {gamma > 0} of the LCP (eq. LCPdef), assuming strict complementarity,
 *   dU/dF = M - M D_A (D_A^T M D_A)^{-1} D_A^T M,
 * so dL/dF = v - M^T D_A lambda with v = M^T dL/dU and
 * (D_A^T M D_A)^T lambda = D_A^T v, solved by GMRES on contact vectors
 * (gmres_tol, gmres_max); every application of M^T is an adjoint mobility
 * solve (identity mobility: none).  If dL_dpos (n x 3 device) is not NULL it
 * receives dL/dc for the centres, with the radii and the contact, active and
 * near sets held fixed: (dL/dU - D_A mu)^T (dM/dc) (F + D gamma) plus the
 * terms of Phi and the normals in D, mu the active-set solution above (one
 * more forward and adjoint mobility solve).  stats->n_active = |A|, stats->ir_sweeps = iterations
 * of the active-set solve.  The paper has no adjoint.  Errors as
 * sps_resolve_collisions; NOT_CONVERGED if a solve hit its cap. */
int sps_collision_adjoint(sps_ctx* ctx, int n, const double* pos, const double* radii,
                          const double* FT_ext, double dt, const double* dL_dU, double* UO,
                          double* dL_dFT, double* dL_dpos, sps_stats* stats);

/* Contact set of sps_build_contacts for callers that cannot allocate device
 * memory when they need it: code embedded in a host whose own memory pool has
 * reserved the device (a framework's caching allocator, an MPS client with a
 * hard memory limit), where a cudaMalloc outside that pool fails or fragments
 * it, and time-stepping loops that must not pay for, or risk failing on, an
 * allocation in the middle of a step.  The paper has no counterpart: it is an
 * allocation-free variant of sps_build_contacts, computed without a context
 * and without any cudaMalloc / cudaFree.
 *
 * Threshold: the absolute delta only, i.e. the list of sps_build_contacts with
 * delta_rel = 0 (the relative part delta_rel (a_i + a_j) is not supported).
 * Search: all pairs, one thread per sphere i testing every j > i, so the cost
 * is n (n - 1) / 2 pair tests (3.4e10 at the size limit) and the work per
 * thread falls from n - 1 to 0 across the grid; the context builder's cell
 * list is the one for large n.
 *
 * Scratch: a fixed device array inside the library (one counter per sphere,
 * about 1 MB) that every GPU loading the library keeps until the process
 * exits.  n <= 262,144 spheres (larger n returns SPS_ERR_CAPACITY).  The first
 * call on a device looks up that array's device address (once per device,
 * with that device current).  All calls share the array and it keeps the
 * last call's contents: calls that overlap on the GPU (different streams or
 * threads at the same time) race and must not be issued.  Every counter a
 * call reads is written by the same call first.
 *
 * pos (n x 3), radii (n): device inputs.  ij (max_contacts x 2 int32), phi
 * (max_contacts), normals (max_contacts x 3): device outputs, written in the
 * order of sps_build_contacts (bit-identical values).  *n_contacts_out (host)
 * receives n_c; if n_c > max_contacts the call returns SPS_ERR_CAPACITY and
 * writes no output array.  stream: cudaStream_t (NULL = legacy default).  The
 * call reads the count back to the host and synchronises the stream before
 * returning. */
int sps_build_contacts_noalloc(int n, const double* pos, const double* radii, double a_c_scale,
                               double delta, int max_contacts, int* ij, double* phi,
                               double* normals, int* n_contacts_out, void* stream);

/* Phase timers (CUDA events recorded on the context's stream around each
 * kernel of a phase; the paper's Sec. 6.5 timing categories, refined). */
typedef enum {
  SPS_PH_FAR_K = 0,    /* far-field traction N-body kernel ("Far Traction")  */
  SPS_PH_FAR_S = 1,    /* far-field single-layer N-body kernel ("Far SL")    */
  SPS_PH_FAR_AUX = 2,  /* FP32 conversion and split reduction of the far field */
  SPS_PH_NEAR_K = 3,   /* near-pair VSH traction ("Near Correction")         */
  SPS_PH_NEAR_S = 4,   /* near-pair VSH velocity                             */
  SPS_PH_SELF = 5,     /* VSH analysis, self synthesis, near coefficients    */
  SPS_PH_KRYLOV = 6,   /* GMRES orthogonalisation and vector updates, L, rho */
  SPS_PH_CONTACT = 7,  /* contact set, D, D^T                                */
  SPS_PH_BBPGD = 8,    /* BBPGD vector kernels                               */
  SPS_PH_GEOM = 9,     /* surface nodes and near lists ("Far/Near Setup")    */
  SPS_PH_BB_D = 10,    /* identity mobility: per-sphere pass of a BBPGD step
                          (projected step and D)                             */
  SPS_PH_BB_DT = 11,   /* identity mobility: per-contact pass (D^T, + q and
                          the step's statistics)                             */
  SPS_PH_FAR_DW = 12,  /* far field in double-float (SPS_FP64_DW and the
                          mixed path's refinement), S and K                  */
  SPS_PH_COUNT = 13
} sps_phase;

/* enable != 0 starts recording (and clears the totals); 0 stops. */
int sps_profile(sps_ctx* ctx, int enable);
/* Synchronises the stream and writes, per phase, the summed event time in
 * milliseconds (ms[SPS_PH_COUNT]) and the number of kernel launches timed
 * (launches[SPS_PH_COUNT]); either may be NULL. */
int sps_profile_read(sps_ctx* ctx, double* ms, long long* launches);

/* Host-only tables (no GPU needed), for checking the library's spherical
 * harmonic set-up: P = (p+1)(2p+2) unit-sphere nodes and weights, and the
 * real VSH analysis matrix (rows 6*NC, NC = (p+1)(p+2)/2, row index
 * ((type*NC + n(n+1)/2 + m)*2 + re_im), type 0/1/2 = V/W/X, m >= 0; columns
 * c*P + k).  Analysis gives the multipliers of V, W, X in eq. rhoshexp.
 * Any output may be NULL. */
int sps_unit_tables(int p, double* nodes /*3*P planes*/, double* weights /*P*/,
                    double* analysis /*6NC x 3P row-major*/,
                    double* synthesis /*3P x 6NC row-major*/);

#ifdef __cplusplus
}
#endif
#endif /* SPS_H */
