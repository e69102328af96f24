/*
 * gbi.h -- C ABI of the GB300 Galerkin boundary-integral library for N active
 * spheres (Singh, Ghose & Adhikari, "Many-body microhydrodynamics of colloidal
 * particles with active boundary layers").
 *
 * Problem statement (Sec. II, Eq. boundary_conditions; Sec. III): N spheres of
 * radius a in an unbounded fluid of viscosity eta, centres R_n, with active slip
 * described by the one-body velocities V^a_n, Omega^a_n and the higher velocity
 * coefficients V^(l sigma)_n; external forces F^e_n and torques T^e_n.  Outputs:
 * the rigid-body motion V_n, Omega_n (Eq. genralized_active_stokes_law) and the
 * solved flow coefficients Q^(l sigma)_n (Eq. generalized_Qlsigma).
 *
 * Conventions shared by every call:
 *  - All array arguments are DEVICE pointers owned by the caller (for example
 *    torch tensors), unless the function name ends in _host.  They must not alias.
 *  - Row-major, double precision.  Vectors are [N][3] (x, y, z).
 *  - Packed higher coefficients VH, QH are [N][h] with h = gbi_h(trunc).  The
 *    modes follow each other in the order 2s 3t | 3a 3s 4t | 4a 4s 5t (l<=2 keeps
 *    the first two, l<=3 the first five, l<=4 all eight).  A mode whose
 *    irreducible tensor has rank k takes 2k+1 slots: the coordinates of that
 *    symmetric traceless tensor in the orthonormal basis U_mu (mu = -k..k) with
 *    U_mu . x^k = N_k r^k Y_{k mu}(x), real spherical harmonics without the
 *    Condon-Shortley phase, N_k^2 = 4 pi k!/(2k+1)!!.  For k = 1 this is
 *    (y, z, x).  The tensors are those of Sec. III, Eq. irred_velocity_coefficients:
 *    V^(L) = V^(L0) - (L-1)/L Delta(eps.V^(L1)) + L(L-1)/(2(2L-1)) Delta(delta V^(L2)).
 *  - Calls are asynchronous on the context's stream (gbi_set_stream) except where
 *    noted; the library allocates only inside its context workspace, which grows
 *    on the first call for a given size and is then reused.
 *  - Errors are returned as gbi_status; no call aborts the process.  A CUDA
 *    error is returned as GBI_ERR_CUDA and its text is kept for gbi_last_error().
 */
#ifndef GBI_H
#define GBI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GBI_OK = 0,
  GBI_ERR_ARG = 1,            /* invalid argument (NULL pointer, N < 0, bad truncation, NaN input) */
  GBI_ERR_OVERLAP = 2,        /* two centres closer than params.min_sep * a (nothing computed)      */
  GBI_ERR_NOT_CONVERGED = 3,  /* iteration cap reached; outputs hold the best iterate               */
  GBI_ERR_TIMEOUT = 4,        /* a bounded device wait gave up                                      */
  GBI_ERR_CUDA = 5,           /* CUDA runtime error (see gbi_last_error)                            */
  GBI_ERR_NOMEM = 6           /* workspace allocation failed                                        */
} gbi_status;

typedef struct gbi_ctx gbi_ctx;

typedef struct {
  double a;          /* sphere radius                                                    */
  double eta;        /* viscosity                                                        */
  int trunc;         /* 2, 3 or 4: mode set 1s 2a | 2s 3t (+3a 3s 4t) (+4a 4s 5t)        */
  int precision;     /* 0: FP64 pair sums throughout; 1: FP32 pair sums inside GMRES,     */
                     /*    FP64 right-hand side, residuals and outputs (iterative         */
                     /*    refinement); 2: as 1 but those FP64 passes run in double-float */
                     /*    arithmetic (pairs of floats, ~48-bit significand) on the FP32  */
                     /*    pipe; 3: as 2 but the right-hand side and the output pass in   */
                     /*    FP32 too (only the refinement residual in double-float), so    */
                     /*    V and Omega carry FP32 pair-sum rounding (~1e-7 relative) while */
                     /*    the traction solve still meets rtol for that right-hand side. */
                     /*    Arnoldi, Givens and the solution update stay FP64.             */
  double rtol;       /* target relative residual ||b - A q|| / ||b|| of the traction solve */
  int restart;       /* GMRES restart length (Krylov vectors per cycle), 1..128          */
  int max_iter;      /* cap on inner GMRES iterations over the whole solve               */
  int max_refine;    /* cap on refinement sweeps (precision 1..3; 0 = 8)                 */
  double inner_rtol; /* relative tolerance of each inner FP32 solve (precision 1..3;     */
                     /*    0 = 1e-5); loosened to 0.1 rtol |b| / |r| when that is larger */
  double min_sep;    /* overlap guard: reject pairs closer than min_sep * a (0 = off)    */
} gbi_params;

typedef struct {
  int iters;                 /* inner GMRES iterations                                   */
  int refinements;           /* FP64 residual evaluations after the first                */
  int matvecs_f32;           /* FP32 pair passes                                         */
  int matvecs_f64;           /* FP64 or double-float pair passes                         */
  double rel_residual;       /* final ||b - A q|| / ||b|| in FP64                        */
  double min_separation;     /* smallest centre distance seen, in units of a             */
  long long pair_interactions; /* ordered pairs evaluated, summed over all pair passes   */
} gbi_info;

/* Library handle.  gbi_create binds the calling thread's device `device`
 * (cudaSetDevice) and creates no stream: work goes to the legacy default stream
 * until gbi_set_stream is called.  Returns GBI_ERR_ARG for a NULL `out`. */
gbi_status gbi_create(gbi_ctx** out, int device);
gbi_status gbi_destroy(gbi_ctx* ctx);
/* stream: a cudaStream_t (may be NULL = default stream). */
gbi_status gbi_set_stream(gbi_ctx* ctx, void* stream);
/* Block until all work queued by the context has finished. */
gbi_status gbi_synchronize(gbi_ctx* ctx);
const char* gbi_status_string(int status);
/* Text of the last CUDA error seen by this context ("" if none). */
const char* gbi_last_error(gbi_ctx* ctx);

/* Number of packed H components per sphere (8, 25, 48) or all components
 * including the six rigid-body ones (14, 31, 54); -1 for an invalid truncation. */
int gbi_h(int trunc);
int gbi_d(int trunc);

/* Internal coordinate scale c per packed component (length gbi_d(trunc), host
 * pointer): x = c * y, where x are the coordinates in which the pair operator of
 * gbi_apply is symmetric.  The first six are 1s (y,z,x) then 2a (y,z,x). */
gbi_status gbi_component_scales(int trunc, double* out_host);
/* One-body self scalars g (units 1/a, host pointer, length gbi_d(trunc)):
 * 8 pi eta V^(l sigma) = -(g/a) Q^(l sigma) for an isolated sphere. */
gbi_status gbi_self_scalars(int trunc, double* out_host);

/* Pair operator (Sec. III, Eq. single_layer_yl_matrix_element, m != n) in internal
 * coordinates: for every sphere n and every row component p,
 *     y[p][n] = alpha * ( sum_{m != n} sum_q G_nm[p][q] x[q][m] + add_self * (g_p/a) x[p][n] )
 *               + beta * y[p][n].
 * x, y are component-major: x[q*N + m].  rows / cols select the components:
 * 0 = all (gbi_d), 1 = rigid-body (first 6), 2 = higher (last gbi_h); x and y point
 * at the first component of their set.  add_self requires rows == cols.
 * precision 0 = FP64 arithmetic, 1 = FP32 arithmetic, 2 = double-float arithmetic on the
 * FP32 pipe (not for rows = cols = 0); inputs and outputs FP64 in every case.
 * R: [N][3] centres.  Cost: N(N-1) pair interactions. */
gbi_status gbi_apply(gbi_ctx* ctx, int N, int trunc, double a, int rows, int cols, int precision,
                     const double* R, const double* x, double* y, double alpha, double beta, int add_self);

/* Full Galerkin solve (Sec. II, Eq. many_body_active_passive_stresses and
 * Eq. many_body_active_VL, in the flow-coefficient form): solves
 *     G^HH Q^H = -8 pi eta V^H - G^HL F^L
 * by restarted GMRES (FP64 Arnoldi and Givens least squares; FP32 or FP64 pair
 * sums per params.precision), then
 *     8 pi eta (V - V^a, 2a (Omega - Omega^a)) = -G^LL F^L - G^LH Q^H,
 * with F^(1) = -F^e and F^(21) = -T^e / a.
 * Inputs R, Va, Oa, Fe, Te: [N][3]; VH: [N][h] packed.  Outputs V, Omega: [N][3];
 * QH: [N][h] packed (may be NULL unless warm_start).  If warm_start != 0, QH is
 * also read as the initial guess.  info may be NULL.  Synchronous.
 * On a non-default stream with profiling off, a mixed-precision solve (precision 1..3)
 * without warm start is captured as one CUDA graph the second time a call repeats the
 * previous call's sizes, parameters, tuning and workspace, and replayed afterwards (see
 * gbi_solve_graph_replays); the caller's arrays are copied in and out around the graph,
 * so they may differ from call to call.  Results are identical either way. */
gbi_status gbi_solve(gbi_ctx* ctx, const gbi_params* params, int N,
                     const double* R, const double* Va, const double* Oa, const double* VH,
                     const double* Fe, const double* Te,
                     double* V, double* Omega, double* QH, int warm_start, gbi_info* info);

/* Batched solve of nsys independent suspensions in one set of launches (the
 * batched workload: many suspensions of uneven N).  offsets_host (host array of
 * nsys+1 ints, offsets_host[0] = 0, non-decreasing) splits the spheres into
 * systems; all other arrays are as in gbi_solve, concatenated over the systems.
 * Every system has its own GMRES state (Krylov basis slice, Hessenberg matrix,
 * Givens rotations, tolerance test) and its own refinement flag; spheres of
 * different systems do not interact.  info aggregates over the systems: iters is
 * the number of lock-step inner iterations, rel_residual the largest system
 * residual.  Returns GBI_ERR_NOT_CONVERGED if any system missed the tolerance.
 * Synchronous. */
gbi_status gbi_batch_solve(gbi_ctx* ctx, const gbi_params* params, int nsys, const int* offsets_host,
                           const double* R, const double* Va, const double* Oa, const double* VH,
                           const double* Fe, const double* Te,
                           double* V, double* Omega, double* QH, int warm_start, gbi_info* info);

/* Same as gbi_solve with HOST pointers: copies inputs to the device, solves, copies
 * the outputs back.  Synchronous. */
gbi_status gbi_solve_host(gbi_ctx* ctx, const gbi_params* params, int N,
                          const double* R, const double* Va, const double* Oa, const double* VH,
                          const double* Fe, const double* Te,
                          double* V, double* Omega, double* QH, int warm_start, gbi_info* info);

/* Superposition approximation (Sec. IV, second form of Eq. mobility_matrices and
 * Eq. propulsion_matrices; Sec. V, Eq. trap_eom): every higher coefficient takes
 * its one-body value Q^H = -8 pi eta a V^H / g and only the direct pair sum
 * remains.  params.trunc = 2 uses the closed-form trap kernel (Stokeslet/RPY,
 * rotlet, stresslet and potential dipole with their finite-size terms);
 * trunc 3, 4 use the general pair operator.  Arguments as gbi_solve (no QH).
 * params.precision selects FP32 (1 or 3) or FP64 (0) pair arithmetic; 2 selects FP64 for
 * the closed-form kernel and double-float for the general one.  Asynchronous. */
gbi_status gbi_superpose(gbi_ctx* ctx, const gbi_params* params, int N,
                         const double* R, const double* Va, const double* Oa, const double* VH,
                         const double* Fe, const double* Te, double* V, double* Omega);

/* Superposition approximation above a plane no-slip wall z = 0 (fluid z > 0; every
 * centre must have z > 0): Sec. VI extends the method to other geometries through their
 * Green's function, here Blake's (the Oseen tensor plus its image system at the mirror
 * point).  V, Omega = the unbounded superposition of gbi_superpose (params.trunc must be
 * 2) plus, at every centre, the image flows of every sphere's force Fe, torque Te and
 * stresslet S = (20/3) pi eta a^2 V^(2s) (the force dipole it exerts on the fluid), its
 * own images included, at the point-singularity level (V += u, Omega += curl u / 2).
 * The image of the potential dipole V^(3t) and the finite-size terms of the images are
 * not included.  params.precision 0 or 2: FP64 images; 1 or 3: FP32.  Arguments as
 * gbi_superpose.  Asynchronous. */
gbi_status gbi_wall_superpose(gbi_ctx* ctx, const gbi_params* params, int N, const double* R, const double* Va,
                              const double* Oa, const double* VH, const double* Fe, const double* Te, double* V,
                              double* Omega);

/* Superposition approximation in a periodic cube of side L (point forces): Sec. VI
 * notes that the flow sum of a periodic domain converges only conditionally; the limit
 * taken is Hasimoto's (zero mean flow over the cell).  V_n = Va_n + Fe_n / (6 pi eta a) +
 * [sum_{m != n} G^per(R_n - R_m) Fe_m + G^per_self Fe_n] / (8 pi eta), G^per the Oseen
 * tensor summed over the lattice by Ewald's method.  Real space: a cell list of M^3 cells
 * (cost ~ N^2 / M^3) or every pair by the minimum image.  Wave space: either directly over
 * the wave vectors kept (structure factors, cost ~ N n_k; with the split balanced the
 * whole sum grows as N^1.5), or on a K^3 mesh (smooth particle-mesh Ewald, order-8
 * B-splines, cost ~ N + K^3 log K, so ~ N log N overall).  Positions may lie anywhere
 * (they are wrapped into the cell).  Rotation rates, force dipoles and finite-size terms
 * are not included.  params.precision 1 or 3: FP32 sums (truncation ~1e-6 of the
 * velocities, direct or mesh); 0 or 2: FP64 (direct: ~1e-13; a mesh, only when imposed,
 * is limited by K: ~1e-6 at K = 5 xi L, falling as K^-10).
 * *cells_per_side in: 0 chooses the split by the work estimate, a value >= 3 imposes that
 * many cells per side, a negative value every pair by the minimum image (NULL: choose);
 * out: the cells used (0 for every pair).
 * *mesh in: 0 chooses between the direct and the mesh form by the work estimate (FP32
 * only; FP64 keeps the direct sum), a power of 2 in [16, 512] imposes that mesh (with the
 * cells imposed, at most 128 per side, or else the most cells per side, at least 3, that
 * it resolves), a negative value the direct sum (NULL: choose); out: the mesh used (0 for
 * the direct sum).  Other values of *mesh, or a mesh with every pair: GBI_ERR_ARG.
 * xi (the splitting parameter) and n_wave (the wave vectors of the direct sum in a half
 * space, or K^3 for the mesh) report the plan and may be NULL.  R, Va, Fe, V are [N][3]
 * device arrays.  The mesh form's spreading adds with atomics: its last bits depend on
 * timing.  Synchronizes the stream. */
gbi_status gbi_periodic_superpose(gbi_ctx* ctx, const gbi_params* params, int N, double L, const double* R,
                                  const double* Va, const double* Fe, double* V, int* cells_per_side, int* mesh,
                                  double* xi, long long* n_wave);

/* One-body flow coefficients of the higher modes, the Q^H of the superposition
 * approximation (Sec. IV): QH = -8 pi eta a VH / g per component (g the self scalars
 * of the truncation, gbi_self_scalars, for a unit sphere).  VH, QH are [N][h] device
 * arrays (QH may not alias VH).  Used as a warm start of gbi_solve, alone or with the
 * learned correction (gbi_mlp_correct_qh).  Asynchronous. */
gbi_status gbi_qh_onebody(gbi_ctx* ctx, const gbi_params* params, int N, const double* VH, double* QH);

/* Superposition approximation of gbi_superpose for a batch of independent
 * suspensions laid out as in gbi_batch_solve (system s = spheres [offsets_host[s],
 * offsets_host[s+1])); pairs are summed within each system only.  Every truncation
 * uses the general pair operator (trunc 2 included).  Asynchronous. */
gbi_status gbi_batch_superpose(gbi_ctx* ctx, const gbi_params* params, int nsys, const int* offsets_host,
                               const double* R, const double* Va, const double* Oa, const double* VH,
                               const double* Fe, const double* Te, double* V, double* Omega);

/* Inputs of the harmonic-trap model (Sec. V, Eq. trap_eom) from centres R and unit
 * orientations p ([N][3] device arrays): F^e = -k_trap R, T^e = 0, V^a = vs p,
 * Omega^a = 0, packed V^(2s) = s0 (pp - I/3), V^(3t) = d0 p, other higher modes 0.
 * Outputs Fe, Te, Va, Oa: [N][3]; VH: [N][gbi_h(trunc)].  Asynchronous. */
gbi_status gbi_trap_inputs(gbi_ctx* ctx, int N, int trunc, double k_trap, double vs, double s0, double d0,
                           const double* R, const double* p, double* Fe, double* Te, double* Va, double* Oa,
                           double* VH);

/* Harmonic-trap dynamics (Sec. V, Eq. trap_eom): nsteps forward-Euler steps of
 *     R <- R + dt V,  p <- normalise(p + dt Omega x p),
 * with F^e = -k_trap R, T^e = 0, V^a = vs p, Omega^a = 0, V^(2s) = s0 (pp - I/3),
 * V^(3t) = d0 p and every other higher mode zero, V and Omega re-evaluated every
 * step by gbi_superpose (superposition != 0) or gbi_solve (superposition == 0).  With
 * params.precision 0 each solve starts from the previous step's traction coefficients
 * Q^H, also across calls on the same context with the same N and truncation (the first
 * call, or one after a failed solve, starts from zero); mixed-precision solves start
 * from zero (a warm start would cost one more high-precision residual pass and save no
 * refinement sweep).  Results differ only within the solve tolerance.
 * R, p: [N][3] device arrays updated in place.  info (may be NULL) accumulates
 * over the steps.  A step whose solve fails (overlap guard, tolerance not met) leaves
 * R and p as they were and ends the call with that status.  Synchronous when
 * superposition == 0.  When the solve is replayed as a graph (see gbi_solve), the
 * step's input evaluation and update are captured with it; the graph then also depends
 * on R, p, dt and the trap parameters. */
gbi_status gbi_trap_step(gbi_ctx* ctx, const gbi_params* params, int N, double dt, double k_trap,
                         double vs, double s0, double d0, int superposition, int nsteps,
                         double* R, double* p, gbi_info* info);

/* Squirmers (Sec. V, Lighthill-Blake slip with the first two modes): the active slip
 * v^a = (nn - I).[B1 p + B2 (pp - I/3).n] has the tensorial-harmonic coefficients
 * V^a = 2 B1 p / 3, V^(2s) = -3/5 B2 (pp - I/3), V^(3t) = 10/3 B1 p and
 * V^(4t) = 7 B2 (pp - I/3) (every other mode zero; 4t is kept for trunc >= 3).
 * gbi_squirmer_inputs writes them with the trap forcing F^e = -k_trap R, T^e = 0,
 * Omega^a = 0 (layouts as gbi_trap_inputs); gbi_squirmer_step is gbi_trap_step with
 * these inputs re-evaluated from (R, p) at every step.  The paper prints 15/2 V^a and
 * 140/3 B2 for the 3t and 4t coefficients; the values here are the projection of the
 * printed slip onto the modes as this library normalises them. */
gbi_status gbi_squirmer_inputs(gbi_ctx* ctx, int N, int trunc, double k_trap, double B1, double B2,
                               const double* R, const double* p, double* Fe, double* Te, double* Va, double* Oa,
                               double* VH);
gbi_status gbi_squirmer_step(gbi_ctx* ctx, const gbi_params* params, int N, double dt, double k_trap, double B1,
                             double B2, int superposition, int nsteps, double* R, double* p, gbi_info* info);

/* Flow field (Sec. III, Eq. flow_expression / galerkin_representation_flow_yl): the
 * velocity at M points X [M][3] in the fluid around a solved suspension,
 *   v(x) = -(1/(8 pi eta)) sum_m [F^l' grad^(l') G](x - R_m) . Q_m,   Q^L = F^L,
 * the single-layer flow of every sphere's modes with its flow coefficients (F^(1s) =
 * -F^e, F^(2a) from -T^e; Q^H as returned by gbi_solve for the same R, F^e, T^e and
 * truncation).  R, Fe, Te: [N][3]; QH: [N][gbi_h(trunc)]; U: [M][3] output.  The
 * representation holds in the fluid: a point inside a sphere (|x - R_m| < a) gets NaN
 * and is counted in *n_inside (host pointer, may be NULL; when given the call
 * synchronizes the stream to return it).  params: a, eta, trunc; precision 0 evaluates
 * in FP64, any other value in FP32 (two-float centres).  Asynchronous otherwise. */
gbi_status gbi_flow(gbi_ctx* ctx, const gbi_params* params, int N, const double* R, const double* Fe,
                    const double* Te, const double* QH, int M, const double* X, double* U, int* n_inside);

/* gbi_trap_step for a batch of independent suspensions (the layout of gbi_batch_solve:
 * system s holds spheres [offsets_host[s], offsets_host[s+1]); each system has its own
 * trap centred at the origin of the coordinates).  Every step evaluates all systems
 * together (gbi_batch_superpose, or one lock-step gbi_batch_solve); a repeated
 * mixed-precision call on a non-default stream runs each step -- trap inputs, the whole
 * batched solve and the Euler update of every system -- as one replayed CUDA graph.  A
 * step in which any system's solve fails updates no system and ends the call with that
 * status.  Same arguments otherwise; R, p: [offsets_host[nsys]][3]. */
gbi_status gbi_batch_trap_step(gbi_ctx* ctx, const gbi_params* params, int nsys, const int* offsets_host,
                               double dt, double k_trap, double vs, double s0, double d0, int superposition,
                               int nsteps, double* R, double* p, gbi_info* info);

/* gbi_solve without any allocation.  For callers that cannot allocate device memory
 * while they run -- code inside a framework that owns every allocation, a real-time
 * loop that forbids cudaMalloc/cudaFree, or a host that pre-plans its memory -- this
 * entry point performs the same solve as gbi_solve (same arguments and results) but
 * takes every scratch buffer from one static device array of the library (about
 * 2.9 MB, held by every GPU that loads the library until the process exits) and its
 * read-back scalars from a static host array (one per device).  It needs no context: work is queued
 * on `stream` (a cudaStream_t, NULL = default stream) of the current device.
 * The paper has no counterpart; it is an engineering entry point.
 * Limits: N <= 1024, N * gbi_h(trunc) <= 8192, params.restart <= 32 (a value <= 0
 * selects 32); anything larger returns GBI_ERR_ARG before any work.
 * The first call on a device looks up the array's device address (set-up); make that
 * first call before any stream capture on the device.  All calls on one device share
 * that device's array and read-back area: two calls on the same device that overlap
 * (other threads or streams) race; calls on different devices do not.  Each call
 * re-initialises whatever must start at zero.  Synchronous. */
gbi_status gbi_solve_static(void* stream, const gbi_params* params, int N,
                            const double* R, const double* Va, const double* Oa, const double* VH,
                            const double* Fe, const double* Te,
                            double* V, double* Omega, double* QH, int warm_start, gbi_info* info);

/* ---- Learned near-field correction (an engineering addition; the paper has no
 * network).  A pairwise network approximates, for every ordered pair (n, m) of the
 * same system closer than 4a, the part of sphere n's velocity and angular velocity
 * that the Galerkin solution (Sec. II, Eq. many_body_active_passive_stresses, l <= 4)
 * adds to the superposition approximation (Sec. IV) for force- and torque-free
 * spheres with active modes V^a and V^(2s) = s0 (pp - I/3).
 *
 * Pair frame (rho = R_n - R_m, r = |rho|):  e_z = rho / r;  e_x = the part of p_n
 * normal to e_z, normalised (if its squared length is <= 1e-12: that of p_m; if that
 * is also degenerate: the coordinate axis with the smallest |e_z| component, first
 * such, made normal to e_z);  e_y = e_z x e_x.
 * Features (9):  2a/r, (2a/r)^3, d, ln d, p_n.e_z, p_n.e_x, p_m.e_x, p_m.e_y, p_m.e_z,
 * with d = max(r/a - 2, 0.01).
 * Network: tanh(W1 f + b1) -> tanh(W2 . + b2) -> tanh(W3 . + b3) -> W4 . + b4, widths
 * 9, 128, 128, 128, 6; outputs o_0..2 (velocity) and o_3..5 (angular velocity) in the
 * pair frame.  The correction of sphere n is (s0 / sigma) sum_m sum_c o_c e_c (and
 * o_(3+c) e_c for Omega), summed over n's pairs in increasing m.
 * Flat parameters (GBI_MLP_NPARAM floats): W1[128][9], b1[128], W2[128][128], b2[128],
 * W3[128][128], b3[128], W4[6][128], b4[6].
 * Inference multiplies BF16 weights and BF16 layer inputs on the tensor cores with
 * FP32 accumulation and evaluates tanh with the hardware approximation (relative
 * error about 2^-11, below the bf16 rounding of the activation); training (FP32 CUDA
 * cores, tanh to FP32 accuracy) multiplies the same rounded values and updates FP32
 * master weights with Adam (beta1 0.9, beta2 0.999, eps 1e-8).
 *
 * gbi_pairs: ordered pairs (n, m), n != m, of the same system with |R_n - R_m| < rcut a
 * (decided in FP64 as (dx dx + dy dy) + dz dz), grouped by n and sorted by m; systems
 * as in gbi_batch_solve (nsys <= 1 and offsets NULL: one system).  One system of more
 * than 4096 spheres uses a cell list and fails with GBI_ERR_ARG if a sphere has more
 * than 64 such neighbours.  *npairs receives the count; gbi_pairs_get copies the last
 * list into device arrays tg (targets n), sr (sources m) of *npairs ints.
 * Synchronizes the stream.
 * gbi_mlp_set / gbi_mlp_get: load (host FP32, resets Adam) / read the weights and the
 * label scale sigma > 0.
 * gbi_mlp_features: features [P][9] and frames [P][9] (rows e_x, e_y, e_z), FP32, of
 * the pairs (tg[k], sr[k]) (device arrays).
 * gbi_mlp_forward: network outputs for P feature rows; FR == NULL gives pair-frame
 * outputs [P][6], otherwise the rotated (lab-frame) ones.
 * gbi_mlp_correct: builds the 4a pairs of R, evaluates the network and ADDS the
 * corrections to V, Omega ([N][3], device).  *npairs (may be NULL) = pairs evaluated.
 * gbi_mlp_labels: labels [N][6] = sigma/s0 ((Vx, Ox) - (Vs, Os)) from exact (x) and
 * superposition (s) velocities; if *sigma <= 0 it is first set to the power of two
 * nearest 1 / rms((x - s)/s0).
 * gbi_mlp_loss_grad: loss = sum_n |P_n - labels_n|^2 / (6N) over all spheres (P_n the
 * summed rotated outputs) and its gradient (device, GBI_MLP_NPARAM floats), no update.
 * gbi_mlp_adam: one Adam step with the given gradient (device) and learning rate.
 * gbi_mlp_train: epochs passes over the systems in order, minibatches of batch_systems
 * consecutive systems (loss normalised per minibatch), learning rate geometric from
 * lr0 to lr1 over all steps; loss_hist (host, may be NULL) receives each epoch's mean
 * minibatch loss.  Synchronous.
 *
 * Second head (gbi_mlp_set_head, per context; 0 = the velocity head above, the default):
 * head 1 predicts the correction of the strain-mode flow coefficient Q^(2s) of sphere n
 * (the first five packed components of Q^H, Sec. III Eq. generalized_Qlsigma) beyond its
 * one-body value (gbi_qh_onebody).  Outputs o_0..4 are the packed symmetric traceless
 * tensor S' in the pair frame, taken to the lab as sum_kl S'_kl e_k e_l and packed
 * again (the same orthonormal packing as V^H); o_5 is trained toward zero and unused.
 * Forward, loss, gradient and training take the head of the context.  The guess it
 * gives, Q^H = one-body + (s0/sigma) sum_m rotated o, is a warm start of gbi_solve:
 * the solve, not the network, decides the result.
 * gbi_mlp_correct_qh: builds the 4a pairs of R and ADDS the head-1 correction to
 * QH[n][0..4] (rows of h >= 5 doubles, device).  gbi_mlp_correct needs head 0 and
 * gbi_mlp_correct_qh head 1 (GBI_ERR_ARG otherwise).
 * gbi_mlp_labels_qh: labels [N][6] = sigma/s0 (QHx - QH1)[n][0..4], 0, from the solve's
 * (x) and the one-body (1) Q^H (rows of h); sigma as for gbi_mlp_labels. */
#define GBI_MLP_NPARAM 35078
gbi_status gbi_pairs(gbi_ctx* ctx, int N, const double* R, double a, double rcut, int nsys, const int* offsets_host,
                     int* npairs);
gbi_status gbi_pairs_get(gbi_ctx* ctx, int* tg, int* sr);
gbi_status gbi_mlp_set(gbi_ctx* ctx, const float* theta_host, double sigma);
gbi_status gbi_mlp_get(gbi_ctx* ctx, float* theta_host, double* sigma);
gbi_status gbi_mlp_features(gbi_ctx* ctx, int P, const double* R, const double* p, const int* tg, const int* sr,
                            double a, float* F, float* FR);
gbi_status gbi_mlp_forward(gbi_ctx* ctx, int P, const float* F, const float* FR, float* out);
/* Engine of the network kernels.  Inference (gbi_mlp_forward / gbi_mlp_correct): 0 =
 * warp-level mma.sync m16n8k16 (64 pairs per tile), 1 = tcgen05.mma with the accumulator in
 * tensor memory (128 pairs per tile; default); both multiply the same bf16 values with FP32
 * accumulation.  Training (gbi_mlp_loss_grad / gbi_mlp_train): 0 = the FP32 CUDA cores (the
 * forward with exact tanh, FP32 gradients), 1 = tcgen05 (the inference kernel's forward,
 * then a backward kernel whose GEMMs take bf16 operands, dZ rounded to bf16, with FP32
 * accumulation and the weight gradients accumulated in tensor memory; default).  The
 * tcgen05 kernels bound their completion waits; if one gave up it records it on the device
 * and gbi_mlp_status (synchronizes the stream) returns GBI_ERR_TIMEOUT once and clears the
 * record; outputs of that call are not valid. */
gbi_status gbi_mlp_set_engine(gbi_ctx* ctx, int engine);
gbi_status gbi_mlp_status(gbi_ctx* ctx);
gbi_status gbi_mlp_correct(gbi_ctx* ctx, int N, const double* R, const double* p, double a, double s0, int nsys,
                           const int* offsets_host, double* V, double* Omega, int* npairs);
gbi_status gbi_mlp_labels(gbi_ctx* ctx, int N, double s0, const double* Vx, const double* Ox, const double* Vs,
                          const double* Os, double* sigma, double* labels);
gbi_status gbi_mlp_loss_grad(gbi_ctx* ctx, int N, const double* R, const double* p, double a, int nsys,
                             const int* offsets_host, const double* labels, double* loss, float* grad);
gbi_status gbi_mlp_adam(gbi_ctx* ctx, const float* grad, double lr);
gbi_status gbi_mlp_train(gbi_ctx* ctx, int N, const double* R, const double* p, double a, int nsys,
                         const int* offsets_host, const double* labels, int epochs, int batch_systems, double lr0,
                         double lr1, double* loss_hist);
gbi_status gbi_mlp_set_head(gbi_ctx* ctx, int head);
gbi_status gbi_mlp_correct_qh(gbi_ctx* ctx, int N, const double* R, const double* p, double a, double s0, int nsys,
                              const int* offsets_host, int h, double* QH, int* npairs);
gbi_status gbi_mlp_labels_qh(gbi_ctx* ctx, int N, int h, double s0, const double* QHx, const double* QH1,
                             double* sigma, double* labels);

/* Tuning of the pair kernel (engineering; the paper has no counterpart).  The FP32
 * and double-float pair passes run in one of two forms.  Streaming: one block per
 * target sphere whose WPT warps split the sources; WPT in {2, 4, 8, 16} (8 at most for
 * trunc 4 and double-float) trades parallelism at small N against per-target
 * reduction work.  Tiled (code WPT = 1, one system only, not batches): lanes are 32
 * target spheres, source records are staged in shared memory by the TMA unit and read
 * by all lanes at once, and the (targets, source) work is split evenly over one block
 * per SM; the blocks' partial sums are added in a fixed order, so results do not
 * depend on timing.  Both forms sum the same pairs (in different fixed orders).
 * gbi_tune times every WPT for the six FP32 / double-float passes of the mixed-precision
 * solves -- rows H / columns H in FP32 and in double-float, H/L and L/all in
 * double-float, H/L and L/all in FP32 -- on synthetic
 * input of the given layout: nsys systems, system s holding spheres
 * [offsets[s], offsets[s+1]) (host array of nsys + 1 increasing ints, offsets[0] = 0;
 * nsys = 1 describes one suspension, nsys > 1 a gbi_batch_solve batch).  Spheres sit
 * on a cubic lattice of spacing 3a; each candidate runs once to warm up and then reps
 * times (reps = 0 selects 5) between CUDA events on the context's stream.  The fastest
 * WPT is kept in the context for every later pass of the same truncation, pass,
 * precision, batching and floor(log2(total spheres)).  chosen (host, may be NULL)
 * receives the 6 choices in the order above.  Allocates and frees its own device
 * buffers and synchronizes the stream (not capturable).
 * gbi_set_wpt forces one WPT for every later pass (0 = back to tuned/default).
 * gbi_pass_wpt returns the WPT a pass with these parameters would use (0 for the
 * FP64 tiled pass, -1 for invalid arguments).
 * Split tail (streaming form, one system; off by default): when the N target blocks do not
 * fill whole waves of the resident block slots, the targets of the last, partly filled
 * wave have their sources split into 2..8 blocks each (the count that best fills the
 * slots), whose rows are added in part order by the last part to finish -- the result does
 * not depend on timing, only the summation order of those targets changes.  On GB300 at
 * N = 1024 (l <= 3, H/H) it measured slower in FP32 (each part's reduction costs as much
 * as the pairs it takes over) and within 3% in double-float, so it is off unless asked for.
 * gbi_set_split_tail(ctx, 1) turns it on (0 off); gbi_tune times with the setting in
 * force. */
gbi_status gbi_tune(gbi_ctx* ctx, int trunc, int nsys, const int* offsets, int reps, int* chosen);
gbi_status gbi_set_wpt(gbi_ctx* ctx, int wpt);
gbi_status gbi_set_split_tail(gbi_ctx* ctx, int on);
int gbi_pass_wpt(gbi_ctx* ctx, int trunc, int rows, int cols, int precision, int N, int batched);

/* Bounded waits of the tiled pair passes (engineering; the paper has no counterpart).
 * Each wait of a tiled pass for its shared-memory stage gives up after `rounds`
 * mbarrier try_wait rounds (default 2^24, far beyond any copy's latency); the pass
 * then records the failure on the device, waits with the default bound for the copies
 * it has in flight and returns without storing.  gbi_solve and the calls built on it
 * read the record after the solve and return GBI_ERR_TIMEOUT (outputs not valid); the
 * context stays usable.  gbi_set_wait_limit(ctx, r): r >= 0 sets the bound (0 makes
 * every such wait give up at once: a test of this path), r = -1 restores the default.
 * gbi_pass_status synchronizes the stream and returns GBI_ERR_TIMEOUT once if a pair
 * pass launched since the last check (gbi_apply included) gave up, else GBI_OK. */
gbi_status gbi_set_wait_limit(gbi_ctx* ctx, long long rounds);
gbi_status gbi_pass_status(gbi_ctx* ctx);

/* Instrumentation.  gbi_kernel_launches: number of CUDA kernels this context has
 * launched since creation.  gbi_set_profiling(ctx, 1) resets the per-class
 * statistics and from then on records a CUDA event pair on the context's stream
 * around every pair pass; gbi_kernel_stats returns, for one class, the summed
 * event time in ms, the number of launches and the algorithmic flops (the
 * per-pair count of the implemented closed form times N(N-1)).  Pair passes that the
 * device-side GMRES launched after it had stopped (they return at once) are not
 * counted as launches; their few microseconds stay in the summed time.  Class ids:
 * precision * 9 + rows * 3 + cols for gbi_apply-style passes (precision 0 = FP64,
 * 1 = FP32, 2 = double-float; rows/cols 0 = all, 1 = rigid-body, 2 = higher),
 * 27 = closed-form trap pass in FP64, 28 = in FP32, 29 = flow field (gbi_flow) in FP64,
 * 30 = in FP32, 31 = wall images (gbi_wall_superpose) in FP64, 32 = in FP32 (flops: the
 * dual-number arithmetic per (target, source) term times N^2).  gbi_kernel_stats synchronizes
 * on the recorded events. */
long long gbi_kernel_launches(gbi_ctx* ctx);
/* Number of solves this context has run as one replayed CUDA graph (-1 for a NULL
 * context).  A mixed-precision solve (precision 1..3, zero initial guess) on a
 * non-default stream, with profiling off, is captured as one graph the second time a
 * call repeats the previous call's sizes, parameters, tuning and workspace, and
 * replayed while they stay the same; the refinement sweeps, GMRES restarts and Arnoldi
 * steps then loop on the device (nested conditional graph nodes) and the call waits for
 * the GPU once.  Results are identical to the host-driven sequence.  No counterpart in
 * the paper. */
long long gbi_solve_graph_replays(gbi_ctx* ctx);
gbi_status gbi_set_profiling(gbi_ctx* ctx, int on);
gbi_status gbi_kernel_stats(gbi_ctx* ctx, int kernel_class, double* total_ms, long long* launches,
                            double* flops);

#ifdef __cplusplus
}
#endif

#endif /* GBI_H */
