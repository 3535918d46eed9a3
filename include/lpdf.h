/*
 * lpdf.h -- C ABI of the GB300 particle time step of the fully Lagrangian joint
 * velocity-frequency-scalar PDF method (Bakosi, Franzese & Boybeyi, arXiv:1006.0549).
 *
 * The method (Section "Governing equations"): a large number of Lagrangian particles carry
 * position X, velocity U, turbulent frequency omega and scalar compositions psi_alpha, governed
 * by Eq. 2 (position), Eq. 4 (generalized Langevin model), Eq. 5/6 (frequency) and Eq. 9
 * (micromixing: IEM, <phi|V> -> <phi>, or IECM with a reactive source); they are advanced by forward Euler,
 * Eulerian statistics are evaluated at particle positions, and an unstructured grid is used to
 * extract statistics, to solve for Eulerian quantities, and to track particles (Introduction,
 * items i-iii).
 *
 * Conventions for every call:
 *   - Return value: LPDF_OK (0) or a negative LPDF_ERR_* code; lpdf_last_error() gives a
 *     message for the calling thread's last error. Nothing is thrown across the ABI.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA device memory of the
 *     current device (for example torch CUDA tensors). The caller owns every pointer it passes;
 *     the library owns the objects it creates (lpdf_mesh, lpdf_ctx) and their device memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream). Calls marked
 *     "async" only enqueue work on that stream; calls marked "sync" return after the work ends.
 *   - Floating-point particle state is FP32 structure-of-arrays; gridpoint moment sums are FP64.
 */
#ifndef LPDF_H
#define LPDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LPDF_OK 0
#define LPDF_ERR_ARG (-1)           /* null pointer, bad size, bad enum */
#define LPDF_ERR_MESH (-2)          /* non-CCW or degenerate element, non-manifold or unpaired edge */
#define LPDF_ERR_LOST_PARTICLE (-3) /* the neighbour walk hit its hop cap or a wall (see lpdf_status) */
#define LPDF_ERR_NONFINITE (-4)     /* NaN or Inf in the particle state */
#define LPDF_ERR_CG_NOCONV (-5)     /* a conjugate-gradient solve did not converge */
#define LPDF_ERR_CUDA (-6)          /* a CUDA runtime call failed */
#define LPDF_ERR_OVERFLOW (-7)      /* fixed-point moment accumulator range exceeded */
#define LPDF_ERR_UNSUPPORTED (-8)   /* e.g. more scalars than compiled for */

#define LPDF_MAX_SOURCES 8
#define LPDF_MAX_SCALARS 4

/* Edge tags (edge k of an element runs from its vertex k to vertex (k+1) % 3). */
#define LPDF_EDGE_INTERIOR 0
#define LPDF_EDGE_WALL 1        /* no-slip wall, U_w = 0 */
#define LPDF_EDGE_MOVING_WALL 2 /* the lid: U_w = (lid_u, 0, 0) */
#define LPDF_EDGE_PERIODIC 3

/* Node-field columns of the table that pdf_step reads (per node, FP32; row stride nfp,
 * nfp = 4 * ceil((22 + ns) / 4)). Names follow Eq. 4, 5, 6 and 9. */
#define LPDF_F_U 0      /* <U>, <V>, <W>: columns 0..2 */
#define LPDF_F_DUDX 3   /* d<U>/dx, d<U>/dy, d<V>/dx, d<V>/dy, d<W>/dx, d<W>/dy: 3..8 */
#define LPDF_F_LAPU 9   /* laplacian of <U>, <V>, <W>: 9..11 */
#define LPDF_F_DPDX 12  /* d<P>/dx / rho, d<P>/dy / rho: 12..13 */
#define LPDF_F_G11 14   /* G11, G12, G21, G22, G33: 14..18 (planar flow, G13 = G23 = G31 = G32 = 0) */
#define LPDF_F_C0EPS 19 /* C_0 * epsilon */
#define LPDF_F_OMEGA 20 /* <omega> */
#define LPDF_F_SOMEGA 21 /* S_omega of Eq. 6 */
#define LPDF_F_PHI0 22  /* <phi_alpha>, alpha = 0..ns-1 */

/* Model and run parameters. The paper prints no constants; the defaults that
 * lpdf_params_default() writes are the literature values of the cited models. */
typedef struct {
    double nu;      /* kinematic viscosity */
    double dt;      /* forward-Euler time step */
    double C3, C4;  /* Eq. 5 */
    double Cphi;    /* IEM: 1/t_m = Cphi <omega> / 2 */
    double C0;      /* Eq. 4 constant (elliptic relaxation and the simplified Langevin model) */
    double Comega1, Comega2; /* Eq. 6 */
    double CL, Ceta;         /* elliptic-relaxation length scale L = CL max(k^1.5/eps, Ceta nu^0.75/eps^0.25) */
    double lid_u;   /* tangential velocity of LPDF_EDGE_MOVING_WALL edges (the top wall) */
    uint64_t seed;  /* Philox4x32-10 key */
    int32_t ns;     /* number of scalars, 1..LPDF_MAX_SCALARS */
    int32_t n_sources;
    float src_x[LPDF_MAX_SOURCES], src_y[LPDF_MAX_SOURCES], src_r[LPDF_MAX_SOURCES];
    int32_t src_alpha[LPDF_MAX_SOURCES]; /* scalar index set to 1 inside source disc s */
    int32_t gmodel;         /* lpdf_elliptic_relax_solve: 0 elliptic relaxation, 1 simplified Langevin model */
    int32_t pressure_solve; /* lpdf_elliptic_relax_solve: 1 solve for the mean pressure,
                               0 gradient = (dpdx0, dpdy0) only */
    int32_t cg_warm_start;  /* lpdf_elliptic_relax_solve: 1 starts the CGs from the previous solution
                               on this mesh (a time loop), 0 from zero */
    double dpdx0, dpdy0;    /* fixed mean pressure gradient added to the solved one (channel: -1, 0) */
    /* Eq. 9 micromixing: 0 IEM (<phi|V> -> <phi>), 1 IECM with the conditional mean estimated
     * linearly in the velocity, <phi_a|V> = <phi_a> + beta_a . (V - <U>) (lpdf_ctx_set_iecm) */
    int32_t mixing;
    /* reactive source of Eq. 9 (none when react_k <= 0): the second-order reaction
     * psi_a + psi_b -> psi_p at rate react_k, S_a = S_b = -react_k psi_a psi_b, S_p = +react_k psi_a psi_b */
    int32_t react_a, react_b, react_p;
    double react_k;
    /* precision of the gridpoint moment sums of lpdf_pdf_step (the statistics at gridpoints,
     * Introduction item i): 0, each term lambda_a q_k formed in FP32 and summed in FP32 over at
     * most 8 particles of a lane and the 32 lanes of a warp (16 lanes, a half-warp per element,
     * when the ensemble averages at most 384 particles per element) before the exact 64-bit
     * fixed-point accumulation (error at most 48 eps32 sum |lambda_a q_k| + 8 eps32 sum kappa_a
     * |q_k|: the FP32 weight lambda_a, a determinant of rounded coordinate differences, is off by
     * about 2 eps32 kappa_a with kappa_a = (|dx_b dy_c| + |dy_b dx_c|) / |2A| from the particle to
     * the other two vertices, of the order of the element's aspect ratio); 1, compensated: the sums of q,
     * dx q and dy q over an element's particles ((dx, dy) from its first vertex, formed exactly)
     * in double-float FP32 arithmetic (error-free products and additions), combined with the
     * element's FP64 barycentric coefficients in FP64 (error at most 1e-9 sum |lambda_a q_k|,
     * about 1e-13 in practice). Both add 2^-33 per fixed-point conversion. Other values:
     * LPDF_ERR_ARG. lpdf_pdf_step_static supports 0 only (LPDF_ERR_UNSUPPORTED). */
    int32_t moment_sums;
} lpdf_params;

typedef struct lpdf_mesh lpdf_mesh;
typedef struct lpdf_ctx lpdf_ctx;

/* Fills *p with C3 = 5, C4 = 0.25, Cphi = 2, C0 = 2.1, Comega1 = 0.5, Comega2 = 0.73,
 * CL = 0.134, Ceta = 72, nu = 1/180, dt = 1e-3, ns = 1, no sources, seed = 1, lid_u = 0,
 * gmodel = 0, pressure_solve = 0, cg_warm_start = 0, dpdx0 = dpdy0 = 0, mixing = 0 (IEM),
 * react_k = 0 (no reaction), react_a = react_b = react_p = 0, moment_sums = 0. */
void lpdf_params_default(lpdf_params* p);

/* Message of the calling thread's last error ("" if none). Owned by the library. */
const char* lpdf_last_error(void);
const char* lpdf_version(void);

/* ---------------------------------------------------------------------------------------
 * lpdf_mesh_load -- the unstructured triangle mesh (Introduction: the grid extracts
 * statistics, solves Eulerian fields and tracks particles). sync.
 *   node_xy  host, 2*n_nodes doubles (x, y); every value must be exactly representable in FP32
 *   tri      host, 3*n_tri int32 node ids, counter-clockwise
 *   edge_tag host, 3*n_tri int32 LPDF_EDGE_* (edge k: vertex k -> vertex (k+1)%3)
 *   period_x > 0: the domain is periodic in x with this period (node columns at x0 and
 *            x0 + period_x are paired by equal y); 0: walls everywhere.
 * The domain is the bounding box of the nodes, taken half-open: [x0, x1) x [y0, y1).
 * Builds element adjacency (periodic edges linked), element geometry, node->element lists and
 * periodic node pairing, and uploads them to the current device.
 * Errors: LPDF_ERR_ARG, LPDF_ERR_MESH (orientation, unpaired periodic edge, edge shared by
 * more than two elements), LPDF_ERR_CUDA.
 * ------------------------------------------------------------------------------------- */
int lpdf_mesh_load(const double* node_xy, int32_t n_nodes, const int32_t* tri, int32_t n_tri,
                   const int32_t* edge_tag, double period_x, lpdf_mesh** out);
void lpdf_mesh_free(lpdf_mesh* mesh);
/* n_nodes, n_tri, box = {x0, x1, y0, y1} (host outputs; any may be NULL). */
int lpdf_mesh_info(const lpdf_mesh* mesh, int32_t* n_nodes, int32_t* n_tri, double* box);
/* host out, 3*n_tri: neighbour across each edge, -1 on walls. sync. */
int lpdf_mesh_neighbors(const lpdf_mesh* mesh, int32_t* out);
/* host out, n_nodes: the node that holds the statistics of each node (periodic pairing). */
int lpdf_mesh_masters(const lpdf_mesh* mesh, int32_t* out);

/* ---------------------------------------------------------------------------------------
 * lpdf_mesh_load_multi -- n_comp independent meshes held as one (their disjoint union), so that
 * many ensembles of uneven size advance in the same kernel launches (the paper has no
 * counterpart: a batching choice of this library). sync.
 *   node_xy, tri, edge_tag, n_nodes, n_tri  as for lpdf_mesh_load, over all components; tri
 *            holds global node ids.
 *   node_off, tri_off  host, n_comp + 1 each: component c owns nodes [node_off[c],
 *            node_off[c + 1]) and elements [tri_off[c], tri_off[c + 1]) (node_off[0] = tri_off[0]
 *            = 0, node_off[n_comp] = n_nodes, tri_off[n_comp] = n_tri); an element may only use
 *            nodes of its own component.
 *   period_x  as for lpdf_mesh_load, shared by every component (> 0: all components are
 *            periodic in x with this period).
 * Each component has its own bounding box as its half-open domain, pairs its periodic edges and
 * nodes within itself and never exchanges particles with another. Node fields and statistics
 * are per node of the union; lpdf_pdf_step_static rejects these meshes.
 * Errors: as lpdf_mesh_load; LPDF_ERR_ARG for offsets that do not cover the mesh.
 * ------------------------------------------------------------------------------------- */
int lpdf_mesh_load_multi(const double* node_xy, int32_t n_nodes, const int32_t* tri, int32_t n_tri,
                         const int32_t* edge_tag, int32_t n_comp, const int32_t* node_off, const int32_t* tri_off,
                         double period_x, lpdf_mesh** out);

/* ---------------------------------------------------------------------------------------
 * lpdf_ctx_create -- particle ensemble on one mesh with room for `capacity` particles
 * (device SoA state x, y, u, v, w, omega, psi[ns], elem, pid, plus the moment accumulators).
 * params->ns must be in 1..LPDF_MAX_SCALARS. sync. The mesh must outlive the context.
 * ------------------------------------------------------------------------------------- */
int lpdf_ctx_create(const lpdf_mesh* mesh, const lpdf_params* params, int64_t capacity, lpdf_ctx** out);
void lpdf_ctx_free(lpdf_ctx* ctx);
/* Replaces the parameters (ns must not change). */
int lpdf_ctx_set_params(lpdf_ctx* ctx, const lpdf_params* params);
int64_t lpdf_ctx_size(const lpdf_ctx* ctx);

/* Per-component Philox key and scalar sources of a multi-component mesh (default: every
 * component takes params->seed and params' sources). */
typedef struct {
    uint64_t seed;
    int32_t n_sources;
    float src_x[LPDF_MAX_SOURCES], src_y[LPDF_MAX_SOURCES], src_r[LPDF_MAX_SOURCES];
    int32_t src_alpha[LPDF_MAX_SOURCES];
} lpdf_component;
/* sync. comps host, n = the mesh's component count. Errors: LPDF_ERR_ARG. */
int lpdf_ctx_set_components(lpdf_ctx* ctx, const lpdf_component* comps, int32_t n);

/* ---------------------------------------------------------------------------------------
 * lpdf_particles_init -- n_per_elem particles per element, pid = e*n_per_elem + j: position
 * uniform in the element, then located exactly; U = <U>(X) + sigma(X) z; omega Erlang(m_erlang)
 * with mean <omega>(X) (gamma-distributed frequency, Section "Governing equations"); psi = 0.
 *   node_init device, n_nodes x 8 FP32: <U>, <V>, <W>, sigma, <omega>, 3 unused.
 * Random numbers: Philox4x32-10 counter (pid, 0, 0, 1<<16 | block), key = seed. async.
 * Errors: LPDF_ERR_ARG (capacity too small, m_erlang outside 1..6).
 * ------------------------------------------------------------------------------------- */
/* lpdf_particles_init_multi -- as lpdf_particles_init with n_per_elem[c] (host, one per
 * component) particles per element of component c. The components' particles follow one another
 * in component order, pids count from 0 within each component, and each component draws with
 * its own seed, so component c starts exactly as a single-mesh context of that component would. */
int lpdf_particles_init_multi(lpdf_ctx* ctx, const int32_t* n_per_elem, const float* node_init, int32_t m_erlang,
                              void* stream);
int lpdf_particles_init(lpdf_ctx* ctx, int32_t n_per_elem, const float* node_init, int32_t m_erlang,
                        void* stream);

/* ---------------------------------------------------------------------------------------
 * lpdf_set_state / lpdf_get_state -- copy the SoA state in or out. `on_device` = 1: the
 * pointers are device memory, 0: host memory. psi is ns rows of n values. set_state sets the
 * ensemble size to n (n <= capacity). async (a host copy is synchronous w.r.t. the host only
 * when the host memory is pageable).
 * ------------------------------------------------------------------------------------- */
int lpdf_set_state(lpdf_ctx* ctx, int64_t n, const float* x, const float* y, const float* u, const float* v,
                   const float* w, const float* omega, const float* psi, const int32_t* elem,
                   const uint32_t* pid, int on_device, void* stream);
int lpdf_get_state(const lpdf_ctx* ctx, float* x, float* y, float* u, float* v, float* w, float* omega,
                   float* psi, int32_t* elem, uint32_t* pid, int on_device, void* stream);

/* ---------------------------------------------------------------------------------------
 * lpdf_pdf_step -- one forward-Euler step of every particle, then the gridpoint moment sums
 * of the new state. async. The step also re-buckets the ensemble by element (a stable counting
 * sort on the new elements, kept as the gather order of the next step), so the order in which
 * lpdf_get_state lists the particles changes from step to step; pid identifies them.
 *   node_fields device, n_nodes x nfp FP32 (columns LPDF_F_*), evaluated at each particle by
 *               the linear shape functions of its element.
 *   step        the step index (part of the Philox counter: (pid, step, 0<<16 | block)).
 * Per particle, with the state at t_n: Eq. 4 for U, Eq. 5 for omega (sqrt(max(omega,0)),
 * then omega <- |omega|), Eq. 9 for psi (IEM, or IECM with params->mixing = 1, plus the reactive
 * source when params->react_k > 0, both from the state at t_n), Eq. 2 for X with the same dW_1, dW_2;
 * periodic wrap; wall reflection (X mirrored, U <- 2 U_w - U): across the frame's sides, or,
 * on a mesh with wall edges off the frame (walls of any shape), across the wall edge that the
 * walk meets, in FP64 rounded to FP32 (an image that rounds back onto the point moves one FP32
 * step along the inward normal; the image is wrapped into the periodic frame again; at most 8
 * mirrorings); exact point location by a barycentric neighbour walk (hop cap 64; a particle
 * that exceeds a cap keeps its old element and is counted as lost); psi_alpha <- 1 inside
 * scalar source discs; then
 * S_k(n) += lambda_n(X') q_k, q = 1, u, v, w, uu, uv, uw, vv, vw, ww, omega, psi_a, psi_a^2.
 * Errors are recorded in the context's device status word (read with lpdf_status); the
 * call itself only reports argument and launch errors.
 * ------------------------------------------------------------------------------------- */
int lpdf_pdf_step(lpdf_ctx* ctx, const float* node_fields, uint64_t step, void* stream);

/* ---------------------------------------------------------------------------------------
 * IECM (Eq. 9): the scalar mean conditional on the particle velocity. Reading: the conditional
 * mean is estimated linearly in the velocity (exact for jointly Gaussian velocity and scalar),
 * <phi_a|V> = <phi_a> + beta_a . (V - <U>), beta_a = R^-1 c_a with R = <u_i u_j> (the Reynolds
 * stresses, 3 x 3) and c_a = <u_i psi_a'> (the scalar fluxes), both at the gridpoints; beta is
 * a node field interpolated to the particle by the linear shape functions.
 *
 * lpdf_grid_flux_statistics -- the scalar fluxes of the state left by the last pdf_step of a
 *   context created with params->mixing = 1 (the step then also sums lambda_n u_i psi_a). async.
 *   out device, n_nodes x 3 ns FP64, per node (u psi_0, v psi_0, w psi_0, u psi_1, ...):
 *   raw = 1 the sums S(n) = sum_p lambda_n(X_p) u_i psi_a; raw = 0 the covariances
 *   S/S_0 - <u_i><psi_a> (zeros where S_0 = 0). Errors: LPDF_ERR_ARG (mixing = 0 at creation).
 * lpdf_iecm_coefficients -- beta from gridpoint statistics (lpdf_grid_statistics raw = 0) and
 *   fluxes (lpdf_grid_flux_statistics raw = 0), both device FP64. async. beta device out,
 *   n_nodes x 3 ns FP32 (beta_0 = (bx, by, bz), beta_1, ...): beta_a = R^-1 c_a in FP64 by
 *   Cramer's rule; beta_a = 0 where det R <= 1e-12 (trace R / 3)^3.
 * lpdf_ctx_set_iecm -- the beta table (device, n_nodes x 3 ns FP32, owned by the caller, read by
 *   every later pdf_step while params->mixing = 1; NULL clears it: IECM then falls back to IEM). */
int lpdf_grid_flux_statistics(lpdf_ctx* ctx, double* out, int raw, void* stream);
int lpdf_iecm_coefficients(const lpdf_mesh* mesh, int32_t ns, const double* stats, const double* flux, float* beta,
                           void* stream);
int lpdf_ctx_set_iecm(lpdf_ctx* ctx, const float* beta);

/* ---------------------------------------------------------------------------------------
 * lpdf_pdf_steps -- nsteps consecutive steps step0, step0 + 1, ... with the same node fields,
 * bit-identical to nsteps lpdf_pdf_step calls. async. Pairs of steps replay a CUDA graph of two
 * whole steps (captured on first use for these fields and this buffer; the step number is read
 * from device memory, so replays need no host work); an odd last step runs as lpdf_pdf_step.
 * lpdf_ctx_set_timing does not record graph-replayed steps. Changing the state, the order, the
 * parameters, the components or the launch configuration drops the graphs.
 * ------------------------------------------------------------------------------------- */
int lpdf_pdf_steps(lpdf_ctx* ctx, const float* node_fields, uint64_t step0, int32_t nsteps, void* stream);

/* ---------------------------------------------------------------------------------------
 * Launch configuration of the step's kernels. Every configuration gives bit-identical results.
 *   adv (advance kernel): 0 = 256 threads per CTA, >= 4 CTAs per SM (64 registers);
 *       1 = 128, >= 10 (48 registers) on a persistent grid (CTAs stride over 128-particle
 *       tiles); 2 = 128, >= 8 (64 registers); 3 = 256, >= 4, persistent; 4 = 64, >= 18
 *       (56 registers), persistent; 5 = 128, >= 10, persistent, each warp taking 64-particle
 *       chunks in order from a counter in the context's scratch.
 *   mom (moments kernel, a warp per element): 0 = 256 threads, >= 2 CTAs per SM; 1 = 128, >= 4;
 *       2 = 512, >= 1; 3 = 256, >= 3.
 * lpdf_ctx_set_tune sets it (LPDF_ERR_ARG outside those ranges). lpdf_ctx_autotune times every
 * advance variant, then every moments variant with the best advance variant. A trial is one
 * warm-up step and steps_per_trial timed steps (CUDA events on `stream`) of this context's own
 * ensemble and fields; every variant is tried once per round, `rounds` rounds interleaved (odd
 * rounds in reverse order, so that no variant is always timed right after the same one), and
 * a variant's time is its fastest trial (the ensemble keeps changing while it is timed). The
 * fastest variants are kept. The trial steps are real steps, numbered from step0: *steps_used
 * (host, may be NULL) tells how many were taken. choice (host, 2 ints, may be NULL) = (adv,
 * mom); trial_ms (host, 10 doubles, may be NULL) = milliseconds per step of each variant (6
 * advance, then 4 moments variants). sync.
 * ------------------------------------------------------------------------------------- */
int lpdf_ctx_set_tune(lpdf_ctx* ctx, int32_t adv, int32_t mom);
int lpdf_ctx_autotune(lpdf_ctx* ctx, const float* node_fields, uint64_t step0, int32_t steps_per_trial,
                      int32_t rounds, int32_t* choice, double* trial_ms, int32_t* steps_used, void* stream);

/* ---------------------------------------------------------------------------------------
 * lpdf_sort -- physically re-buckets the ensemble by element: afterwards the particles of every
 * element are contiguous in the buffer lpdf_get_state reads, ordered by element and then by
 * their previous position (a deterministic counting sort; pid travels with each particle).
 * Particles are never lost or duplicated; the per-particle results of later steps do not depend
 * on the order. lpdf_pdf_step keeps its own element order, so this is only needed to read the
 * state in element order. async. Uses the context's second state buffer.
 * ------------------------------------------------------------------------------------- */
int lpdf_sort(lpdf_ctx* ctx, void* stream);

/* ---------------------------------------------------------------------------------------
 * lpdf_status -- sync. Reads and clears the device status: out[0] error bits (1 lost
 * particle, 2 non-finite state, 4 fixed-point overflow, 8 a bounded wait on a bulk copy gave up, 16 an internal
 * consistency check of the step kernel failed),
 * out[1] number of lost particles,
 * out[2] pid of one lost particle (-1 if none), out[3] total walk hops of the last step.
 * Returns LPDF_ERR_LOST_PARTICLE / LPDF_ERR_NONFINITE / LPDF_ERR_OVERFLOW when the
 * corresponding bit was set (LPDF_ERR_CUDA for bits 8 and 16), else LPDF_OK.
 * ------------------------------------------------------------------------------------- */
int lpdf_status(lpdf_ctx* ctx, int64_t* out, void* stream);

/* ---------------------------------------------------------------------------------------
 * lpdf_ctx_set_timing / lpdf_ctx_timings -- device time of the kernels of lpdf_pdf_step, from
 * CUDA events recorded on the step's stream (the paper has no counterpart: a measurement aid).
 *   set_timing: enable = 1 records four events around the kernels of every following step,
 *               0 stops recording.
 *   timings:    sync; out_ms (host, 3 doubles) = summed milliseconds of the advance kernel, of
 *               the re-bucketing kernels (histogram, scans, record and particle scatter) and of
 *               the moments kernel over the steps recorded since the previous call; *steps (host,
 *               may be NULL) = their number. The sums restart after each call.
 * ------------------------------------------------------------------------------------- */
int lpdf_ctx_set_timing(lpdf_ctx* ctx, int enable);
int lpdf_ctx_timings(lpdf_ctx* ctx, double* out_ms, int64_t* steps);

/* ---------------------------------------------------------------------------------------
 * lpdf_grid_statistics -- gridpoint statistics of the state left by the last pdf_step
 * (statistics estimated at the gridpoints of the mesh, Section "Governing equations"). async.
 *   out device, n_nodes x (11 + 2 ns) FP64.
 *   raw = 1: the sums S_k(n) = sum_p lambda_n(X_p) q_k(p).
 *   raw = 0: S_0, <u>, <v>, <w>, <u'u'>, <u'v'>, <u'w'>, <v'v'>, <v'w'>, <w'w'>, <omega>,
 *            <psi_a> (ns), <psi_a'^2> (ns); mean = S_q/S_0, central moment = S_qq/S_0 - mean^2;
 *            a node with S_0 = 0 gets zeros.
 * Periodic partner nodes hold identical values.
 * ------------------------------------------------------------------------------------- */
int lpdf_grid_statistics(lpdf_ctx* ctx, double* out, int raw, void* stream);

/* ---------------------------------------------------------------------------------------
 * lpdf_elliptic_relax_solve -- the gridpoint side: node fields for lpdf_pdf_step from gridpoint
 * statistics (Introduction, item ii: Eulerian quantities are solved on the grid). sync (the
 * conjugate-gradient convergence tests read residual norms back to the host).
 *   stats   device, n_nodes x (11 + 2 ns) FP64 as lpdf_grid_statistics(raw = 0) writes them
 *   fields  device out, n_nodes x nfp FP32 (columns LPDF_F_*)
 *   tol     relative residual of each conjugate gradient: |r| <= tol |r_ref|, r_ref the residual
 *           of the start with a zero interior (with cg_warm_start the CG starts from the previous
 *           solution on this mesh, so a slowly changing problem needs few iterations)
 *   maxit   iteration cap of each conjugate gradient
 *   iters   host out (may be NULL), 2 ints: iterations of the elliptic-relaxation solve (its
 *           four components at once) and of the pressure solve (0 when not run)
 * With P1 finite elements on the mesh (periodic partners merged into one unknown):
 *   gradients of <U_i> recovered at the nodes by area-weighted averaging of element gradients,
 *   Laplacians as the recovered divergence of the recovered gradient; k = <u_i u_i>/2,
 *   eps = k <omega> (the paragraph before Eq. 5); S_omega = C_omega2 - C_omega1 P/eps with
 *   P = -<u_i u_j> d<U_i>/dx_j (Eq. 6); G_ij (the paragraph after Eq. 4): gmodel 0 solves
 *   (M + L^2 K) wp = M (-3/4 C0 eps delta) with wp_ij = -4.5 eps n_i n_j on wall nodes,
 *   L = CL max(k^1.5/eps, Ceta nu^0.75/eps^0.25), then G_ij = (wp_ij - eps delta_ij/2)/k and
 *   C0 eps = max(0, -2/3 (eps + <u_i u_j> G_ij)); gmodel 1 gives G_ij = -(1/2 + 3/4 C0) <omega>
 *   delta_ij and C0 eps. pressure_solve 1 solves the weak form of lap p = -d_i d_j (<U_i><U_j> +
 *   <u_i u_j>) (natural boundary condition, zero mean) and adds (dpdx0, dpdy0) to its
 *   recovered gradient. All arithmetic is FP64; the output is rounded to FP32.
 * The first call on a mesh builds and uploads its finite-element tables (kept until
 * lpdf_mesh_free). Calls on the same mesh share its scratch: serialise them.
 * Errors: LPDF_ERR_ARG, LPDF_ERR_UNSUPPORTED (ns), LPDF_ERR_CG_NOCONV (iters still filled in),
 * LPDF_ERR_CUDA.
 * ------------------------------------------------------------------------------------- */
int lpdf_elliptic_relax_solve(const lpdf_mesh* mesh, const lpdf_params* params, const double* stats,
                              float* fields, double tol, int32_t maxit, int32_t* iters, void* stream);

/* ---------------------------------------------------------------------------------------
 * lpdf_tc_gemm_bf16 -- the tensor-core tile of the learned relaxation surrogate, exposed to
 * test it: D = A B^T on the fifth-generation
 * tensor cores (tcgen05, BF16 inputs, FP32 accumulation in tensor memory). The paper has no
 * counterpart. sync.
 *   A  device, M x K BF16 row-major; B device, N x K BF16 row-major; D device, M x N FP32.
 *   M >= 1; N a multiple of 16 in 16..256; K a multiple of 16 in 16..128.
 * Errors: LPDF_ERR_ARG (shape, NULL), LPDF_ERR_CUDA (launch, or a bounded wait for the MMAs
 * gave up).
 * ------------------------------------------------------------------------------------- */
int lpdf_tc_gemm_bf16(const void* A, const void* B, float* D, int32_t M, int32_t N, int32_t K, void* stream);

/* =======================================================================================
 * The learned surrogate of lpdf_elliptic_relax_solve. The paper has no counterpart: its G_ij
 * comes from the elliptic relaxation (the paragraph after Eq. 4); here a small network maps
 * local quantities at each gridpoint to the same outputs, is trained on fields that the plain
 * solve generates, and is checked against the plain solve at a fixed cadence, falling back to
 * it when the error exceeds a threshold.
 *
 * Network: 8 inputs -> 128 -> 128 -> 128 (tanh) -> 7 linear outputs. Inputs are standardised
 * with per-column means and deviations, outputs are standardised targets. The three hidden
 * layers and the output layer run on the fifth-generation tensor cores with BF16 operands
 * (inputs, weights, activations and, in the backward pass, the error signals are rounded to
 * BF16) and FP32 accumulation; biases, tanh, the loss and the optimiser are FP32.
 *
 * Parameter vector (LPDF_MLP_NPARAMS floats, in this order): W1 [128][8], b1 [128],
 * W2 [128][128], b2 [128], W3 [128][128], b3 [128], W4 [7][128], b4 [7]; W [out][in] row-major,
 * layer l computes z = W a + b.
 * Standardisation block (LPDF_MLP_NNORM floats): feature means [8], feature deviations [8],
 * loss weights [7], target means [7], target deviations [7].
 * Inputs (per gridpoint): wall distance, ln k, ln <omega>, b11, b22, b12, II_b = b_ij b_ij and
 * ln(eps_w / eps), with b_ij = <u_i u_j> / (2 k) - delta_ij / 3 (b = 0 where k <= 1e-12), eps =
 * k <omega> and eps_w its value at the nearest wall point (linear along the wall edge; 0 input
 * without walls); the logarithms take max(., 1e-12).
 * Targets: G11, G12, G21, G22, G33 divided by <omega>, C0 eps / (k <omega>), and the relaxed trace
 * wp_ii = k G_ii + 3 eps / 2 over its local value -9/4 C0 eps (1 where eps <= 1e-12; this last
 * output is a diagnostic of the wall effect and is not used by the step); <omega> and k below
 * 1e-12 are taken as 1e-12 in the divisions.
 * Loss: sum over rows and outputs of w_j (y_j - t_j)^2 / (7 B), y and t standardised.
 * ===================================================================================== */
#define LPDF_MLP_IN 8
#define LPDF_MLP_OUT 7
#define LPDF_MLP_HIDDEN 128
#define LPDF_MLP_NPARAMS 35079
#define LPDF_MLP_NNORM 37

typedef struct lpdf_mlp lpdf_mlp;

/* lpdf_mlp_create -- a network with zero parameters, identity standardisation (means 0,
 * deviations 1, weights 1), and the fallback policy check_every = 50, threshold = 0.02.
 * max_batch: the largest batch of lpdf_mlp_gradient and lpdf_mlp_train (>= 1).
 * Errors: LPDF_ERR_ARG, LPDF_ERR_CUDA. */
int lpdf_mlp_create(int64_t max_batch, lpdf_mlp** out);
void lpdf_mlp_free(lpdf_mlp* m);

/* lpdf_mlp_set_params -- sync. params host, LPDF_MLP_NPARAMS floats (layout above); norm host,
 * LPDF_MLP_NNORM floats, or NULL to keep the current block. Resets the optimiser state. */
int lpdf_mlp_set_params(lpdf_mlp* m, const float* params, const float* norm);
/* lpdf_mlp_get_params -- sync. params and norm host out (either may be NULL). */
int lpdf_mlp_get_params(lpdf_mlp* m, float* params, float* norm);

/* lpdf_mlp_fit_norm -- async. Sets the feature and target means and deviations of the
 * standardisation block from a data set (feat device B x 8, tgt device B x 7, FP32); a deviation
 * below 1e-6 max(1, |mean|) is taken as 1. The loss weights are kept. */
int lpdf_mlp_fit_norm(lpdf_mlp* m, const float* feat, const float* tgt, int64_t B, void* stream);

/* lpdf_mlp_forward -- async. out device, B x 7 FP32: the outputs in target units (standardised
 * output times the target deviation plus the target mean). feat device, B x 8 FP32. Any B >= 0. */
int lpdf_mlp_forward(lpdf_mlp* m, const float* feat, int64_t B, float* out, void* stream);

/* lpdf_mlp_gradient -- sync. The gradient of the loss on the batch (feat device B x 8, tgt device
 * B x 7, 1 <= B <= max_batch) with respect to the parameters: grad host, LPDF_MLP_NPARAMS floats
 * (layout above); loss host (may be NULL). The per-tile partial gradients are summed in a fixed
 * order, so the result is bit-reproducible. */
int lpdf_mlp_gradient(lpdf_mlp* m, const float* feat, const float* tgt, int64_t B, float* grad, double* loss,
                      void* stream);

/* lpdf_mlp_train -- sync at the end. `steps` Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, bias
 * correction, learning rate lr) on minibatches of `batch` rows: step s uses rows
 * [c batch, (c + 1) batch) with c = s mod floor(B / batch) (shuffle the data set beforehand).
 * feat device B x 8, tgt device B x 7; 1 <= batch <= min(B, max_batch). losses host (may be
 * NULL): the minibatch loss before each step. The step count of the bias correction continues
 * across calls until lpdf_mlp_set_params. */
int lpdf_mlp_train(lpdf_mlp* m, const float* feat, const float* tgt, int64_t B, int64_t batch, int32_t steps,
                   float lr, double* losses, void* stream);

/* lpdf_surrogate_features -- async. Per geometric node of the mesh: feat device n_nodes x 8
 * (the inputs above) from stats (device, n_nodes x (11 + 2 ns) FP64 as lpdf_grid_statistics
 * raw = 0 writes them); with fields != NULL (device, n_nodes x nfp, e.g. from
 * lpdf_elliptic_relax_solve) also tgt device n_nodes x 7 (the targets above; params->C0 is used).
 * The wall distance is the distance to the nearest LPDF_EDGE_WALL or LPDF_EDGE_MOVING_WALL edge
 * (in a periodic mesh also to their images one period away), computed on first use. */
int lpdf_surrogate_features(const lpdf_mesh* mesh, const lpdf_params* params, const double* stats,
                            const float* fields, float* feat, float* tgt, void* stream);

/* lpdf_mlp_set_policy -- the fallback policy of lpdf_surrogate_relax_solve: every check_every-th
 * call (the first call included; 0: never) also runs the plain solve and compares. */
int lpdf_mlp_set_policy(lpdf_mlp* m, int32_t check_every, double threshold);
/* lpdf_mlp_request_check -- the next lpdf_surrogate_relax_solve call checks (for example after
 * the network was trained further on the fields of a failed check), whatever the cadence. */
int lpdf_mlp_request_check(lpdf_mlp* m);

/* lpdf_surrogate_relax_solve -- lpdf_elliptic_relax_solve (gmodel 0) with G_ij and C0 eps from
 * the network. sync. Everything else (gradients, Laplacians, pressure, S_omega) is computed as
 * in the plain solve. On a checking call the plain solve runs too, the error
 * e = |F_net - F_plain| / |F_plain| (Frobenius norms over the node columns G11..G33 and C0 eps)
 * is measured, the plain fields are returned, and the network is used on the following calls
 * only if e <= threshold; otherwise the plain solve runs until the next checking call.
 *   info host out (may be NULL), 4 doubles: 1 if this call checked, e (-1 when not checked),
 *   1 if the returned fields come from the plain solve, the call count so far.
 * Errors: as lpdf_elliptic_relax_solve; LPDF_ERR_ARG when params->gmodel != 0. */
int lpdf_surrogate_relax_solve(const lpdf_mesh* mesh, lpdf_mlp* m, const lpdf_params* params, const double* stats,
                               float* fields, double tol, int32_t maxit, double* info, void* stream);

/* ---------------------------------------------------------------------------------------
 * lpdf_pdf_step_static -- the same particle step as lpdf_pdf_step for callers that cannot
 * allocate device memory (the paper has no counterpart: this is an interface choice of the
 * library). Hosts that own every device buffer through their own pool or arena, or that
 * forbid cudaMalloc inside their time loop, keep the state in their own buffers and call this
 * without an lpdf_ctx. The call allocates nothing: its scratch (fixed-point gridpoint
 * accumulators and four status words) is a static device array of at most 2^21 accumulators,
 * i.e. n_nodes * (11 + 2 ns) <= 2,097,152 (16 MiB, held by every GPU that loads the library
 * until the process exits); larger meshes are rejected with LPDF_ERR_ARG.
 *   mesh, params    as for lpdf_ctx_create (the mesh itself was built by lpdf_mesh_load); IEM
 *                   only (mixing = 0, react_k <= 0), one component, walls on the frame's sides:
 *                   other settings are rejected with LPDF_ERR_UNSUPPORTED
 *   x..pid          device, n particles (psi: ns rows of n), advanced in place
 *   node_fields     device, n_nodes x nfp FP32 (see lpdf_pdf_step)
 *   moments         device out, n_nodes x (11 + 2 ns) FP64 raw sums S_k(n) of the new state
 *   status_out      host, 4 words as lpdf_status; NULL: the call is asynchronous and the status
 *                   is not read; non-NULL: the call synchronises `stream` and returns
 *                   LPDF_ERR_LOST_PARTICLE / NONFINITE / OVERFLOW as lpdf_status does.
 * The first call on a device looks up the static array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture. Every call shares the one array and clears it
 * on entry, so calls that overlap on the GPU (different streams, threads or processes sharing
 * the context) race: serialise them.
 * ------------------------------------------------------------------------------------- */
int lpdf_pdf_step_static(const lpdf_mesh* mesh, const lpdf_params* params, int64_t n, float* x, float* y,
                         float* u, float* v, float* w, float* omega, float* psi, int32_t* elem,
                         const uint32_t* pid, const float* node_fields, uint64_t step, double* moments,
                         int64_t* status_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LPDF_H */
