/*
 * dgw.h -- C ABI of the GB300 library for the WENO-stabilized RKDG method of
 * Vedral, "Dissipative WENO stabilization of high-order discontinuous Galerkin methods
 * for hyperbolic problems" (arXiv 2309.12019).
 *
 * Problem (Sec. 2, Eq. pde/ivp): a scalar conservation law u_t + div F(u) = 0 on a
 * Cartesian box in 1D or 2D, discretized by modal tensor-Legendre DG of degree p
 * (Eq. fesol; Q_p on quadrilaterals), the local Lax-Friedrichs flux (Sec. 2), the
 * dissipative stabilization gamma_e nu_e int grad(phi).grad(U_h) (Sec. 3, Eq. astab,
 * with Eq. visc for nu_e) driven by the WENO sensor of Sec. 4 (Eq. sensor / gensensor),
 * and advanced by the optimal SSP-RK3 scheme (Eq. ssp).  Also the Euler equations of gas
 * dynamics (Sec. 5.6) in 1D and 2D with the same scheme and a density-driven sensor.
 *
 * Conventions shared by every entry point
 *  - State arrays ("U") are device arrays owned by the caller, mode-major
 *    (structure of arrays): U[k*E + e] with element e = iy*nx + ix and mode
 *    k = i + (p+1)*j (i: Legendre degree in x, j: in y; 1D: k = i).  K = (p+1)^dim
 *    modes, E = nx (1D) or nx*ny (2D) elements.  The Euler system stacks its dim + 2
 *    components: row comp*(p+1)^dim + k holds mode k of rho (comp 0), the momentum
 *    components (1 .. dim) and rho E (dim + 1), so K = (dim + 2)(p+1)^dim rows.  The element type is double for
 *    DGW_FP64 contexts and float for DGW_FP32 contexts.  Base addresses must be
 *    aligned to 16 bytes.
 *  - Every call is asynchronous on the given stream (a cudaStream_t passed as
 *    void*; NULL is the legacy default stream) unless stated otherwise.  Argument
 *    errors are returned synchronously and nothing is enqueued.  Device-side
 *    conditions (non-finite results) set a flag in the context that
 *    dgw_sync_status() reads.
 *  - Return values are dgw_status codes; dgw_last_error() gives a thread-local
 *    message for the last failing call of the calling thread.
 *  - A context is bound to the CUDA device that was current at dgw_create; call
 *    it with that device current.  A context may be used from one thread at a
 *    time; calls on different streams that touch the same U race.
 */
#ifndef DGW_H
#define DGW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DGW_OK = 0,
    DGW_EINVAL = -1,        /* bad argument (null pointer, size, alignment, range) */
    DGW_ENOMEM = -2,        /* device or host allocation failed */
    DGW_ECUDA = -3,         /* a CUDA runtime call failed (message has the CUDA error) */
    DGW_EUNSUPPORTED = -4,  /* valid but not built (e.g. p > 3, non-square 2D cells) */
    DGW_ETIMEOUT = -5,      /* a bounded device-side wait gave up */
    DGW_ENONFINITE = -6     /* a kernel produced a NaN or Inf */
} dgw_status;

/* Boundary treatment of one side of the box (Sec. 2: weak inflow conditions). */
typedef enum {
    DGW_BC_PERIODIC = 0,
    DGW_BC_INFLOW_ZERO = 1, /* ghost U+ = 0 where F'(U-).n < 0, U+ = U- elsewhere
                               (scalar laws only) */
    DGW_BC_OUTFLOW = 2,     /* ghost U+ = U- */
    DGW_BC_REFLECT = 3,     /* Euler system only: reflecting wall, ghost state with the
                               normal momentum mirrored, (rho, m - 2 (m.n) n, rho E) */
    DGW_BC_STATE = 4        /* 2D Euler system only: prescribed ghost states (the double Mach
                               reflection of Sec. 5.6): at each face point the ghost is
                               dgw_flux.bstate[0] or [1] or a reflecting wall, by whether the
                               point's coordinate along the side (y on the x-sides, x on the
                               y-sides) lies below bsplit + bspeed t (see dgw_flux) */
} dgw_bc;

/* Cartesian mesh of [x0,x1] (1D) or [x0,x1]x[y0,y1] (2D) with nx (x ny) equal cells.
 * 2D cells must be square (the scaled seminorm of Sec. 4 uses one h_e per cell).
 * bc: sides -x, +x, -y, +y; periodic sides must come in pairs. */
typedef struct {
    int dim;
    int nx, ny;
    double x0, x1, y0, y1;
    int bc[4];
} dgw_mesh;

/* Flux functions of the paper's scalar examples (Sec. 5). */
typedef enum {
    DGW_FLUX_ADVECT = 0,    /* F = (a0, a1) u                                  */
    DGW_FLUX_ROTATION = 1,  /* F = omega (cy - y, x - cx) u   (solid body)      */
    DGW_FLUX_BURGERS = 2,   /* F = (a0, a1) u^2 / 2                            */
    DGW_FLUX_KPP = 3,       /* F = (sin u, cos u)                              */
    DGW_FLUX_EULER = 4      /* Euler system (Sec. 5.6), 1D or 2D: U = (rho, rho v, rho E),
                               F(U) n = (rho v.n, rho v (v.n) + p n, (rho E + p) v.n),
                               p = (gas_gamma - 1)(rho E - rho |v|^2 / 2); the LLF speed
                               s+ is the larger |v.n| + c of the two states; the sensor is
                               computed from the density and applied to every component;
                               no positivity safeguard: a negative density or pressure
                               gives non-finite results (dgw_sync_status) */
} dgw_flux_kind;

typedef struct {
    int kind;               /* dgw_flux_kind */
    double a[2];
    double center[2];
    double omega;
    double lambda_nu;       /* > 0: fixed lambda_e in nu_e = lambda_e h / (2p) (the paper
                               uses 2.0 for KPP); 0: max |F'(U_h)|_2 over the element's
                               volume and face Gauss points (Euler: max |v| + c over the
                               same points, the element's own values on its faces) */
    double gas_gamma;       /* Euler system: ratio of heat capacities (> 1; the paper and
                               dgw_defaults use 1.4); ignored by the scalar fluxes */
    /* DGW_BC_STATE sides: two prescribed conservative states (rho, rho vx, rho vy, rho E);
     * per side (-x, +x, -y, +y) the position along the side where the ghost changes at
     * t = 0, its speed, and the ghost below / from it: 0 or 1 for bstate[0] or bstate[1],
     * 2 for a reflecting wall.  t is the context's time (dgw_set_time); each stage of a
     * step sees its stage time (SSP-RK3: t, t + dt, t + dt / 2). */
    double bstate[2][4];
    double bsplit[4];
    double bspeed[4];
    int bbelow[4];
    int babove[4];
} dgw_flux;

typedef enum { DGW_STAB_DG = 0, DGW_STAB_LO = 1, DGW_STAB_WENO = 2, DGW_STAB_ZHAO = 3 } dgw_stab;

/* DGW_FP64: every operation in double.  DGW_FP32: state, residual and RK update in
 * float with float accumulation; operator tables are built in double and rounded. */
typedef enum { DGW_FP64 = 0, DGW_FP32 = 1 } dgw_prec;

/* Stabilization and sensor parameters (Sec. 3-5). */
typedef struct {
    int stab;               /* dgw_stab: DG (none), LO (gamma = 1), WENO (Eq. sensor), ZHAO
                               (the comparison sensor of Zhao et al. that Sec. 5.6 restates:
                               gamma = sum_l |w_l / lin_l - 1|^theta / (|1 / min lin - 1|^theta
                               + m_e) over the same candidates and weights; 0 without
                               neighbours; q and b do not apply; needs w_nbr > 0) */
    double q;               /* sensor exponent, Eq. (sensor); the paper uses 1 */
    double b;               /* threshold of Eq. (gensensor): gamma = 0 where the ratio
                               ||U - U*||_e / ||U||_e is below b; 0 recovers Eq. (sensor).
                               dgw_defaults sets 0.1, the tolerance of the remark in Sec. 4
                               with which the scalar problems' WENO errors equal DG's on
                               smooth data (Tables 1-2); the Euler runs of Sec. 5.6 use 0 */
    double w_nbr;           /* linear weight of each neighbour candidate (paper: 1e-2);
                               the cell's own candidate gets 1 - m_e * w_nbr */
    double eps_w;           /* nonlinear weights w_l ~ lin_l / (eps_w + beta_l)^2 (1e-6) */
    double eps_s;           /* ||U - U*||_e <= eps_s gives gamma = 0 (1e-12) */
    int prec;               /* dgw_prec */
    double theta;           /* exponent of the ZHAO sensor (> 0); the paper uses 1 */
    int rk_order;           /* SSP Runge-Kutta of dgw_rk_step / dgw_rk_step_host / the no-alloc
                               step: 3 = Eq. (ssp) (default), 2 = the two-stage SSP method,
                               4 = Ketcheson's ten-stage SSP method (Sec. 5 uses order p + 1;
                               the paper names no scheme).  The adjoint and the batch step
                               implement order 3 only and refuse the others. */
} dgw_params;

typedef struct dgw_ctx dgw_ctx;

/* Fills *m, *f, *s with the defaults above (periodic unit interval, advection with
 * a = (1, 0), WENO with q = 1, b = 0.1, w_nbr = 1e-2, eps_w = 1e-6, eps_s = 1e-12, FP64).
 * Any argument may be NULL. */
void dgw_defaults(dgw_mesh* m, dgw_flux* f, dgw_params* s);

/* Creates a context for degree p (1..3) on the current device: checks the arguments
 * (DGW_BC_REFLECT only with DGW_FLUX_EULER and DGW_BC_INFLOW_ZERO only without it, else
 * DGW_EINVAL),
 * builds the operator tables (Gauss rule of p+2 points, Legendre values, Hermite
 * shift matrices, seminorm Gram matrix, stiffness) in double, uploads them, and
 * allocates the two RK stage buffers (2*K*E elements) plus small scratch.
 * *out receives the context; release it with dgw_destroy. */
dgw_status dgw_create(const dgw_mesh* mesh, int p, const dgw_flux* flux,
                      const dgw_params* params, dgw_ctx** out);

/* Frees the context and its device memory (synchronizes the device first). NULL is
 * accepted. */
dgw_status dgw_destroy(dgw_ctx* ctx);

/* Sizes: *E elements, *K modes per element, *elem_bytes bytes per coefficient.  Any
 * pointer may be NULL. */
dgw_status dgw_sizes(const dgw_ctx* ctx, int64_t* E, int* K, int* elem_bytes);

/* Replaces the stabilization parameters (same precision).  Synchronous, cheap. */
dgw_status dgw_set_params(dgw_ctx* ctx, const dgw_params* params);

/* L2 projection of initial data onto V_p (Sec. 2, Eq. fesol).  samples (device,
 * double, E * nq^dim values): f at the nq-point Gauss-Legendre points of each
 * element, sample t = a + nq*b at x = xc + h/2 g_a, y = yc + h/2 g_b.  nq in 1..8.
 * U (device, context precision, K*E) receives c_k = int f phi_k / int phi_k^2.  Euler
 * system: (dim + 2) * E * nq^dim samples, those of each conserved variable one after
 * the other. */
dgw_status dgw_project(dgw_ctx* ctx, int nq, const double* samples, void* U, void* stream);

/* Semi-discrete right-hand side L = M^{-1} R_stab(U) (Eq. weak2 with s_h^e of Sec. 3):
 * volume term, LLF face term, and -gamma_e nu_e times the element stiffness applied to
 * U_h (gamma_e = 0 for DG, 1 for LO, Eq. sensor for WENO).  U and L: device, K*E,
 * context precision, must not overlap. */
dgw_status dgw_residual(dgw_ctx* ctx, const void* U, void* L, void* stream);

/* WENO sensor gamma_e (Sec. 4, Eq. sensor / gensensor) of every element.
 * gamma: device double[E].  Computed in the context precision, stored as double. */
dgw_status dgw_sensor(dgw_ctx* ctx, const void* U, double* gamma, void* stream);

/* nsteps steps of the optimal SSP-RK3 scheme (Eq. ssp) with step dt, in place on U
 * (device, K*E).  Each stage recomputes the sensor from the stage state.  The stage
 * states live in the context's buffers.  Launch sequence is replayed from a CUDA graph
 * cached per (U, dt, nsteps, stream) unless the stream is being captured.  nsteps = 0
 * does nothing; a negative nsteps or a non-finite dt is DGW_EINVAL. */
dgw_status dgw_rk_step(dgw_ctx* ctx, void* U, double dt, int nsteps, void* stream);

/* As dgw_rk_step for a state held in HOST memory: copies U_in (host, K*E elements,
 * pinned for asynchronous copies) to the device, runs nsteps steps and copies the
 * result to U_out (host; may equal U_in).  Returns after the stream has finished.
 * For the scalar laws on 2D meshes not periodic in y (at least two tile rows high), with
 * rk_order 3, the first and the last step run as a pipeline over bands of rows,
 * overlapping the input copy, the three stages and the output copy; the context then
 * uses streams of its own, ordered after the work already on `stream` and joined back to
 * it.  Otherwise the whole state is copied in, stepped and copied out.  nsteps >= 1. */
dgw_status dgw_rk_step_host(dgw_ctx* ctx, const void* U_in, void* U_out, double dt,
                            int nsteps, void* stream);

/* Total mass sum_e int_{K_e} U_h dx = sum_e |K_e| c_0^e (Euler: of the density) in
 * double, by a fixed-order tree (bitwise reproducible).  Blocks until the result is on
 * the host. */
dgw_status dgw_mass(dgw_ctx* ctx, const void* U, double* host_mass, void* stream);

/* The context's time t, which DGW_BC_STATE sides read (the paper's double Mach
 * reflection moves its top boundary's switch with time): dgw_set_time sets it (ordered on
 * the stream), each step of dgw_rk_step / dgw_rk_step_host advances it by dt on the
 * device, and dgw_residual / dgw_sensor evaluate at it.  dgw_get_time synchronizes the
 * stream and returns it.  A new context starts at t = 0. */
dgw_status dgw_set_time(dgw_ctx* ctx, double t, void* stream);
dgw_status dgw_get_time(dgw_ctx* ctx, double* t, void* stream);

/* Reads and clears the context's device-side error flags.  Synchronizes the stream.
 * DGW_ETIMEOUT: a stage kernel's bounded wait for its TMA tile copy gave up, so that
 * tile was skipped and the output is incomplete; DGW_ENONFINITE: a stage produced a
 * NaN or Inf; else DGW_OK. */
dgw_status dgw_sync_status(dgw_ctx* ctx, void* stream);

/* Diagnostic: poll limit of the stage kernels' bounded waits on their TMA copies (2D
 * meshes whose rows are 16-byte multiples).  0 restores the default (2^22 polls); a
 * negative value makes every such wait give up at once: the kernel then still waits
 * (bounded) for its copy to land, sets the flag that dgw_sync_status reports as
 * DGW_ETIMEOUT and skips the tile.  Exists so that tests can exercise that path without
 * a hang.  Drops the context's cached graphs. */
dgw_status dgw_debug(dgw_ctx* ctx, int wait_limit);

/* Which kernel runs the context's whole-mesh stage launches on 2D FP32 meshes whose rows
 * are 16-byte multiples: 0 (the default) the persistent kernel (one 512-thread CTA per
 * SM walking tiles of 32 x 32 cells, the next tile's data loaded during the current
 * one's arithmetic) when the mesh has at least four such tiles per SM, else the tile
 * kernel (one CTA per 32 x 16-cell tile); 1 always the tile kernel; 2 the persistent
 * kernel wherever it applies.  The two kernels give bitwise the same results.  Any
 * other choice is DGW_EINVAL.  Drops the context's cached graphs. */
dgw_status dgw_set_stage_kernel(dgw_ctx* ctx, int choice);

/* ------------------------------------------------------------------------------------
 * Discrete adjoint (the paper has no counterpart: it differentiates the discrete scheme
 * of Sec. 2-4).  Built for periodic meshes with the advection and Burgers fluxes;
 * other contexts return DGW_EUNSUPPORTED.  Non-smooth points use subgradients:
 * d min(1, r)/dr = [r < 1], d|x| = sign(x) (sign(0) = 0), a maximum picks its first
 * maximising argument, and the eps_s guard / b threshold are constant pieces.  The
 * context allocates 4 + 2*dim state-sized buffers on first use.  The Euler system and
 * the ZHAO sensor return DGW_EUNSUPPORTED.
 * ---------------------------------------------------------------------------------- */

/* out = J_L(U)^T lam, the transpose Jacobian of L = M^{-1} R_stab (Eq. weak2 with the
 * stabilization of Sec. 3 and the sensor of Sec. 4) at U, applied to lam.  All three
 * device arrays K*E; out must not overlap U or lam. */
dgw_status dgw_residual_vjp(dgw_ctx* ctx, const void* U, const void* lam, void* out, void* stream);

/* Reverse of one SSP-RK3 step (Eq. ssp) from the state U_n at the start of the step:
 * lam_n = (dU^{n+1}/dU^n)^T lam_np1.  The two stage states are recomputed from U_n.
 * lam_n may equal lam_np1. */
dgw_status dgw_adjoint_step(dgw_ctx* ctx, const void* U_n, const void* lam_np1, void* lam_n, double dt,
                            void* stream);

/* One SSP-RK3 step (Eq. ssp) from U that keeps its two stage states: U1 = U + dt L(U)
 * and U2 = 3/4 U + 1/4 (U1 + dt L(U1)) are written to the caller's arrays (device, K*E),
 * and U^{n+1} to U_next when it is not NULL (U_next may equal U; NULL skips the third
 * stage).  U1 and U2 must not overlap U, U_next or each other.  For checkpointed
 * gradients: the recomputation of a segment stores the stage states, and the reverse
 * step then takes them (dgw_adjoint_step_stages) instead of recomputing them. */
dgw_status dgw_rk_step_stages(dgw_ctx* ctx, const void* U, double dt, void* U1, void* U2, void* U_next,
                              void* stream);

/* As dgw_adjoint_step, with the step's stage states U1, U2 given (as dgw_rk_step_stages
 * writes them from U_n) rather than recomputed; the result is the same bits. */
dgw_status dgw_adjoint_step_stages(dgw_ctx* ctx, const void* U_n, const void* U1, const void* U2,
                                   const void* lam_np1, void* lam_n, double dt, void* stream);

/* Misfit J = 1/2 int (U_h - U_target,h)^2 dx (exact: mass-matrix weighted) in double,
 * and optionally grad = dJ/dU = M (U - U_target) (device, K*E, may be NULL).  Blocks
 * until *host_J is set. */
dgw_status dgw_misfit(dgw_ctx* ctx, const void* U, const void* U_target, double* host_J, void* grad,
                      void* stream);

/* ------------------------------------------------------------------------------------
 * Batched ensemble: many independent meshes (their own size, degree, flux, time step)
 * advanced together.  The paper has no counterpart; each instance is the scalar problem
 * above.  The instances form groups by (dimension, degree); each group's persistent
 * kernel takes work items (stage, instance, chunk of tiles) in order, and an item waits,
 * with a bounded spin, only for its own instance's previous stage, so instances of
 * different sizes overlap.  The groups' kernels run side by side on streams the batch
 * owns, forked from and joined back into the caller's stream.
 * Fluxes: advection and Burgers (others return DGW_EUNSUPPORTED; reflecting walls
 * DGW_EINVAL).  Stabilization parameters and precision are common.
 * ---------------------------------------------------------------------------------- */
typedef struct dgw_batch dgw_batch;

/* Creates a batch of n instances (meshes[i], ps[i], fluxes[i]); allocates two stage
 * buffers of the packed state and small counters.  Time steps: dgw_batch_set_dt. */
dgw_status dgw_batch_create(int n, const dgw_mesh* meshes, const int* ps, const dgw_flux* fluxes,
                            const dgw_params* params, dgw_batch** out);
dgw_status dgw_batch_destroy(dgw_batch* b);

/* Packed state: one device array of *total coefficients; instance i occupies
 * [offsets[i], offsets[i] + K_i E_i) in the layout of a single context (mode-major).
 * Offsets are multiples of 4 elements. */
dgw_status dgw_batch_sizes(const dgw_batch* b, int64_t* total, int64_t* offsets);

/* Time step of every instance (host array of n doubles).  Synchronous. */
dgw_status dgw_batch_set_dt(dgw_batch* b, const double* dt);

/* L2 projection of instances first .. first+count-1 from samples at the nq-point Gauss
 * points (dgw_project layout, nq in 1..8), concatenated in instance order (device,
 * double, sum of E_i nq^dim_i values). */
dgw_status dgw_batch_project(dgw_batch* b, int nq, int first, int count, const double* samples,
                             void* U, void* stream);

/* nsteps SSP-RK3 steps (Eq. ssp) of every instance, in place on the packed state U. */
dgw_status dgw_batch_rk_step(dgw_batch* b, void* U, int nsteps, void* stream);

/* For each group alone, times `steps` steps for every tile height built (2D float: tiles
 * 32 cells wide and 2, 4 or 8 rows high; 2D double: 4 rows; 1D: 128 x 1) and every
 * work-item size (1, 2, 4, 8, 16 tiles) on a copy of U, and keeps the fastest pair for
 * that group.  *chosen_chunk (may be NULL) receives the work-item size of the group with
 * the most cells.  Allocates a temporary copy of U.  The schedule changes no result. */
dgw_status dgw_batch_autotune(dgw_batch* b, void* U, int steps, int* chosen_chunk, void* stream);

/* Schedule of the group of instances of dimension dim and degree p: the tile height of its
 * kernel (*rows) and the tiles per work item (*chunk).  Either pointer may be NULL.  Until
 * an autotune or dgw_batch_set_schedule: 1D items of 2 tiles; 2D float tiles of 8 rows and
 * items of 16 tiles; 2D double tiles of 4 rows and items of 16 tiles. */
dgw_status dgw_batch_schedule(const dgw_batch* b, int dim, int p, int* rows, int* chunk);

/* Sets that schedule (a tile height that is built, chunk >= 1; DGW_EINVAL otherwise), e.g.
 * one an earlier autotune found.  Synchronous.  The schedule changes no result. */
dgw_status dgw_batch_set_schedule(dgw_batch* b, int dim, int p, int rows, int chunk);

/* Reads and clears the batch's error flag: DGW_ETIMEOUT if a wait gave up,
 * DGW_ENONFINITE for a non-finite result.  Synchronizes the stream. */
dgw_status dgw_batch_sync_status(dgw_batch* b, void* stream);

/* Diagnostic: spin limit of the waits, and (unreachable != 0) make every dependent
 * wait ask for one tile more than exists, so that it gives up: tests the bounded-wait
 * path without a hang. */
dgw_status dgw_batch_debug(dgw_batch* b, long long wait_limit, int unreachable);

/* SSP-RK3 steps for callers that cannot allocate device memory (the paper has no
 * counterpart; this is a deployment convenience).  Such callers include applications
 * whose device memory all belongs to another allocator (a framework's pool that leaves
 * nothing to cudaMalloc), and real-time or safety-critical code that may not allocate
 * after start-up, where an allocation can block or fail at an arbitrary point.
 * The arguments combine those of dgw_create and dgw_rk_step, and the result equals
 * theirs, but nothing is allocated: the two stage states live in one file-scope
 * device array of 2 x 8 MiB (+256 bytes) that every GPU loading the library keeps
 * until the process exits.  K*E*elem_bytes must not exceed 8,388,608 bytes
 * (e.g. 256^2 cells of Q2 in FP64); larger states return DGW_EINVAL with a message.
 * The first call on a device, and the first for each (precision, dimension, degree)
 * there, looks up the array's device address and uploads the operator tables
 * synchronously: make those calls before any stream capture.  Later calls only
 * enqueue kernels on the stream.  All calls share the array, so calls whose work
 * overlaps on the GPU (other streams, other threads) race and corrupt each other:
 * order them on one stream.  Device-side conditions are not reported by this entry
 * point (there is no context to hold the flag): neither non-finite results nor a
 * bounded TMA wait that gave up, after which a tile is skipped and its output keeps
 * whatever the array held before.  Scalar laws only: the Euler system returns
 * DGW_EUNSUPPORTED. */
dgw_status dgw_rk_step_noalloc(const dgw_mesh* mesh, int p, const dgw_flux* flux,
                               const dgw_params* params, void* U, double dt, int nsteps,
                               void* stream);

/* Diagnostic: the float sin/cos the FP32 kernels use for the KPP flux (Sec. 5 KPP
 * problem, F = (sin u, cos u)), applied to n device floats x; results in s and c
 * (device).  Exists so that tests can bound its error against double precision. */
dgw_status dgw_selftest_sincos(const float* x, float* s, float* c, int64_t n, void* stream);

/* Diagnostic: the volume term of the KPP problem at Q3 (Eq. weak2, F = (sin u, cos u) at
 * the 5 x 5 Gauss points) for ntiles tiles of 128 cells, by the packed-FP32 CUDA-core code
 * of the stage kernel (variant 0) or on the tensor cores (variant 1: tcgen05.mma
 * kind::tf32 in three passes, hi.hi + hi.lo + lo.hi of a TF32 split, accumulators in
 * tensor memory).  U: device float[16][ntiles * 128] (mode-major, k = i + 4 j); out: the
 * same shape, acc_k = sum over the Gauss points of W grad(phi_k).F in reference units.
 * Synchronous; *ms (host, may be NULL) receives the kernel's duration from CUDA events
 * on the stream.  Exists so that tests and the benchmark can compare the two on the same
 * work; DGW_ETIMEOUT if a bounded wait of variant 1 gave up. */
dgw_status dgw_selftest_tc_volume(const float* U, float* out, int64_t ntiles, int variant, float* ms,
                                  void* stream);

/* Message of the last failing call on this thread ("" if none). */
const char* dgw_last_error(void);

/* Library version string. */
const char* dgw_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DGW_H */
