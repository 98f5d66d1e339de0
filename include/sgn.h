/*
 * sgn.h - C ABI of libsgn.so: the split-form summation-by-parts (SBP)
 * semi-discretization of the 2D hyperbolized Serre-Green-Naghdi (SGN)
 * equations with variable bathymetry (arXiv 2601.02540), fused with classical
 * fourth-order Runge-Kutta stages, on one NVIDIA B300 GPU (sm_103a).
 *
 * The operations and the passages of the paper that define them:
 *   sgn_rhs          the right-hand side of eq. (sd_periodic_2D_SGN) (periodic,
 *                    Sec. 4.1) or eq. (semi_2D) (reflecting walls with SATs,
 *                    Sec. 4.2), with the second-order SBP operators and SATs of
 *                    the remark "Concrete SBP operators and SATs" (Sec. 4).
 *   sgn_init_aux     eq. (initialization) of Sec. 6: eta = h and
 *                    w = -h (D_x u + D_y v) + 3/2 (u D_x b + v D_y b).
 *   sgn_step         classical RK4 with a fixed time step applied to that RHS.
 *   sgn_mass_energy  total mass 1^T M h and energy 1^T M E of Thm. 4.1/4.2 and
 *                    the semi-discrete energy rate <d_q E, q_t>_M of eq.
 *                    (splitcondition).
 *   sgn_mms_exact, sgn_mms_source, sgn_step_mms   the manufactured solution
 *                    of Sec. 6.1.2 and RK4 with its source terms.
 *   sgn_step_sponge  RK4 with the relaxation zones of the wave-tank
 *                    experiments (Sec. 6).
 *   sgn_step_relaxed energy-conserving relaxation RK4 (named as future work
 *                    in the paper's conclusions; energy of Thm. 4.1).
 *   sgn_step_adaptive  adaptive time integration with an embedded
 *                    five-stage third-order FSAL pair and step-size control
 *                    (Sec. 6).
 *   sgn_rhs_vjp, sgn_step_record, sgn_step_vjp, sgn_step_record_tape,
 *   sgn_step_vjp_tape   the discrete adjoint of the RHS and of one RK4 step
 *                    (no counterpart in the paper).
 *
 * Data layout.  A state is five planes (h, u, v, w, eta), each plane nx*ny
 * values, x fastest: element (f, j, i) at index f*nx*ny + j*nx + i.  Node
 * (i, j) sits at x_i = xmin + i*dx, y_j = ymin + j*dy, where
 *   periodic:   dx = (xmax - xmin) / nx       (x_max is the image of x_min)
 *   reflecting: dx = (xmax - xmin) / (nx - 1) (both walls are nodes)
 * and likewise in y.  The bathymetry b is one plane.
 *
 * Precision (sgn_params.prec):
 *   SGN_F64         state, RHS and stage states in double.
 *   SGN_F32         state, RHS and stage states in float.
 *   SGN_F32_F64ACC  the caller's state q (= q_n) and the RK accumulator are
 *                   double; the RHS and the intermediate stage states are
 *                   float.
 *   SGN_DF64        the state and the RK accumulator are double; the RHS is
 *                   evaluated, and the intermediate stage states are stored,
 *                   in double-word arithmetic (a float pair hi + lo, about 48
 *                   significant bits, relative rounding ~2^-48) on the FP32
 *                   units, which on this GPU outnumber the FP64 units 64 to
 *                   one.  The adjoint, relaxed, manufactured and
 *                   relaxation-zone entry points need SGN_F64; the adaptive
 *                   integrator takes SGN_F64 or SGN_DF64.
 *   "state type" below means double for SGN_F64, SGN_F32_F64ACC and SGN_DF64,
 *   float for SGN_F32.  Bathymetry arguments are always double.  Diagnostics are always
 *   accumulated in double.
 *
 * Memory and streams.  Every pointer named *_dev is device memory of the
 * current CUDA device, owned by the caller, contiguous in the layout above,
 * aligned to at least 16 bytes and not overlapping any other argument unless
 * stated.  The context owns its own scratch (RK registers, reduction
 * partials), allocated in sgn_create.  `stream` is a cudaStream_t (NULL = the
 * legacy default stream).  Calls are asynchronous on `stream` except
 * sgn_create, sgn_destroy, sgn_mass_energy and sgn_check, which synchronize.
 * A context may be used by one stream at a time.
 *
 * Errors.  Every call returns a status; nothing is thrown and nothing exits.
 * Invalid arguments return SGN_E_INVAL without launching any kernel.  Kernels
 * latch a device flag when a stage input has h <= 0 (SGN_E_NONPOSITIVE_H) or a
 * non-finite h (SGN_E_NONFINITE); the flag is reported (and cleared) by the
 * next synchronizing call.  sgn_last_error() returns a message for the last
 * failure of the calling thread.
 */
#ifndef SGN_H
#define SGN_H

#include <stddef.h>

#if defined(__GNUC__)
#define SGN_API __attribute__((visibility("default")))
#else
#define SGN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SGN_OK = 0,
    SGN_E_INVAL = 1,          /* bad argument: null pointer, size, parameter */
    SGN_E_NOMEM = 2,          /* device or pinned-host allocation failed */
    SGN_E_CUDA = 3,           /* a CUDA runtime call failed */
    SGN_E_NONPOSITIVE_H = 4,  /* a stage input had h <= 0 (dry state; excluded by the paper) */
    SGN_E_NONFINITE = 5,      /* a stage input had a non-finite h */
    SGN_E_TIMEOUT = 6,        /* a bounded device wait gave up */
    SGN_E_UNSUPPORTED = 7     /* valid request the library does not implement */
} sgn_status;

typedef enum { SGN_BC_PERIODIC = 0, SGN_BC_REFLECTING = 1 } sgn_bc;
typedef enum { SGN_F64 = 0, SGN_F32 = 1, SGN_F32_F64ACC = 2, SGN_DF64 = 3 } sgn_prec;

typedef struct {
    int nx, ny;                    /* nodes per direction, each >= 3; ny <= 524280
                                      (65535 rows of 8-node blocks: the launch grid's
                                      y limit); nx*ny < 2^32 except for SGN_F64 */
    double xmin, xmax, ymin, ymax; /* domain, xmax > xmin, ymax > ymin */
    int bc;                        /* sgn_bc, both directions */
    double g;                      /* gravitational acceleration, > 0 */
    double lambda;                 /* relaxation parameter, >= 0 */
    int prec;                      /* sgn_prec */
} sgn_params;

typedef struct sgn_ctx sgn_ctx;

/* Create a context for one grid.  Validates `p`, allocates the scratch and
 * copies the bathymetry b_dev (double, nx*ny, device) into the context.
 * Synchronizes.  On failure *out is NULL.  SGN_F64 contexts pick the tile
 * height of their stage kernels (32 x 8, 32 x 16 or 32 x 24) for the SM count
 * of the current device: the one with the least FP64 work on the most loaded
 * SM; the results are the same at every height. */
SGN_API sgn_status sgn_create(const sgn_params* p, const void* b_dev, sgn_ctx** out);

/* Free the context and its scratch.  Synchronizes.  NULL is a no-op. */
SGN_API sgn_status sgn_destroy(sgn_ctx* ctx);

/* Replace the bathymetry (double, nx*ny, device).  Asynchronous on stream. */
SGN_API sgn_status sgn_set_bathymetry(sgn_ctx* ctx, const void* b_dev, void* stream);

/* Initialize the auxiliary variables in place (eq. (initialization)): reads
 * h, u, v of q_dev (state type) and writes w and eta, evaluated in double. */
SGN_API sgn_status sgn_init_aux(sgn_ctx* ctx, void* q_dev, void* stream);

/* dq_dev = RHS(q_dev): both state type, five planes, no overlap.  In
 * SGN_F32_F64ACC the inputs are rounded to float and the RHS is evaluated in
 * float, then widened. */
SGN_API sgn_status sgn_rhs(sgn_ctx* ctx, const void* q_dev, void* dq_dev, void* stream);

/* Advance q_dev (state type, in place) by nsteps >= 0 classical RK4 steps of
 * size dt (finite, > 0): 4 fused RHS+stage launches per step (SGN_F32: 2, two
 * stages per launch, unless sgn_set_stage_fusion turns that off).  On grids of at
 * most 2^21 nodes (launch-bound) runs of 50 steps are replayed from a CUDA
 * graph, captured on the context's first such call for this (q_dev, dt) on a
 * private stream; the launches and results are those of the direct path.
 * When `stream` is itself capturing, the steps are launched directly. */
SGN_API sgn_status sgn_step(sgn_ctx* ctx, void* q_dev, double dt, int nsteps, void* stream);

/* sgn_step that also monitors every new state: the fourth stage launch of
 * each step (which produces q_{n+1}) reduces its mass 1^T M h, energy 1^T M E
 * and shifted energy 1^T M E' (Thm. 4.1; as out[0..2] of sgn_mass_energy, and
 * equal to them bit for bit: the same per-node arithmetic on the stored
 * double state and the same fixed-order reduction).  out (host, 3*nsteps
 * doubles) receives {mass, energy, shifted energy} after each step.  The
 * energy rate (which needs one more RHS evaluation) is not monitored.
 * Synchronizes `stream` at the end and reports a latched h <= 0 / non-finite
 * flag.  The first call with more steps than before allocates 4 doubles per
 * step of device scratch. */
SGN_API sgn_status sgn_step_diag(sgn_ctx* ctx, void* q_dev, double dt, int nsteps, double* out, void* stream);

/* The end-to-end path for a state in host memory: copies the five planes at
 * q_host ([5][ny][nx], x fastest, state type of prec, as q_dev elsewhere)
 * into device memory owned by the context, advances them nsteps >= 0 RK4
 * steps of size dt as sgn_step, or as sgn_step_diag when out is non-NULL
 * (host, 3*nsteps doubles: mass, energy and shifted energy after each step),
 * and copies the result back over q_host.  One copy each way per call, on
 * `stream`; page-locked q_host moves at the link rate, pageable memory goes
 * through the CUDA runtime's staging buffers.  Synchronizes `stream` and reports a latched
 * h <= 0 / non-finite flag (the state is not copied back when the steps
 * report an error).  q_host in device memory is SGN_E_INVAL.  The first call
 * allocates the device state (5 planes), kept until sgn_destroy; calls on one
 * context do not overlap. */
SGN_API sgn_status sgn_step_host(sgn_ctx* ctx, void* q_host, double dt, int nsteps, double* out, void* stream);

/* Diagnostics of q_dev (state type), accumulated in double in a fixed order:
 * per-node values summed over 32 x 8 node bands, then the band sums in band
 * order.  The order depends on the grid only (not on the precision mode or
 * the kernels' tile shape), so the results are bitwise reproducible, and the
 * mass and energies of a given double state agree bit for bit across
 * contexts, the batched path and sgn_mass_energy_noalloc:
 *   out[0] = 1^T M h       out[1] = 1^T M E      out[2] = 1^T M E'
 *   out[3] = <d_q E, RHS(q)>_M
 * with E = h((u^2+v^2)/2 + w^2/6 + g/2 (h + 2b) + lambda/6 (eta/h - 1)^2)
 * and E' = E + g b^2/2 (the same energy shifted by a constant in time).
 * out is host memory of 4 doubles.  Synchronizes `stream`, then reports any
 * latched device flag. */
SGN_API sgn_status sgn_mass_energy(sgn_ctx* ctx, const void* q_dev, double* out, void* stream);

/* The diagnostics of sgn_mass_energy for callers that may not allocate device
 * memory: code embedded in a framework whose allocator owns every byte of the
 * device, latency-critical loops where cudaMalloc/cudaFree would implicitly
 * synchronize the device, plugins that are not allowed to allocate.  There is
 * no counterpart in the paper; it is a second way to run the same reduction.
 *
 * Needs no context: p describes the grid (prec must be SGN_F64, else
 * SGN_E_UNSUPPORTED), b_dev is the bathymetry (double, nx*ny, device), q_dev
 * the state (double, five planes, device, 16-byte aligned), out 4 doubles of
 * host memory, filled as by sgn_mass_energy.  Calls no allocating routine:
 * the per-band partial sums live in a 2 MiB array of static device memory
 * that every GPU which loads the library keeps until the process exits.  That
 * limits the grid to 32768 blocks of 32x16 nodes (16,777,216 nodes, e.g.
 * 4096x4096); larger grids return SGN_E_INVAL.  The first call on a device
 * looks up the array's device address and sets the kernel's shared-memory
 * limit (make that first call before any stream capture).  All calls share
 * the one array: calls that overlap on the GPU (other streams, other threads)
 * race and must be serialized by the caller.  Synchronizes `stream`; reports a
 * non-positive or non-finite h like sgn_mass_energy. */
SGN_API sgn_status sgn_mass_energy_noalloc(const sgn_params* p, const void* b_dev, const void* q_dev,
                                           double* out, void* stream);

/* Adjoint of the RHS (the paper has no adjoint; this is the exact transpose of
 * the Jacobian of the discrete RHS of eqs. (sd_periodic_2D_SGN) / (semi_2D) as
 * sgn_rhs evaluates it):
 *   qbar_dev  = J(q)^T abar            (overwritten, five planes)
 *   bbar_dev += (d RHS / d b)^T abar   (accumulated, one plane)
 * All double, device; qbar_dev must not overlap q_dev or abar_dev.  SGN_F64
 * contexts only (else SGN_E_UNSUPPORTED).  Three launches: the tape of the
 * RHS at q (its intermediate values, SGN_TAPE_PLANES planes, written by the
 * FP64 stage kernel), then the two adjoint passes, which read it.  The first
 * adjoint call of a context allocates 99 planes of scratch (SGN_E_NOMEM if
 * that fails).  Asynchronous. */
SGN_API sgn_status sgn_rhs_vjp(sgn_ctx* ctx, const void* q_dev, const void* abar_dev, void* qbar_dev,
                               void* bbar_dev, void* stream);

/* Like sgn_step, and records every step's stage states for the adjoint:
 * before step n the stash slot n (20 planes at stash_dev + 20*n*nx*ny doubles)
 * receives [q_n | Q2 | Q3 | Q4] with Q2 = q_n + dt/2 k1, Q3 = q_n + dt/2 k2,
 * Q4 = q_n + dt k3.  stash_dev holds nsteps slots (caller-owned, device,
 * double).  SGN_F64 only.  Asynchronous. */
SGN_API sgn_status sgn_step_record(sgn_ctx* ctx, void* q_dev, double dt, int nsteps, void* stash_dev,
                                   void* stream);

/* Adjoint of one classical RK4 step of size dt, using one stash slot written
 * by sgn_step_record: on entry qbar_dev holds the cotangent of q_{n+1}, on
 * return that of q_n:  k4bar = dt/6 qbar', Q4bar = J(Q4)^T k4bar,
 * k3bar = dt/3 qbar' + dt Q4bar, Q3bar = J(Q3)^T k3bar, k2bar = dt/3 qbar' +
 * dt/2 Q3bar, Q2bar = J(Q2)^T k2bar, k1bar = dt/6 qbar' + dt/2 Q2bar,
 * Q1bar = J(q_n)^T k1bar, qbar = qbar' + Q1bar + Q2bar + Q3bar + Q4bar, and
 * bbar_dev += sum_s (d RHS / d b)(Q_s)^T ks_bar.  Nine launches: the tape
 * of the RHS at each Q_s, and the two adjoint passes per stage, the second
 * pass of stages 4, 3, 2 fused with the first pass of the stage before it.
 * Internally the stage cotangents are carried with the scales
 * dt/6, dt^2/6, dt^3/12, dt^4/24 factored out; a dt for which dt^4/24 is not a
 * normal double returns SGN_E_INVAL.  The first adjoint call of a context
 * allocates 99 planes of scratch (SGN_E_NOMEM if that fails).  SGN_F64 only.
 * Asynchronous. */
SGN_API sgn_status sgn_step_vjp(sgn_ctx* ctx, const void* stash_dev, void* qbar_dev, void* bbar_dev,
                                double dt, void* stream);

/* Planes of the tape of one RHS evaluation: per node, intermediate values of
 * the RHS (1/h, -P2/h, the unscaled differences of h, u, v, w, eta + 3/2 b,
 * u^2, v^2, the continuity fluxes A_x, A_y, D_x(hu) - A_x, D_y(hv) - A_y and
 * the RHS of u, v, w), which the adjoint passes read instead of recomputing. */
#define SGN_TAPE_PLANES 21

/* Like sgn_step_record, and the stage kernels also write the tapes of the
 * step's four RHS evaluations: before step n the tape slot n
 * (4 * SGN_TAPE_PLANES planes at tape_dev + 4 * SGN_TAPE_PLANES * n * nx*ny
 * doubles) receives [T(q_n) | T(Q2) | T(Q3) | T(Q4)].  The stage states and
 * q_{n+1} are those of sgn_step_record bit for bit.  tape_dev: caller-owned,
 * device, double, nsteps slots, 16-byte aligned; NULL with nsteps > 0 is
 * SGN_E_INVAL.  SGN_F64 only.  Asynchronous. */
SGN_API sgn_status sgn_step_record_tape(sgn_ctx* ctx, void* q_dev, double dt, int nsteps, void* stash_dev,
                                        void* tape_dev, void* stream);

/* sgn_step_vjp with the step's tapes from sgn_step_record_tape (one tape slot,
 * 4 * SGN_TAPE_PLANES planes): five launches (the second pass of stages 4, 3
 * and 2 each fused with the first pass of the stage before it) and the same
 * results as sgn_step_vjp bit for bit.  NULL tape_dev is SGN_E_INVAL. */
SGN_API sgn_status sgn_step_vjp_tape(sgn_ctx* ctx, const void* stash_dev, const void* tape_dev,
                                     void* qbar_dev, void* bbar_dev, double dt, void* stream);

/* ---- Manufactured solution (Sec. 6.1.2) ----------------------------------
 * The paper verifies the full 2D scheme, both boundary treatments, with the
 * manufactured solution
 *   b   = 0.08 (cos 2pi x cos 2pi y + 1/2 cos 4pi x cos 4pi y)
 *   h   = 2 + 1/2 sin 2pi x sin 2pi y cos 2pi t - b
 *   u   = 0.3 sin 2pi x sin 2pi t,  v = 0.3 sin 2pi y sin 2pi t
 *   eta = h,  w = -h (u_x + v_y) + 3/2 (u b_x + v b_y)
 * (on [-1,1]^2 with lambda = 500 to t = 1), made exact by source terms
 * S = q_t - F(q), F the continuum right-hand side of eq. (2D_hyperbolic_SGN)
 * in primitive variables.  Node (i, j) of the context's grid sits at
 * (xmin + i dx, ymin + j dy).  All double, device, five planes.
 *
 * sgn_mms_exact: q_dev <- the manufactured state at time t; b_dev (one
 *   plane, or NULL) <- b.  Asynchronous.
 * sgn_mms_source: s_dev <- S at every node at time t.  Asynchronous.
 * sgn_step_mms: nsteps classical RK4 steps of size dt from time t0 of
 *   q' = RHS(q) + S(t), the source evaluated at the stage times t_n,
 *   t_n + dt/2, t_n + dt/2, t_n + dt inside the four fused stage launches.
 *   SGN_F64 contexts only (else SGN_E_UNSUPPORTED).  Asynchronous; the
 *   context's bathymetry should be the manufactured b (sgn_mms_exact then
 *   sgn_set_bathymetry). */
SGN_API sgn_status sgn_mms_exact(sgn_ctx* ctx, double t, void* q_dev, void* b_dev, void* stream);
SGN_API sgn_status sgn_mms_source(sgn_ctx* ctx, double t, void* s_dev, void* stream);
SGN_API sgn_status sgn_step_mms(sgn_ctx* ctx, void* q_dev, double t0, double dt, int nsteps, void* stream);

/* Relaxation zones (Sec. 6, the wave-tank experiments: zones at the ends of
 * the domain absorb outgoing waves): nsteps classical RK4 steps of size dt of
 *   q' = RHS(q) - sigma(x, y) (q - q0)
 * on q_dev (double, in place), q0_dev the rest state (double, five planes, not
 * overlapping q_dev).  sigma rises quadratically from 0 at the inner edge of a
 * zone to sigma_max at the domain boundary: with d = min(x - xmin, xmax - x),
 * sigma_x = sigma_max ((width_x - d) / width_x)^2 for d < width_x, else 0;
 * likewise in y; corners take sigma_x + sigma_y; a width of 0 disables that
 * direction.  The source is evaluated at the stage inputs inside the four
 * fused stage launches.  SGN_F64 contexts only (else SGN_E_UNSUPPORTED).
 * Asynchronous. */
SGN_API sgn_status sgn_step_sponge(sgn_ctx* ctx, void* q_dev, double dt, int nsteps, const void* q0_dev,
                                   double width_x, double width_y, double sigma_max, void* stream);

/* Relaxation RK4: nsteps energy-conserving steps of nominal size dt > 0 on
 * q_dev (double, in place).  The paper names relaxation Runge-Kutta methods as
 * future work and shows that plain RK does not conserve the energy 1^T M E of
 * Thm. 4.1 / 4.2 in the fully discrete scheme.  Each step computes the plain
 * RK4 update q1 (the four fused stage launches of sgn_step), then the root
 * gamma near 1 of E(q + gamma (q1 - q)) = E(q), and sets q <- q + gamma (q1 - q);
 * the step advances time by gamma dt.  The energy change is summed per node in
 * a form without cancellation, reduced in a fixed order, and gamma is found by
 * Newton's method on the host (one reduction per step, a second only when
 * |gamma - 1| > 1e-3).  gammas (host, nsteps doubles, or NULL) receives gamma
 * per step, *t_out (or NULL) the time advanced.  Synchronizes `stream` every
 * step.  SGN_F64 contexts only (else SGN_E_UNSUPPORTED).  The first call of a
 * context allocates 5 planes of scratch.  A stage input with h <= 0 returns
 * SGN_E_NONPOSITIVE_H (non-finite: SGN_E_NONFINITE); no root near 1 returns
 * SGN_E_NONFINITE. */
SGN_API sgn_status sgn_step_relaxed(sgn_ctx* ctx, void* q_dev, double dt, int nsteps, double* gammas,
                                    double* t_out, void* stream);

/* The Runge-Kutta pairs of sgn_step_adaptive. */
typedef enum { SGN_PAIR_P5S3 = 0, SGN_PAIR_BS3 = 1 } sgn_pair;

/* Adaptive time integration of q_dev (double, in place) from t0 to t_end
 * (Sec. 6: an explicit third-order, five-stage Runge-Kutta method with the
 * first-same-as-last (FSAL) property and an embedded error estimator,
 * optimized for stability-limited hyperbolic problems, rtol = atol = 1e-6;
 * the paper does not print its coefficients).  `pair` selects
 *   SGN_PAIR_P5S3  a five-stage third-order FSAL pair with those properties,
 *                  constructed for this library: Butcher matrix of the
 *                  two-register form a_ij = b_j (j < i-1) with
 *                  a21 = 0.3464, a32 = 0.5544, a43 = 0.3078,
 *                  a54 = 0.25084211224332113157,
 *                  b = (-0.077114705798502101362, 0.51296293729322573879,
 *                       -0.53636230691175187515, 0.69586264419699749322,
 *                       0.40465143122003074449),
 *                  embedded second-order weights over k1..k5 and
 *                  k6 = f(q_{n+1}): bhat = (0.14576960111557976478,
 *                  0.13123039888442023522, 0.103, 0.1816, 0.1978, 0.2406);
 *                  stability polynomial 1 + z + z^2/2 + z^3/6 + 0.0324 z^4 +
 *                  0.006 z^5, stable on the imaginary axis up to |z| = 3.8798.
 *                  k_i = f(q_n + dt sum_{j<i} a_ij k_j), q_{n+1} = q_n +
 *                  dt sum b_i k_i, e = dt sum_{i<=6} (b_i - bhat_i) k_i.
 *                  Step size with the limiter rho(x) = 1 + atan(x - 1) and
 *                  eps = 0.9 / max(err, 1e-10): after an accepted attempt
 *                  dt_next = dt rho(eps^(0.7/3) eps_prev^(-0.4/3)) (Gustafsson's
 *                  PI control; eps_prev that of the previous accepted attempt,
 *                  1 before the first), after a rejected one
 *                  dt_next = dt rho(eps^(1/3)).  Five fused RHS launches per attempt.
 *   SGN_PAIR_BS3   the Bogacki-Shampine 3(2) FSAL pair: k2 = f(q_n + dt/2 k1),
 *                  k3 = f(q_n + 3dt/4 k2), q_{n+1} = q_n + dt (2/9 k1 + 1/3 k2 +
 *                  4/9 k3), k4 = f(q_{n+1}), e = dt (-5/72 k1 + 1/12 k2 + 1/9 k3
 *                  - 1/8 k4); dt_next = dt min(10, max(0.2, 0.9 err^(-1/3)))
 *                  (10 when err = 0).  Three fused RHS launches per attempt.
 * In both, k1 = f(q_n) is the FSAL slope of the previous accepted step; an
 * attempt is accepted when
 *   err = sqrt(mean over all 5 nx ny values of (e / (atol + rtol max(|q_n|, |q_{n+1}|)))^2) <= 1;
 * a rejected attempt is retried from q_n; a step that would pass t_end is cut
 * to land on it.  An attempt whose stage inputs have h <= 0 or a non-finite h
 * counts as rejected with err = +inf.  The first attempt has size dt0 > 0;
 * rtol, atol >= 0, not both 0; at most max_attempts attempts; an unknown pair
 * returns SGN_E_INVAL.  One reduction per attempt; the host reads err after
 * each attempt (synchronizes `stream` every attempt).
 * hist (host, 3*max_attempts doubles, or NULL) receives {dt, err, accepted}
 * per attempt; stats (host, 5 doubles) receives {accepted, rejected, t
 * reached, next dt, attempts}.  SGN_F64 or SGN_DF64 contexts (the RHS in
 * double or in float pairs; the state, the error norm in double; else
 * SGN_E_UNSUPPORTED).  The first call of a context allocates 40 planes of
 * 8-byte scratch (SGN_E_NOMEM if that fails).  An initial state with h <= 0 or
 * a non-finite h returns SGN_E_NONPOSITIVE_H / SGN_E_NONFINITE without an
 * attempt. */
SGN_API sgn_status sgn_step_adaptive(sgn_ctx* ctx, void* q_dev, double t0, double t_end, double dt0,
                                     double rtol, double atol, int max_attempts, int pair, double* hist,
                                     double* stats, void* stream);

/* ---- Ragged ensembles ----------------------------------------------------
 * Many independent grids (each its own size, boundary treatment, parameters
 * and fixed time step) advanced together: one launch per RK4 stage (SGN_F32:
 * per two stages and boundary class, see sgn_batch_set_stage_fusion) covers a
 * tile list spanning every instance, and sgn_batch_step replays CUDA graphs of
 * 26 steps.  The arithmetic per node is the single-grid kernel's, in the same
 * order, so each instance evolves exactly as with sgn_step.
 *
 * Packed layout: instance i owns nx_i*ny_i nodes starting at node offset
 * off_i = sum_{k<i} nx_k*ny_k.  Bathymetry: one plane per instance at off_i
 * (double).  State: five planes per instance at 5*off_i (state type of prec),
 * each plane nx_i*ny_i values, x fastest. */
typedef struct {
    int nx, ny;                    /* >= 3; ny <= 524280 and nx*ny < 2^32 (the batched
                                      precisions other than SGN_F64) as in sgn_params */
    double xmin, xmax, ymin, ymax;
    int bc;                        /* sgn_bc */
    double g, lambda;
    double dt;                     /* this instance's fixed RK4 step, > 0 */
} sgn_instance;

typedef struct sgn_batch sgn_batch;

/* Copy the instance table and the packed bathymetry, build the tile lists and
 * allocate the RK registers.  Synchronizes. */
SGN_API sgn_status sgn_batch_create(const sgn_instance* inst, int ninst, int prec, const void* b_dev,
                                    sgn_batch** out);
SGN_API sgn_status sgn_batch_destroy(sgn_batch* batch);
/* total nodes of all instances (the packed plane length), or -1 */
SGN_API long long sgn_batch_cells(const sgn_batch* batch);
/* eq. (initialization) for every instance, in place on the packed state */
SGN_API sgn_status sgn_batch_init_aux(sgn_batch* batch, void* q_dev, void* stream);
/* nsteps RK4 steps of every instance (each with its own dt), in place */
SGN_API sgn_status sgn_batch_step(sgn_batch* batch, void* q_dev, int nsteps, void* stream);
/* per-instance diagnostics as sgn_mass_energy: out[4*i + k], host, 4*ninst
 * doubles.  Synchronizes; reports a latched h <= 0 / non-finite flag. */
SGN_API sgn_status sgn_batch_mass_energy(sgn_batch* batch, const void* q_dev, double* out, void* stream);
/* Tile height 8*rows, rows in {1, 2, 4} (default 2). */
SGN_API sgn_status sgn_batch_set_rows(sgn_batch* batch, int rows);
/* on = 1: run the four RK4 stages with the persistent kernel (a grid of
 * resident blocks, resident blocks per SM x SMs, that walks the tile list and
 * prefetches the next tile's inputs into shared memory with cp.async while it
 * evaluates the current one); on = 0: one block per tile (default).  The same
 * arithmetic either way (equal results bit for bit).  The persistent kernel
 * serves the float compute types (SGN_F32, SGN_F32_F64ACC) and tile heights
 * 8 and 16 (rows 1, 2); otherwise on = 1 returns SGN_E_UNSUPPORTED. */
SGN_API sgn_status sgn_batch_set_persistent(sgn_batch* batch, int on);
/* SGN_F32 ensembles: on = 1 (default) advances sgn_batch_step two RK4 stages
 * per launch over 32 x 16 tiles (as sgn_set_stage_fusion for one grid; the
 * same states bit for bit, q_{n+1} alternately in q_dev and batch scratch,
 * an odd step count ends with one copy), one launch per boundary class
 * present (the periodic instances' tiles, then the reflecting ones, each
 * kernel with the registers of its own boundary treatment), so two or four
 * launches per step; on = 0 one launch per stage with the
 * tiling of sgn_batch_set_rows / sgn_batch_set_persistent; the persistent
 * kernel, when selected, takes precedence.  Other precisions: on = 1 is
 * SGN_E_UNSUPPORTED. */
SGN_API sgn_status sgn_batch_set_stage_fusion(sgn_batch* batch, int on);
SGN_API sgn_status sgn_batch_stage_fusion(const sgn_batch* batch, int* on);
/* The current tiling: *rows (1, 2, 4) and *persistent (0, 1). */
SGN_API sgn_status sgn_batch_tiling(const sgn_batch* batch, int* rows, int* persistent);
/* Time 8 steps of each tiling -- rows 1, 2, 4 with one block per tile, for
 * the float compute types rows 1, 2 with the persistent kernel, and for
 * SGN_F32 two stages per launch -- on a copy of q_dev (allocated and freed
 * here), in three rounds; keep the tiling with the fastest round and return
 * its rows in *rows_out (or NULL; see sgn_batch_tiling and
 * sgn_batch_stage_fusion for the kernel).  Synchronizes. */
SGN_API sgn_status sgn_batch_autotune(sgn_batch* batch, const void* q_dev, int* rows_out, void* stream);

/* Synchronize `stream` and report (and clear) the latched device flag. */
SGN_API sgn_status sgn_check(sgn_ctx* ctx, void* stream);

/* The tile height of an SGN_F64 context's stage kernels: 32 x (8 rows), rows
 * in {1, 2, 3}; sgn_create picks it (see there), sgn_set_tile_rows overrides
 * it (a height whose launch grid would exceed 65535 rows of tiles is
 * SGN_E_INVAL; other precisions: SGN_E_UNSUPPORTED).  Every height gives the
 * same results bit for bit.  Not thread-safe against launches on the
 * context. */
SGN_API sgn_status sgn_set_tile_rows(sgn_ctx* ctx, int rows);
SGN_API sgn_status sgn_tile_rows(const sgn_ctx* ctx, int* rows);

/* SGN_F32 contexts: on = 1 (default) advances sgn_step two RK4 stages per
 * launch (stages 1-2 and 3-4: the first stage of each pair is evaluated on
 * the tile grown by one node and its result stays in shared memory), 37
 * plane accesses per node and step instead of 74; on = 0 runs one launch
 * per stage.  The same states bit for bit either way.  The fused step
 * writes q_{n+1} alternately to q and to context scratch, so an odd step
 * count ends with one device copy into q.  sgn_step_diag always runs one
 * launch per stage.  Other precisions: SGN_E_UNSUPPORTED.  Not thread-safe
 * against launches on the context. */
SGN_API sgn_status sgn_set_stage_fusion(sgn_ctx* ctx, int on);

/* Human-readable name of a status, and the last error message of the calling
 * thread (never NULL). */
SGN_API const char* sgn_status_str(sgn_status s);
SGN_API const char* sgn_last_error(void);

/* Kernel launches issued by this library since load (all contexts). */
SGN_API unsigned long long sgn_launch_count(void);

/* The FP64 fused multiply-add rate of the current device, for the roofline of
 * the FP64 kernels (no counterpart in the paper).  One launch of 8 blocks of
 * 256 threads per SM; every thread runs 16 independent chains x <- x a + c
 * (0 < a < 1, so the values stay bounded) for `iters` iterations, a multiple
 * of 4 in [4, 2^20] (else SGN_E_INVAL).  *fma_count receives the number of
 * FMAs executed and *seconds the launch's duration, timed with CUDA events on
 * `stream` (rate = *fma_count / *seconds; a B300 SM completes 2 per clock).
 * Allocates and frees its small output buffer; synchronizes. */
SGN_API sgn_status sgn_measure_fp64_fma(int iters, double* fma_count, double* seconds, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SGN_H */
