/*
 * es.h -- C ABI of the GB300 locally relaxed entropy-stable RK step.
 *
 * Method: Ranocha, Dalcin & Parsani, "Fully-discrete explicit locally
 * entropy-stable schemes for the compressible Euler and Navier--Stokes
 * equations" (2020).  The library advances u' = f(u) (Eq. (ode)) where f is
 * the SBP-SAT semidiscretisation of Eq. (compressible_ns_diss) on a Cartesian
 * mesh of LGL hexahedra (periodic, or with the Dirichlet-penalty boundaries of
 * es_set_boundary), with an explicit Runge--Kutta method
 * (Eq. (RK-step)) and the local relaxation of Eq. (relaxation-local-gamma)
 * with gamma = min_kappa gamma_kappa (Theorem 2.3).
 *
 * Conventions (every entry point):
 *  - Return 0 (ES_OK) or a negative ES_ERR_* code.  Argument errors are
 *    detected on the host before anything is launched.
 *  - Device pointers are CUDA device memory of the current device; they are
 *    owned by the caller and never freed by the library.  The context owns its
 *    workspace and frees it in es_destroy.
 *  - Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL is the
 *    legacy default stream).  Errors found on the device (non-physical state,
 *    no relaxation root) are sticky bits read by es_status.
 *  - State layout ("SoA"): double q[5][K][Np], variable v = rho, rho u1,
 *    rho u2, rho u3, rho E; element e = ex + nx (ey + ny ez); node
 *    n = i + (p+1) (j + (p+1) k) with (i, j, k) the LGL indices along
 *    (x1, x2, x3).  K = nx ny nz, Np = (p+1)^3.
 *  - Not thread-safe per context: one host thread drives a context at a time.
 */
#ifndef ES_H
#define ES_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ES_OK 0
#define ES_ERR_INVALID (-1)     /* bad argument or unsupported configuration */
#define ES_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define ES_ERR_NONPHYSICAL (-3) /* rho <= 0 or p <= 0 met at some node */
#define ES_ERR_NO_ROOT (-4)     /* an element had r'(0) >= 0: no positive gamma_kappa */
#define ES_ERR_NOMEM (-6)       /* device or host allocation failed */
#define ES_ERR_TOO_LARGE (-7)   /* problem exceeds the fixed scratch of es_rhs_noalloc */

#define ES_RK_BS3 0 /* Bogacki--Shampine 3(2), b = (2/9, 1/3, 4/9, 0) */
#define ES_RK_RK4 1 /* classical RK(4,4) */
#define ES_RK_RK65 2 /* Butcher's six-stage fifth-order method, b = (7, 0, 32, 12, 32, 7)/90
                       (Section 4 pairs p = 4 with a fifth-order BSRK(8,5) whose coefficients
                       it does not print; es_set_tableau loads any explicit tableau) */

#define ES_FP64 0  /* every operation in FP64 */
#define ES_MIXED 1 /* FP32 fluxes/SATs/viscous terms; FP64 state, stage states,
                      entropy-variable increments, entropy sums and gamma solve */
#define ES_FP64X 2 /* fluxes/SATs/viscous terms in float-float arithmetic on the FP32 pipe
                      (hi + lo pairs of floats, ~2^-47 relative per operation, FP32 exponent
                      range), and so are the stage states, entropy-variable increments,
                      element sums and the gamma solve (joined to FP64 once per element);
                      FP64 state.  Meets the FP64 parity bars with the float-float rounding
                      unit.  es_rhs_noalloc evaluates such a configuration with the FP64
                      kernels. */
#define ES_MIXED_FF 3 /* FP32 fluxes/SATs/viscous terms as ES_MIXED; the stage states,
                      entropy-variable increments, the per-element sums and the gamma
                      solve in float-float on the FP32 pipe (FP64 state, FP64 gamma). */

#define ES_RELAX_NONE 0  /* baseline RK, gamma = 1 */
#define ES_RELAX_LOCAL 1 /* gamma = min_kappa gamma_kappa (Theorem 2.3) */
#define ES_RELAX_GLOBAL 2 /* one gamma per instance for eta = sum_kappa eta_kappa
                             (Eqs. (u-n-gamma), (t-n-gamma)); gamma_elem reports it */

typedef struct es_ctx es_ctx;

typedef struct {
  int p;                /* LGL degree, 2..5 */
  int nx, ny, nz;       /* elements per direction, each >= 1 */
  double lo[3], hi[3];  /* periodic box */
  double gamma_gas;     /* ratio of specific heats, > 1 */
  double mu;            /* dynamic viscosity; 0 = Euler (no viscous terms) */
  double Pr;            /* Prandtl number (mu > 0) */
  double R;             /* gas constant, p = rho R T */
  int interface_diss;   /* 0: entropy-conservative SAT^I; 1: + Rusanov diss^I;
                           2: + matrix diss^I in entropy variables,
                           (1/2) R |Lambda| T R^T [[w]] (Barth-scaled eigenvectors) */
  int relax;            /* ES_RELAX_* */
  int rk;               /* ES_RK_* */
  int precision;        /* ES_FP64, ES_MIXED, ES_FP64X or ES_MIXED_FF */
  double delta_floor;   /* elements whose RMS relative change over the step is
                           <= delta_floor are unconstrained (gamma_kappa = +inf);
                           <= 0 selects 1e-8 (ES_FP64, ES_FP64X) or 4e-6 (ES_MIXED,
                           ES_MIXED_FF:
                           64 eps_32, above the FP32 right-hand side's rounding noise) */
  double visc_diss;     /* diss^V coefficient alpha >= 0 (used when mu > 0; 0 = off):
                           interior penalty on the entropy-variable jump at every face,
                           alpha (2/h_m)(1/omega_0) (C_mm(q-) + C_mm(q+))/2 (w- - w+)
                           added to the interface flux, C_mm the viscous-flux block
                           of dw/dx_m (symmetric positive semidefinite) */
  double root_rtol;     /* stop of the gamma_kappa root solve (Section 4 leaves the
                           solver open): a Newton step |s| <= root_rtol gamma ends it
                           (the updated iterate is returned), as does a bracket of
                           width <= 4 2^-52 max(1, gamma).  In [0, 1); 0 selects 1e-8,
                           whose quadratic convergence leaves an error near 1e-16 gamma.
                           The float-float solves (ES_FP64X, ES_MIXED_FF) use at least
                           2^-40 and stop at a bracket of width 2^-44 max(1, gamma). */
} es_config;

/* Mesh, LGL/SBP tables (Section 3.1: diagonal-norm SBP on LGL nodes) and
 * device workspace for one configuration.  Allocates device memory on the
 * current device.  On error *out is NULL. */
int es_create(const es_config* cfg, es_ctx** out);

/* Frees the workspace; NULL is a no-op. Synchronises the device. */
void es_destroy(es_ctx* ctx);

/* f(q) of Eq. (ode): dqdt[5][K][Np] = the right-hand side of
 * Eq. (compressible_ns_diss) (volume flux differencing 2 D o F 1, SAT^I
 * (+ diss^I), BR1 viscous terms and SAT^V when mu > 0, + diss^V when also
 * visc_diss > 0).  If E_elem is not
 * NULL, E_elem[K] = (eta_kappa' f)(q) = sum_n P_n w(q_n).dqdt_n
 * (the integrand of Eq. (eta-est-1-RK)).  q and dqdt must not overlap. */
int es_rhs(es_ctx* ctx, const double* q, double* dqdt, double* E_elem, void* stream);

/* eta_elem[K] = eta_kappa(q) = 1^T P S_kappa (Section 3.2), S = -rho s/(gamma-1). */
int es_entropy(es_ctx* ctx, const double* q, double* eta_elem, void* stream);

/* Boundary treatment of direction dir (0, 1, 2 = x1, x2, x3) of a context
 * (Section 4.1.2 prescribes boundary data by penalising the numerical solution
 * against a given state; the penalty form is not printed).  Every direction is
 * periodic after es_create.  For kind != ES_BC_PERIODIC the faces x_dir = lo and
 * x_dir = hi are Dirichlet-penalty boundaries: the inviscid SAT uses the
 * interface flux between the element's trace and the prescribed exterior state
 * q_b (f_num(q_b, q) on the lo side, f_num(q, q_b) on the hi side), the BR1
 * gradient lifts toward (w + w(q_b))/2, and the viscous boundary flux is the
 * interior one.  q_b is evaluated on the device at each stage's time
 * t + c_i dt (es_advance: t is its time argument; es_rhs: the time set by
 * es_set_time, initially 0).
 *   ES_BC_STATE          params[10] = q_b on the lo side, then on the hi side
 *                        (conserved variables, physical).
 *   ES_BC_VISCOUS_SHOCK  params[4] = {Mach > 1, Reynolds > 0, Prandtl > 0,
 *                        speed}: the viscous-shock solution of Section 4.1.2
 *                        along dir (shock-frame upstream rho = u = 1,
 *                        p = 1/(gamma M^2), mu = 1/Re, V(x) from its implicit
 *                        solution, total enthalpy constant; exact for Pr = 3/4
 *                        and mu, Pr of the context equal to these), seen from a
 *                        frame moving with velocity speed: the shock is at
 *                        x_dir = speed t (speed = -1: upstream gas at rest).
 * Batches are periodic.  Errors: ES_ERR_INVALID for a bad direction, kind or
 * parameter list; ES_ERR_NOMEM if the boundary workspace cannot be allocated. */
#define ES_BC_PERIODIC 0
#define ES_BC_STATE 1
#define ES_BC_VISCOUS_SHOCK 2
int es_set_boundary(es_ctx* ctx, int dir, int kind, const double* params, int nparams);

/* Sets the time at which es_rhs evaluates prescribed boundary states (host value;
 * synchronous).  ES_ERR_INVALID for a non-finite t. */
int es_set_time(es_ctx* ctx, double t);

/* Replaces the context's Runge--Kutta method (Eq. (RK-step)) by the explicit tableau
 * with s <= 10 stages: a (host, s x s row-major, a[i*s + j] = a_ij, zero on and above
 * the diagonal), weights b[s] and stage times c[s] (host; copied, the caller keeps
 * ownership).  Requirements, else ES_ERR_INVALID: finite entries, a strictly lower
 * triangular, sum_j a_ij = c_i and sum_i b_i = 1 (1e-13), and b_i >= 0 unless the
 * context relaxes nothing (the entropy estimate Eq. (eta-est-1-RK) needs b_i >= 0).
 * Trailing stages with b_i = 0 are not evaluated.  Stage buffers are allocated here
 * (ES_ERR_NOMEM).  Takes effect with the next es_advance; no check of the order. */
int es_set_tableau(es_ctx* ctx, int s, const double* a, const double* b, const double* c);

/* One relaxation (last row of Eq. (relaxation-local-gamma), Theorem 2.3):
 * for every element the root gamma_elem[e] > 0 of
 *   eta_e(u_old + g (u_new - u_old)) - eta_e(u_old) - g d_eta[e] = 0,
 * then *gamma = min_e gamma_elem[e] (1 if no element is constrained) and
 * u_out = u_old + gamma (u_new - u_old).  All pointers are device memory;
 * u_out may alias u_new but not u_old.  Unconstrained elements report +inf. */
int es_relax_step(es_ctx* ctx, const double* u_old, const double* u_new, const double* d_eta,
                  double* gamma_elem, double* gamma, double* u_out, void* stream);

/* nsteps relaxed RK steps of size dt (Eq. (RK-step) + Eq. (eta-est-1-RK) +
 * Eq. (relaxation-local-gamma)), in place on q (device).  *t (device scalar)
 * advances by gamma dt per step (Eq. (t-n-gamma)).  gamma_hist[nsteps]
 * (device) receives each step's gamma if not NULL; gamma_elem[K] (device)
 * receives the last step's gamma_kappa if not NULL. */
int es_advance(es_ctx* ctx, double* q, int nsteps, double dt, double* t, double* gamma_hist,
               double* gamma_elem, void* stream);

/* One relaxed step (es_advance with nsteps = 1) that also returns both sides of
 * the local entropy inequality of Theorem 2.3,
 *   eta_kappa(u^n) <= eta_kappa(u^{n-1}) + gamma (eta_kappa^new - eta_kappa(u^{n-1})),
 * per element, all device arrays of K doubles (any may be NULL):
 *   eta_old[e]  = eta_kappa(u^{n-1}) = sum_n P_n S(u_n) (as es_entropy computes it);
 *   deta[e]     = eta_kappa^new - eta_kappa(u^{n-1}) = dt sum_i b_i (eta_kappa' f)(y^i),
 *                 the estimate of Eq. (eta-est-1-RK) formed from the step's own stage
 *                 values (those the relaxation used: FP32 right-hand sides in the
 *                 mixed modes) as sum_n P_n w(u_n).d_n - A_kappa in FP64;
 *   eta_new[e]  = eta_kappa(u^n) after the relaxed update (es_entropy of q);
 *   gamma_elem  = the step's gamma_kappa (+inf where unconstrained), *gamma (device
 *                 scalar) the step's gamma.
 * q (device, in place) and *t (device, may be NULL) advance as in es_advance.  With
 * ES_RELAX_NONE the estimate is still formed (gamma = 1), so the baseline step's
 * inequality can be checked too. */
int es_step_estimate(es_ctx* ctx, double* q, double dt, double* t, double* gamma, double* gamma_elem,
                     double* eta_old, double* deta, double* eta_new, void* stream);

/* es_advance on HOST buffers: copies q_host (5 K Np doubles) and *t_host to
 * the context's device buffers, advances, and copies q, t and gamma_hist
 * (nsteps doubles, may be NULL) back; returns after the stream completes.
 * Pinned host memory makes the copies asynchronous DMA. */
int es_advance_host(es_ctx* ctx, double* q_host, int nsteps, double dt, double* t_host,
                    double* gamma_hist_host, void* stream);

/* Node coordinates xyz[3][K][Np] (host memory), in the state layout. */
int es_node_coords(const es_ctx* ctx, double* xyz_host);

/* Synchronises `stream`, returns the first sticky device error
 * (ES_ERR_NONPHYSICAL, ES_ERR_NO_ROOT) or ES_ERR_CUDA, and clears the bits. */
int es_status(es_ctx* ctx, void* stream);

/* Number of kernel launches the context has enqueued since es_create. */
long long es_launch_count(const es_ctx* ctx);

/* Per-kernel timing (instrumentation, not part of the method).  While enabled,
 * every launch of the context is bracketed by CUDA events recorded on the
 * launching stream.  es_profile_read synchronises the device and returns,
 * per kernel kind (ES_KERNEL_*), the summed event time in ms and the launch
 * count since the last read, then resets them.  Arrays hold ES_KERNEL_COUNT
 * entries. */
#define ES_KERNEL_PREP 0    /* stage state + parameter vector */
#define ES_KERNEL_FACE 1    /* interface fluxes */
#define ES_KERNEL_GRAD 2    /* BR1 gradients + viscous flux */
#define ES_KERNEL_VOLUME 3  /* flux differencing, SATs, viscous divergence */
#define ES_KERNEL_RELAX 4   /* gamma_kappa root solve */
#define ES_KERNEL_OTHER 5   /* scalar bookkeeping, final update, entropy */
#define ES_KERNEL_COUNT 6
int es_profile_enable(es_ctx* ctx, int enable);
int es_profile_read(es_ctx* ctx, double* ms, long long* launches);

/* Right-hand side without a context: for callers that cannot call cudaMalloc
 * (code running where the allocator is off limits, e.g. inside another
 * library's allocation-free region or a host framework that owns all device
 * memory).  The paper has no counterpart; it is the same operation as es_rhs
 * (same kernels, same results) with the caller passing only inputs and
 * outputs: q and dqdt (device, [5][K][Np]) and optionally E_elem (device, [K]).
 * A config describes a periodic mesh: boundaries set with es_set_boundary
 * belong to a context and do not apply here.
 *
 * It allocates nothing: the kernels' scratch is one fixed array of
 * ES_NOALLOC_SCRATCH_BYTES (32 MiB) of device memory compiled into the
 * library, which every GPU that loads the library holds until the process
 * exits.  Problems whose scratch (es_rhs_noalloc_scratch_bytes) exceeds it are
 * rejected with ES_ERR_TOO_LARGE before any work is enqueued; invalid
 * configurations return ES_ERR_INVALID.
 *
 * The first call on each device runs a one-time set-up (it looks up the
 * array's device address with the device current and sets kernel attributes);
 * make that first call before any stream capture.  All calls share the array
 * and the status word inside it, so calls that overlap on the GPU (different
 * streams, or different host threads) race: serialise them.  Device-side
 * errors (non-physical states) are not reported by this call.
 * CUDA errors: if the calling thread already has a pending CUDA error from
 * earlier work, the call returns ES_ERR_CUDA before enqueueing anything and
 * leaves that error pending (it stays the caller's to read).  A runtime call or
 * launch of this entry point that fails returns ES_ERR_CUDA and clears the
 * error it raised, so it is not reported again by a later call. */
#define ES_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int es_rhs_noalloc(const es_config* cfg, const double* q, double* dqdt, double* E_elem, void* stream);
/* Scratch bytes es_rhs_noalloc needs for cfg (0 if cfg is invalid). */
size_t es_rhs_noalloc_scratch_bytes(const es_config* cfg);

/* Volume-kernel tile autotuning for this context: times every usable variant
 * (es_volume_variant) on two stages of the state q (device, [5][K][Np]; q is not
 * changed) and keeps the fastest for later calls.  Synchronises. */
int es_autotune(es_ctx* ctx, const double* q, void* stream);

/* The tile variant in use: 0..2 run the stage as k_prep + k_face + k_volume with one
 * of three (elements per CTA x threads) tiles of the flux-differencing kernel; 3..5
 * use the same tiles with the interface fluxes evaluated inside the flux-differencing
 * kernel from the neighbours' parameter vectors, so the face-flux kernel and its
 * round trip through memory drop out (available for FP32 fluxes, ES_MIXED and
 * ES_MIXED_FF, on periodic Euler meshes; each face's flux is then evaluated by both
 * of its elements).  Every variant gives bit-identical results; 0 is the default.  es_set_volume_variant returns
 * ES_ERR_INVALID for a variant outside 0..5 or a fused one the context cannot use;
 * es_autotune picks among all usable variants. */
int es_volume_variant(const es_ctx* ctx);
int es_set_volume_variant(es_ctx* ctx, int variant);

/* ---- Batches: many independent instances advanced together -------------
 * Instances may differ in LGL degree and element counts (and box) but share
 * the physics and method fields of es_config (gamma_gas, mu, Pr, R,
 * interface_diss, relax, rk, precision, delta_floor); otherwise
 * ES_ERR_INVALID.  Instances of one degree form one group stored as one SoA
 * over the group's elements; each step of all groups is captured once in a
 * CUDA graph (one kernel per phase and degree, groups on parallel branches)
 * and replayed.  Every instance has its own dt, gamma (= min over its own
 * elements, Theorem 2.3) and t.  The batch owns the states (device memory). */
typedef struct es_batch es_batch;
int es_batch_create(const es_config* cfgs, int count, es_batch** out);
void es_batch_destroy(es_batch* b);
/* nodes of instance inst, or of the whole batch for inst = -1; -1 on error */
long long es_batch_nodes(const es_batch* b, int inst);
/* node coordinates xyz[3][K_i][Np_i] of instance inst (host) */
int es_batch_node_coords(const es_batch* b, int inst, double* xyz_host);
/* copy instance inst's state [5][K_i][Np_i] in from / out to host memory (synchronous) */
int es_batch_set_state(es_batch* b, int inst, const double* q_host);
int es_batch_get_state(es_batch* b, int inst, double* q_host);
/* per-instance time steps dt_host[count] (> 0); required before es_batch_advance */
int es_batch_set_dt(es_batch* b, const double* dt_host);
/* tile autotuning per degree group on the current states (invalidates the graph) */
int es_batch_autotune(es_batch* b, void* stream);
/* es_set_tableau for every instance of the batch (same arguments and errors;
 * synchronises the device and invalidates the graph) */
int es_batch_set_tableau(es_batch* b, int s, const double* a, const double* bw, const double* c);
/* the volume tile variant chosen for instance inst's group */
int es_batch_volume_variant(const es_batch* b, int inst);
/* nsteps relaxed steps of every instance (graph replay), ordered after prior
 * work on `stream`; later work on `stream` waits for it */
int es_batch_advance(es_batch* b, int nsteps, void* stream);
/* es_step_estimate for every instance of the batch: one relaxed step of all
 * instances (the same kernels as es_batch_advance, launched on `stream` instead of
 * replaying the graph) that keeps each element's eta_kappa(u^{n-1}), estimate
 * deta_kappa and eta_kappa(u^n) in the batch (allocated on the first call,
 * ES_ERR_NOMEM).  es_batch_get_estimate copies instance inst's values and its last
 * gamma_kappa to host arrays of K_i doubles (any may be NULL; synchronises;
 * ES_ERR_INVALID before the first es_batch_step_estimate). */
int es_batch_step_estimate(es_batch* b, void* stream);
int es_batch_get_estimate(es_batch* b, int inst, double* eta_old_host, double* deta_host, double* eta_new_host,
                          double* gamma_elem_host);
/* per-instance t and last gamma (host arrays of count, either may be NULL); synchronises */
int es_batch_times(es_batch* b, double* t_host, double* gamma_host);
int es_batch_status(es_batch* b, void* stream);
/* kernels enqueued (graph replays count every kernel of the step) */
long long es_batch_launch_count(const es_batch* b);

/* out[i] = 1/x[i] (device arrays) with the library's FP64 reciprocal: the
 * hardware approximation refined by one third-order step r (1 + e + e^2),
 * e = 1 - x r (within one ulp, not correctly rounded), used in the
 * flux, thermodynamics and relaxation kernels in place of IEEE division.
 * Exposed so that it can be checked against IEEE division; x must be normal. */
int es_reciprocal(const double* x, double* out, long long n, void* stream);

/* ALU throughput of this GPU (instrumentation, not part of the method): *tflops =
 * the rate at which independent fused multiply-adds retire on every SM, FP64 if fp64
 * is nonzero, else FP32 (2 flops per FMA; eight independent chains per thread, 64
 * warps per SM, one warm-up launch, five launches timed with CUDA events on
 * `stream`).  It is the measured denominator of the roofline of the ALU-bound
 * kernels.  Allocates and frees a small output buffer; synchronises `stream`. */
int es_fma_peak(int fp64, double* tflops, void* stream);

/* Static message for an ES_* code. */
const char* es_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* ES_H */
