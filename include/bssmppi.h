/*
 * bssmppi.h - C ABI of the GB300 (sm_103a) BSS-MPPI library.
 *
 * BSS-MPPI (Yin, Tsiotras, Berntorp, "Chance-Constrained Information-Theoretic Stochastic Model
 * Predictive Control with Safety Shielding") solves, at every control step, the chance-constrained
 * stochastic optimal control problem of Sec. III (problem "BSSMPPIProblemformulation"): minimise the
 * expected trajectory cost over the nominal control sequence v subject to disturbed dynamics
 * x_{k+1} = f(x_k, u_k, w_k) and per-step chance constraints Pr(x_k in F) > 1 - P_fail. One solve
 * is Algorithm 1's body: K perturbed control sequences are each rolled out over M disturbance
 * particles for T steps (Algorithm 2 gives the particle mean and covariance of every step), the
 * belief barrier of Eq. "DCBF" and the penalty of Eq. "cbfpenalty" enter the cost, and the costs
 * give the weights of Eq. "Weights" and the update of Eq. "MPPI update law".
 *
 * Notation bridge to the paper: K here = the paper's M (control samples), M here = the paper's N
 * (particles per sample), T here = the paper's K (horizon), gamma here = the paper's beta (DCBF
 * decay rate, factor (1 - gamma)), ctrl_w = the paper's gamma (control-cost weight of Eq.
 * "TrajectoryCost"), delta = the per-boundary chance level epsilon of Eq. "track chance constraint".
 *
 * Conventions (all entry points):
 *  - Pointers named d_* are device pointers (global memory of the current CUDA device); h_* are host
 *    pointers. All arrays are dense, row-major, float32 unless stated. The caller owns every pointer
 *    it passes; the library never frees or keeps them beyond the call (except where stated).
 *  - A handle owns its device buffers and runs all work on the CUDA stream given at create time.
 *    Calls taking d_* pointers only enqueue work (stream-ordered, asynchronous) unless stated.
 *  - Return value: BSSMPPI_OK (0) or a negative bssmppi_status. Arguments are validated on the host
 *    before any launch; on error nothing is enqueued and bssmppi_last_error() explains why.
 *  - There is no CPU fallback: without a usable CUDA device every compute call fails with
 *    BSSMPPI_ECUDA.
 */
#ifndef BSSMPPI_H
#define BSSMPPI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BSSMPPI_ABI_VERSION 3u
#define BSSMPPI_NU 2          /* controls: [steer delta (rad), acceleration (m/s^2)] */
#define BSSMPPI_NX_MAX 8          /* states: 6 (bicycle), 4 (double integrator), 8 (wheel speeds) */
#define BSSMPPI_K_MAX (1 << 20)
#define BSSMPPI_M_MAX 256
#define BSSMPPI_T_MAX 256
#define BSSMPPI_NTRACK_MAX 16384
#define BSSMPPI_NDIAG 4       /* diagnostics: {beta = min S, eta = sum of omega, ESS = eta^2 / sum omega^2,
                                 free energy beta - lambda ln(eta / K)} */

typedef enum bssmppi_status {
    BSSMPPI_OK = 0,
    BSSMPPI_EINVAL = -1,   /* invalid argument or parameter */
    BSSMPPI_ENOMEM = -2,   /* device or pinned-host allocation failed */
    BSSMPPI_ECUDA = -3,    /* a CUDA runtime call failed (no device, launch error, ...) */
    BSSMPPI_ETIMEOUT = -4, /* a bounded device wait gave up */
    BSSMPPI_EBUSY = -5,    /* resource temporarily exhausted */
    BSSMPPI_ENOTSUP = -6   /* valid but unsupported combination */
} bssmppi_status;

typedef enum bssmppi_model {
    BSSMPPI_MODEL_BICYCLE6 = 0,  /* dynamic single-track vehicle, x = [v_x, v_y, r, e_psi, e_y, s] */
    BSSMPPI_MODEL_DOUBLE_INT4 = 1, /* planar double integrator, x = [p_x, p_y, v_x, v_y] (test model) */
    BSSMPPI_MODEL_WHEELS8 = 2     /* single-track vehicle with wheel speeds and friction-ellipse combined
                                     slip (Sec. V-A's plant), x = [v_x, v_y, r, omega_F, omega_R, e_psi,
                                     e_y, s], u = [steer, throttle]; M <= 128 */
} bssmppi_model;

/* Which internal buffer of the last solve bssmppi_read() copies. */
typedef enum bssmppi_buffer {
    BSSMPPI_BUF_S = 0,     /* K trajectory costs S_k (Eq. "TrajectoryCost" with the augmented costs) */
    BSSMPPI_BUF_W = 1,     /* K normalised weights omega_k / sum omega (Eq. "Weights") */
    BSSMPPI_BUF_EPS = 2,   /* K*T*2 effective perturbations u_{k,t} - v_t (u clamped to the bounds) */
    BSSMPPI_BUF_MEAN = 3,  /* K*(T+1)*nx particle means per step (record_moments=1 only) */
    BSSMPPI_BUF_VAR = 4,   /* K*(T+1)*nx unbiased particle variances per step (record_moments=1 only) */
    BSSMPPI_BUF_DIAG = 5,  /* BSSMPPI_NDIAG floats */
    BSSMPPI_BUF_V = 6      /* T*2 resident nominal control sequence */
} bssmppi_buffer;

/*
 * Problem parameters, copied at create. Sec. III states the problem: initial state x_0 (and its
 * covariance Sigma_{x_0}, Algorithm 1), control noise covariance Sigma_eps (Sec. II), disturbance
 * law w ~ N(0, Sigma_w) (Sec. V-A), chance level delta (Eq. "track chance constraint"), DCBF decay
 * rate gamma (Eq. "DCBF_constraint2") and temperature lambda (Eq. "Weights").
 */
typedef struct bssmppi_params {
    int32_t K, M, T;      /* samples (1..BSSMPPI_K_MAX), particles (2..BSSMPPI_M_MAX), horizon (1..BSSMPPI_T_MAX) */
    int32_t n_sub;        /* explicit-Euler substeps per dt (bicycle model), 1..64 */
    int32_t model;        /* bssmppi_model */
    int32_t ey_index;     /* state component bounded by |x_i| <= w_T (4 = e_y for the bicycle) */
    float dt, mass, Iz, lf, lr, tire_B, tire_C, mu, g, vx_floor; /* model constants (SI units) */
    /* wheel-speed model only: wheel radius R, axle wheel inertia I_w, longitudinal friction mu_x (mu is the
       lateral one), rear drive torque at full throttle, and the speed floor of the slip denominators */
    float wheel_radius, wheel_inertia, mu_x, tau_max, slip_floor;
    float u_min[2], u_max[2];  /* control bounds; sampled controls are clamped to them */
    float lambda;         /* temperature, > 0 */
    float delta;          /* per-boundary chance level, 0 < delta < 0.5; nu from `backoff` below */
    float gamma;          /* DCBF decay rate, 0 < gamma < 1 */
    float ctrl_w;         /* weight of v_t^T Sigma_eps^-1 u_t in S */
    float C_safe;         /* weight C of the safe-condition violation cost */
    float C_obs;          /* collision penalty added when |mean e_y| > w_T */
    float w_T;            /* track half-width */
    float x_goal[8], Q[8], Qf[8]; /* quadratic running and terminal cost (diagonal weights; first nx used) */
    float track_len;      /* length of the closed centre line (m), > 0 */
    int32_t n_track;      /* curvature table size, a power of two in 2..BSSMPPI_NTRACK_MAX */
    const float* track_kappa; /* host pointer to n_track curvature samples kappa(i * track_len / n_track); copied */
    double Sigma_eps[4];  /* 2x2 SPD control-noise covariance */
    double Sigma_w[64];   /* nx x nx PSD disturbance covariance (leading dimension nx) */
    uint64_t seed;        /* Philox key */
    int32_t crn_disturbance; /* 1: disturbance draws shared by all K samples (common random numbers) */
    int32_t compensated;  /* 1: Welford/Chan moments and Kahan sums; 0: naive sums (precision study) */
    int32_t record_moments; /* 1: keep per-step particle means and variances (BSSMPPI_BUF_MEAN/VAR) */
    int32_t resample;     /* 0: persistent particles x^n_{k+1} = f(x^n_k, u_k) + w (Sec. IV-C propagation);
                             1: Algorithm 2 read literally: before every step k >= 1 the particles are
                             re-drawn from N(mean_k, Sigma_k), the Monte-Carlo moments of step k (full
                             covariance, PSD Cholesky), with Philox stream 4. Needs compensated = 1; not
                             available to the shield repair or the server (BSSMPPI_ENOTSUP there). */
    int32_t backoff;      /* back-off of the racing barrier (Remark 1): 0 Gaussian nu = sqrt(2) erfinv(1 - 2 delta),
                             exact for a Gaussian belief; 1 Cantelli nu = sqrt((1 - delta) / delta), which holds
                             for any belief with that mean and variance */
    int32_t clamp_margin; /* 0: h = (w_T - nu sigma)^2 - mean_ey^2 as Eq. "DCBF" writes it (it grows again once
                             nu sigma > w_T); 1: h = max(w_T - nu sigma, 0)^2 - mean_ey^2, non-increasing in sigma */
} bssmppi_params;

/*
 * General constraint set (Assumption 1 and Eqs. "chance_constraint2", "deterministic_chance_constraint",
 * "DCBFchoice0", "DCBFchoice"). Each constraint c_q(x) < 0 is held with probability at least 1 - p_q.
 * Its deterministic form backs off by nu_q sqrt(eta_q^T Sigma eta_q), with eta_q = grad c_q at the
 * belief mean and nu_q from Remark 1. The barrier becomes h = min_q [-c_q(mean) - nu_q
 * sqrt(eta_q^T Sigma eta_q)], with Sigma the full Monte-Carlo covariance. The collision penalty C_obs
 * is charged when the mean breaks a constraint (some c_q(mean) > 0).
 */
#define BSSMPPI_MAX_CONSTRAINTS 8
typedef enum bssmppi_constraint_kind {
    BSSMPPI_CON_HALFSPACE = 0, /* c(x) = a^T x - b */
    BSSMPPI_CON_DISK = 1       /* c(x) = r^2 - (x_i - center_0)^2 - (x_j - center_1)^2: an obstacle */
} bssmppi_constraint_kind;
typedef enum bssmppi_backoff {
    BSSMPPI_BACKOFF_GAUSSIAN = 0, /* nu = sqrt(2) erfinv(1 - 2p), 0 < p < 0.5 */
    BSSMPPI_BACKOFF_CANTELLI = 1  /* nu = sqrt((1 - p) / p), 0 < p < 1; holds for any distribution */
} bssmppi_backoff;
typedef struct bssmppi_constraint {
    int32_t kind;         /* bssmppi_constraint_kind */
    int32_t backoff;      /* bssmppi_backoff */
    int32_t i, j;         /* DISK: the two (distinct) state components of the obstacle's plane */
    float p;              /* chance level p_q of this constraint */
    float b;              /* HALFSPACE: offset b */
    float a[8];           /* HALFSPACE: normal a (entries past nx ignored) */
    float center[2];      /* DISK: centre in the (x_i, x_j) plane */
    float radius;         /* DISK: radius r > 0 */
    int32_t reserved;     /* 0 */
} bssmppi_constraint;

typedef struct bssmppi_ctx* bssmppi_t;

/* Library identification. bssmppi_params_size() lets bindings check their struct layout. */
uint32_t bssmppi_abi_version(void);
size_t bssmppi_params_size(void);

/*
 * Create a controller handle for one problem (Sec. III). `cuda_stream` is a cudaStream_t (NULL = the
 * legacy default stream) on the current device; all of the handle's work runs on it. Allocates the
 * handle's device buffers (sample costs, weights, perturbations, the resident nominal sequence v
 * (zero-initialised), the device-resident solve counter (0) and the reduction scratch) and copies
 * the curvature table. Synchronous. Returns EINVAL for out-of-range parameters, ENOMEM or ECUDA.
 * On success *out is a new handle; on failure *out is NULL and bssmppi_last_error(NULL) says why.
 * The particles' placement in lanes depends on K, M and the device's SM count (from 8 to 32
 * particles, two per lane once the solve fills about 12 warps per SM); the random draws do not, so
 * two placements give the same solve up to the rounding order of the particle sums.
 */
int bssmppi_create(const bssmppi_params* params, void* cuda_stream, bssmppi_t* out);

/*
 * One BSS-MPPI solve (one iteration of Algorithm 1's outer loop, from the state estimate through
 * OptimalControl, with Algorithm 2 for the mean and covariance propagation), as one kernel launch:
 *   d_x0     [nx]      state estimate x_bar_0 (device).
 *   d_Sigma0 [nx*nx]   covariance Sigma_{x_0} of the estimate, or NULL for a known state. When given,
 *                      the particles start at x_bar_0 + L_0 xi with L_0 its Cholesky factor.
 *   d_v      [T*2]     in: nominal sequence v; out: updated sequence v+ (Eq. "MPPI update law").
 *                      NULL: use and update the handle's resident nominal sequence instead.
 *   d_u0     [2]       out: first control v+_0 to execute, or NULL.
 * The handle's resident sequence always ends equal to v+. The solve uses the device-resident
 * counter for its random numbers and then increments it on the device. Asynchronous.
 */
int bssmppi_solve(bssmppi_t h, const float* d_x0, const float* d_Sigma0, float* d_v, float* d_u0);

/*
 * A solve on the resident nominal followed, in the same launch, by the warm-start shift of
 * bssmppi_shift: the resident nominal ends as v+ shifted left by n steps with its last element
 * repeated (v[t] <- v+[min(t + n, T - 1)]), and d_u0 (device, 2, or NULL for the handle's) receives
 * v+_0 from before the shift. Equivalent to bssmppi_solve(h, d_x0, d_Sigma0, NULL, d_u0) followed by
 * bssmppi_shift(h, NULL, n), in one launch instead of two. 0 <= n <= T. Asynchronous.
 */
int bssmppi_solve_shift(bssmppi_t h, const float* d_x0, const float* d_Sigma0, float* d_u0, int32_t n);

/*
 * The same solve with host buffers: stages h_x0, h_v (NULL = resident) and h_Sigma0 (if non-NULL)
 * in the handle's pinned buffer and copies them to the device in one transfer, solves, reads v+ and
 * the first control back in one transfer into h_v and h_u0 (each if non-NULL), and waits for the
 * stream. Synchronous; the host pointers may be pageable. The two copies and the kernel are
 * captured once per combination of the optional buffers as a CUDA graph and replayed (rebuilt
 * after bssmppi_set_constraints or bssmppi_set_sample_range); while timing events are requested
 * (bssmppi_timing) they are issued one by one instead.
 */
int bssmppi_solve_host(bssmppi_t h, const float* h_x0, const float* h_Sigma0, float* h_v, float* h_u0);

/*
 * Warm start (Algorithm 1, "v <- v_safe", followed by the usual receding-horizon shift): shift the
 * sequence left by n steps, repeating its last element: v[t] <- v[min(t + n, T - 1)].
 * d_v [T*2] device sequence, or NULL for the resident one. 0 <= n <= T. Asynchronous.
 */
int bssmppi_shift(bssmppi_t h, float* d_v, int32_t n);

/*
 * Replaces the racing barrier of Eq. "DCBF" with the general constraint set `cons[0..n)` (host
 * array, copied; n <= BSSMPPI_MAX_CONSTRAINTS); n = 0 restores the racing barrier. The back-off
 * coefficients are computed here in double precision. For the bicycle, s is the absolute path
 * coordinate of the track (no wrap at the lap). Needs compensated = 1. Waits for the handle's stream,
 * then selects the full-belief kernel variant (all means and the whole covariance every step).
 * Returns BSSMPPI_EINVAL for a bad kind, back-off, chance level, disk state pair or non-finite
 * value, leaving the handle's set unchanged. The shield repair and the server do not use it.
 */
int bssmppi_set_constraints(bssmppi_t h, const bssmppi_constraint* cons, int32_t n);

/*
 * Sample-sharded solve: G handles (typically one per GPU) split the K_total samples of one solve
 * into disjoint ranges. All have the same parameters, seed, nominal, state and counter. Samples
 * are independent until the weights (Eq. "Weights"), so each shard rolls out its own range and
 * reduces it to a log-sum-exp partial of 3 + 2T floats {beta_g = min S, eta_g = sum omega,
 * q_g = sum omega^2, N_g = sum omega eps_eff}, with omega = exp(-(S - beta_g)/lambda). One
 * exchange of the partials (an all-gather of (3 + 2T) G floats) and a merge give every shard the
 * whole solve's update: beta = min beta_g, f_g = exp(-(beta_g - beta)/lambda),
 * v+ = v + sum f_g N_g / sum f_g eta_g (Eq. "MPPI update law").
 *
 * bssmppi_set_sample_range: this handle's K samples are samples [k_begin, k_begin + K) of K_total;
 * their random streams are keyed by the global sample index, so the shards together draw exactly
 * the numbers one handle with K_total samples would draw. Waits for the handle's stream.
 * BSSMPPI_EINVAL unless 0 <= k_begin, k_begin + K <= K_total <= BSSMPPI_K_MAX.
 *
 * bssmppi_solve_partial: as bssmppi_solve, but writes the partial to d_partial (device, 3 + 2T
 * floats) and leaves v, u0, the weights and the diagnostics unchanged; the counter advances.
 * d_v (device, T*2, or NULL for the resident nominal) is the nominal the shard samples around.
 * Asynchronous.
 *
 * bssmppi_merge_partials: merges G partials (device, G x (3 + 2T) floats; G <= 256) into the
 * resident nominal (and d_v, device T*2, if not NULL), u0 (d_u0, or the handle's), the diagnostics
 * (free energy with K_total samples) and the normalised weights of this handle's own samples
 * (BSSMPPI_BUF_W), from the costs of its last bssmppi_solve_partial. Asynchronous.
 */
int bssmppi_set_sample_range(bssmppi_t h, int32_t k_begin, int32_t K_total);
int bssmppi_solve_partial(bssmppi_t h, const float* d_x0, const float* d_Sigma0, const float* d_v, float* d_partial);
int bssmppi_merge_partials(bssmppi_t h, const float* d_partials, int32_t G, float* d_v, float* d_u0);

/* Free the handle and its device buffers after waiting for its stream. NULL is accepted. */
int bssmppi_destroy(bssmppi_t h);

/* Human-readable reason for the last failure on this handle (h = NULL: the last failed create on
 * this thread). The string stays valid until the next call on the same handle / thread. */
const char* bssmppi_last_error(bssmppi_t h);

/* Solve counter (the Philox counter word that distinguishes solves). set: stream-ordered write;
 * get: waits for the stream, then reads. */
int bssmppi_set_counter(bssmppi_t h, uint32_t counter);
int bssmppi_get_counter(bssmppi_t h, uint32_t* counter);

/* Overwrite the resident nominal sequence from d_v [T*2] (device). Asynchronous. */
int bssmppi_set_nominal(bssmppi_t h, const float* d_v);

/*
 * Copy an internal buffer of the last solve (bssmppi_buffer `which`) into the device array d_dst of
 * `bytes` bytes (must be at least the buffer's size; see bssmppi_buffer). Asynchronous. MEAN and VAR
 * need record_moments = 1 (else ENOTSUP).
 */
int bssmppi_read(bssmppi_t h, int32_t which, void* d_dst, size_t bytes);

/*
 * Shield repair objective and its gradient by a hand-written adjoint. Shield-MPPI minimises the
 * violation of the DCBF condition with path-integral and gradient-based steps (Sec. II; the
 * LocalRepair step of Algorithm 1); the gradient step uses this objective, the belief-barrier
 * penalty of Eq. "cbfpenalty" along the rollout of the nominal sequence itself:
 *   J_r(v) = sum_{t=1..T} C max(-h_t + (1 - gamma) h_{t-1}, 0),  h_t = (w_T - nu sigma_t)^2 - mean_t^2,
 * with the M particles driven by u_t = v_t (no control noise) and the disturbance draws of sample
 * 0 of the current solve counter, so J_r is a deterministic function of v (common random numbers).
 *   d_x0 [nx] (device). d_v [T*2] (device; NULL = the resident sequence).
 *   d_grad [T*2] out: dJ_r/dv (device). d_J [1] out: J_r (device, or NULL).
 * Needs M <= 256 (one thread per particle). Asynchronous. FP32 throughout; the forward pass takes
 * the heading's and the steering angle's sine and cosine from the hardware after reducing them into
 * [-pi, pi] (absolute error at most 2^-21.4), which shortens its serial chain.
 */
int bssmppi_repair_grad(bssmppi_t h, const float* d_x0, const float* d_v, float* d_grad, float* d_J);

/*
 * Local repair: `iters` projected gradient steps v <- clamp(v - step dJ_r/dv, u_min, u_max) on the
 * objective of bssmppi_repair_grad, in one launch. d_v [T*2] in/out (device; NULL = resident).
 * d_J [iters + 1] out: J_r before each step and after the last (device, or NULL).
 * 1 <= iters <= 1000, step >= 0. Asynchronous.
 */
int bssmppi_repair(bssmppi_t h, const float* d_x0, float* d_v, int32_t iters, float step, float* d_J);

/*
 * Kernel timing with CUDA events recorded on the handle's stream around the single launch of every
 * solve (rollout, costs, and the weights/update fused into that kernel's tail).
 * bssmppi_timing(h, n) with n > 0 starts recording the next n solves (older records are dropped;
 * n <= 4096), n = 0 stops. bssmppi_timing_read waits for the recorded events and writes up to `max`
 * durations in milliseconds (rollout_ms[i]: the whole launch; update_ms[i]: always 0, the update
 * has no launch of its own; either array may be NULL) for the solves recorded so far; *count
 * receives how many.
 */
int bssmppi_timing(bssmppi_t h, int32_t n);
int bssmppi_timing_read(bssmppi_t h, float* h_rollout_ms, float* h_update_ms, int32_t max, int32_t* count);

/* ------------------------------------------------------------------------------------------------
 * Serving: many controllers, requests batched continuously.
 *
 * A server keeps every registered controller's problem, curvature table, warm-start nominal
 * sequence (T_max x 2) and solve counter resident on the device. Each request is one solve of
 * Algorithm 1 for one controller with its own K, M, T and state estimate; after it, the
 * controller's nominal becomes v+ shifted by one step (the receding-horizon warm start) and its
 * counter advances, exactly as bssmppi_solve followed by bssmppi_shift(h, NULL, 1) would leave them.
 * A newer request of a controller replaces its older pending one (reported with status
 * BSSMPPI_EBUSY). A scheduler thread admits requests in arrival order while the batch has room
 * and the slot's share of hbm_budget_bytes holds their buffers (K*T*2 + 2K floats each); requests
 * that arrive while a batch runs are admitted into the other slot and run beside it on the device.
 * Batches run as captured CUDA graphs (use_graphs = 1) of persistent batched kernels. Controllers
 * whose problem constants agree in everything but their seed and track form one constants class; a
 * batch holds requests of one class (the oldest pending request's), whose constants the batched
 * kernels take as a parameter, so requests of another class wait for a batch of their own. With
 * max_batch = 1 and slots = 1 the server runs one solve at a time (the one-launch-per-solve path).
 * ---------------------------------------------------------------------------------------------- */
typedef struct bssmppi_server* bssmppi_server_t;

typedef struct bssmppi_server_config {
    int32_t max_controllers;   /* controller table size, 1..65536 */
    int32_t max_batch;         /* requests per batch, 1..4096 */
    int32_t T_max;             /* largest horizon of any request, 1..BSSMPPI_T_MAX */
    int32_t slots;             /* batches in flight, 1..8 */
    int32_t use_graphs;        /* 1: replay one captured CUDA graph per batch */
    int32_t reserved;          /* must be 0 */
    size_t hbm_budget_bytes;   /* device memory for the in-flight requests' buffers (split over slots) */
    int64_t max_batch_work;    /* particle-steps (sum of K*M*T) per batch, 0 = no limit; a batch always
                                  takes its oldest request, so the limit bounds batch duration */
} bssmppi_server_config;

typedef struct bssmppi_result {
    uint64_t req_id;           /* the id given at submit */
    int32_t ctrl_id;
    int32_t status;            /* BSSMPPI_OK, or BSSMPPI_EBUSY: replaced by a newer request */
    float u0[2];               /* first control of v+ (valid when status = OK) */
    float beta;                /* minimum trajectory cost of the solve */
    int32_t K, M, T;
    double t_submit_us, t_start_us, t_done_us; /* server clock; t_start = batch launch (-1 if replaced) */
} bssmppi_result;

typedef struct bssmppi_server_stats {
    int64_t submitted, superseded, admitted, completed, batches, max_batch_seen, queued;
    double now_us;             /* server clock at the call */
} bssmppi_server_stats;

/* Create a server on the current device. Allocates the controller table, the slots' descriptors,
 * results and HBM arenas, captures the batch graphs and starts the scheduler thread. */
int bssmppi_server_create(const bssmppi_server_config* cfg, bssmppi_server_t* out);
/* Register a controller (bicycle model, compensated; K, M, T of params are ignored: each request
 * brings its own). Its nominal starts at zero and its counter at 0. *ctrl_id receives its index. */
int bssmppi_server_add_controller(bssmppi_server_t s, const bssmppi_params* params, int32_t* ctrl_id);
/* Queue a solve for controller ctrl_id from state h_x0 [6] (host; copied). 2 <= M <= 128,
 * 1 <= T <= T_max. Thread-safe; returns immediately. */
int bssmppi_server_submit(bssmppi_server_t s, int32_t ctrl_id, const float* h_x0, int32_t K, int32_t M, int32_t T,
                          uint64_t req_id);
/* Move up to max finished results (completed or replaced) into out; *n receives how many. */
int bssmppi_server_poll(bssmppi_server_t s, bssmppi_result* out, int32_t max, int32_t* n);
/* Wait until no request is queued or in flight (ETIMEOUT after timeout_ms). */
int bssmppi_server_drain(bssmppi_server_t s, int32_t timeout_ms);
/* Read or overwrite a controller's resident nominal (h_v [T_max*2], host) and counter; EBUSY while
 * the controller has work queued or in flight. Synchronous. */
int bssmppi_server_get_state(bssmppi_server_t s, int32_t ctrl_id, float* h_v, uint32_t* counter);
int bssmppi_server_set_state(bssmppi_server_t s, int32_t ctrl_id, const float* h_v, uint32_t counter);
int bssmppi_server_get_stats(bssmppi_server_t s, bssmppi_server_stats* out);
/* Inspect one served solve (Algorithm 1's sample costs S, the normalised weights of Eq. "Weights"
 * and the clamped perturbations eps_eff = u - v that Eq. "MPPI_update_law" averages): the next
 * request of controller ctrl_id to complete has its S[K], w[K] and eps_eff[K][T][2] (row-major)
 * copied, in that order, into the caller's host buffer h_out of cap_floats floats before its slot is
 * reused, and *h_written receives K (2 + 2T), or -1 when that does not fit (nothing is copied), or -2
 * on a CUDA error. *h_written is 0 until then; read it after bssmppi_server_drain. The buffer and
 * *h_written must stay valid until the request completes. One-shot: a capture serves one request.
 * EBUSY while the controller has work queued or in flight. Costs the copy's time in the scheduler
 * thread; meant for checking and logging, not for the serving loop. */
int bssmppi_server_capture(bssmppi_server_t s, int32_t ctrl_id, float* h_out, int64_t cap_floats, int64_t* h_written);
const char* bssmppi_server_last_error(bssmppi_server_t s);
/* Stop the scheduler, wait for the device and free everything. NULL is accepted. */
int bssmppi_server_destroy(bssmppi_server_t s);

/*
 * Weights and update (the same computation as the second half of bssmppi_solve) for callers that
 * cannot allocate device memory. Some callers cannot call cudaMalloc once they run: hard real-time
 * control loops that forbid allocation after start-up (an allocation can block and synchronise the
 * device within a control period), and plugins hosted by a process whose memory manager owns the
 * device memory. This entry point allocates nothing: its scratch (partial sums and arrival ticket)
 * is one fixed array of 303,360 bytes in the library's device memory, held by every GPU that loads
 * the library until the process exits. The paper has no counterpart; it is an interface addition.
 *   d_S [K] costs, d_eps [K*T*2] effective perturbations (inputs, device).
 *   d_v [T*2] nominal in, v+ out (device). d_w [K] normalised weights out (device).
 *   d_u0 [2], d_diag [BSSMPPI_NDIAG], d_counter [1] (incremented by one): optional, NULL to skip.
 *   K in [1, BSSMPPI_K_MAX], T in [1, BSSMPPI_T_MAX]; larger sizes are rejected with EINVAL (the
 *   scratch holds at most 148 x 512 partial sums). lambda > 0. compensated: 1 = Kahan sums.
 * The first call on a device looks up the array's device address (once per device, with that
 * device current), and under lazy module loading (CUDA's default) the first launch also loads the
 * library's kernels, which places the array in device memory and can synchronise the device. So
 * make one warm-up call per device at start-up, before the allocation-free phase begins and before
 * any stream capture; later calls do neither. Every call shares the one array
 * and the ticket is cleared at the start of each call, so calls that overlap on the GPU (on
 * different streams, or from different threads) race and must be serialised by the caller.
 * Asynchronous on `cuda_stream`; errors are reported through bssmppi_last_error(NULL).
 */
int bssmppi_update_noalloc(const float* d_S, const float* d_eps, float* d_v, float* d_w, float* d_u0,
                           float* d_diag, uint32_t* d_counter, int32_t K, int32_t T, float lambda,
                           int32_t compensated, void* cuda_stream);

/*
 * Model step x_{k+1} = f(x_k, u_k) + w_k (Eq. "DeterministicNonlinearSystem" / "DisturbedNonlinearSystem";
 * n_sub Euler substeps of the handle's model) for n independent states: d_x [n*nx], d_u [n*2],
 * d_w [n*nx] additive disturbance or NULL for none, d_x_next [n*nx], device. Used to check the model
 * on its own and to step a simulated plant. Asynchronous.
 */
int bssmppi_model_step(bssmppi_t h, const float* d_x, const float* d_u, const float* d_w, float* d_x_next, int64_t n);

/*
 * Philox4x32-10 (Salmon et al., SC'11), the counter-based generator of every random number the solve
 * draws: d_out[4i..4i+3] = Philox(counter d_ctr[4i..4i+3], key (seed & 0xffffffff, seed >> 32)) for
 * i < n. Device arrays of 4n uint32. Runs on `cuda_stream` (cudaStream_t, NULL = default).
 */
int bssmppi_philox4x32_10(const uint32_t* d_ctr, uint64_t seed, uint32_t* d_out, int64_t n, void* cuda_stream);

/*
 * Box-Muller Gaussians as the solve draws them: for each word pair (a, b) = d_words[2i], d_words[2i+1],
 * u1 = ((a >> 8) + 1) 2^-24, u2 = (b >> 8) 2^-24, d_z[2i] = sqrt(-2 ln u1) cos(2 pi u2),
 * d_z[2i+1] = sqrt(-2 ln u1) sin(2 pi u2). n pairs; device arrays.
 */
int bssmppi_box_muller(const uint32_t* d_words, float* d_z, int64_t n, void* cuda_stream);

/*
 * The slip-angle arctangent as the bicycle substep evaluates it: d_y[i] = atan(d_t[i])
 * for n values; device arrays. For |t| <= 1/2 an odd polynomial of degree 11 (within one FP32 ulp), beyond
 * it the library's atanf. Exported so that its error can be checked against an exact reference.
 */
int bssmppi_slip_atan(const float* d_t, float* d_y, int64_t n, void* cuda_stream);

/*
 * The tyre curve of the simplified Pacejka law as the bicycle substep evaluates it (Sec. V-A's
 * vehicle model, reading R3: F_y = mu F_z sin(C atan(B alpha))): d_y[i] = sin(C atan(d_x[i])) for
 * the handle's C, n values (x = B alpha); device arrays. For |x| <= 1 a degree-9 polynomial in x^2
 * fitted to the curve on the host for that C; beyond, the library's atanf and the hardware sine.
 * Exported so that its error can be checked against an exact reference. Asynchronous.
 */
int bssmppi_tyre_curve(bssmppi_t h, const float* d_x, float* d_y, int64_t n, void* cuda_stream);

/*
 * The rear tyre's curve as the bicycle substep evaluates it where one or two particles share a lane
 * (Sec. V-A's vehicle model, readings R3 and R4: the rear slip angle is -atan t for the slip argument
 * t = (v_y - l_r r) / v_x, so F_y,r / D_r = sin(C atan(-B atan t))): d_y[i] for d_t[i], the handle's
 * B and C, n values; device arrays, taken in pairs through the packed form as in the solve. For
 * |t| <= tau (tau = tan(1/B), or 1/2 if that is less) a degree-9 polynomial in (t / tau)^2 fitted
 * on the host; beyond, slip_atan and the library's atanf and hardware sine. Exported so that its
 * error can be checked against an exact reference. Asynchronous.
 */
int bssmppi_rear_tyre(bssmppi_t h, const float* d_t, float* d_y, int64_t n, void* cuda_stream);

/*
 * The coefficients c_0..c_9 (h_c, host, n >= 10 floats) of the rear tyre's polynomial for B > 0 and
 * C > 0 and its domain's half-width (*h_tau): sin(C atan(-B atan t)) = x sum_i c_i x^(2i) with
 * x = t / tau on |t| <= tau, interpolating at ten Chebyshev points in double precision. Host only.
 * EINVAL for B <= 0, C <= 0, n < 10 or a NULL output.
 */
int bssmppi_rear_tyre_coefficients(double B, double C, float* h_c, int32_t n, double* h_tau);

/*
 * The coefficients c_0..c_9 (h_c, host, n >= 10 floats) of the tyre curve's polynomial for a tyre shape factor
 * C > 0: sin(C atan x) = x sum_i c_i x^(2i) on |x| <= 1, interpolating at ten Chebyshev points in
 * double precision. Host only (no device is needed). EINVAL for C <= 0 or n < 10.
 */
int bssmppi_tyre_curve_coefficients(double C, float* h_c, int32_t n);

/*
 * Measured FP32 arithmetic peak of the current device (no counterpart in the paper: the
 * denominator of the rollout kernel's roofline, which is bound by FP32 issue, not by memory or
 * tensor cores). Runs a grid of (blocks per SM at full occupancy) x SMs blocks of 256 threads, each
 * thread with 16 independent fused multiply-add chains of `iters` steps (packed = 1: the same chains
 * as 8 register pairs through the packed .f32x2 form), once to warm up and once timed with CUDA
 * events on cuda_stream (NULL = the legacy default stream). Writes the timed launch's duration
 * (*h_ms), its rate counting a multiply-add as two operations (*h_tflops, 1e12 per second) and the
 * SM count (*h_sms). Allocates and frees one float. EINVAL if iters is outside [1, 2^24] or an
 * output is NULL; ECUDA on a CUDA error. Synchronous.
 */
int bssmppi_fp32_peak(int32_t packed, int32_t iters, void* cuda_stream, float* h_ms, double* h_tflops,
                      int32_t* h_sms);

#ifdef __cplusplus
}
#endif
#endif /* BSSMPPI_H */
