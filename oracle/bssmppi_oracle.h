/*
 * FP64 reference oracle for the BSS-MPPI solve (Yin, Tsiotras, Berntorp, "Chance-Constrained
 * Information-Theoretic Stochastic Model Predictive Control with Safety Shielding").
 *
 * TEST INFRASTRUCTURE ONLY. This plain, slow C code (single-threaded unless a caller asks for
 * OpenMP threads over the samples) exists to check the CUDA
 * path. Only the test suite, the smoke check and the benchmark's CPU-baseline leg may load it. It
 * shares no code, header, constant or helper with the CUDA library; the two receive the same
 * seeded inputs and nothing else.
 *
 * Everything is computed in double precision in the paper's order:
 *   Algorithm 1 (sample control sequences, roll out, accumulate the augmented cost, update),
 *   Algorithm 2 (propagate N particles, Monte-Carlo mean and unbiased covariance),
 *   Eq. "MPPI update law" and Eq. "Weights" (max-subtracted exponential weighting),
 *   Eq. "DCBF" (racing belief barrier h = (w_T - nu sigma_y)^2 - e_y^2),
 *   Eq. "cbfpenalty" / "modified state-dependent costs" (C_safe on the augmented belief state).
 * Random numbers come from Philox4x32-10 (Salmon et al., SC'11) with the counter layout described
 * in bssmppi_oracle.c, so the oracle draws the same integers as the CUDA path.
 *
 * Notation bridge: K = number of control samples (the paper's M), M = particles per sample (the
 * paper's N), T = horizon steps (the paper's K), gamma = DCBF decay rate (the paper's beta in
 * (1 - beta)), ctrl_w = control-cost weight (the paper's gamma in the trajectory cost).
 */
#ifndef BSSMPPI_ORACLE_H
#define BSSMPPI_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* One constraint c(x) < 0 of the feasible set (Assumption 1) with its chance level p
 * (Pr(c(x) >= 0) <= p, Eq. "chance_constraint2") and back-off rule (Remark 1).
 *   kind 0, half-space: c(x) = a^T x - b.
 *   kind 1, disk obstacle in the plane of states (i, j): c(x) = r^2 - (x_i - o_0)^2 - (x_j - o_1)^2.
 *   backoff 0: nu = sqrt(2) erfinv(1 - 2p) (Gaussian); 1: nu = sqrt((1 - p) / p) (Cantelli). */
typedef struct orc_constraint {
    int kind, backoff, i, j;
    double p, b, a[8], center[2], radius;
} orc_constraint;

typedef struct orc_problem {
    int K, M, T, n_sub, model; /* model 0: dynamic bicycle (nx=6); 1: double integrator (nx=4);
                                  2: single-track model with wheel speeds and combined slip (nx=8) */
    double dt, mass, Iz, lf, lr, tire_B, tire_C, mu, g, vx_floor;
    double wheel_radius, wheel_inertia, mu_x, tau_max, slip_floor; /* model 2 only */
    double u_min[2], u_max[2];
    double Sigma_eps[4];  /* 2x2 row-major, SPD */
    double Sigma_w[64];   /* nx x nx row-major (leading dimension nx), PSD */
    double lambda, delta, gamma, ctrl_w, C_safe, C_obs, w_T;
    double x_goal[8], Q[8], Qf[8];
    int ey_index;         /* component bounded by |x_i| <= w_T (e_y) */
    const double* kappa;  /* curvature table, n_track entries over [0, track_len) */
    int n_track;
    double track_len;
    uint64_t seed;
    int crn_disturbance;  /* 1: disturbance draws shared by all K samples */
    int resample;         /* 1: Algorithm 2 read literally: before every step k >= 1 the particles are
                             re-drawn from N(xbar_k, Sigma_k) (stream 4); 0: persistent particles */
    int n_con;            /* 0: the racing barrier of Eq. "DCBF"; > 0: the general set, Eq. "DCBFchoice" */
    const orc_constraint* con;
    int backoff;          /* racing barrier's nu (Remark 1): 0 Gaussian, 1 Cantelli */
    int clamp_margin;     /* 1: h = max(w_T - nu sigma, 0)^2 - mean_ey^2; 0: as Eq. "DCBF" writes it */
} orc_problem;

/* Per-solve outputs; any pointer may be NULL. Sizes: S[K], u[K*T*2] (clamped samples), w[K]
 * (normalised weights), v_plus[T*2], mean[K*(T+1)*nx], cov[K*(T+1)*nx*nx], margin[K]
 * (min over steps of ||mean e_y| - w_T|, or of |c_i(mean)| over the constraints of a general set),
 * h[K*(T+1)], diag[4] = {beta, eta, ESS, free energy
 * beta - lambda ln(eta / K)}. */
typedef struct orc_outputs {
    double *S, *u, *w, *v_plus, *mean, *cov, *margin, *h, *diag;
} orc_outputs;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_philox4x32_10_batch(int64_t n, const uint32_t* ctr, const uint32_t key[2], uint32_t* out);
void orc_gaussian_pair(uint32_t a, uint32_t b, double z[2]);
double orc_backoff_gaussian(double p);  /* sqrt(2) erfinv(1 - 2p) */
double orc_backoff_cantelli(double p);  /* sqrt((1 - p) / p) */
int orc_nx(const orc_problem* p);
double orc_track_kappa(const orc_problem* p, double s);
/* Deterministic model step x_{k+1} = f(x_k, u_k) (n_sub Euler substeps for the bicycle). */
void orc_model_step(const orc_problem* p, const double* x, const double* u, double* x_next);
/* Rollout and cost of samples [k_begin, k_end) (Algorithm 1's inner loop with Algorithm 2). */
int orc_rollout(const orc_problem* p, const double* x0, const double* Sigma0, const double* v,
                uint32_t solve_ctr, int k_begin, int k_end, const orc_outputs* out);
/* The same with the samples spread over n_threads OpenMP threads (whole samples per thread, so
 * every output is the one-thread result bit for bit; one thread when built without OpenMP). */
int orc_rollout_threads(const orc_problem* p, const double* x0, const double* Sigma0, const double* v,
                        uint32_t solve_ctr, int k_begin, int k_end, const orc_outputs* out, int n_threads);
/* OptimalControl: weights and v+ = sum w u / sum w from costs S[K] and clamped samples u. */
void orc_optimal_control(int K, int T, double lambda, const double* S, const double* u,
                         double* w, double* v_plus, double* diag);
/* The weights/update split over disjoint sample subsets (one per GPU when K is sharded):
 * part[3 + 2T] = {beta_g, eta_g, q_g = sum omega^2, U_g[2T] = sum omega u} of samples [k_begin, k_end),
 * and the merge of G such partials into v+ and diag (K_total samples in all). */
void orc_lse_partial(int k_begin, int k_end, int T, double lambda, const double* S, const double* u, double* part);
void orc_lse_merge(int G, int T, double lambda, int K_total, const double* parts, double* v_plus, double* diag);
/* Full solve = orc_rollout over all samples + orc_optimal_control. Returns 0 or -1 (bad args). */
int orc_solve(const orc_problem* p, const double* x0, const double* Sigma0, const double* v,
              uint32_t solve_ctr, const orc_outputs* out);
int orc_solve_threads(const orc_problem* p, const double* x0, const double* Sigma0, const double* v,
                      uint32_t solve_ctr, const orc_outputs* out, int n_threads);
/* Warm start with a one-step shift: v[t] <- v[t+1], last element repeated. */
void orc_shift(int T, double* v);

/* Shield repair objective J_r(v) = sum_{t=1..T} C_safe,t of the M-particle rollout of the
 * nominal sequence v (no control noise, disturbance draws of sample 0) and its gradient dJ/dv
 * by a reverse sweep (adjoint). grad [T*2] and args_out [T+1] (the hinge arguments
 * -h_t + (1 - gamma) h_{t-1}, entry 0 unused) may be NULL. Returns J, or NaN for the wheel-speed
 * model (model 2, which has no adjoint here), M < 2 or T < 1.
 * The paper leaves the repair step undefined, so this objective is a reading of it. Its value is
 * pinned to the barrier penalty that orc_rollout's own h gives for the same nominal (no control
 * noise, common random numbers); its gradient by central finite differences of J_r. */
double orc_repair_objective(const orc_problem* p, const double* x0, const double* v,
                            uint32_t solve_ctr, double* grad, double* args_out);

#ifdef __cplusplus
}
#endif
#endif
