/*
 * FP64 reference oracle for the BSS-MPPI solve. TEST INFRASTRUCTURE ONLY: loaded by the tests,
 * the smoke check and the benchmark's CPU-baseline leg; never by the product path. See
 * bssmppi_oracle.h for the interface and the notation bridge.
 *
 * Random-number layout (both sides implement it independently from this description):
 *   key     = (seed & 0xffffffff, seed >> 32)
 *   counter = (c0, c1, c2, c3) with
 *     c0 = step index t | (call index j << 16)
 *     c1 = particle index n (0 for control noise)
 *     c2 = sample index k (0 for every sample when disturbance draws are shared)
 *     c3 = (stream << 28) | (solve counter & 0x0fffffff);
 *     streams: 0 control noise, 1 state disturbance, 3 initial particles, 4 per-step re-draws of
 *     the particles (only when the problem asks for Algorithm 2's re-sampling). For 6 states the
 *     disturbance pairs particles n and n + H, H = 2^ceil(log2 M) / 2, on one counter whose word 1
 *     is the lower index (see draw_disturbance).
 *   Uniforms from two 32-bit words a, b: u1 = ((a >> 8) + 1) 2^-24 in (0, 1],
 *   u2 = (b >> 8) 2^-24 in [0, 1); Box-Muller z = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2).
 *   Gaussian pair i of a draw comes from call i/2, words (2(i%2), 2(i%2)+1).
 */
#include "bssmppi_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the 4x32 Philox S-box with  */
/* multipliers 0xD2511F53, 0xCD9E8D57 and key bumps by the Weyl constants 0x9E3779B9,           */
/* 0xBB67AE85 between rounds.                                                                    */
/* ------------------------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void orc_philox4x32_10_batch(int64_t n, const uint32_t* ctr, const uint32_t key[2], uint32_t* out)
{
    for (int64_t i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

void orc_gaussian_pair(uint32_t a, uint32_t b, double z[2])
{
    const double two_m24 = 1.0 / 16777216.0;
    double u1 = (double)((a >> 8) + 1u) * two_m24;
    double u2 = (double)(b >> 8) * two_m24;
    double rad = sqrt(-2.0 * log(u1));
    const double two_pi = 6.283185307179586476925286766559;
    z[0] = rad * cos(two_pi * u2);
    z[1] = rad * sin(two_pi * u2);
}

/* Remark 1: Gaussian back-off nu = sqrt(2) erfinv(1 - 2p). erfinv by bisection on libm erf
 * (slow and plainly correct: erf is strictly increasing). */
double orc_backoff_gaussian(double p)
{
    double target = 1.0 - 2.0 * p;
    double lo = -10.0, hi = 10.0;
    for (int i = 0; i < 200; ++i) {
        double mid = 0.5 * (lo + hi);
        if (erf(mid) < target) lo = mid; else hi = mid;
    }
    return sqrt(2.0) * 0.5 * (lo + hi);
}

double orc_backoff_cantelli(double p) { return sqrt((1.0 - p) / p); }

int orc_nx(const orc_problem* p) { return p->model == 0 ? 6 : (p->model == 2 ? 8 : 4); }

/* Cholesky factor L (lower, row-major n x n) of a symmetric PSD matrix; a zero pivot gives a
 * zero column (a component with no noise). */
static void cholesky_psd(int n, const double* A, double* L)
{
    memset(L, 0, sizeof(double) * n * n);
    for (int j = 0; j < n; ++j) {
        double d = A[j * n + j];
        for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
        if (d <= 1e-300) continue;
        double ljj = sqrt(d);
        L[j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = s / ljj;
        }
    }
}

/* Curvature kappa(s): linear interpolation of the periodic table. */
double orc_track_kappa(const orc_problem* p, double s)
{
    double x = s / p->track_len * (double)p->n_track;
    double fl = floor(x);
    double f = x - fl;
    long n = p->n_track;
    long i0 = (long)fl % n;
    if (i0 < 0) i0 += n;
    long i1 = (i0 + 1) % n;
    return (1.0 - f) * p->kappa[i0] + f * p->kappa[i1];
}

static double track_dkappa_ds(const orc_problem* p, double s)
{
    double x = s / p->track_len * (double)p->n_track;
    long n = p->n_track;
    long i0 = (long)floor(x) % n;
    if (i0 < 0) i0 += n;
    long i1 = (i0 + 1) % n;
    return (p->kappa[i1] - p->kappa[i0]) * (double)n / p->track_len;
}

/* Dynamic single-track model in the road-aligned (Frenet) frame, state
 * [v_x, v_y, yaw rate r, e_psi, e_y, s], input [steer delta, accel a], simplified Pacejka lateral
 * tyre forces F_y = mu F_z sin(C atan(B alpha)) with static axle loads. */
static void bicycle_rhs(const orc_problem* p, const double* x, const double* u, double* dx)
{
    double vx = x[0], vy = x[1], r = x[2], epsi = x[3], ey = x[4], s = x[5];
    double steer = u[0], acc = u[1];
    double vxh = fmax(vx, p->vx_floor);
    double alpha_f = steer - atan2(vy + p->lf * r, vxh);
    double alpha_r = -atan2(vy - p->lr * r, vxh);
    double Fzf = p->mass * p->g * p->lr / (p->lf + p->lr);
    double Fzr = p->mass * p->g * p->lf / (p->lf + p->lr);
    double Fyf = p->mu * Fzf * sin(p->tire_C * atan(p->tire_B * alpha_f));
    double Fyr = p->mu * Fzr * sin(p->tire_C * atan(p->tire_B * alpha_r));
    double kap = orc_track_kappa(p, s);
    double sdot = (vx * cos(epsi) - vy * sin(epsi)) / (1.0 - kap * ey);
    dx[0] = acc - Fyf * sin(steer) / p->mass + vy * r;
    dx[1] = (Fyf * cos(steer) + Fyr) / p->mass - vx * r;
    dx[2] = (p->lf * Fyf * cos(steer) - p->lr * Fyr) / p->Iz;
    dx[3] = r - kap * sdot;
    dx[4] = vx * sin(epsi) + vy * cos(epsi);
    dx[5] = sdot;
}

/* Vector-Jacobian product of bicycle_rhs: given g = dL/dF, accumulate dL/dx into gx and dL/du
 * into gu. */
static void bicycle_rhs_vjp(const orc_problem* p, const double* x, const double* u, const double* g,
                            double* gx, double* gu)
{
    double vx = x[0], vy = x[1], r = x[2], epsi = x[3], ey = x[4], s = x[5];
    double steer = u[0];
    double m = p->mass, Iz = p->Iz, lf = p->lf, lr = p->lr, B = p->tire_B, C = p->tire_C;
    double vxh = fmax(vx, p->vx_floor);
    double yf = vy + lf * r, yr = vy - lr * r;
    double alpha_f = steer - atan2(yf, vxh);
    double alpha_r = -atan2(yr, vxh);
    double Dfz = p->mu * m * p->g * lr / (lf + lr);
    double Drz = p->mu * m * p->g * lf / (lf + lr);
    double tf = atan(B * alpha_f), tr = atan(B * alpha_r);
    double Fyf = Dfz * sin(C * tf);  /* the rear force enters the adjoint only through dFr */
    double dFf = Dfz * cos(C * tf) * C * B / (1.0 + B * alpha_f * B * alpha_f);
    double dFr = Drz * cos(C * tr) * C * B / (1.0 + B * alpha_r * B * alpha_r);
    double kap = orc_track_kappa(p, s), dkap = track_dkappa_ds(p, s);
    double sp = sin(epsi), cp = cos(epsi), sd = sin(steer), cd = cos(steer);
    double num = vx * cp - vy * sp, den = 1.0 - kap * ey;
    double sdot = num / den;

    double gFf = g[0] * (-sd / m) + g[1] * (cd / m) + g[2] * (lf * cd / Iz);
    double gFr = g[1] / m - g[2] * (lr / Iz);
    double gsdot = -g[3] * kap + g[5];
    double gkap = -g[3] * sdot + gsdot * num * ey / (den * den);
    double gnum = gsdot / den;
    double gey = gsdot * num * kap / (den * den);
    double gvx = gnum * cp, gvy = -gnum * sp, gepsi = gnum * (-vx * sp - vy * cp);
    double gr = 0.0, gsteer = 0.0, gacc = g[0];
    gvy += g[0] * r; gr += g[0] * vy; gsteer += g[0] * (-Fyf * cd / m);
    gsteer += g[1] * (-Fyf * sd / m); gvx += -g[1] * r; gr += -g[1] * vx;
    gsteer += g[2] * (-lf * Fyf * sd / Iz);
    gr += g[3];
    gvx += g[4] * sp; gvy += g[4] * cp; gepsi += g[4] * (vx * cp - vy * sp);
    double gs = gkap * dkap;
    double gaf = gFf * dFf, gar = gFr * dFr;
    double qf = vxh * vxh + yf * yf, qr = vxh * vxh + yr * yr;
    gsteer += gaf;
    double gyf = -gaf * vxh / qf, gyr = -gar * vxh / qr;
    double gvxh = gaf * yf / qf + gar * yr / qr;
    gvy += gyf + gyr; gr += lf * gyf - lr * gyr;
    if (vx > p->vx_floor) gvx += gvxh;
    gx[0] += gvx; gx[1] += gvy; gx[2] += gr; gx[3] += gepsi; gx[4] += gey; gx[5] += gs;
    gu[0] += gsteer; gu[1] += gacc;
}

/* Single-track model with wheel speeds and combined slip (Sec. V-A's plant: state
 * [v_x, v_y, r, omega_F, omega_R, e_psi, e_y, s], input [steer, throttle]). Lateral slip angles as in
 * the bicycle model; longitudinal slip kappa = (R omega - v_w) / max(|v_w|, slip_floor) with v_w the
 * wheel's forward speed; one magic-formula curve on the combined slip s = sqrt(kappa^2 + alpha^2),
 * g = sin(C atan(B s)), split along the slip direction and scaled by the friction ellipse's axes:
 * F_x = mu_x F_z g kappa / s, F_y = mu F_z g alpha / s (so (F_x / mu_x F_z)^2 + (F_y / mu F_z)^2 = g^2 <= 1).
 * Rear-wheel drive torque tau_max * throttle; static axle loads. */
static void wheels8_rhs(const orc_problem* p, const double* x, const double* u, double* dx)
{
    double vx = x[0], vy = x[1], r = x[2], wf = x[3], wr = x[4], epsi = x[5], ey = x[6], s = x[7];
    double steer = u[0], thr = u[1];
    double vxh = fmax(vx, p->vx_floor);
    double alpha_f = steer - atan2(vy + p->lf * r, vxh);
    double alpha_r = -atan2(vy - p->lr * r, vxh);
    double vwf = vx * cos(steer) + (vy + p->lf * r) * sin(steer);
    double vwr = vx;
    double kf = (p->wheel_radius * wf - vwf) / fmax(fabs(vwf), p->slip_floor);
    double kr = (p->wheel_radius * wr - vwr) / fmax(fabs(vwr), p->slip_floor);
    double L = p->lf + p->lr;
    double Fz[2] = {p->mass * p->g * p->lr / L, p->mass * p->g * p->lf / L};
    double kap[2] = {kf, kr}, alp[2] = {alpha_f, alpha_r}, Fx[2], Fy[2];
    for (int w = 0; w < 2; ++w) {
        double sl = sqrt(kap[w] * kap[w] + alp[w] * alp[w]);
        /* g(s) / s, which tends to C B as s -> 0 */
        double ratio = sl > 1e-12 ? sin(p->tire_C * atan(p->tire_B * sl)) / sl : p->tire_C * p->tire_B;
        Fx[w] = p->mu_x * Fz[w] * ratio * kap[w];
        Fy[w] = p->mu * Fz[w] * ratio * alp[w];
    }
    double FXf = Fx[0] * cos(steer) - Fy[0] * sin(steer);
    double FYf = Fx[0] * sin(steer) + Fy[0] * cos(steer);
    double kp = orc_track_kappa(p, s);
    double sdot = (vx * cos(epsi) - vy * sin(epsi)) / (1.0 - kp * ey);
    dx[0] = (FXf + Fx[1]) / p->mass + vy * r;
    dx[1] = (FYf + Fy[1]) / p->mass - vx * r;
    dx[2] = (p->lf * FYf - p->lr * Fy[1]) / p->Iz;
    dx[3] = -p->wheel_radius * Fx[0] / p->wheel_inertia;
    dx[4] = (p->tau_max * thr - p->wheel_radius * Fx[1]) / p->wheel_inertia;
    dx[5] = r - kp * sdot;
    dx[6] = vx * sin(epsi) + vy * cos(epsi);
    dx[7] = sdot;
}

void orc_model_step(const orc_problem* p, const double* x, const double* u, double* x_next)
{
    if (p->model == 2) {
        double h = p->dt / p->n_sub, xs[8], dx[8];
        memcpy(xs, x, sizeof xs);
        for (int j = 0; j < p->n_sub; ++j) {
            wheels8_rhs(p, xs, u, dx);
            for (int i = 0; i < 8; ++i) xs[i] += h * dx[i];
        }
        memcpy(x_next, xs, sizeof xs);
    } else if (p->model == 0) {
        double h = p->dt / p->n_sub, xs[6], dx[6];
        memcpy(xs, x, sizeof xs);
        for (int j = 0; j < p->n_sub; ++j) {
            bicycle_rhs(p, xs, u, dx);
            for (int i = 0; i < 6; ++i) xs[i] += h * dx[i];
        }
        memcpy(x_next, xs, sizeof xs);
    } else {
        /* planar double integrator, exact zero-order-hold discretisation */
        double dt = p->dt;
        x_next[0] = x[0] + dt * x[2] + 0.5 * dt * dt * u[0];
        x_next[1] = x[1] + dt * x[3] + 0.5 * dt * dt * u[1];
        x_next[2] = x[2] + dt * u[0];
        x_next[3] = x[3] + dt * u[1];
    }
}

/* Reverse of orc_model_step: cotangent gx_next of x_{k+1} -> adds dL/dx_k to gx, dL/du to gu. */
static void model_step_vjp(const orc_problem* p, const double* x, const double* u,
                           const double* gx_next, double* gx, double* gu)
{
    if (p->model == 0) {
        int ns = p->n_sub;
        double h = p->dt / ns;
        double* xs = (double*)malloc(sizeof(double) * 6 * (size_t)(ns + 1));
        memcpy(xs, x, sizeof(double) * 6);
        for (int j = 0; j < ns; ++j) {
            double dx[6];
            bicycle_rhs(p, xs + 6 * j, u, dx);
            for (int i = 0; i < 6; ++i) xs[6 * (j + 1) + i] = xs[6 * j + i] + h * dx[i];
        }
        double g[6];
        memcpy(g, gx_next, sizeof g);
        for (int j = ns - 1; j >= 0; --j) {
            double hg[6], gxs[6] = {0, 0, 0, 0, 0, 0};
            for (int i = 0; i < 6; ++i) hg[i] = h * g[i];
            bicycle_rhs_vjp(p, xs + 6 * j, u, hg, gxs, gu);
            for (int i = 0; i < 6; ++i) g[i] += gxs[i];
        }
        for (int i = 0; i < 6; ++i) gx[i] += g[i];
        free(xs);
    } else {
        double dt = p->dt;
        gx[0] += gx_next[0];
        gx[1] += gx_next[1];
        gx[2] += dt * gx_next[0] + gx_next[2];
        gx[3] += dt * gx_next[1] + gx_next[3];
        gu[0] += 0.5 * dt * dt * gx_next[0] + dt * gx_next[2];
        gu[1] += 0.5 * dt * dt * gx_next[1] + dt * gx_next[3];
    }
}

static void philox_words(const orc_problem* p, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t stream,
                         uint32_t solve_ctr, uint32_t w[4])
{
    uint32_t key[2] = {(uint32_t)(p->seed & 0xffffffffu), (uint32_t)(p->seed >> 32)};
    uint32_t ctr[4] = {c0, c1, c2, (stream << 28) | (solve_ctr & 0x0fffffffu)};
    orc_philox4x32_10(ctr, key, w);
}

/* n standard normals of one (step t, particle n, sample k) draw of a stream. */
static void draw_normals(const orc_problem* p, int n_out, uint32_t t, uint32_t n, uint32_t k,
                         uint32_t stream, uint32_t solve_ctr, double* z)
{
    uint32_t w[4];
    int pairs = (n_out + 1) / 2;
    for (int i = 0; i < pairs; ++i) {
        if (i % 2 == 0) philox_words(p, t | ((uint32_t)(i / 2) << 16), n, k, stream, solve_ctr, w);
        double pair[2];
        orc_gaussian_pair(w[2 * (i % 2)], w[2 * (i % 2) + 1], pair);
        z[2 * i] = pair[0];
        if (2 * i + 1 < n_out) z[2 * i + 1] = pair[1];
    }
}

/* The state disturbance of particle n at step t. For 6 states, particles n and n + H with
 * H = 2^ceil(log2 M) / 2 share one counter (word 1 = n mod H, the lower index): calls 0-2 give six
 * Gaussian pairs, pairs 0-2 to the lower particle and pairs 3-5 to the upper one, so no word is
 * drawn unused. Other state counts draw per particle (4 or 8 normals use whole calls). */
static void draw_disturbance(const orc_problem* p, int nx, uint32_t t, uint32_t n, uint32_t kk, uint32_t solve_ctr,
                             double* z)
{
    if (nx != 6) {
        draw_normals(p, nx, t, n, kk, 1, solve_ctr, z);
        return;
    }
    uint32_t pw = 1;
    while (pw < (uint32_t)p->M) pw <<= 1;
    const uint32_t H = pw / 2;
    const uint32_t half = n >= H ? 1u : 0u, q = n - half * H;
    double pairs[12];
    for (int i = 0; i < 6; ++i) {
        uint32_t w[4];
        philox_words(p, t | ((uint32_t)(i / 2) << 16), q, kk, 1, solve_ctr, w);
        orc_gaussian_pair(w[2 * (i % 2)], w[2 * (i % 2) + 1], pairs + 2 * i);
    }
    for (int i = 0; i < 6; ++i) z[i] = pairs[6 * half + i];
}

/* Belief barrier, Eq. "DCBF": h = (w_T - nu sigma_y)^2 - mean_ey^2 with sigma_y^2 the (e_y, e_y)
 * entry of the covariance (eta = gradient of the boundary constraint = unit vector on e_y). With
 * clamp_margin the margin w_T - nu sigma_y is taken as 0 once the back-off exceeds the half-width. */
static double belief_h(const orc_problem* p, double nu, const double* mean, const double* cov, int nx)
{
    int e = p->ey_index;
    double sig = sqrt(fmax(cov[e * nx + e], 0.0));
    double b = p->w_T - nu * sig;
    if (p->clamp_margin && b < 0.0) b = 0.0;
    return b * b - mean[e] * mean[e];
}

/* Remark 1: the back-off of the racing barrier for the chance level delta. */
static double racing_nu(const orc_problem* p)
{
    return p->backoff ? orc_backoff_cantelli(p->delta) : orc_backoff_gaussian(p->delta);
}

/* c_i(x) of one constraint and its gradient eta = grad c_i(x) (Assumption 1). */
static double constraint_value(const orc_constraint* c, const double* x, int nx, double* eta)
{
    for (int l = 0; l < nx; ++l) eta[l] = 0.0;
    if (c->kind == 0) {
        double v = -c->b;
        for (int l = 0; l < nx; ++l) {
            v += c->a[l] * x[l];
            eta[l] = c->a[l];
        }
        return v;
    }
    double di = x[c->i] - c->center[0], dj = x[c->j] - c->center[1];
    eta[c->i] = -2.0 * di;
    eta[c->j] = -2.0 * dj;
    return c->radius * c->radius - di * di - dj * dj;
}

/* General belief barrier, Eq. "DCBFchoice0" and Eq. "DCBFchoice": h = min_i h_i with
 * h_i = -c_i(mean) - nu_i sqrt(eta_i^T Sigma eta_i), eta_i = grad c_i(mean), nu_i from Remark 1. */
static double general_h(const orc_problem* p, const double* mean, const double* cov, int nx)
{
    double h = INFINITY;
    for (int q = 0; q < p->n_con; ++q) {
        const orc_constraint* c = p->con + q;
        double eta[8];
        double cv = constraint_value(c, mean, nx, eta);
        double quad = 0.0;
        for (int a = 0; a < nx; ++a)
            for (int b = 0; b < nx; ++b) quad += eta[a] * cov[a * nx + b] * eta[b];
        double nu = c->backoff == 0 ? orc_backoff_gaussian(c->p) : orc_backoff_cantelli(c->p);
        double hi = -cv - nu * sqrt(fmax(quad, 0.0));
        if (hi < h) h = hi;
    }
    return h;
}

/* Running cost, Eq. "CostFunction": (x - x_g)^T Q (x - x_g) + C_obs when the mean breaks a
 * constraint (|e_y| > w_T for the racing barrier; c_i(mean) > 0 for some i for the general set). */
static double state_cost(const orc_problem* p, const double* W, const double* xm, int nx)
{
    double c = 0.0;
    for (int i = 0; i < nx; ++i) {
        double d = xm[i] - p->x_goal[i];
        c += W[i] * d * d;
    }
    if (p->n_con == 0) {
        if (fabs(xm[p->ey_index]) > p->w_T) c += p->C_obs;
    } else {
        int broken = 0;
        for (int q = 0; q < p->n_con; ++q) {
            double eta[8];
            if (constraint_value(p->con + q, xm, nx, eta) > 0.0) broken = 1;
        }
        if (broken) c += p->C_obs;
    }
    return c;
}

/* Eq. "cbfpenalty": C_safe(z_k) = C max(-h(z_k^(1)) + (1 - gamma) h(z_k^(2)), 0). */
static double c_safe(const orc_problem* p, double h_now, double h_prev)
{
    double a = -h_now + (1.0 - p->gamma) * h_prev;
    return p->C_safe * (a > 0.0 ? a : 0.0);
}

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

int orc_rollout_threads(const orc_problem* p, const double* x0, const double* Sigma0, const double* v,
                        uint32_t solve_ctr, int k_begin, int k_end, const orc_outputs* out, int n_threads)
{
    const int nx = orc_nx(p), M = p->M, T = p->T;
    if (M < 2 || T < 1 || k_begin < 0 || k_end > p->K || k_begin > k_end) return -1;
    double L_eps[4], L_w[64], L_0[64], Sinv[4];
    cholesky_psd(2, p->Sigma_eps, L_eps);
    cholesky_psd(nx, p->Sigma_w, L_w);
    if (Sigma0) cholesky_psd(nx, Sigma0, L_0);
    double det = p->Sigma_eps[0] * p->Sigma_eps[3] - p->Sigma_eps[1] * p->Sigma_eps[2];
    Sinv[0] = p->Sigma_eps[3] / det; Sinv[1] = -p->Sigma_eps[1] / det;
    Sinv[2] = -p->Sigma_eps[2] / det; Sinv[3] = p->Sigma_eps[0] / det;
    const double nu = racing_nu(p);

    /* The samples are independent until the weights (Algorithm 1 rolls each one out on its own),
     * so with n_threads > 1 (and an OpenMP build) threads take whole samples; every sample's
     * arithmetic is the same as with one thread. */
#pragma omp parallel num_threads(n_threads > 1 ? n_threads : 1)
    {
        double* X = (double*)malloc(sizeof(double) * (size_t)M * nx);      /* particles x^n_k */
        double* xbar = (double*)malloc(sizeof(double) * (size_t)(T + 1) * nx);
        double* Sig = (double*)malloc(sizeof(double) * (size_t)(T + 1) * nx * nx);
        double* hz = (double*)malloc(sizeof(double) * (size_t)(T + 1));
        double* u = (double*)malloc(sizeof(double) * (size_t)T * 2);

#pragma omp for schedule(dynamic, 4)
        for (int m = k_begin; m < k_end; ++m) {
            /* Algorithm 1: initialise the belief state z_0 = (z_0, z_{-1} = z_0) from the estimate. */
            memcpy(xbar, x0, sizeof(double) * nx);
            for (int i = 0; i < nx * nx; ++i) Sig[i] = Sigma0 ? Sigma0[i] : 0.0;
            uint32_t kk = p->crn_disturbance ? 0u : (uint32_t)m;
            for (int n = 0; n < M; ++n) {
                for (int i = 0; i < nx; ++i) X[n * nx + i] = x0[i];
                if (Sigma0) {
                    double xi[8];
                    draw_normals(p, nx, 0, (uint32_t)n, kk, 3, solve_ctr, xi);
                    for (int i = 0; i < nx; ++i)
                        for (int j = 0; j <= i; ++j) X[n * nx + i] += L_0[i * nx + j] * xi[j];
                }
            }
            /* Sample the control perturbation sequence eps^m ~ N(0, Sigma_eps). */
            for (int k = 0; k < T; ++k) {
                double z[2];
                draw_normals(p, 2, (uint32_t)k, 0, (uint32_t)m, 0, solve_ctr, z);
                double e0 = L_eps[0] * z[0];
                double e1 = L_eps[2] * z[0] + L_eps[3] * z[1];
                u[2 * k + 0] = clampd(v[2 * k + 0] + e0, p->u_min[0], p->u_max[0]);
                u[2 * k + 1] = clampd(v[2 * k + 1] + e1, p->u_min[1], p->u_max[1]);
            }
            /* Roll out: Algorithm 2 propagates the particles, then the augmented cost accumulates. */
            hz[0] = p->n_con ? general_h(p, xbar, Sig, nx) : belief_h(p, nu, xbar, Sig, nx);
            double S = 0.0;
            for (int k = 0; k < T; ++k) {
                const double* uk = u + 2 * k;
                if (p->resample && k > 0) {
                    /* Algorithm 2's sampling of the particles, x^n_k ~ N(xbar_k, Sigma_k), drawn as
                     * xbar_k + L_k xi^n with L_k the (PSD) Cholesky factor of the Monte-Carlo covariance
                     * of step k and xi^n from stream 4. At k = 0 the initial particles above are the draw. */
                    double Lk[64];
                    cholesky_psd(nx, Sig + (size_t)k * nx * nx, Lk);
                    const double* mk = xbar + (size_t)k * nx;
                    for (int n = 0; n < M; ++n) {
                        double xi[8];
                        draw_normals(p, nx, (uint32_t)k, (uint32_t)n, kk, 4, solve_ctr, xi);
                        for (int i = 0; i < nx; ++i) {
                            double x = mk[i];
                            for (int j = 0; j <= i; ++j) x += Lk[i * nx + j] * xi[j];
                            X[n * nx + i] = x;
                        }
                    }
                }
                for (int n = 0; n < M; ++n) {
                    double xn[8], w[8], z[8];
                    orc_model_step(p, X + n * nx, uk, xn);
                    draw_disturbance(p, nx, (uint32_t)k, (uint32_t)n, kk, solve_ctr, z);
                    for (int i = 0; i < nx; ++i) {
                        w[i] = 0.0;
                        for (int j = 0; j <= i; ++j) w[i] += L_w[i * nx + j] * z[j];
                    }
                    for (int i = 0; i < nx; ++i) X[n * nx + i] = xn[i] + w[i];
                }
                double* mk = xbar + (size_t)(k + 1) * nx;
                double* Sk = Sig + (size_t)(k + 1) * nx * nx;
                for (int i = 0; i < nx; ++i) {
                    double s = 0.0;
                    for (int n = 0; n < M; ++n) s += X[n * nx + i];
                    mk[i] = s / M;
                }
                for (int i = 0; i < nx; ++i)
                    for (int j = 0; j < nx; ++j) {
                        double s = 0.0;
                        for (int n = 0; n < M; ++n) s += (X[n * nx + i] - mk[i]) * (X[n * nx + j] - mk[j]);
                        Sk[i * nx + j] = s / (M - 1);
                    }
                hz[k + 1] = p->n_con ? general_h(p, mk, Sk, nx) : belief_h(p, nu, mk, Sk, nx);
                /* S += q(xbar_k) + ctrl_w v_k^T Sigma_eps^-1 u_k + C_safe(z_k), with h_{-1} = h_0. */
                double vSu = v[2 * k] * (Sinv[0] * uk[0] + Sinv[1] * uk[1])
                           + v[2 * k + 1] * (Sinv[2] * uk[0] + Sinv[3] * uk[1]);
                double h_prev = (k == 0) ? hz[0] : hz[k - 1];
                S += state_cost(p, p->Q, xbar + (size_t)k * nx, nx) + p->ctrl_w * vSu + c_safe(p, hz[k], h_prev);
            }
            /* Terminal: phi(xbar_T) + C_safe(z_T). */
            S += state_cost(p, p->Qf, xbar + (size_t)T * nx, nx) + c_safe(p, hz[T], hz[T > 0 ? T - 1 : 0]);

            if (out->S) out->S[m] = S;
            if (out->u) memcpy(out->u + (size_t)m * T * 2, u, sizeof(double) * T * 2);
            if (out->mean) memcpy(out->mean + (size_t)m * (T + 1) * nx, xbar, sizeof(double) * (T + 1) * nx);
            if (out->cov) memcpy(out->cov + (size_t)m * (T + 1) * nx * nx, Sig, sizeof(double) * (T + 1) * nx * nx);
            if (out->h) memcpy(out->h + (size_t)m * (T + 1), hz, sizeof(double) * (T + 1));
            if (out->margin) {
                double mg = INFINITY;
                for (int k = 0; k <= T; ++k) {
                    if (p->n_con == 0) {
                        double d = fabs(fabs(xbar[(size_t)k * nx + p->ey_index]) - p->w_T);
                        if (d < mg) mg = d;
                    } else {
                        for (int q = 0; q < p->n_con; ++q) {
                            double eta[8];
                            double d = fabs(constraint_value(p->con + q, xbar + (size_t)k * nx, nx, eta));
                            if (d < mg) mg = d;
                        }
                    }
                }
                out->margin[m] = mg;
            }
        }
        free(X); free(xbar); free(Sig); free(hz); free(u);
    }
    return 0;
}

int orc_rollout(const orc_problem* p, const double* x0, const double* Sigma0, const double* v,
                uint32_t solve_ctr, int k_begin, int k_end, const orc_outputs* out)
{
    return orc_rollout_threads(p, x0, Sigma0, v, solve_ctr, k_begin, k_end, out, 1);
}

/* Eq. "Weights" and Eq. "MPPI update law": beta = min S, w = exp(-(S - beta)/lambda),
 * v+ = sum_m w_m u^m / sum_m w_m. */
void orc_optimal_control(int K, int T, double lambda, const double* S, const double* u,
                         double* w, double* v_plus, double* diag)
{
    double beta = INFINITY;
    for (int m = 0; m < K; ++m) if (S[m] < beta) beta = S[m];
    double* om = (double*)malloc(sizeof(double) * (size_t)K);
    double eta = 0.0;
    for (int m = 0; m < K; ++m) { om[m] = exp(-(S[m] - beta) / lambda); eta += om[m]; }
    if (v_plus && u) {
        for (int i = 0; i < 2 * T; ++i) {
            double acc = 0.0;
            for (int m = 0; m < K; ++m) acc += om[m] * u[(size_t)m * 2 * T + i];
            v_plus[i] = acc / eta;
        }
    }
    double sq = 0.0;
    for (int m = 0; m < K; ++m) {
        double wh = om[m] / eta;
        if (w) w[m] = wh;
        sq += wh * wh;
    }
    if (diag) { diag[0] = beta; diag[1] = eta; diag[2] = 1.0 / sq; diag[3] = beta - lambda * log(eta / K); }
    free(om);
}

/* Eq. "Weights" and Eq. "MPPI update law" restricted to the samples [k_begin, k_end): the
 * log-sum-exp partial {beta_g = min S, eta_g = sum omega, q_g = sum omega^2, U_g[2T] = sum omega u}
 * with omega = exp(-(S - beta_g)/lambda) over that subset. */
void orc_lse_partial(int k_begin, int k_end, int T, double lambda, const double* S, const double* u, double* part)
{
    double beta = INFINITY;
    for (int m = k_begin; m < k_end; ++m) if (S[m] < beta) beta = S[m];
    double eta = 0.0, q = 0.0;
    for (int i = 0; i < 2 * T; ++i) part[3 + i] = 0.0;
    for (int m = k_begin; m < k_end; ++m) {
        double om = exp(-(S[m] - beta) / lambda);
        eta += om;
        q += om * om;
        for (int i = 0; i < 2 * T; ++i) part[3 + i] += om * u[(size_t)m * 2 * T + i];
    }
    part[0] = beta; part[1] = eta; part[2] = q;
}

/* Merge of G partials (a disjoint cover of the samples): beta = min_g beta_g, each partial rescaled
 * by f_g = exp(-(beta_g - beta)/lambda), eta = sum f_g eta_g, v+ = sum f_g U_g / eta; diag as in
 * orc_optimal_control with K_total samples (ESS = eta^2 / sum f_g^2 q_g). */
void orc_lse_merge(int G, int T, double lambda, int K_total, const double* parts, double* v_plus, double* diag)
{
    const int stride = 3 + 2 * T;
    double beta = INFINITY;
    for (int g = 0; g < G; ++g) if (parts[g * stride] < beta) beta = parts[g * stride];
    double eta = 0.0, q = 0.0;
    for (int i = 0; i < 2 * T; ++i) v_plus[i] = 0.0;
    for (int g = 0; g < G; ++g) {
        const double* pg = parts + (size_t)g * stride;
        double f = exp(-(pg[0] - beta) / lambda);
        eta += f * pg[1];
        q += f * f * pg[2];
        for (int i = 0; i < 2 * T; ++i) v_plus[i] += f * pg[3 + i];
    }
    for (int i = 0; i < 2 * T; ++i) v_plus[i] /= eta;
    if (diag) { diag[0] = beta; diag[1] = eta; diag[2] = eta * eta / q; diag[3] = beta - lambda * log(eta / K_total); }
}

int orc_solve_threads(const orc_problem* p, const double* x0, const double* Sigma0, const double* v,
                      uint32_t solve_ctr, const orc_outputs* out, int n_threads)
{
    orc_outputs o = *out;
    double* S = o.S ? o.S : (double*)malloc(sizeof(double) * (size_t)p->K);
    double* u = o.u ? o.u : (double*)malloc(sizeof(double) * (size_t)p->K * p->T * 2);
    o.S = S; o.u = u;
    int rc = orc_rollout_threads(p, x0, Sigma0, v, solve_ctr, 0, p->K, &o, n_threads);
    if (rc == 0) orc_optimal_control(p->K, p->T, p->lambda, S, u, o.w, o.v_plus, o.diag);
    if (!out->S) free(S);
    if (!out->u) free(u);
    return rc;
}

int orc_solve(const orc_problem* p, const double* x0, const double* Sigma0, const double* v,
              uint32_t solve_ctr, const orc_outputs* out)
{
    return orc_solve_threads(p, x0, Sigma0, v, solve_ctr, out, 1);
}

void orc_shift(int T, double* v)
{
    for (int k = 0; k + 1 < T; ++k) { v[2 * k] = v[2 * k + 2]; v[2 * k + 1] = v[2 * k + 3]; }
}

/* Shield repair objective and its adjoint. J_r(v) = sum_{t=1..T} C_safe(z_t) of the belief
 * rollout of the nominal controls v (no control noise; the disturbance draws of sample 0, so the
 * draws are common to every evaluation). The reverse sweep differentiates the Monte-Carlo mean
 * and unbiased variance of e_y, the barrier h and the hinge of C_safe, then the dynamics. */
double orc_repair_objective(const orc_problem* p, const double* x0, const double* v,
                            uint32_t solve_ctr, double* grad, double* args_out)
{
    const int nx = orc_nx(p), M = p->M, T = p->T, e = p->ey_index;
    /* The adjoint covers the bicycle and the double integrator only (model_step_vjp). */
    if (p->model == 2 || M < 2 || T < 1) return NAN;
    double L_w[64];
    cholesky_psd(nx, p->Sigma_w, L_w);
    const double nu = racing_nu(p);
    double* X = (double*)malloc(sizeof(double) * (size_t)(T + 1) * M * nx);
    double* mean = (double*)calloc((size_t)(T + 1), sizeof(double));
    double* sig = (double*)calloc((size_t)(T + 1), sizeof(double));
    double* hz = (double*)calloc((size_t)(T + 1), sizeof(double));
    double* arg = (double*)calloc((size_t)(T + 1), sizeof(double));
    for (int n = 0; n < M; ++n)
        for (int i = 0; i < nx; ++i) X[(size_t)n * nx + i] = x0[i];
    mean[0] = x0[e];
    sig[0] = 0.0;
    hz[0] = (p->w_T) * (p->w_T) - x0[e] * x0[e];
    for (int t = 0; t < T; ++t) {
        for (int n = 0; n < M; ++n) {
            double xn[8], z[8];
            const double* xc = X + ((size_t)t * M + n) * nx;
            double* xo = X + ((size_t)(t + 1) * M + n) * nx;
            orc_model_step(p, xc, v + 2 * t, xn);
            draw_disturbance(p, nx, (uint32_t)t, (uint32_t)n, 0u, solve_ctr, z);
            for (int i = 0; i < nx; ++i) {
                double w = 0.0;
                for (int j = 0; j <= i; ++j) w += L_w[i * nx + j] * z[j];
                xo[i] = xn[i] + w;
            }
        }
        double s = 0.0;
        for (int n = 0; n < M; ++n) s += X[((size_t)(t + 1) * M + n) * nx + e];
        double mu_e = s / M, q = 0.0;
        for (int n = 0; n < M; ++n) {
            double d = X[((size_t)(t + 1) * M + n) * nx + e] - mu_e;
            q += d * d;
        }
        mean[t + 1] = mu_e;
        sig[t + 1] = sqrt(q / (M - 1));
        double b = p->w_T - nu * sig[t + 1];
        if (p->clamp_margin && b < 0.0) b = 0.0;
        hz[t + 1] = b * b - mu_e * mu_e;
    }
    double J = 0.0;
    for (int t = 1; t <= T; ++t) {
        arg[t] = -hz[t] + (1.0 - p->gamma) * hz[t - 1];
        J += c_safe(p, hz[t], hz[t - 1]);
    }
    if (args_out)
        for (int t = 0; t <= T; ++t) args_out[t] = arg[t];
    if (grad) {
        double* G = (double*)calloc((size_t)M * nx, sizeof(double));   /* dJ/dx^n_t */
        for (int i = 0; i < 2 * T; ++i) grad[i] = 0.0;
        for (int t = T; t >= 1; --t) {
            double gh = 0.0;
            if (arg[t] > 0.0) gh += -p->C_safe;
            if (t + 1 <= T && arg[t + 1] > 0.0) gh += p->C_safe * (1.0 - p->gamma);
            if (gh != 0.0) {
                double dh_dmean = -2.0 * mean[t];
                double margin = p->w_T - nu * sig[t];
                if (p->clamp_margin && margin < 0.0) margin = 0.0;  /* the clamped margin has no slope in sigma */
                double dh_dsig = -2.0 * nu * margin;
                for (int n = 0; n < M; ++n) {
                    double en = X[((size_t)t * M + n) * nx + e];
                    double g = dh_dmean / M;
                    if (sig[t] > 0.0) g += dh_dsig * (en - mean[t]) / ((M - 1) * sig[t]);
                    G[(size_t)n * nx + e] += gh * g;
                }
            }
            for (int n = 0; n < M; ++n) {
                double gx[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                model_step_vjp(p, X + ((size_t)(t - 1) * M + n) * nx, v + 2 * (t - 1),
                               G + (size_t)n * nx, gx, grad + 2 * (t - 1));
                memcpy(G + (size_t)n * nx, gx, sizeof(double) * nx);
            }
        }
        free(G);
    }
    free(X); free(mean); free(sig); free(hz); free(arg);
    return J;
}
