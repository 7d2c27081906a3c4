// Host runtime of the C ABI declared in include/bssmppi.h: parameter validation, derived
// constants (Cholesky factors, Sigma_eps^-1, back-off nu), device buffers and kernel launches.
#include "../../include/bssmppi.h"
#include "device.cuh"
#include "internal.h"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

struct bssmppi_ctx {
    bssmppi_params prm{};
    bss::DevParams dp{};
    int P = 1;            // particles per lane (1, 2, 4 or 8)
    bss::RollLaunch roll; // persistent rollout launch shape
    bss::ConSet cons{};   // general constraint set (n = 0: the racing barrier)
    int nx = 6;           // 4, 6 or 8 states
    cudaStream_t stream = nullptr;
    int device = 0;
    float* d_kappa = nullptr;
    float* d_S = nullptr;
    float* d_w = nullptr;
    float* d_eps = nullptr;
    float* d_mean = nullptr;
    float* d_var = nullptr;
    float* d_v = nullptr;
    float* d_in = nullptr;      // device staging of the host-buffer solve: x0 (8) | v (2T) | Sigma0 (64)
    float* d_x0 = nullptr;      // = d_in
    float* d_Sigma0 = nullptr;  // = d_in + 8 + 2T
    float* d_u0 = nullptr;
    float* d_diag = nullptr;
    uint32_t* d_ctr = nullptr;
    float* d_tail_part = nullptr;  // block partials of the rollout's fused weights/update tail
    unsigned int* d_ticket = nullptr;
    float* d_repair_X = nullptr;  // stored particle states of the repair rollout
    float* d_repair_J = nullptr;  // objective of the last repair_grad call
    float* h_stage = nullptr;   // pinned host staging: x0 (8) | v (2T) | Sigma0 (64) || v+ (2T) | u0 (2)
    // The host-buffer solve as CUDA graphs (H2D copy, solve kernel, D2H copy), one per combination
    // of the optional buffers, captured on first use on a private stream and replayed on `stream`.
    // Dropped whenever the kernel's by-value parameters change (sample range, constraint set).
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t host_graph[8] = {};
    // timing ring: 2 events per recorded solve
    cudaEvent_t* ev = nullptr;
    int ev_cap = 0, ev_count = 0;
    std::string err;
};

namespace {

thread_local std::string g_create_error;

int fail(bssmppi_ctx* h, int code, const std::string& msg)
{
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

int cuda_fail(bssmppi_ctx* h, cudaError_t e, const char* what)
{
    return fail(h, BSSMPPI_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define BSS_CUDA(h, call)                                               \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);        \
    } while (0)

// PSD-tolerant Cholesky (lower, row-major) in double; zero pivots give zero columns.
// Returns false if the matrix is not symmetric positive semidefinite (within a tolerance).
bool cholesky_psd(int n, const double* A, double* L)
{
    double scale = 0.0;
    for (int i = 0; i < n; ++i) scale = std::fmax(scale, std::fabs(A[i * n + i]));
    const double tol = 1e-12 * (scale > 0 ? scale : 1.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (std::fabs(A[i * n + j] - A[j * n + i]) > tol) return false;
    std::memset(L, 0, sizeof(double) * n * n);
    for (int j = 0; j < n; ++j) {
        double d = A[j * n + j];
        for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
        if (d < -tol) return false;
        if (d <= tol) {
            // zero pivot: the rest of the column must vanish for the matrix to be PSD
            for (int i = j + 1; i < n; ++i) {
                double s = A[i * n + j];
                for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
                if (std::fabs(s) > 1e-9 * (scale > 0 ? scale : 1.0)) return false;
            }
            continue;
        }
        const double ljj = std::sqrt(d);
        L[j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = s / ljj;
        }
    }
    return true;
}

// erfinv(y) for |y| < 1: Winitzki's closed-form approximation (S. Winitzki, "A handy
// approximation for the error function and its inverse", 2008) refined by Newton steps on
// std::erf, whose derivative is 2/sqrt(pi) exp(-x^2).
double inverse_erf(double y)
{
    const double a = 0.147, pi = 3.14159265358979323846;
    const double ln = std::log((1.0 - y) * (1.0 + y));
    const double t = 2.0 / (pi * a) + 0.5 * ln;
    double x = std::copysign(std::sqrt(std::sqrt(t * t - ln / a) - t), y);
    for (int i = 0; i < 6; ++i) {
        const double f = std::erf(x) - y;
        x -= f / (2.0 / std::sqrt(pi) * std::exp(-x * x));
    }
    return x;
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

int validate(const bssmppi_params* p, std::string& why)
{
    auto bad = [&](const char* m) { why = m; return BSSMPPI_EINVAL; };
    if (!p) return bad("params is NULL");
    if (p->K < 1 || p->K > BSSMPPI_K_MAX) return bad("K out of range [1, 2^20]");
    if (p->M < 2 || p->M > BSSMPPI_M_MAX) return bad("M out of range [2, 256] (an unbiased variance needs M >= 2)");
    if (p->T < 1 || p->T > BSSMPPI_T_MAX) return bad("T out of range [1, 256]");
    if (p->model != BSSMPPI_MODEL_BICYCLE6 && p->model != BSSMPPI_MODEL_DOUBLE_INT4 && p->model != BSSMPPI_MODEL_WHEELS8)
        return bad("unknown model");
    if (p->model == BSSMPPI_MODEL_BICYCLE6 && p->ey_index != 4) return bad("bicycle model constrains e_y: ey_index must be 4");
    if (p->model != BSSMPPI_MODEL_DOUBLE_INT4 &&
        (!(p->tire_B > 0.0f) || !(p->tire_C > 0.0f) || !std::isfinite(p->tire_B) || !std::isfinite(p->tire_C)))
        return bad("the tyre curve needs finite B > 0 and C > 0");
    if (p->model == BSSMPPI_MODEL_WHEELS8 && p->ey_index != 6) return bad("wheel-speed model constrains e_y: ey_index must be 6");
    if (p->model == BSSMPPI_MODEL_WHEELS8 && p->M > 128) return bad("the wheel-speed model takes M <= 128");
    if (p->model == BSSMPPI_MODEL_WHEELS8 &&
        !(p->wheel_radius > 0 && p->wheel_inertia > 0 && p->mu_x > 0 && p->tau_max >= 0 && p->slip_floor > 0))
        return bad("wheel constants must be > 0 (tau_max >= 0)");
    if (p->model == BSSMPPI_MODEL_DOUBLE_INT4 && p->ey_index != 1) return bad("double integrator constrains p_y: ey_index must be 1");
    if (p->n_sub < 1 || p->n_sub > 64) return bad("n_sub out of range [1, 64]");
    if (!(p->dt > 0.0f)) return bad("dt must be > 0");
    if (p->model != BSSMPPI_MODEL_DOUBLE_INT4) {
        if (!(p->mass > 0 && p->Iz > 0 && p->lf > 0 && p->lr > 0 && p->g > 0 && p->vx_floor > 0)) return bad("model constants must be > 0");
        if (!p->track_kappa) return bad("track_kappa is NULL");
        if (!is_pow2(p->n_track) || p->n_track < 2 || p->n_track > BSSMPPI_NTRACK_MAX) return bad("n_track must be a power of two in [2, 16384]");
        if (!(p->track_len > 0.0f)) return bad("track_len must be > 0");
    }
    for (int j = 0; j < 2; ++j)
        if (!(p->u_min[j] < p->u_max[j])) return bad("u_min must be < u_max");
    if (!(p->lambda > 0.0f) || !std::isfinite(p->lambda)) return bad("lambda must be finite and > 0");
    if (!(p->delta > 0.0f && p->delta < 0.5f)) return bad("delta must be in (0, 0.5)");
    if (!(p->gamma > 0.0f && p->gamma < 1.0f)) return bad("gamma must be in (0, 1)");
    if (!(p->w_T > 0.0f)) return bad("w_T must be > 0");
    if (p->resample != 0 && p->resample != 1) return bad("resample must be 0 or 1");
    if (p->resample && !p->compensated) return bad("resample needs compensated = 1");
    const double* Se = p->Sigma_eps;
    if (!(Se[0] > 0 && Se[3] > 0 && Se[0] * Se[3] - Se[1] * Se[2] > 0 && std::fabs(Se[1] - Se[2]) <= 1e-12 * (Se[0] + Se[3])))
        return bad("Sigma_eps must be symmetric positive definite");
    return BSSMPPI_OK;
}

template <typename T>
int alloc(bssmppi_ctx* h, T** ptr, size_t count)
{
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(ptr), count * sizeof(T));
    if (e != cudaSuccess) {
        *ptr = nullptr;
        return fail(h, e == cudaErrorMemoryAllocation ? BSSMPPI_ENOMEM : BSSMPPI_ECUDA,
                    std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    return BSSMPPI_OK;
}

void release(bssmppi_ctx* h)
{
    // d_x0 and d_Sigma0 live in d_in, d_u0 in d_v
    void* ptrs[] = {h->d_kappa, h->d_S, h->d_w, h->d_eps, h->d_mean, h->d_var, h->d_v, h->d_in,
                    h->d_diag, h->d_ctr, h->d_ticket, h->d_repair_X, h->d_repair_J,
                    h->d_tail_part};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (h->h_stage) cudaFreeHost(h->h_stage);
    for (cudaGraphExec_t& g : h->host_graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    h->cap_stream = nullptr;
    for (int i = 0; i < 2 * h->ev_cap; ++i) cudaEventDestroy(h->ev[i]);
    delete[] h->ev;
    h->ev = nullptr;
    h->ev_cap = 0;
}

}  // namespace

void bss::set_thread_error(const char* msg) { g_create_error = msg ? msg : ""; }

// SM count of the current device (the lane mapping's occupancy rule); without one, a count so large
// that the rule keeps one particle per lane.
static int device_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms < 1) {
        (void)cudaGetLastError();
        return 1 << 20;
    }
    return sms;
}

// The even-polynomial interpolation behind both tyre fits: c_0..c_9 such that f(x) ~ sum_i c_i x^(2i)
// on |x| <= 1, f even (given as g(x) = f(x) for x in (0, 1]). p(z) interpolates q(z) = f(sqrt z) at
// the ten Chebyshev points z_k = (1 + cos(pi (k + 1/2) / 10)) / 2 of [0, 1]. The Chebyshev
// coefficients come from the discrete cosine sums; the three-term recurrence
// T_{j+1} = 2u T_j - T_{j-1} turns them into powers of u = 2z - 1, and the binomial expansion into
// powers of z. Everything is in double precision; the coefficients are rounded to FP32 at the end.
// The tyre curve's q(z) = sin(C atan sqrt z) / sqrt z is analytic on [0, 1] with its nearest
// singularity at z = -1, so the interpolant is within about 4e-8 of it. The rear tyre's, in x = t / tau
// with tau = tan(1/B) (or 1/2 if less), q(z) = sin(C atan(-B atan(tau sqrt z))) / sqrt z, has its
// nearest singularity where B atan(tau x) = +-i, at z = -tanh(1/B)^2 / tau^2 (about -0.99 at B = 10),
// no nearer in relative terms.
template <typename G>
static void even_poly_fit(G g, float* c)
{
    constexpr int N = bss::kTyreDeg + 1;
    const double pi = 3.14159265358979323846;
    double f[N], a[N];
    for (int k = 0; k < N; ++k) {
        const double z = 0.5 * (1.0 + std::cos(pi * (k + 0.5) / N));
        f[k] = g(std::sqrt(z));
    }
    for (int j = 0; j < N; ++j) {
        double sum = 0.0;
        for (int k = 0; k < N; ++k) sum += f[k] * std::cos(pi * j * (k + 0.5) / N);
        a[j] = (j == 0 ? 1.0 : 2.0) * sum / N;
    }
    double pu[N] = {}, t0[N] = {}, t1[N] = {}, t2[N];
    t0[0] = 1.0;
    t1[1] = 1.0;
    for (int i = 0; i < N; ++i) pu[i] = a[0] * t0[i] + a[1] * t1[i];
    for (int j = 2; j < N; ++j) {
        for (int i = 0; i < N; ++i) t2[i] = (i > 0 ? 2.0 * t1[i - 1] : 0.0) - t0[i];
        for (int i = 0; i < N; ++i) {
            pu[i] += a[j] * t2[i];
            t0[i] = t1[i];
            t1[i] = t2[i];
        }
    }
    double pz[N] = {};
    for (int i = 0; i < N; ++i) {  // pu_i (2z - 1)^i = pu_i sum_m binom(i, m) 2^m z^m (-1)^(i - m)
        double binom = 1.0;
        for (int m = 0; m <= i; ++m) {
            pz[m] += pu[i] * binom * std::ldexp(1.0, m) * (((i - m) & 1) ? -1.0 : 1.0);
            binom = binom * (i - m) / (m + 1);
        }
    }
    for (int i = 0; i < N; ++i) c[i] = (float)pz[i];
}

void bss::tyre_curve_fit(double C, float* c)
{
    even_poly_fit([&](double x) { return std::sin(C * std::atan(x)) / x; }, c);
}

double bss::rear_tyre_tau(double B)
{
    const double half = 0.5;
    return 1.0 / B < std::atan(half) ? std::tan(1.0 / B) : half;
}

void bss::rear_tyre_fit(double B, double C, float* c)
{
    const double tau = rear_tyre_tau(B);
    even_poly_fit([&](double x) { return std::sin(C * std::atan(-B * std::atan(tau * x))) / x; }, c);
}

// Validates the parameters and derives the kernels' constants: lane mapping (seg, spw, P),
// Cholesky factors, Sigma_eps^-1, the back-off nu, the Philox round keys and the model constants.
int bss::derive_params(const bssmppi_params* p, DevParams& d, int& P, std::string& why)
{
    int rc = validate(p, why);
    if (rc != BSSMPPI_OK) return rc;
    const int nx = p->model == BSSMPPI_MODEL_BICYCLE6 ? 6 : (p->model == BSSMPPI_MODEL_WHEELS8 ? 8 : 4);
    double Lw[64], Le[4];
    if (!cholesky_psd(nx, p->Sigma_w, Lw)) {
        why = "Sigma_w must be symmetric positive semidefinite";
        return BSSMPPI_EINVAL;
    }
    if (!cholesky_psd(2, p->Sigma_eps, Le)) {
        why = "Sigma_eps must be symmetric positive definite";
        return BSSMPPI_EINVAL;
    }
    // Mapping of particles to lanes: a segment of seg lanes (a power of two) per sample, P particles
    // per lane (lane l holds particles l, l + seg, ...). From 8 to 32 particles, two per lane in half
    // as many lanes when that still gives about 12 warps per SM (K M / 64 warps: about 1,800 on 152
    // SMs): the pairs run packed and the per-step merge and cost work is shared by two particles, but
    // fewer warps hide less latency (at 3-7 warps per SM it was 40 % slower). Otherwise seg is the
    // next power of two >= M up to a warp, and P covers the rest.
    int seg = 1;
    int seg2 = 1;
    while (2 * seg2 < p->M) seg2 <<= 1;
    const long warps2 = ((long)p->K * seg2 + 31) / 32;  // sample groups of 32 / seg2 samples
    if (p->M >= 8 && p->M <= 32 && warps2 >= 12L * device_sms()) {
        seg = seg2;
        P = 2;
    } else {
        while (seg < p->M && seg < 32) seg <<= 1;
        const int ppl = (p->M + seg - 1) / seg;
        P = 1;
        while (P < ppl) P <<= 1;
    }
    d.K = p->K; d.M = p->M; d.T = p->T; d.nx = nx;
    d.seg = seg; d.spw = 32 / seg;
    d.dist_half = seg * P / 2;  // = 2^ceil(log2 M) / 2 for every M (seg P is the next power of two)
    d.uniform = (p->M == seg * P) ? 1 : 0;
    d.n_sub = p->model == BSSMPPI_MODEL_DOUBLE_INT4 ? 1 : p->n_sub;
    d.ey = p->ey_index; d.crn = p->crn_disturbance ? 1 : 0; d.record = p->record_moments ? 1 : 0;
    d.resample = p->resample ? 1 : 0;
    if (p->backoff != BSSMPPI_BACKOFF_GAUSSIAN && p->backoff != BSSMPPI_BACKOFF_CANTELLI) {
        why = "backoff must be 0 (Gaussian) or 1 (Cantelli)";
        return BSSMPPI_EINVAL;
    }
    if (p->clamp_margin != 0 && p->clamp_margin != 1) {
        why = "clamp_margin must be 0 or 1";
        return BSSMPPI_EINVAL;
    }
    d.k_off = 0;
    d.K_norm = p->K;
    d.key0 = (uint32_t)(p->seed & 0xffffffffu); d.key1 = (uint32_t)(p->seed >> 32);
    for (int r = 0; r < 10; ++r) {  // Philox key schedule: k + r (0x9E3779B9, 0xBB67AE85)
        d.rk0[r] = d.key0 + (uint32_t)r * 0x9E3779B9u;
        d.rk1[r] = d.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    d.dt = p->dt; d.h = p->dt / (float)d.n_sub;
    d.inv_m = 1.0f / p->mass; d.inv_Iz = 1.0f / p->Iz; d.lf = p->lf; d.lr = p->lr;
    d.tB = p->tire_B; d.tC = p->tire_C;
    d.Df = (float)((double)p->mu * p->mass * p->g * p->lr / ((double)p->lf + p->lr));
    d.Dr = (float)((double)p->mu * p->mass * p->g * p->lf / ((double)p->lf + p->lr));
    d.vx_floor = p->vx_floor;
    if (p->model == BSSMPPI_MODEL_WHEELS8) {
        const double L = (double)p->lf + p->lr;
        d.Dxf = (float)((double)p->mu_x * p->mass * p->g * p->lr / L);
        d.Dxr = (float)((double)p->mu_x * p->mass * p->g * p->lf / L);
        d.Rw = p->wheel_radius;
        d.inv_Iw = 1.0f / p->wheel_inertia;
        d.tau_max = p->tau_max;
        d.slip_floor = p->slip_floor;
    }
    d.umin0 = p->u_min[0]; d.umin1 = p->u_min[1]; d.umax0 = p->u_max[0]; d.umax1 = p->u_max[1];
    d.Le00 = (float)Le[0]; d.Le10 = (float)Le[2]; d.Le11 = (float)Le[3];
    const double* Se = p->Sigma_eps;
    const double det = Se[0] * Se[3] - Se[1] * Se[2];
    d.Si00 = (float)(Se[3] / det); d.Si01 = (float)(-Se[1] / det);
    d.Si10 = (float)(-Se[2] / det); d.Si11 = (float)(Se[0] / det);
    for (int i = 0; i < 36; ++i) d.Lw[i] = 0.0f;
    d.lw_diag = 1;
    for (int i = 0; i < nx; ++i)
        for (int j = 0; j <= i; ++j) {
            d.Lw[i * (i + 1) / 2 + j] = (float)Lw[i * nx + j];
            if (j < i && d.Lw[i * (i + 1) / 2 + j] != 0.0f) d.lw_diag = 0;
        }
    d.lambda = p->lambda;
    d.inv_lambda = 1.0f / p->lambda;
    d.nu = p->backoff == BSSMPPI_BACKOFF_CANTELLI
             ? (float)std::sqrt((1.0 - (double)p->delta) / (double)p->delta)
             : (float)(std::sqrt(2.0) * inverse_erf(1.0 - 2.0 * (double)p->delta));
    d.clamp_margin = p->clamp_margin ? 1 : 0;
    d.one_m_gamma = 1.0f - p->gamma;
    d.ctrl_w = p->ctrl_w; d.Csafe = p->C_safe; d.Cobs = p->C_obs; d.wT = p->w_T;
    d.mean_mask = 0;
    for (int i = 0; i < 8; ++i) {
        d.xg[i] = p->x_goal[i];
        d.Q[i] = i < nx ? p->Q[i] : 0.0f;
        d.Qf[i] = i < nx ? p->Qf[i] : 0.0f;
        if (i < nx && (d.Q[i] != 0.0f || d.Qf[i] != 0.0f || i == p->ey_index || p->record_moments)) d.mean_mask |= 1 << i;
    }
    const bool track = p->model != BSSMPPI_MODEL_DOUBLE_INT4;
    const int ntab = track ? p->n_track : 2;
    d.n_track_mask = ntab - 1;
    d.track_scale = track ? (float)((double)ntab / p->track_len) : 0.0f;
    d.Mf = (float)p->M; d.invM = 1.0f / (float)p->M; d.invM1 = 1.0f / (float)(p->M - 1);
    d.Df_m = (float)((double)d.Df / p->mass);
    d.lfDf_Iz = (float)((double)p->lf * d.Df / p->Iz);
    d.fold[kFoldH] = d.h; d.fold[kFoldNH] = -d.h; d.fold[kFoldLf] = d.lf; d.fold[kFoldNLr] = -d.lr;
    d.fold[kFoldTB] = d.tB; d.fold[kFoldNTB] = -d.tB; d.fold[kFoldTC] = d.tC;
    d.fold[kFoldNDrM] = (float)(-(double)d.Dr / p->mass);
    d.fold[kFoldNLrDrIz] = (float)(-(double)p->lr * d.Dr / p->Iz);
    if (p->model == BSSMPPI_MODEL_WHEELS8) {
        d.fold[kFoldWRw] = d.Rw;
        d.fold[kFoldWDxf] = d.Dxf;
        d.fold[kFoldWDf] = d.Df;
        d.fold[kFoldWInvM] = d.inv_m;
        d.fold[kFoldWNInvM] = -d.inv_m;
        d.fold[kFoldWDxrM] = (float)((double)d.Dxr / p->mass);
        d.fold[kFoldWDrM] = (float)((double)d.Dr / p->mass);
        d.fold[kFoldWLfIz] = (float)((double)p->lf / p->Iz);
        d.fold[kFoldWLrDrIz] = (float)((double)p->lr * d.Dr / p->Iz);
        d.fold[kFoldWNhRwIw] = (float)(-(double)d.h * p->wheel_radius / p->wheel_inertia);
        d.fold[kFoldWNRwDxrIw] = (float)(-(double)p->wheel_radius * d.Dxr / p->wheel_inertia);
    }
    d.fold[kFoldTB2] = (float)((double)p->tire_B * p->tire_B);
    float tyre[kTyreDeg + 1];
    tyre_curve_fit(p->tire_C, tyre);
    for (int i = 0; i <= kTyreDeg; ++i) d.fold[kFoldTy0 + i] = tyre[i];
    rear_tyre_fit(p->tire_B, p->tire_C, tyre);
    for (int i = 0; i <= kTyreDeg; ++i) d.fold[kFoldRy0 + i] = tyre[i];
    d.fold[kFoldRInv] = (float)(1.0 / rear_tyre_tau(p->tire_B));
    for (int i = kFoldOne; i < kFoldN; ++i) d.fold[i] = fold_fixed(i);
    for (int i = 0; i < kFoldN; ++i) d.fold2[i] = make_float2(d.fold[i], d.fold[i]);
    return BSSMPPI_OK;
}

extern "C" {

uint32_t bssmppi_abi_version(void) { return BSSMPPI_ABI_VERSION; }
size_t bssmppi_params_size(void) { return sizeof(bssmppi_params); }

const char* bssmppi_last_error(bssmppi_t h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int bssmppi_create(const bssmppi_params* p, void* cuda_stream, bssmppi_t* out)
{
    if (!out) return fail(nullptr, BSSMPPI_EINVAL, "out is NULL");
    *out = nullptr;
    std::string why;
    bss::DevParams dp{};
    int P = 1;
    int rc = bss::derive_params(p, dp, P, why);
    if (rc != BSSMPPI_OK) return fail(nullptr, rc, why);
    const int nx = dp.nx;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(nullptr, BSSMPPI_ECUDA, std::string("no usable CUDA device: ") + cudaGetErrorString(e));

    auto* h = new bssmppi_ctx();
    h->prm = *p;
    h->prm.track_kappa = nullptr;
    h->nx = nx;
    h->device = dev;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->P = P;
    h->dp = dp;
    const int ntab = dp.n_track_mask + 1;

    const size_t K = p->K, T = p->T;
    rc = BSSMPPI_OK;
    if (rc == BSSMPPI_OK) rc = alloc(h, &h->d_kappa, ntab + 1);
    if (rc == BSSMPPI_OK) rc = alloc(h, &h->d_S, K);
    if (rc == BSSMPPI_OK) rc = alloc(h, &h->d_w, K);
    if (rc == BSSMPPI_OK) rc = alloc(h, &h->d_eps, K * T * 2);
    if (rc == BSSMPPI_OK && p->record_moments) rc = alloc(h, &h->d_mean, K * (T + 1) * nx);
    if (rc == BSSMPPI_OK && p->record_moments) rc = alloc(h, &h->d_var, K * (T + 1) * nx);
    // the resident nominal and u0 side by side, so a host solve reads both back with one copy
    if (rc == BSSMPPI_OK) rc = alloc(h, &h->d_v, T * 2 + 2);
    if (rc == BSSMPPI_OK) h->d_u0 = h->d_v + 2 * T;
    if (rc == BSSMPPI_OK) rc = alloc(h, &h->d_in, 8 + 2 * T + 64);
    if (rc == BSSMPPI_OK) {
        h->d_x0 = h->d_in;
        h->d_Sigma0 = h->d_in + 8 + 2 * T;
    }
    if (rc == BSSMPPI_OK) rc = alloc(h, &h->d_diag, BSSMPPI_NDIAG);
    if (rc == BSSMPPI_OK) rc = alloc(h, &h->d_ctr, 1);
    if (rc == BSSMPPI_OK) rc = alloc(h, &h->d_ticket, 1);
    if (rc == BSSMPPI_OK) rc = alloc(h, &h->d_tail_part, (size_t)bss::kTailMaxBlocks * (3 + 2 * T));
    const bool repairable = p->M <= 256 && p->model != BSSMPPI_MODEL_WHEELS8;  // the repair has no 8-state adjoint
    if (rc == BSSMPPI_OK && repairable) rc = alloc(h, &h->d_repair_X, bss::repair_scratch_floats(h->dp));
    if (rc == BSSMPPI_OK) rc = alloc(h, &h->d_repair_J, 1);
    if (rc == BSSMPPI_OK) {
        e = cudaMallocHost(reinterpret_cast<void**>(&h->h_stage), sizeof(float) * (8 + 2 * T + 64 + 2 * T + 2));
        if (e != cudaSuccess) {
            h->h_stage = nullptr;
            rc = fail(h, BSSMPPI_ENOMEM, std::string("cudaMallocHost: ") + cudaGetErrorString(e));
        }
    }
    if (rc == BSSMPPI_OK) {
        std::string step;
        e = cudaSuccess;
        if (p->model != BSSMPPI_MODEL_DOUBLE_INT4) {  // the track models read the curvature table
            float* tab = new float[ntab + 1];
            std::memcpy(tab, p->track_kappa, sizeof(float) * ntab);
            tab[ntab] = tab[0];
            e = cudaMemcpy(h->d_kappa, tab, sizeof(float) * (ntab + 1), cudaMemcpyHostToDevice);
            delete[] tab;
        } else {
            e = cudaMemset(h->d_kappa, 0, sizeof(float) * (ntab + 1));
        }
        if (e == cudaSuccess) e = cudaMemset(h->d_v, 0, sizeof(float) * T * 2);
        if (e == cudaSuccess) e = cudaMemset(h->d_ctr, 0, sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMemset(h->d_ticket, 0, sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMemset(h->d_diag, 0, sizeof(float) * BSSMPPI_NDIAG);
        if (e == cudaSuccess) e = bss::rollout_prepare(h->dp, h->P, p->compensated != 0, h->dp.resample != 0, h->roll);
        if (e == cudaSuccess && repairable) e = bss::repair_prepare(h->dp);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = cuda_fail(h, e, "create");
    }
    h->dp.kappa = h->d_kappa;
    if (rc != BSSMPPI_OK) {
        g_create_error = h->err;
        release(h);
        delete h;
        return rc;
    }
    *out = h;
    return BSSMPPI_OK;
}

namespace {

// One solve launch: the rollout reads the nominal from v_in; the tail writes v+ to the resident
// nominal and the first control to u0.
int launch_solve(bssmppi_t h, const float* d_x0, const float* d_Sigma0, const float* v_in, float* u0, int shift_n = 0,
                 cudaStream_t st = nullptr, bool timed = true)
{
    if (!st) st = h->stream;
    cudaEvent_t* ev = (timed && h->ev_count < h->ev_cap) ? h->ev + 2 * h->ev_count : nullptr;
    if (ev) BSS_CUDA(h, cudaEventRecord(ev[0], st));
    // One launch: rollout, costs, and (in its tail) weights, update, u0, diagnostics, counter.
    bss::TailIO tail{h->d_tail_part, h->d_ticket, h->d_w, u0, h->d_diag, h->d_ctr, h->d_v, nullptr, shift_n};
    BSS_CUDA(h, bss::rollout_launch(h->dp, h->P, h->prm.compensated != 0, h->roll, d_x0, d_Sigma0, v_in, h->d_ctr,
                                    h->d_S, h->d_eps, h->d_mean, h->d_var, tail, h->cons, st));
    if (ev) {
        BSS_CUDA(h, cudaEventRecord(ev[1], st));
        ++h->ev_count;
    }
    return BSSMPPI_OK;
}

void drop_host_graphs(bssmppi_t h)
{
    for (cudaGraphExec_t& g : h->host_graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

// Records the host-buffer solve's three operations (H2D of n_in staged floats, the solve, D2H of
// v+ | u0 when `out`) on the private capture stream and instantiates them as one graph.
int capture_host_graph(bssmppi_t h, size_t n_in, bool with_v, bool with_S0, bool out, cudaGraphExec_t* ex)
{
    if (!h->cap_stream) BSS_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    cudaStream_t cs = h->cap_stream;
    const int T = h->prm.T;
    float* sout = h->h_stage + 8 + 2 * T + 64;
    BSS_CUDA(h, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemcpyAsync(h->d_in, h->h_stage, sizeof(float) * n_in, cudaMemcpyHostToDevice, cs);
    int rc = BSSMPPI_OK;
    if (e == cudaSuccess)
        rc = launch_solve(h, h->d_x0, with_S0 ? h->d_Sigma0 : nullptr, with_v ? h->d_in + 8 : h->d_v, h->d_u0, 0, cs,
                          false);
    if (e == cudaSuccess && rc == BSSMPPI_OK && out)
        e = cudaMemcpyAsync(sout, h->d_v, sizeof(float) * (2 * T + 2), cudaMemcpyDeviceToHost, cs);
    cudaGraph_t g = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(cs, &g);  // always ends the capture
    if (rc != BSSMPPI_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e == cudaSuccess) e = e_end;
    if (e == cudaSuccess) e = cudaGraphInstantiate(ex, g, 0);
    if (g) cudaGraphDestroy(g);
    return e == cudaSuccess ? BSSMPPI_OK : cuda_fail(h, e, "host-buffer solve graph");
}

}  // namespace

int bssmppi_solve(bssmppi_t h, const float* d_x0, const float* d_Sigma0, float* d_v, float* d_u0)
{
    if (!h) return fail(nullptr, BSSMPPI_EINVAL, "handle is NULL");
    if (!d_x0) return fail(h, BSSMPPI_EINVAL, "x0 is NULL");
    const size_t vbytes = sizeof(float) * 2 * h->prm.T;
    if (d_v) BSS_CUDA(h, cudaMemcpyAsync(h->d_v, d_v, vbytes, cudaMemcpyDeviceToDevice, h->stream));
    const int rc = launch_solve(h, d_x0, d_Sigma0, h->d_v, d_u0 ? d_u0 : h->d_u0);
    if (rc != BSSMPPI_OK) return rc;
    if (d_v) BSS_CUDA(h, cudaMemcpyAsync(d_v, h->d_v, vbytes, cudaMemcpyDeviceToDevice, h->stream));
    return BSSMPPI_OK;
}

int bssmppi_solve_shift(bssmppi_t h, const float* d_x0, const float* d_Sigma0, float* d_u0, int32_t n)
{
    if (!h) return fail(nullptr, BSSMPPI_EINVAL, "handle is NULL");
    if (!d_x0) return fail(h, BSSMPPI_EINVAL, "x0 is NULL");
    if (n < 0 || n > h->prm.T) return fail(h, BSSMPPI_EINVAL, "shift n must be in [0, T]");
    return launch_solve(h, d_x0, d_Sigma0, h->d_v, d_u0 ? d_u0 : h->d_u0, n);
}

int bssmppi_solve_host(bssmppi_t h, const float* h_x0, const float* h_Sigma0, float* h_v, float* h_u0)
{
    if (!h) return fail(nullptr, BSSMPPI_EINVAL, "handle is NULL");
    if (!h_x0) return fail(h, BSSMPPI_EINVAL, "x0 is NULL");
    const int nx = h->nx, T = h->prm.T;
    // inputs in one pinned block, copied with one H2D: x0 (8) | v (2T) | Sigma0 (64)
    float* sx0 = h->h_stage;
    float* sv = sx0 + 8;
    float* sS0 = sv + 2 * T;
    float* sout = sS0 + 64;  // v+ (2T) | u0 (2), read back with one D2H
    std::memcpy(sx0, h_x0, sizeof(float) * nx);
    if (h_v) std::memcpy(sv, h_v, sizeof(float) * 2 * T);
    if (h_Sigma0) std::memcpy(sS0, h_Sigma0, sizeof(float) * nx * nx);
    const size_t n_in = h_Sigma0 ? (size_t)(8 + 2 * T + nx * nx) : (h_v ? (size_t)(8 + 2 * T) : (size_t)nx);
    const bool out = h_v || h_u0;
    if (h->ev_count < h->ev_cap) {  // timing events requested: plain launches, so each solve records its own
        BSS_CUDA(h, cudaMemcpyAsync(h->d_in, sx0, sizeof(float) * n_in, cudaMemcpyHostToDevice, h->stream));
        const int rc = launch_solve(h, h->d_x0, h_Sigma0 ? h->d_Sigma0 : nullptr, h_v ? h->d_in + 8 : h->d_v, h->d_u0);
        if (rc != BSSMPPI_OK) return rc;
        if (out)
            BSS_CUDA(h, cudaMemcpyAsync(sout, h->d_v, sizeof(float) * (2 * T + 2), cudaMemcpyDeviceToHost, h->stream));
    } else {  // one graph launch: the copies and the kernel run back to back without host round trips
        cudaGraphExec_t& ex = h->host_graph[(h_v ? 1 : 0) | (h_Sigma0 ? 2 : 0) | (out ? 4 : 0)];
        if (!ex) {
            const int rc = capture_host_graph(h, n_in, h_v != nullptr, h_Sigma0 != nullptr, out, &ex);
            if (rc != BSSMPPI_OK) return rc;
        }
        BSS_CUDA(h, cudaGraphLaunch(ex, h->stream));
    }
    BSS_CUDA(h, cudaStreamSynchronize(h->stream));
    if (h_v) std::memcpy(h_v, sout, sizeof(float) * 2 * T);
    if (h_u0) std::memcpy(h_u0, sout + 2 * T, sizeof(float) * 2);
    return BSSMPPI_OK;
}

int bssmppi_set_sample_range(bssmppi_t h, int32_t k_begin, int32_t K_total)
{
    if (!h) return fail(nullptr, BSSMPPI_EINVAL, "handle is NULL");
    if (k_begin < 0 || K_total < h->prm.K || K_total > BSSMPPI_K_MAX || k_begin > K_total - h->prm.K)
        return fail(h, BSSMPPI_EINVAL, "need 0 <= k_begin and k_begin + K <= K_total <= BSSMPPI_K_MAX");
    BSS_CUDA(h, cudaStreamSynchronize(h->stream));  // solves in flight keep the old range
    h->dp.k_off = k_begin;
    h->dp.K_norm = K_total;
    drop_host_graphs(h);
    return BSSMPPI_OK;
}

int bssmppi_solve_partial(bssmppi_t h, const float* d_x0, const float* d_Sigma0, const float* d_v, float* d_partial)
{
    if (!h) return fail(nullptr, BSSMPPI_EINVAL, "handle is NULL");
    if (!d_x0 || !d_partial) return fail(h, BSSMPPI_EINVAL, "x0 and partial must be non-NULL");
    const size_t vbytes = sizeof(float) * 2 * h->prm.T;
    if (d_v) BSS_CUDA(h, cudaMemcpyAsync(h->d_v, d_v, vbytes, cudaMemcpyDeviceToDevice, h->stream));
    bss::TailIO tail{h->d_tail_part, h->d_ticket, h->d_w, nullptr, nullptr, h->d_ctr, h->d_v, d_partial, 0};
    BSS_CUDA(h, bss::rollout_launch(h->dp, h->P, h->prm.compensated != 0, h->roll, d_x0, d_Sigma0, h->d_v, h->d_ctr,
                                    h->d_S, h->d_eps, h->d_mean, h->d_var, tail, h->cons, h->stream));
    return BSSMPPI_OK;
}

int bssmppi_merge_partials(bssmppi_t h, const float* d_partials, int32_t G, float* d_v, float* d_u0)
{
    if (!h) return fail(nullptr, BSSMPPI_EINVAL, "handle is NULL");
    if (!d_partials) return fail(h, BSSMPPI_EINVAL, "partials are NULL");
    if (G < 1 || G > bss::kTailMaxBlocks) return fail(h, BSSMPPI_EINVAL, "G must be in [1, 256]");
    bss::TailIO tail{nullptr, nullptr, h->d_w, d_u0 ? d_u0 : h->d_u0, h->d_diag, nullptr, h->d_v, nullptr, 0};
    BSS_CUDA(h, bss::merge_partials_launch(h->dp, G, d_partials, h->prm.compensated != 0, h->d_S, tail, h->stream));
    const size_t vbytes = sizeof(float) * 2 * h->prm.T;
    if (d_v) BSS_CUDA(h, cudaMemcpyAsync(d_v, h->d_v, vbytes, cudaMemcpyDeviceToDevice, h->stream));
    return BSSMPPI_OK;
}

int bssmppi_set_constraints(bssmppi_t h, const bssmppi_constraint* cons, int32_t n)
{
    if (!h) return fail(nullptr, BSSMPPI_EINVAL, "handle is NULL");
    if (n < 0 || n > BSSMPPI_MAX_CONSTRAINTS) return fail(h, BSSMPPI_EINVAL, "constraint count must be in [0, 8]");
    if (n > 0 && !cons) return fail(h, BSSMPPI_EINVAL, "constraints are NULL");
    if (n > 0 && !h->prm.compensated) return fail(h, BSSMPPI_EINVAL, "a constraint set needs compensated = 1");
    bss::ConSet cs{};
    cs.n = n;
    for (int q = 0; q < n; ++q) {
        const bssmppi_constraint& c = cons[q];
        const double pq = c.p;
        if (c.backoff == BSSMPPI_BACKOFF_GAUSSIAN) {
            if (!(pq > 0.0 && pq < 0.5)) return fail(h, BSSMPPI_EINVAL, "Gaussian back-off needs 0 < p < 0.5");
            cs.nu[q] = (float)(std::sqrt(2.0) * inverse_erf(1.0 - 2.0 * pq));
        } else if (c.backoff == BSSMPPI_BACKOFF_CANTELLI) {
            if (!(pq > 0.0 && pq < 1.0)) return fail(h, BSSMPPI_EINVAL, "Cantelli back-off needs 0 < p < 1");
            cs.nu[q] = (float)std::sqrt((1.0 - pq) / pq);
        } else {
            return fail(h, BSSMPPI_EINVAL, "unknown back-off rule");
        }
        if (c.kind == BSSMPPI_CON_HALFSPACE) {
            cs.kind[q] = 0;
            cs.b[q] = c.b;
            for (int l = 0; l < 8; ++l) {
                if (!std::isfinite(c.a[l])) return fail(h, BSSMPPI_EINVAL, "half-space normal must be finite");
                cs.a[q][l] = l < h->nx ? c.a[l] : 0.0f;
            }
            if (!std::isfinite(c.b)) return fail(h, BSSMPPI_EINVAL, "half-space offset must be finite");
        } else if (c.kind == BSSMPPI_CON_DISK) {
            if (c.i < 0 || c.i >= h->nx || c.j < 0 || c.j >= h->nx || c.i == c.j)
                return fail(h, BSSMPPI_EINVAL, "disk states i, j must be distinct states");
            if (!(c.radius > 0.0f) || !std::isfinite(c.radius) || !std::isfinite(c.center[0]) ||
                !std::isfinite(c.center[1]))
                return fail(h, BSSMPPI_EINVAL, "disk radius must be positive and its centre finite");
            cs.kind[q] = 1;
            cs.b[q] = c.radius * c.radius;
            cs.a[q][c.i] = 1.0f;
            cs.a[q][c.j] = 1.0f;
            cs.o[q][c.i] = c.center[0];
            cs.o[q][c.j] = c.center[1];
        } else {
            return fail(h, BSSMPPI_EINVAL, "unknown constraint kind");
        }
    }
    bss::RollLaunch L;
    const bool full = h->dp.resample != 0 || n > 0;
    BSS_CUDA(h, cudaStreamSynchronize(h->stream));  // no solve may still read the old set's launch shape
    BSS_CUDA(h, bss::rollout_prepare(h->dp, h->P, h->prm.compensated != 0, full, L, &cs));
    h->roll = L;
    h->cons = cs;
    drop_host_graphs(h);
    return BSSMPPI_OK;
}

int bssmppi_shift(bssmppi_t h, float* d_v, int32_t n)
{
    if (!h) return fail(nullptr, BSSMPPI_EINVAL, "handle is NULL");
    if (n < 0 || n > h->prm.T) return fail(h, BSSMPPI_EINVAL, "shift n must be in [0, T]");
    if (n == 0) return BSSMPPI_OK;
    BSS_CUDA(h, bss::shift_launch(d_v ? d_v : h->d_v, h->prm.T, n, h->stream));
    return BSSMPPI_OK;
}

int bssmppi_destroy(bssmppi_t h)
{
    if (!h) return BSSMPPI_OK;
    cudaStreamSynchronize(h->stream);
    release(h);
    delete h;
    return BSSMPPI_OK;
}

int bssmppi_timing(bssmppi_t h, int32_t n)
{
    if (!h) return fail(nullptr, BSSMPPI_EINVAL, "handle is NULL");
    if (n < 0 || n > 4096) return fail(h, BSSMPPI_EINVAL, "timing slots must be in [0, 4096]");
    BSS_CUDA(h, cudaStreamSynchronize(h->stream));
    for (int i = 0; i < 2 * h->ev_cap; ++i) cudaEventDestroy(h->ev[i]);
    delete[] h->ev;
    h->ev = nullptr;
    h->ev_cap = 0;
    h->ev_count = 0;
    if (n == 0) return BSSMPPI_OK;
    h->ev = new cudaEvent_t[2 * (size_t)n];
    for (int i = 0; i < 2 * n; ++i) {
        cudaError_t e = cudaEventCreate(&h->ev[i]);
        if (e != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaEventDestroy(h->ev[j]);
            delete[] h->ev;
            h->ev = nullptr;
            return cuda_fail(h, e, "cudaEventCreate");
        }
    }
    h->ev_cap = n;
    return BSSMPPI_OK;
}

int bssmppi_timing_read(bssmppi_t h, float* h_rollout_ms, float* h_update_ms, int32_t max, int32_t* count)
{
    if (!h) return fail(nullptr, BSSMPPI_EINVAL, "handle is NULL");
    const int n = h->ev_count < max ? h->ev_count : (max > 0 ? max : 0);
    for (int i = 0; i < n; ++i) {
        cudaEvent_t* ev = h->ev + 2 * i;
        BSS_CUDA(h, cudaEventSynchronize(ev[1]));
        float a = 0.0f;
        BSS_CUDA(h, cudaEventElapsedTime(&a, ev[0], ev[1]));
        if (h_rollout_ms) h_rollout_ms[i] = a;
        if (h_update_ms) h_update_ms[i] = 0.0f;  // fused into the rollout launch
    }
    if (count) *count = n;
    return BSSMPPI_OK;
}

int bssmppi_repair_grad(bssmppi_t h, const float* d_x0, const float* d_v, float* d_grad, float* d_J)
{
    if (!h) return fail(nullptr, BSSMPPI_EINVAL, "handle is NULL");
    if (!d_x0 || !d_grad) return fail(h, BSSMPPI_EINVAL, "x0 and grad must be non-NULL");
    if (!h->d_repair_X) return fail(h, BSSMPPI_ENOTSUP, "repair needs M <= 256 and the bicycle or linear model");
    if (h->prm.resample) return fail(h, BSSMPPI_ENOTSUP, "repair differentiates persistent particles (resample = 0)");
    if (h->cons.n > 0) return fail(h, BSSMPPI_ENOTSUP, "repair differentiates the racing barrier (no constraint set)");
    const float* v = d_v ? d_v : h->d_v;
    BSS_CUDA(h, bss::repair_launch(h->dp, d_x0, const_cast<float*>(v), h->d_ctr, h->d_repair_X, d_grad,
                                   d_J ? d_J : h->d_repair_J, 0, 0.0f, h->stream));
    return BSSMPPI_OK;
}

int bssmppi_repair(bssmppi_t h, const float* d_x0, float* d_v, int32_t iters, float step, float* d_J)
{
    if (!h) return fail(nullptr, BSSMPPI_EINVAL, "handle is NULL");
    if (!d_x0) return fail(h, BSSMPPI_EINVAL, "x0 is NULL");
    if (iters < 1 || iters > 1000) return fail(h, BSSMPPI_EINVAL, "iters must be in [1, 1000]");
    if (!(step >= 0.0f) || !std::isfinite(step)) return fail(h, BSSMPPI_EINVAL, "step must be finite and >= 0");
    if (!h->d_repair_X) return fail(h, BSSMPPI_ENOTSUP, "repair needs M <= 256 and the bicycle or linear model");
    if (h->prm.resample) return fail(h, BSSMPPI_ENOTSUP, "repair differentiates persistent particles (resample = 0)");
    if (h->cons.n > 0) return fail(h, BSSMPPI_ENOTSUP, "repair differentiates the racing barrier (no constraint set)");
    BSS_CUDA(h, bss::repair_launch(h->dp, d_x0, d_v ? d_v : h->d_v, h->d_ctr, h->d_repair_X, nullptr, d_J, iters,
                                   step, h->stream));
    return BSSMPPI_OK;
}

int bssmppi_set_counter(bssmppi_t h, uint32_t counter)
{
    if (!h) return fail(nullptr, BSSMPPI_EINVAL, "handle is NULL");
    uint32_t* stage = reinterpret_cast<uint32_t*>(h->h_stage);
    BSS_CUDA(h, cudaStreamSynchronize(h->stream));
    stage[0] = counter;
    BSS_CUDA(h, cudaMemcpyAsync(h->d_ctr, stage, sizeof(uint32_t), cudaMemcpyHostToDevice, h->stream));
    BSS_CUDA(h, cudaStreamSynchronize(h->stream));
    return BSSMPPI_OK;
}

int bssmppi_get_counter(bssmppi_t h, uint32_t* counter)
{
    if (!h) return fail(nullptr, BSSMPPI_EINVAL, "handle is NULL");
    if (!counter) return fail(h, BSSMPPI_EINVAL, "counter is NULL");
    BSS_CUDA(h, cudaMemcpyAsync(counter, h->d_ctr, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream));
    BSS_CUDA(h, cudaStreamSynchronize(h->stream));
    return BSSMPPI_OK;
}

int bssmppi_set_nominal(bssmppi_t h, const float* d_v)
{
    if (!h) return fail(nullptr, BSSMPPI_EINVAL, "handle is NULL");
    if (!d_v) return fail(h, BSSMPPI_EINVAL, "v is NULL");
    BSS_CUDA(h, cudaMemcpyAsync(h->d_v, d_v, sizeof(float) * 2 * h->prm.T, cudaMemcpyDeviceToDevice, h->stream));
    return BSSMPPI_OK;
}

int bssmppi_read(bssmppi_t h, int32_t which, void* d_dst, size_t bytes)
{
    if (!h) return fail(nullptr, BSSMPPI_EINVAL, "handle is NULL");
    if (!d_dst) return fail(h, BSSMPPI_EINVAL, "destination is NULL");
    const size_t K = h->prm.K, T = h->prm.T, nx = h->nx;
    const void* src = nullptr;
    size_t need = 0;
    switch (which) {
    case BSSMPPI_BUF_S: src = h->d_S; need = K; break;
    case BSSMPPI_BUF_W: src = h->d_w; need = K; break;
    case BSSMPPI_BUF_EPS: src = h->d_eps; need = K * T * 2; break;
    case BSSMPPI_BUF_MEAN: src = h->d_mean; need = K * (T + 1) * nx; break;
    case BSSMPPI_BUF_VAR: src = h->d_var; need = K * (T + 1) * nx; break;
    case BSSMPPI_BUF_DIAG: src = h->d_diag; need = BSSMPPI_NDIAG; break;
    case BSSMPPI_BUF_V: src = h->d_v; need = T * 2; break;
    default: return fail(h, BSSMPPI_EINVAL, "unknown buffer");
    }
    if (!src) return fail(h, BSSMPPI_ENOTSUP, "buffer not kept (record_moments = 0)");
    need *= sizeof(float);
    if (bytes < need) return fail(h, BSSMPPI_EINVAL, "destination too small");
    BSS_CUDA(h, cudaMemcpyAsync(d_dst, src, need, cudaMemcpyDeviceToDevice, h->stream));
    return BSSMPPI_OK;
}

int bssmppi_model_step(bssmppi_t h, const float* d_x, const float* d_u, const float* d_w, float* d_x_next, int64_t n)
{
    if (!h) return fail(nullptr, BSSMPPI_EINVAL, "handle is NULL");
    if (n < 0 || (n > 0 && (!d_x || !d_u || !d_x_next))) return fail(h, BSSMPPI_EINVAL, "bad arrays");
    BSS_CUDA(h, bss::model_step_launch(h->dp, d_x, d_u, d_w, d_x_next, n, h->stream));
    return BSSMPPI_OK;
}

int bssmppi_philox4x32_10(const uint32_t* d_ctr, uint64_t seed, uint32_t* d_out, int64_t n, void* cuda_stream)
{
    if (n < 0 || (n > 0 && (!d_ctr || !d_out))) return fail(nullptr, BSSMPPI_EINVAL, "bad arrays");
    if ((reinterpret_cast<uintptr_t>(d_ctr) | reinterpret_cast<uintptr_t>(d_out)) & 15u)
        return fail(nullptr, BSSMPPI_EINVAL, "arrays must be 16-byte aligned");
    cudaError_t e = bss::philox_launch(d_ctr, seed, d_out, n, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? BSSMPPI_OK : cuda_fail(nullptr, e, "philox");
}

int bssmppi_box_muller(const uint32_t* d_words, float* d_z, int64_t n, void* cuda_stream)
{
    if (n < 0 || (n > 0 && (!d_words || !d_z))) return fail(nullptr, BSSMPPI_EINVAL, "bad arrays");
    if ((reinterpret_cast<uintptr_t>(d_words) | reinterpret_cast<uintptr_t>(d_z)) & 7u)
        return fail(nullptr, BSSMPPI_EINVAL, "arrays must be 8-byte aligned");
    cudaError_t e = bss::box_muller_launch(d_words, d_z, n, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? BSSMPPI_OK : cuda_fail(nullptr, e, "box_muller");
}

int bssmppi_slip_atan(const float* d_t, float* d_y, int64_t n, void* cuda_stream)
{
    if (n < 0 || (n > 0 && (!d_t || !d_y))) return fail(nullptr, BSSMPPI_EINVAL, "bad arrays");
    cudaError_t e = bss::slip_atan_launch(d_t, d_y, n, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? BSSMPPI_OK : cuda_fail(nullptr, e, "slip_atan");
}

int bssmppi_tyre_curve(bssmppi_t h, const float* d_x, float* d_y, int64_t n, void* cuda_stream)
{
    if (!h) return fail(nullptr, BSSMPPI_EINVAL, "NULL handle");
    if (n < 0 || (n > 0 && (!d_x || !d_y))) return fail(h, BSSMPPI_EINVAL, "tyre_curve: bad arguments");
    cudaError_t e = bss::tyre_curve_launch(h->dp, d_x, d_y, n, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? BSSMPPI_OK : cuda_fail(h, e, "tyre_curve");
}

int bssmppi_rear_tyre(bssmppi_t h, const float* d_t, float* d_y, int64_t n, void* cuda_stream)
{
    if (!h) return fail(nullptr, BSSMPPI_EINVAL, "NULL handle");
    if (n < 0 || (n > 0 && (!d_t || !d_y))) return fail(h, BSSMPPI_EINVAL, "rear_tyre: bad arguments");
    cudaError_t e = bss::rear_tyre_launch(h->dp, d_t, d_y, n, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? BSSMPPI_OK : cuda_fail(h, e, "rear_tyre");
}

int bssmppi_rear_tyre_coefficients(double B, double C, float* h_c, int32_t n, double* h_tau)
{
    if (!h_c || !h_tau || n < bss::kTyreDeg + 1 || !(B > 0.0) || !(C > 0.0) || !std::isfinite(B) || !std::isfinite(C))
        return fail(nullptr, BSSMPPI_EINVAL, "rear_tyre_coefficients: needs B, C > 0 and room for 10 coefficients");
    float c[bss::kTyreDeg + 1];
    bss::rear_tyre_fit(B, C, c);
    for (int i = 0; i <= bss::kTyreDeg; ++i) h_c[i] = c[i];
    *h_tau = bss::rear_tyre_tau(B);
    return BSSMPPI_OK;
}

int bssmppi_tyre_curve_coefficients(double C, float* h_c, int32_t n)
{
    if (!h_c || n < bss::kTyreDeg + 1 || !(C > 0.0) || !std::isfinite(C))
        return fail(nullptr, BSSMPPI_EINVAL, "tyre_curve_coefficients: needs C > 0 and room for 10 coefficients");
    float c[bss::kTyreDeg + 1];
    bss::tyre_curve_fit(C, c);
    for (int i = 0; i <= bss::kTyreDeg; ++i) h_c[i] = c[i];
    return BSSMPPI_OK;
}

}  // extern "C"
