// Device building blocks of the BSS-MPPI hot path (sm_103a): the counter-based random numbers,
// the vehicle model, and the particle-moment merges. FP32 throughout; no FP64 on the device.
#pragma once

#include <type_traits>

#include <cstdint>
#include <cuda_runtime.h>

namespace bss {

constexpr int kWarp = 32;
constexpr int kNxMax = 8;
// States of each model (0: bicycle, 1: double integrator, 2: wheel speeds) and the index of the
// path coordinate s (-1: none).
__host__ __device__ constexpr int model_nx(int model) { return model == 0 ? 6 : (model == 2 ? 8 : 4); }
__host__ __device__ constexpr int model_s_index(int model) { return model == 0 ? 5 : (model == 2 ? 7 : -1); }

// Sets of states as bit masks (bit i: state i). A rollout compiled for a fixed set of cost-weighted
// states (the racing cost weights v_x, e_psi and e_y of the bicycle) merges and costs only those
// belief means; mask 0 stands for a set known at run time only.
constexpr int kRacingCostMask = (1 << 0) | (1 << 3) | (1 << 4);
// A general constraint set on the road plane touches e_y and s only; with the racing cost, the
// full-belief rollout then keeps the means of v_x, e_psi, e_y and s and the covariance of (e_y, s).
constexpr int kPlaneConMask = (1 << 4) | (1 << 5);
constexpr int kPlaneMeanMask = kRacingCostMask | kPlaneConMask;
__host__ __device__ constexpr int mask_count(int m)
{
    int n = 0;
    for (int i = 0; i < 32; ++i) n += (m >> i) & 1;
    return n;
}
__host__ __device__ constexpr int mask_nth(int m, int j)  // index of the j-th set bit of m (-1: none)
{
    for (int i = 0; i < 32; ++i)
        if ((m >> i) & 1) {
            if (j == 0) return i;
            --j;
        }
    return -1;
}

// Everything a solve's kernels need, derived on the host at create time and passed by value
// (kernel parameter space), so several controllers can run concurrently without global state.
// Constant operands of the bicycle substep: the model's h, -h, l_f, -l_r, B, -B, C, -D_r / m,
// -l_r D_r / I_z, then fixed numbers: 1, -1, the heading-rotation series' 1/24, -1/2, 1/120,
// -1/6, the slip-angle arctangent's coefficients (slip_atan below), highest degree first, and the
// heading series' 1/9!, -1/7!, -1/10!, 1/8! and -1/6! (sincos_series).
// The wheel-speed model adds R_w, D_xf = mu_x F_zf, D_f, 1/m, -1/m, D_xr / m, D_r / m, l_f / I_z,
// l_r D_r / I_z, -h R_w / I_w and -R_w D_xr / I_w (kFoldW*). B^2 and the coefficients c_0..c_9 of
// the tyre curve's polynomial (tyre_curve below) follow, then 1 / tau and the coefficients of the
// rear tyre's polynomial (rear_tyre below).
constexpr int kTyreDeg = 9;  // degree in x^2 of the tyre curve's polynomial
enum : int {
    kFoldH, kFoldNH, kFoldLf, kFoldNLr, kFoldTB, kFoldNTB, kFoldTC, kFoldNDrM, kFoldNLrDrIz,
    kFoldWRw, kFoldWDxf, kFoldWDf, kFoldWInvM, kFoldWNInvM, kFoldWDxrM, kFoldWDrM, kFoldWLfIz, kFoldWLrDrIz,
    kFoldWNhRwIw, kFoldWNRwDxrIw, kFoldTB2, kFoldTy0, kFoldTyLast = kFoldTy0 + kTyreDeg,
    kFoldRInv, kFoldRy0, kFoldRyLast = kFoldRy0 + kTyreDeg,
    kFoldOne, kFoldM1, kFoldC24, kFoldMHalf, kFoldC120, kFoldM6, kFoldSa0, kFoldSaLast = kFoldSa0 + 4,
    kFoldS9, kFoldS7, kFoldC10, kFoldC8, kFoldC6, kFoldN
};

// Coefficients of the slip-angle arctangent's polynomial p (slip_atan), highest degree first.
__host__ __device__ constexpr float slip_atan_coef(int i)
{
    return i == 0 ? -5.1325989538e-2f : i == 1 ? 1.0160016107e-1f : i == 2 ? -1.4175010834e-1f
         : i == 3 ? 1.9994226694e-1f : -3.3333234306e-1f;
}

// The fixed numbers among them (i >= kFoldOne).
__host__ __device__ constexpr float fold_fixed(int i)
{
    return i == kFoldOne ? 1.0f : i == kFoldM1 ? -1.0f : i == kFoldC24 ? 4.1666667e-2f : i == kFoldMHalf ? -0.5f
         : i == kFoldC120 ? 8.3333333e-3f : i == kFoldM6 ? -1.6666667e-1f
         : (i >= kFoldSa0 && i <= kFoldSaLast) ? slip_atan_coef(i - kFoldSa0)
         : i == kFoldS9 ? 2.7557319e-6f : i == kFoldS7 ? -1.9841270e-4f : i == kFoldC10 ? -2.7557319e-7f
         : i == kFoldC8 ? 2.4801587e-5f : i == kFoldC6 ? -1.3888889e-3f : 0.0f;
}

struct DevParams {
    int K, M, T, n_sub, nx;
    int seg;          // lanes per control sample (power of two <= 32)
    int spw;          // control samples per warp (32 / seg)
    int uniform;      // 1: every lane of a segment holds exactly P valid particles
    int ey, crn, record, n_track_mask;
    int mean_mask;    // bit i: the cost needs the belief mean of state i (always all when recording)
    int resample;     // 1: particles re-drawn from N(mean, cov) before every step k >= 1 (Algorithm 2 literal)
    int k_off;        // global index of the handle's first sample (a shard of a larger K); 0 otherwise
    int K_norm;       // samples of the whole (possibly sharded) solve: K unless sharded
    int lw_diag;      // 1: Sigma_w is diagonal, so its Cholesky factor is (the disturbance needs nx products)
    int dist_half;    // H = 2^ceil(log2 M) / 2: particles n and n + H share a disturbance counter (6 states)
    int clamp_margin; // 1: the racing barrier's margin w_T - nu sigma is clamped at 0
    uint32_t key0, key1;
    uint32_t rk0[10], rk1[10];       // Philox round keys k + r W (the key schedule, precomputed)
    float dt, h, inv_m, inv_Iz, lf, lr, tB, tC, Df, Dr, vx_floor;
    float umin0, umin1, umax0, umax1;
    float Le00, Le10, Le11;          // Cholesky factor of Sigma_eps
    float Si00, Si01, Si10, Si11;    // Sigma_eps^-1
    float Lw[36];                    // Cholesky factor of Sigma_w, packed lower triangle by rows
    float lambda, inv_lambda, nu, one_m_gamma, ctrl_w, Csafe, Cobs, wT;
    float xg[8], Q[8], Qf[8];
    // wheel-speed model: mu_x F_z per axle, wheel radius, 1 / wheel inertia, full-throttle drive
    // torque, slip-denominator speed floor
    float Dxf, Dxr, Rw, inv_Iw, tau_max, slip_floor;
    float track_scale;               // n_track / track_len
    float Mf, invM, invM1;           // M, 1/M, 1/(M-1)
    float Df_m, lfDf_Iz;             // D_f / m and l_f D_f / I_z (per-step force factors)
    // Constant operands of the bicycle substep (kFold* indices), alone and as (v, v) pairs for the
    // packed two-particle form.
    float fold[kFoldN];
    float2 fold2[kFoldN];
    const float* kappa;              // device curvature table, n_track + 1 entries (last = first)
};

// ---------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC'11): ten rounds of the 4x32 S-box (two 32x32->64 multiplies by 0xD2511F53 and 0xCD9E8D57,
// xors with the other words and the round key), the key advanced by the Weyl increments
// 0x9E3779B9 and 0xBB67AE85 between rounds. Kept entirely in registers.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// The same ten rounds with the key schedule taken from precomputed round keys (kernel parameters),
// which saves the two key additions of every round. Each 32x32 -> 64-bit product is written as one
// widening multiply, so its high and low halves come from a single instruction.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t* rk0, const uint32_t* rk1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
        c = make_uint4(hi1 ^ c.y ^ rk0[round], lo1, hi0 ^ c.w ^ rk1[round], lo0);
    }
    return c;
}

// Counter layout of the solve's streams: word 0 = step | (call << 16), word 1 = particle,
// word 2 = sample, word 3 = (stream << 28) | (solve counter & 0x0fffffff).
enum : uint32_t { kStreamControl = 0u, kStreamDisturbance = 1u, kStreamInitial = 3u, kStreamResample = 4u };

// PP: any parameter object with the Philox round keys rk0, rk1 (DevParams, or a serving item).
template <typename PP>
__device__ __forceinline__ uint4 draw_words(const PP& P, uint32_t step, uint32_t call, uint32_t particle,
                                            uint32_t sample, uint32_t stream, uint32_t ctr)
{
    return philox4x32_10_rk(make_uint4(step | (call << 16), particle, sample, (stream << 28) | (ctr & 0x0fffffffu)),
                            P.rk0, P.rk1);
}

// Box-Muller from two 32-bit words: u1 in (0, 1], u2 in [0, 1) from their top 24 bits (exact in
// FP32), z = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2). The angle is taken centred,
// theta = 2 pi (u2 - 1/2) in [-pi, pi) (u2 - 1/2 is exact), where the hardware sine and cosine are
// accurate to 2^-21.4 absolute; (cos, sin)(2 pi u2) = -(cos, sin)(theta). The radius is taken as
// t rsqrt(t), t = -2 ln u1, within a few ulp of the square root (t = 0 at u1 = 1 gives 0); the
// smallest positive t is about 2^-23, far from the subnormal range.
__device__ __forceinline__ float2 box_muller(uint32_t a, uint32_t b)
{
    const float two_m24 = 5.9604644775390625e-08f;
    const float u1 = (float)((a >> 8) + 1u) * two_m24;
    const float theta = 6.28318530717958647692f * ((float)(b >> 8) * two_m24 - 0.5f);
    const float t = -2.0f * logf(u1);
    const float rad = t > 0.0f ? t * rsqrtf(t) : 0.0f;
    float sn, cs;
    __sincosf(theta, &sn, &cs);
    return make_float2(-rad * cs, -rad * sn);
}

// Standard normals of one draw (Gaussian pair i from call i/2, words 2(i%2), 2(i%2)+1).
template <int NX, typename PP>
__device__ __forceinline__ void draw_normals(const PP& P, uint32_t step, uint32_t particle, uint32_t sample,
                                             uint32_t stream, uint32_t ctr, float (&z)[NX])
{
    const uint4 w0 = draw_words(P, step, 0u, particle, sample, stream, ctr);
    const float2 g0 = box_muller(w0.x, w0.y);
    const float2 g1 = box_muller(w0.z, w0.w);
    z[0] = g0.x; z[1] = g0.y; z[2] = g1.x; z[3] = g1.y;
    if constexpr (NX > 4) {
        const uint4 w1 = draw_words(P, step, 1u, particle, sample, stream, ctr);
        const float2 g2 = box_muller(w1.x, w1.y);
        z[4] = g2.x; z[5] = g2.y;
        if constexpr (NX > 6) {
            const float2 g3 = box_muller(w1.z, w1.w);
            z[6] = g3.x; z[7] = g3.y;
        }
    }
}

// State disturbance of one particle n at a step (stream 1). For 6 states, particles n and n + H
// (H = dist_half) share the counter whose word 1 is the lower index: its calls 0-2 give six Gaussian
// pairs, pairs 0-2 to the lower particle and 3-5 to the upper one, so no word goes unused. Other
// state counts draw per particle.
template <int NX, typename PP>
__device__ __forceinline__ void draw_disturbance(const PP& P, uint32_t step, uint32_t particle, uint32_t sample,
                                                 uint32_t ctr, float (&z)[NX])
{
    if constexpr (NX == 6) {
        const bool upper = particle >= (uint32_t)P.dist_half;
        const uint32_t q = upper ? particle - (uint32_t)P.dist_half : particle;
        const uint4 wa = draw_words(P, step, upper ? 1u : 0u, q, sample, kStreamDisturbance, ctr);
        const uint4 wb = draw_words(P, step, upper ? 2u : 1u, q, sample, kStreamDisturbance, ctr);
        // Select the words, then transform: one Box-Muller per pair whichever half the particle is in.
        const float2 g0 = box_muller(upper ? wa.z : wa.x, upper ? wa.w : wa.y);
        const float2 g1 = box_muller(upper ? wb.x : wa.z, upper ? wb.y : wa.w);
        const float2 g2 = box_muller(upper ? wb.z : wb.x, upper ? wb.w : wb.y);
        z[0] = g0.x; z[1] = g0.y; z[2] = g1.x; z[3] = g1.y; z[4] = g2.x; z[5] = g2.y;
    } else {
        draw_normals<NX>(P, step, particle, sample, kStreamDisturbance, ctr, z);
    }
}

// The disturbances of both particles of one 6-state pair (lower index q, upper q + H) from their
// shared counter: three calls instead of four.
template <typename PP>
__device__ __forceinline__ void draw_disturbance_pair(const PP& P, uint32_t step, uint32_t q, uint32_t sample,
                                                      uint32_t ctr, float (&lo)[6], float (&hi)[6])
{
    const uint4 w0 = draw_words(P, step, 0u, q, sample, kStreamDisturbance, ctr);
    const uint4 w1 = draw_words(P, step, 1u, q, sample, kStreamDisturbance, ctr);
    const uint4 w2 = draw_words(P, step, 2u, q, sample, kStreamDisturbance, ctr);
    float2 g = box_muller(w0.x, w0.y);
    lo[0] = g.x; lo[1] = g.y;
    g = box_muller(w0.z, w0.w);
    lo[2] = g.x; lo[3] = g.y;
    g = box_muller(w1.x, w1.y);
    lo[4] = g.x; lo[5] = g.y;
    g = box_muller(w1.z, w1.w);
    hi[0] = g.x; hi[1] = g.y;
    g = box_muller(w2.x, w2.y);
    hi[2] = g.x; hi[3] = g.y;
    g = box_muller(w2.z, w2.w);
    hi[4] = g.x; hi[5] = g.y;
}

// x += L z with L diagonal (its diagonal entries at the packed positions i (i + 3) / 2).
template <int NX>
__device__ __forceinline__ void add_diagonal(const float* L, const float (&z)[NX], float (&x)[NX])
{
#pragma unroll
    for (int i = 0; i < NX; ++i) x[i] = fmaf(L[i * (i + 3) / 2], z[i], x[i]);
}

// x += L z with L packed lower-triangular by rows.
template <int NX>
__device__ __forceinline__ void add_correlated(const float* L, const float (&z)[NX], float (&x)[NX])
{
#pragma unroll
    for (int i = 0; i < NX; ++i) {
        float w = 0.0f;
#pragma unroll
        for (int j = 0; j <= i; ++j) w = fmaf(L[i * (i + 1) / 2 + j], z[j], w);
        x[i] += w;
    }
}

// ---------------------------------------------------------------------------------------------
// Dynamic single-track vehicle in the road-aligned frame. State [v_x, v_y, r, e_psi, e_y, ds]
// where ds = s - s0 is the progress since the start of the rollout (kept relative so that FP32
// rounding of the progress does not grow with the lap position). Lateral tyre forces follow the
// simplified Pacejka law F_y = D sin(C atan(B alpha)), D = mu F_z with static axle loads.
// ---------------------------------------------------------------------------------------------
struct Control {
    float steer, accel, sin_steer, cos_steer;
};

// sin x and cos x from the hardware sine and cosine after reducing x into [-pi, pi] (x - 2 pi rint(x /
// 2 pi)), where their absolute error is at most 2^-21.4: no branch, and a short dependent chain
// where that matters more than the last bits (the repair's serial forward pass).
__device__ __forceinline__ void sincos_reduced(float x, float* s, float* c)
{
    const float r = fmaf(-6.28318530717958647692f, rintf(x * 0.15915494309189533577f), x);
    __sincosf(r, s, c);
}

// sin x and cos x from their Taylor series through x^9 and x^10 (coefficients 1/n!); for |x| <= pi/4
// the truncation errors are below |x|^11/11! < 2e-9 and |x|^12/12! < 2e-10, under FP32 rounding.
// Outside that range (a spinning vehicle) the library's sincosf.
__device__ __forceinline__ void sincos_series(float x, float* s, float* c)
{
    if (fabsf(x) <= 0.78539816f) {
        const float x2 = x * x;
        float ps = fold_fixed(kFoldS9);           //  1/9!
        ps = fmaf(ps, x2, fold_fixed(kFoldS7));   // -1/7!
        ps = fmaf(ps, x2, fold_fixed(kFoldC120)); //  1/5!
        ps = fmaf(ps, x2, fold_fixed(kFoldM6));   // -1/3!
        *s = fmaf(ps * x2, x, x);
        float pc = fold_fixed(kFoldC10);          // -1/10!
        pc = fmaf(pc, x2, fold_fixed(kFoldC8));   //  1/8!
        pc = fmaf(pc, x2, fold_fixed(kFoldC6));   // -1/6!
        pc = fmaf(pc, x2, fold_fixed(kFoldC24));  //  1/4!
        pc = fmaf(pc, x2, -0.5f);                 // -1/2!
        *c = fmaf(pc, x2, 1.0f);
    } else {
        sincosf(x, s, c);
    }
}

// PP: any parameter object with the track's track_scale and n_track_mask.
template <typename PP>
__device__ __forceinline__ float track_curvature(const PP& P, const float* __restrict__ kap, float s)
{
    const float x = s * P.track_scale;
    const float fl = floorf(x);
    const float f = x - fl;
    const int i = ((int)fl) & P.n_track_mask;
    const float k0 = kap[i], k1 = kap[i + 1];
    return fmaf(f, k1 - k0, k0);
}

// The same lookup from a table of (kappa_i, kappa_{i+1} - kappa_i) pairs (one 8-byte load; the
// difference is the same FP32 subtraction, so the result is bit-identical).
template <typename PP>
__device__ __forceinline__ float track_curvature(const PP& P, const float2* __restrict__ kap, float s)
{
    const float x = s * P.track_scale;
    const float fl = floorf(x);
    const float f = x - fl;
    const float2 k = kap[((int)fl) & P.n_track_mask];
    return fmaf(f, k.y, k.x);
}

// Arithmetic on one particle's value (float) or two particles' values side by side (float2, the
// packed FP32 instructions of the sm_100 family: fma / mul on .f32x2 register pairs, rounded to
// nearest in each half). Every rounding is explicit (fmaf and __fmul_rn are never contracted), so
// each half of a packed result equals the one-particle result bit for bit.
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
template <typename F> __device__ __forceinline__ float each(float a, F f) { return f(a); }
template <typename F> __device__ __forceinline__ float2 each(float2 a, F f) { return make_float2(f(a.x), f(a.y)); }
template <typename F> __device__ __forceinline__ float each(float a, float b, F f) { return f(a, b); }
template <typename F> __device__ __forceinline__ float2 each(float2 a, float2 b, F f)
{
    return make_float2(f(a.x, b.x), f(a.y, b.y));
}
template <typename F> __device__ __forceinline__ float each(float a, float b, float c, F f) { return f(a, b, c); }
template <typename F> __device__ __forceinline__ float2 each(float2 a, float2 b, float2 c, F f)
{
    return make_float2(f(a.x, b.x, c.x), f(a.y, b.y, c.y));
}
template <typename V> __device__ __forceinline__ V splat(float a);
template <> __device__ __forceinline__ float splat<float>(float a) { return a; }
template <> __device__ __forceinline__ float2 splat<float2>(float a) { return make_float2(a, a); }
template <typename V> __device__ __forceinline__ V fold(const DevParams& P, int i);
template <> __device__ __forceinline__ float fold<float>(const DevParams& P, int i)
{
    return i >= kFoldOne ? fold_fixed(i) : P.fold[i];  // fixed numbers as immediate operands
}
template <> __device__ __forceinline__ float2 fold<float2>(const DevParams& P, int i) { return P.fold2[i]; }

// atan t for the slip angles, whose arguments (v_y + l_f r) / v_x and (v_y - l_r r) / v_x
// stay small while the tyres grip. For |t| <= 1/2, atan t = t + t z p(z) with z = t^2 and p of degree 4, its
// coefficients fitted for the least maximum relative error on [0, 1/2] by Lawson's iteratively
// reweighted least squares (fit_slip_atan.py beside this package): 5.3e-9 in exact arithmetic,
// 0.72 FP32 ulp by Horner's rule with fused multiply-adds. Beyond, the library's atanf. The choice
// is made per particle, so a result does not depend on which particles share a warp. Both
// models take it for their slip angles (slip_atans: pairs of particles in packed instructions).
__device__ __forceinline__ float slip_atan(float t)
{
    if (fabsf(t) <= 0.5f) {
        const float z = __fmul_rn(t, t);
        float p = slip_atan_coef(0);
#pragma unroll
        for (int i = 1; i < 5; ++i) p = fmaf(p, z, slip_atan_coef(i));
        return fmaf(__fmul_rn(t, z), p, t);
    }
    return atanf(t);
}

// |x| > lim for one particle's value, or for either of a pair's.
__device__ __forceinline__ bool beyond(float x, float lim) { return fabsf(x) > lim; }
__device__ __forceinline__ bool beyond(float2 x, float lim) { return fabsf(x.x) > lim || fabsf(x.y) > lim; }

// slip_atan's polynomial for two particles side by side (each half rounds as slip_atan does).
__device__ __forceinline__ float2 slip_poly2(const DevParams& P, float2 t)
{
    const float2 z = vmul(t, t);
    float2 p = fold<float2>(P, kFoldSa0);
#pragma unroll
    for (int i = kFoldSa0 + 1; i <= kFoldSaLast; ++i) p = vfma(p, z, fold<float2>(P, i));
    return vfma(vmul(t, z), p, t);
}

// slip_atan of the front and rear slip arguments of one particle, or of two particles side by side:
// for pairs, the polynomial for all four with packed instructions, then the library's atanf for an
// argument beyond |t| = 1/2, entered by the warp only when one of its particles needs it (one vote
// for both tyres).
template <typename V>
__device__ __forceinline__ void slip_atans(const DevParams& P, V tf, V tr, V& yf, V& yr)
{
    if constexpr (std::is_same<V, float>::value) {
        yf = slip_atan(tf);
        yr = slip_atan(tr);
    } else {
        yf = slip_poly2(P, tf);
        yr = slip_poly2(P, tr);
        if (__any_sync(__activemask(), beyond(tf, 0.5f) || beyond(tr, 0.5f))) {
            const auto fix = [](float tv, float yv) { return fabsf(tv) <= 0.5f ? yv : atanf(tv); };
            yf = each(tf, yf, fix);
            yr = each(tr, yr, fix);
        }
    }
}

// Per-step factors (the control is the same for every particle of a sample): steer, a,
// -D_f sin(delta) / m, -D_f cos(delta) / m, l_f D_f cos(delta) / I_z.
template <typename V>
struct SubstepCtl {
    V steer, acc, a1, na2, b1;
};

template <typename V>
__device__ __forceinline__ SubstepCtl<V> substep_ctl(const DevParams& P, const Control& u)
{
    SubstepCtl<V> c;
    c.steer = splat<V>(u.steer);
    c.acc = splat<V>(u.accel);
    c.a1 = splat<V>(__fmul_rn(-P.Df_m, u.sin_steer));
    c.na2 = splat<V>(__fmul_rn(-P.Df_m, u.cos_steer));
    c.b1 = splat<V>(__fmul_rn(P.lfDf_Iz, u.cos_steer));
    return c;
}

// slip_atan of one slip argument per particle (a pair side by side: packed polynomial, then the
// library's atanf for a particle beyond |t| = 1/2, entered by the warp only when one needs it).
template <typename V>
__device__ __forceinline__ V slip_atan_v(const DevParams& P, V t)
{
    if constexpr (std::is_same<V, float>::value) {
        return slip_atan(t);
    } else {
        V y = slip_poly2(P, t);
        if (__any_sync(__activemask(), beyond(t, 0.5f)))
            y = each(t, y, [](float tv, float yv) { return fabsf(tv) <= 0.5f ? yv : atanf(tv); });
        return y;
    }
}

// The heading's sine and cosine carried across the substeps of one step: seeded from the series at
// the step's first substep, then rotated by each substep's increment d = h e_psi' (|d| << 1:
// sin d and cos d from three-term series, errors below |d|^7/7! and |d|^6/6!).
template <typename V>
__device__ __forceinline__ void rotate_heading_v(const DevParams& P, V d, V& sp, V& cp)
{
    const V d2 = vmul(d, d);
    const V cd = vfma(d2, vfma(d2, fold<V>(P, kFoldC24), fold<V>(P, kFoldMHalf)), fold<V>(P, kFoldOne));
    const V sd = vfma(vmul(d, d2), vfma(d2, fold<V>(P, kFoldC120), fold<V>(P, kFoldM6)), d);
    const V s = vfma(sp, cd, vmul(cp, sd));
    cp = vfma(cp, cd, vmul(vmul(sp, sd), fold<V>(P, kFoldM1)));
    sp = s;
}

// sincos_series of one particle's heading, or of two particles' side by side: for pairs, both
// series with packed instructions (each half rounds as sincos_series does), then the library's
// sincosf for a heading beyond pi/4, entered by the warp only when one of its particles needs it.
template <typename V>
__device__ __forceinline__ void sincos_series_v(const DevParams& P, V x, V& s, V& c)
{
    if constexpr (std::is_same<V, float>::value) {
        sincos_series(x, &s, &c);
    } else {
        const V x2 = vmul(x, x);
        V ps = fold<V>(P, kFoldS9);
        ps = vfma(ps, x2, fold<V>(P, kFoldS7));
        ps = vfma(ps, x2, fold<V>(P, kFoldC120));
        ps = vfma(ps, x2, fold<V>(P, kFoldM6));
        s = vfma(vmul(ps, x2), x, x);
        V pc = fold<V>(P, kFoldC10);
        pc = vfma(pc, x2, fold<V>(P, kFoldC8));
        pc = vfma(pc, x2, fold<V>(P, kFoldC6));
        pc = vfma(pc, x2, fold<V>(P, kFoldC24));
        pc = vfma(pc, x2, fold<V>(P, kFoldMHalf));
        c = vfma(pc, x2, fold<V>(P, kFoldOne));
        if (__any_sync(__activemask(), beyond(x, 0.78539816f))) {
            if (fabsf(x.x) > 0.78539816f) sincosf(x.x, &s.x, &c.x);
            if (fabsf(x.y) > 0.78539816f) sincosf(x.y, &s.y, &c.y);
        }
    }
}

// The tyre curve of the simplified Pacejka law, sin(C atan x) for x = B alpha. For |x| <= 1 it is
// x p(x^2), p the degree-9 polynomial that interpolates sin(C atan sqrt z) / sqrt z at the ten
// Chebyshev points of [0, 1] (fitted on the host for the problem's C in double precision; its
// coefficients are of the order of C, so Horner's rule in FP32 stays within about 2e-7 of the curve,
// as accurate as the hardware sine it replaces); beyond, the library's atanf and the hardware sine
// (|C atan x| < C pi / 2 < pi keeps the sine inside the range where its absolute error is at most
// 2^-21.4). The choice is made per particle; the warp enters the library route only when one of its
// particles needs it, so the common case is one uniform branch.
__device__ __forceinline__ float tyre_curve_library(const DevParams& P, float x) { return __sinf(P.tC * atanf(x)); }

template <typename V>
__device__ __forceinline__ V tyre_poly(const DevParams& P, V x)
{
    const V z = vmul(x, x);
    V p = fold<V>(P, kFoldTyLast);
#pragma unroll
    for (int d = kTyreDeg - 1; d >= 0; --d) p = vfma(p, z, fold<V>(P, kFoldTy0 + d));
    return vmul(x, p);
}

template <typename V>
__device__ __forceinline__ V tyre_curve(const DevParams& P, V x)
{
    V g = tyre_poly(P, x);
    if (__any_sync(__activemask(), beyond(x, 1.0f)))
        g = each(x, g, [&](float xv, float gv) { return fabsf(xv) > 1.0f ? tyre_curve_library(P, xv) : gv; });
    return g;
}

// The rear tyre's curve as one function of its slip argument t = (v_y - l_r r) / v_x, whose slip
// angle is -atan t: g_r(t) = sin(C atan(-B atan t)). For |t| <= tau, tau = tan(1/B) (where
// |B atan t| <= 1) or 1/2 if less, it is x q(x^2) with x = t / tau and q the degree-9 polynomial that
// interpolates g_r(tau x) / x at ten Chebyshev points of x^2 in [0, 1], fitted on the host for the
// problem's B and C like the tyre curve's (one polynomial where the slip angle's and the tyre
// curve's took two). Beyond, the slip angle from slip_atan and the curve by the library route.
template <typename V>
__device__ __forceinline__ V rear_tyre_poly(const DevParams& P, V x)
{
    const V z = vmul(x, x);
    V p = fold<V>(P, kFoldRyLast);
#pragma unroll
    for (int d = kTyreDeg - 1; d >= 0; --d) p = vfma(p, z, fold<V>(P, kFoldRy0 + d));
    return vmul(x, p);
}
__device__ __forceinline__ float rear_tyre_beyond(const DevParams& P, float t)
{
    return tyre_curve_library(P, __fmul_rn(-P.tB, slip_atan(t)));
}

// The front tyre's curve at x_f = B alpha_f and the rear tyre's at its slip argument t_r, with one
// vote of the warp for the library routes. The choice is made per particle.
template <typename V>
__device__ __forceinline__ void front_rear_tyres(const DevParams& P, V xf, V tr, V& gf, V& gr)
{
    gf = tyre_poly(P, xf);
    const V xr = vmul(tr, fold<V>(P, kFoldRInv));
    gr = rear_tyre_poly(P, xr);
    if (__any_sync(__activemask(), beyond(xf, 1.0f) || beyond(xr, 1.0f))) {
        gf = each(xf, gf, [&](float x, float g) { return fabsf(x) > 1.0f ? tyre_curve_library(P, x) : g; });
        gr = each(xr, tr, gr, [&](float x, float t, float g) { return fabsf(x) > 1.0f ? rear_tyre_beyond(P, t) : g; });
    }
}

// The rear tyre's curve of one particle or a pair, as the substep evaluates it (checking kernels).
template <typename V>
__device__ __forceinline__ V rear_tyre(const DevParams& P, V tr)
{
    const V xr = vmul(tr, fold<V>(P, kFoldRInv));
    V gr = rear_tyre_poly(P, xr);
    if (__any_sync(__activemask(), beyond(xr, 1.0f)))
        gr = each(xr, tr, gr, [&](float x, float t, float g) { return fabsf(x) > 1.0f ? rear_tyre_beyond(P, t) : g; });
    return gr;
}

// One explicit-Euler substep of one particle (V = float) or of two particles side by side
// (V = float2: one issued instruction does each multiply-add for both). The transcendentals,
// quotients and the curvature lookup are taken per particle. (sp, cp) = (sin e_psi, cos e_psi) on
// entry and on exit. Tab: the curvature table's element (float, or float2 pairs of value and
// difference). The force constants are folded into per-step factors (SubstepCtl), and each state's
// derivative is summed at its own (small) magnitude before one fused multiply-add adds h times it
// to the state: v_x' = v_x + h (a - D_f sin(delta)/m g_f + v_y r), and so on, with g_f, g_r the
// tyre curves' values sin(C atan(B alpha)).
// TP: the object holding the track's scale and mask (P itself, or a serving item).
// POLY: the tyre curve from its polynomial (tyre_curve); otherwise the library's atanf and the
// hardware sine for every particle, which measured faster where four particles share a lane and in
// the server's batched kernels.
template <bool POLY = true, typename V, typename Tab, typename TP>
__device__ __forceinline__ void bicycle_substep(const DevParams& P, const TP& trk, const Tab* __restrict__ kap,
                                                float s0, const SubstepCtl<V>& u, V (&X)[6], V& sp, V& cp)
{
    const V vx = X[0], vy = X[1], r = X[2];
    // v_x >= vx_floor >= 1 and 1 - kappa e_y is near 1, so the fast (2-ulp) quotients are safe.
    const V ivx = each(vx, [&](float a) { return __fdividef(1.0f, fmaxf(a, P.vx_floor)); });
    const V tf = vmul(vfma(fold<V>(P, kFoldLf), r, vy), ivx);    // (v_y + l_f r) / v_x
    const V tr = vmul(vfma(fold<V>(P, kFoldNLr), r, vy), ivx);   // (v_y - l_r r) / v_x
    V gf, gr;  // F_f / D_f, F_r / D_r
    if constexpr (POLY) {
        const V af = vfma(slip_atan_v(P, tf), fold<V>(P, kFoldM1), u.steer);  // alpha_f
        front_rear_tyres(P, vmul(fold<V>(P, kFoldTB), af), tr, gf, gr);        // at B alpha_f, t_r
    } else {
        V atf, atr;
        slip_atans(P, tf, tr, atf, atr);
        const V af = vfma(atf, fold<V>(P, kFoldM1), u.steer);  // alpha_f
        const V bf = vmul(fold<V>(P, kFoldTB), af);            // B alpha_f
        const V br = vmul(fold<V>(P, kFoldNTB), atr);          // B alpha_r
        const auto lib = [&](float a) { return tyre_curve_library(P, a); };
        gf = each(bf, lib);
        gr = each(br, lib);
    }
    const V nk = each(X[5], [&](float a) { return -track_curvature(trk, kap, s0 + a); });  // -kappa(s)
    const V num = vfma(vx, cp, vmul(vmul(vy, sp), fold<V>(P, kFoldM1)));                // v_x cos - v_y sin
    const V den = vfma(nk, X[4], fold<V>(P, kFoldOne));                                 // 1 - kappa e_y
    const V sdot = each(num, den, [](float a, float b) { return __fdividef(a, b); });
    const V dep = vfma(nk, sdot, r);
    const V dey = vfma(vx, sp, vmul(vy, cp));
    const V h = fold<V>(P, kFoldH);
    const V dvx = vfma(gf, u.a1, vfma(vy, r, u.acc));                                            // a - F_f sin / m + v_y r
    const V ndvy = vfma(vx, r, vfma(gf, u.na2, vmul(gr, fold<V>(P, kFoldNDrM))));             // -v_y' (exact sign flip)
    const V dr = vfma(gf, u.b1, vmul(gr, fold<V>(P, kFoldNLrDrIz)));                           // (l_f F_f cos - l_r F_r) / I_z
    X[0] = vfma(h, dvx, vx);
    X[1] = vfma(fold<V>(P, kFoldNH), ndvy, vy);
    X[2] = vfma(h, dr, r);
    X[3] = vfma(h, dep, X[3]);
    X[4] = vfma(h, dey, X[4]);
    X[5] = vfma(h, sdot, X[5]);
    rotate_heading_v(P, vmul(h, dep), sp, cp);
}

// Single-track model with wheel speeds and combined slip, x = [v_x, v_y, r, omega_F, omega_R, e_psi,
// e_y, s - s0], u = [steer, throttle]. Lateral slip angles as in the bicycle model; longitudinal slip
// kappa = (R omega - v_w) / max(|v_w|, slip_floor), v_w the wheel's forward speed; one tyre curve
// g = sin(C atan(B s)) on the combined slip s = sqrt(kappa^2 + alpha^2), split along the slip
// direction and scaled by the friction ellipse's axes: F_x = mu_x F_z g kappa / s,
// F_y = mu F_z g alpha / s. Rear-wheel drive torque tau_max * throttle; static axle loads.
// g(s) / s for the squared combined slip sl2 = s^2, which tends to C B at zero slip. While
// (B s)^2 <= 1 it is B p(B^2 sl2) with the tyre curve's polynomial (g(b) = b p(b^2), b = B s): no
// square root, and C B at zero slip by itself. Beyond, one reciprocal square root gives both
// s = sl2 / sqrt(sl2) and 1 / s for the library arctangent and the hardware sine (|C atan(B s)| <
// C pi / 2 < pi keeps the sine inside its accurate range). The choice is made per particle.
__device__ __forceinline__ float tyre_ratio_beyond(const DevParams& P, float sl2, float z, float r)
{
    if (z > 1.0f) {
        const float rs = rsqrtf(sl2);
        r = __sinf(P.tC * atanf(P.tB * (sl2 * rs))) * rs;
    }
    return r;
}

template <typename V>
__device__ __forceinline__ V tyre_ratio(const DevParams& P, V sl2)
{
    const V z = vmul(fold<V>(P, kFoldTB2), sl2);  // (B s)^2
    V p = fold<V>(P, kFoldTyLast);
#pragma unroll
    for (int d = kTyreDeg - 1; d >= 0; --d) p = vfma(p, z, fold<V>(P, kFoldTy0 + d));
    const V r = vmul(fold<V>(P, kFoldTB), p);
    if constexpr (std::is_same<V, float2>::value) {
        return make_float2(tyre_ratio_beyond(P, sl2.x, z.x, r.x), tyre_ratio_beyond(P, sl2.y, z.y, r.y));
    } else {
        return tyre_ratio_beyond(P, sl2, z, r);
    }
}

// Per-step factors of the wheel-speed substep: steer, cos delta, sin delta, -sin delta and
// tau_max a / I_w.
template <typename V>
struct WheelsCtl {
    V steer, cs, sn, nsn, taw;
};

template <typename V>
__device__ __forceinline__ WheelsCtl<V> wheels_ctl(const DevParams& P, const Control& u)
{
    WheelsCtl<V> c;
    c.steer = splat<V>(u.steer);
    c.cs = splat<V>(u.cos_steer);
    c.sn = splat<V>(u.sin_steer);
    c.nsn = splat<V>(-u.sin_steer);
    c.taw = splat<V>(__fmul_rn(P.tau_max, __fmul_rn(u.accel, P.inv_Iw)));
    return c;
}

// One explicit-Euler substep of the wheel-speed model for one particle (V = float) or two side by
// side (V = float2), as the bicycle substep: explicit roundings, per-particle transcendentals and
// quotients, packed multiply-adds, each derivative summed before h times it is added to the state.
// With F_xf = D_xf g_f kappa_f, F_yf = D_f g_f alpha_f, C = g_r kappa_r, D = -g_r alpha_r and the
// front forces rotated into the body frame, F_X = F_xf cos - F_yf sin, F_Y = F_xf sin + F_yf cos:
//   v_x' = v_x + h (F_X / m + (D_xr / m) C + v_y r),   v_y' = v_y + h (F_Y / m - (D_r / m) D - v_x r),
//   r' = r + h ((l_f / I_z) F_Y + (l_r D_r / I_z) D),   w_F' = w_F - (h R_w / I_w) F_xf,
//   w_R' = w_R + h (tau_max a / I_w - (R_w D_xr / I_w) C).
template <typename V, typename Tab, typename TP>
__device__ __forceinline__ void wheels_substep(const DevParams& P, const TP& trk, const Tab* __restrict__ kap,
                                               float s0, const WheelsCtl<V>& u, V (&X)[8], V& sp, V& cp)
{
    const V vx = X[0], vy = X[1], r = X[2], wf = X[3], wr = X[4];
    const V ivx = each(vx, [&](float a) { return __fdividef(1.0f, fmaxf(a, P.vx_floor)); });
    const V yf = vfma(fold<V>(P, kFoldLf), r, vy);                                         // v_y + l_f r
    V atf, nar;  // atan of the front slip argument; -alpha_r
    slip_atans(P, vmul(yf, ivx), vmul(vfma(fold<V>(P, kFoldNLr), r, vy), ivx), atf, nar);
    const V af = vfma(atf, fold<V>(P, kFoldM1), u.steer);                                  // alpha_f
    const V vwf = vfma(vx, u.cs, vmul(yf, u.sn));                                          // front wheel's speed
    const auto slip = [&](float num, float vw) { return __fdividef(num, fmaxf(fabsf(vw), P.slip_floor)); };
    const V kf = each(vfma(fold<V>(P, kFoldWRw), wf, vmul(vwf, fold<V>(P, kFoldM1))), vwf, slip);
    const V kr = each(vfma(fold<V>(P, kFoldWRw), wr, vmul(vx, fold<V>(P, kFoldM1))), vx, slip);
    const V gf = tyre_ratio(P, vfma(kf, kf, vmul(af, af)));
    const V gr = tyre_ratio(P, vfma(kr, kr, vmul(nar, nar)));
    const V G1 = vmul(vmul(gf, kf), fold<V>(P, kFoldWDxf));                                // F_xf
    const V G2 = vmul(vmul(gf, af), fold<V>(P, kFoldWDf));                                 // F_yf
    const V C = vmul(gr, kr), D = vmul(gr, nar);
    const V FX = vfma(G2, u.nsn, vmul(G1, u.cs));
    const V FY = vfma(G1, u.sn, vmul(G2, u.cs));
    const V nk = each(X[7], [&](float a) { return -track_curvature(trk, kap, s0 + a); });     // -kappa(s)
    const V num = vfma(vx, cp, vmul(vmul(vy, sp), fold<V>(P, kFoldM1)));
    const V den = vfma(nk, X[6], fold<V>(P, kFoldOne));
    const V sdot = each(num, den, [](float a, float b) { return __fdividef(a, b); });
    const V dep = vfma(nk, sdot, r);
    const V dey = vfma(vx, sp, vmul(vy, cp));
    const V h = fold<V>(P, kFoldH);
    const V dvx = vfma(FX, fold<V>(P, kFoldWInvM), vfma(C, fold<V>(P, kFoldWDxrM), vmul(vy, r)));
    const V ndvy = vfma(vx, r, vfma(FY, fold<V>(P, kFoldWNInvM), vmul(D, fold<V>(P, kFoldWDrM))));  // -v_y'
    const V dr = vfma(FY, fold<V>(P, kFoldWLfIz), vmul(D, fold<V>(P, kFoldWLrDrIz)));
    const V dwr = vfma(C, fold<V>(P, kFoldWNRwDxrIw), u.taw);
    X[0] = vfma(h, dvx, vx);
    X[1] = vfma(fold<V>(P, kFoldNH), ndvy, vy);
    X[2] = vfma(h, dr, r);
    X[3] = vfma(G1, fold<V>(P, kFoldWNhRwIw), wf);
    X[4] = vfma(h, dwr, wr);
    X[5] = vfma(h, dep, X[5]);
    X[6] = vfma(h, dey, X[6]);
    X[7] = vfma(h, sdot, X[7]);
    rotate_heading_v(P, vmul(h, dep), sp, cp);
}

// Tape of one bicycle substep: the transcendental results its adjoint needs
// {F_yf, dF_yf/dalpha_f, dF_yr/dalpha_r, sin e_psi, cos e_psi, kappa(s), dkappa/ds}.
constexpr int kTapeFloats = 7;

// The bicycle model's substep for one particle, with the forces written out unfolded, also writing
// its tape (the repair's forward pass records it so that the reverse sweep needs no transcendental
// functions). Its roundings differ from bicycle_substep's folded form by a few FP32 ulps, and its
// heading's sine and cosine come from sincos_reduced (within 2^-21.4 absolute), which shortens the
// serial chain of the repair's forward pass.
__device__ __forceinline__ void bicycle_substep_taped(const DevParams& P, const float* __restrict__ kap, float s0,
                                                      const Control& u, float (&x)[6], float (&tp)[kTapeFloats])
{
    const float vx = x[0], vy = x[1], r = x[2], ep = x[3], ey = x[4];
    const float inv_vx = __fdividef(1.0f, fmaxf(vx, P.vx_floor));
    const float alpha_f = u.steer - atanf((vy + P.lf * r) * inv_vx);
    const float alpha_r = -atanf((vy - P.lr * r) * inv_vx);
    const float bf = P.tB * alpha_f, br = P.tB * alpha_r;
    float sf, cf, sr, cr;
    __sincosf(P.tC * atanf(bf), &sf, &cf);
    __sincosf(P.tC * atanf(br), &sr, &cr);
    const float Ff = P.Df * sf, Fr = P.Dr * sr;
    const float xs = (s0 + x[5]) * P.track_scale;
    const float fl = floorf(xs);
    const int i = ((int)fl) & P.n_track_mask;
    const float k0 = kap[i], k1 = kap[i + 1];
    const float kap_s = fmaf(xs - fl, k1 - k0, k0);
    float sp, cp;
    sincos_reduced(ep, &sp, &cp);
    const float sdot = __fdividef(vx * cp - vy * sp, 1.0f - kap_s * ey);
    const float dvx = u.accel - Ff * u.sin_steer * P.inv_m + vy * r;
    const float dvy = (Ff * u.cos_steer + Fr) * P.inv_m - vx * r;
    const float dr = (P.lf * Ff * u.cos_steer - P.lr * Fr) * P.inv_Iz;
    const float dep = r - kap_s * sdot;
    const float dey = vx * sp + vy * cp;
    tp[0] = Ff;
    tp[1] = __fdividef(P.Df * cf * P.tC * P.tB, 1.0f + bf * bf);
    tp[2] = __fdividef(P.Dr * cr * P.tC * P.tB, 1.0f + br * br);
    tp[3] = sp;
    tp[4] = cp;
    tp[5] = kap_s;
    tp[6] = (k1 - k0) * P.track_scale;
    x[0] = fmaf(P.h, dvx, vx);
    x[1] = fmaf(P.h, dvy, vy);
    x[2] = fmaf(P.h, dr, r);
    x[3] = fmaf(P.h, dep, ep);
    x[4] = fmaf(P.h, dey, ey);
    x[5] = fmaf(P.h, sdot, x[5]);
}

// Reverse mode of one bicycle substep x' = x + h F(x, u) from its tape. On entry g holds dL/dx';
// on exit g holds dL/dx, and dL/du is added to (g_steer, g_accel). The partial derivatives are
// those of the forward formulas: d atan(q)/dq = 1/(1 + q^2), d sin = cos, the quotient rule for
// s', and the piecewise-linear slope of the curvature table.
__device__ __forceinline__ void bicycle_substep_vjp_taped(const DevParams& P, const Control& u, const float (&x)[6],
                                                          const float (&tp)[kTapeFloats], float (&g)[6],
                                                          float& g_steer, float& g_accel)
{
    const float vx = x[0], vy = x[1], r = x[2], ey = x[4];
    const float vxh = fmaxf(vx, P.vx_floor);
    const float yf = vy + P.lf * r, yr = vy - P.lr * r;
    const float Ff = tp[0], dFf = tp[1], dFr = tp[2], sp = tp[3], cp = tp[4], kap_s = tp[5], dkap = tp[6];
    const float num = vx * cp - vy * sp;
    const float inv_den = __fdividef(1.0f, 1.0f - kap_s * ey);
    const float sdot = num * inv_den;

    float a[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) a[j] = P.h * g[j];
    const float gFf = a[0] * (-u.sin_steer * P.inv_m) + a[1] * (u.cos_steer * P.inv_m) + a[2] * (P.lf * u.cos_steer * P.inv_Iz);
    const float gFr = a[1] * P.inv_m - a[2] * (P.lr * P.inv_Iz);
    const float gsdot = -a[3] * kap_s + a[5];
    const float gkap = -a[3] * sdot + gsdot * num * ey * inv_den * inv_den;
    const float gnum = gsdot * inv_den;
    const float gey = gsdot * num * kap_s * inv_den * inv_den;
    float gvx = gnum * cp - a[1] * r + a[4] * sp;
    float gvy = -gnum * sp + a[0] * r + a[4] * cp;
    const float gep = gnum * (-vx * sp - vy * cp) + a[4] * (vx * cp - vy * sp);
    float gr = a[0] * vy - a[1] * vx + a[3];
    g_steer += a[0] * (-Ff * u.cos_steer * P.inv_m) + a[1] * (-Ff * u.sin_steer * P.inv_m)
             + a[2] * (-P.lf * Ff * u.sin_steer * P.inv_Iz);
    g_accel += a[0];
    const float gaf = gFf * dFf, gar = gFr * dFr;
    g_steer += gaf;
    const float inv_qf = __fdividef(1.0f, vxh * vxh + yf * yf);
    const float inv_qr = __fdividef(1.0f, vxh * vxh + yr * yr);
    const float gyf = -gaf * vxh * inv_qf, gyr = -gar * vxh * inv_qr;
    const float gvxh = gaf * yf * inv_qf + gar * yr * inv_qr;
    gvy += gyf + gyr;
    gr += P.lf * gyf - P.lr * gyr;
    if (vx > P.vx_floor) gvx += gvxh;
    g[0] += gvx;
    g[1] += gvy;
    g[2] += gr;
    g[3] += gep;
    g[4] += gey;
    g[5] += gkap * dkap;
}

// Planar double integrator, exact zero-order-hold step.
__device__ __forceinline__ void double_integrator_step(const DevParams& P, const Control& u, float (&x)[4])
{
    const float dt = P.dt, hdt2 = 0.5f * P.dt * P.dt;
    x[0] = fmaf(hdt2, u.steer, fmaf(dt, x[2], x[0]));
    x[1] = fmaf(hdt2, u.accel, fmaf(dt, x[3], x[1]));
    x[2] = fmaf(dt, u.steer, x[2]);
    x[3] = fmaf(dt, u.accel, x[3]);
}

// Reverse mode of the double-integrator step: g (dL/dx') -> dL/dx in place, dL/du added.
__device__ __forceinline__ void double_integrator_step_vjp(const DevParams& P, float (&g)[4], float& g_ax, float& g_ay)
{
    const float dt = P.dt, hdt2 = 0.5f * P.dt * P.dt;
    g_ax += hdt2 * g[0] + dt * g[2];
    g_ay += hdt2 * g[1] + dt * g[3];
    g[2] += dt * g[0];
    g[3] += dt * g[1];
}

// One full model step f(x, u) (n_sub substeps for the bicycle).
template <int MODEL, int NX>
__device__ __forceinline__ void model_step(const DevParams& P, const float* __restrict__ kap, float s0,
                                           const Control& u, float (&x)[NX])
{
    if constexpr (MODEL == 0) {
        float sp, cp;
        sincos_series(x[3], &sp, &cp);
        const SubstepCtl<float> c = substep_ctl<float>(P, u);
        for (int j = 0; j < P.n_sub; ++j) bicycle_substep(P, P, kap, s0, c, x, sp, cp);
    } else if constexpr (MODEL == 2) {
        float sp, cp;
        sincos_series(x[5], &sp, &cp);
        const WheelsCtl<float> c = wheels_ctl<float>(P, u);
        for (int j = 0; j < P.n_sub; ++j) wheels_substep(P, P, kap, s0, c, x, sp, cp);
    } else {
        double_integrator_step(P, u, x);
    }
}

// ---------------------------------------------------------------------------------------------
// Running / terminal cost on the belief mean: (m - x_g)^T W (m - x_g) + C_obs 1[|m_ey| > w_T].
// MM != 0: only the states of MM carry weight (W_i = 0 elsewhere, so the skipped terms add exact
// zeros) and only their means are read.
// ---------------------------------------------------------------------------------------------
template <int NX, int EY, int MM = 0>
__device__ __forceinline__ float state_cost(const DevParams& P, const float* W, const float (&m)[NX])
{
    float c = 0.0f;
#pragma unroll
    for (int i = 0; i < NX; ++i) {
        if (MM != 0 && !((MM >> i) & 1)) continue;
        const float d = m[i] - P.xg[i];
        c = fmaf(W[i] * d, d, c);
    }
    return c + (fabsf(m[EY]) > P.wT ? P.Cobs : 0.0f);
}

// Belief barrier h = (w_T - nu sigma)^2 - m_ey^2.
__device__ __forceinline__ float belief_barrier(const DevParams& P, float mean_ey, float var_ey)
{
    float b = P.wT - P.nu * sqrtf(fmaxf(var_ey, 0.0f));
    if (P.clamp_margin) b = fmaxf(b, 0.0f);
    return b * b - mean_ey * mean_ey;
}

// General constraint set (Assumption 1): constraints c_q(x) < 0, each held with its own chance
// level through the back-off nu_q (Remark 1, computed on the host). A kernel parameter of its own,
// read with constant offsets only (the loops over q are unrolled).
constexpr int kMaxCon = 8;
struct ConSet {
    int n;                  // 0: the racing barrier of Eq. "DCBF"; 1..kMaxCon: this set
    int kind[kMaxCon];      // 0: half-space a^T x - b; 1: disk r^2 - |D (x - o)|^2 on two states
    float nu[kMaxCon];      // back-off coefficient
    float b[kMaxCon];       // half-space offset b; disk: r^2
    float a[kMaxCon][kNxMax];  // half-space normal a; disk: the selector D (1 on its two states)
    float o[kMaxCon][kNxMax];  // disk centre on its two states (0 elsewhere)
};

// c_q(m) and eta = grad c_q(m). CM != 0: the set touches the states of CM only (a and o vanish
// elsewhere, so the skipped terms are exact zeros), and eta is written on CM only.
template <int NX, int CM = 0>
__device__ __forceinline__ float constraint_value(const ConSet& cs, int q, const float (&m)[NX], float (&eta)[NX])
{
    float v;
    if (cs.kind[q] == 0) {
        v = -cs.b[q];
#pragma unroll
        for (int l = 0; l < NX; ++l) {
            if (CM != 0 && !((CM >> l) & 1)) continue;
            v = fmaf(cs.a[q][l], m[l], v);
            eta[l] = cs.a[q][l];
        }
    } else {
        v = cs.b[q];
#pragma unroll
        for (int l = 0; l < NX; ++l) {
            if (CM != 0 && !((CM >> l) & 1)) continue;
            const float d = cs.a[q][l] * (m[l] - cs.o[q][l]);
            v = fmaf(-d, d, v);
            eta[l] = -2.0f * d;
        }
    }
    return v;
}

// Eq. "DCBFchoice0" and Eq. "DCBFchoice": h = min_q -c_q(m) - nu_q sqrt(eta_q^T Sigma eta_q), with the
// covariance packed (lower triangle by rows).
// CM != 0: the set touches the states of CM only; the covariance is read on CM x CM (the terms of
// other states carry eta = 0 and would add exact zeros).
template <int NX, int CM = 0>
__device__ __forceinline__ float general_barrier(const ConSet& cs, const float (&m)[NX], const float (&C)[NX * (NX + 1) / 2])
{
    float h = INFINITY;
#pragma unroll
    for (int q = 0; q < kMaxCon; ++q) {
        if (q >= cs.n) break;
        float eta[NX];
        const float cv = constraint_value<NX, CM>(cs, q, m, eta);
        float quad = 0.0f;
#pragma unroll
        for (int i = 0; i < NX; ++i) {
            if (CM != 0 && !((CM >> i) & 1)) continue;
            float r = 0.5f * C[i * (i + 1) / 2 + i] * eta[i];
#pragma unroll
            for (int j = 0; j < i; ++j)
                if (CM == 0 || ((CM >> j) & 1)) r = fmaf(C[i * (i + 1) / 2 + j], eta[j], r);
            quad = fmaf(2.0f * eta[i], r, quad);
        }
        h = fminf(h, -cv - cs.nu[q] * sqrtf(fmaxf(quad, 0.0f)));
    }
    return h;
}

// The collision indicator of Eq. "CostFunction" for the general set: some c_q(m) > 0.
template <int NX, int CM = 0>
__device__ __forceinline__ bool any_constraint_broken(const ConSet& cs, const float (&m)[NX])
{
    bool broken = false;
#pragma unroll
    for (int q = 0; q < kMaxCon; ++q) {
        if (q >= cs.n) break;
        float eta[NX];
        broken |= constraint_value<NX, CM>(cs, q, m, eta) > 0.0f;
    }
    return broken;
}

// Quadratic part of the running cost, (m - x_g)^T diag(W) (m - x_g).
// MM != 0: W vanishes outside MM (the skipped terms are exact zeros).
template <int NX, int MM = 0>
__device__ __forceinline__ float quad_cost(const DevParams& P, const float* W, const float (&m)[NX])
{
    float c = 0.0f;
#pragma unroll
    for (int i = 0; i < NX; ++i) {
        if (MM != 0 && !((MM >> i) & 1)) continue;
        const float d = m[i] - P.xg[i];
        c = fmaf(W[i] * d, d, c);
    }
    return c;
}

// Neumaier-compensated accumulation: sum + c carries the sum to about twice the working precision.
struct CompSum {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        const float t = s + x;
        c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
        s = t;
    }
    __device__ __forceinline__ float value() const { return s + c; }
};

// Error-free sum of two compensated accumulators (TwoSum of the leading parts).
__device__ __forceinline__ void comp_merge(float& s, float& c, float s2, float c2)
{
    const float t = s + s2;
    const float bp = t - s;
    const float err = (s - (t - bp)) + (s2 - bp);
    s = t;
    c = c + c2 + err;
}

}  // namespace bss
