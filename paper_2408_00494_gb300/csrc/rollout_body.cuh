// Body of the fused belief rollout for one group of control samples, shared by the per-solve kernel
// (rollout.cu) and the batched serving kernels (serve.cu).
//
// Fused belief rollout: for every control sample, draw its perturbed control sequence, roll its M
// disturbance particles through the model for T steps, reduce the particle mean and variance of
// every step across the lanes that hold them, and accumulate the augmented trajectory cost.
//
// Mapping: a segment of `seg` lanes (seg = min(32, next power of two >= M)) owns one control
// sample; lane l of the segment holds particles l, l + seg, ..., l + (P-1) seg in registers.
// Particle states never touch memory. Per step, the moments are merged across the segment by a
// shuffle butterfly (Chan's parallel merge of counts, means and M2 when compensated), so every
// lane ends with the same belief and computes the cost redundantly; lane 0 writes the result.
#pragma once

#include <type_traits>

#include "device.cuh"

namespace bss {

struct RollIO {
    const float* x0;
    const float* Sigma0;
    const float* v;
    const uint32_t* ctr;
    float* S;
    float* eps;
    float* mean;
    float* var;
};

// Moments of the M particles of one sample. x[p] is particle ls + seg p (valid iff < M).
// mean[i] = particle mean, var[i] = unbiased variance 1/(M-1) sum (x - mean)^2 (Algorithm 2);
// var is produced for EY only unless all_var. Means outside the merged set are left lane-local (or,
// with MM != 0, untouched). The merged set: MM when it is nonzero (a kernel compiled for a fixed
// set of cost-weighted states, never recording); otherwise every state with equal counts on every
// lane and no recording, else dp.mean_mask (the states some cost term weights).
// IT: the object holding the sample's sizes (M, uniform, Mf, invM, invM1): dp itself, or a serving item.
template <int NX, int EY, int P, bool COMP, int MM, typename IT>
__device__ __forceinline__ void belief_moments(const DevParams& dp, const IT& it, const float (&x)[P][NX], int ls,
                                               int seg, bool all_var, float (&mean)[NX], float (&var)[NX])
{
    static_assert(MM == 0 || ((MM >> EY) & 1), "the barrier reads the mean of e_y");
    const int mmask = MM != 0 ? MM : dp.mean_mask;
    if constexpr (COMP) {
        // Per lane: exact two-pass mean and M2 over its (at most P) particles.
        float cnt = 0.0f;
        if (it.uniform) {
            cnt = (float)P;
        } else {
#pragma unroll
            for (int p = 0; p < P; ++p) cnt += (ls + seg * p < it.M) ? 1.0f : 0.0f;
        }
        const float inv_cnt = it.uniform ? (1.0f / (float)P) : (cnt > 0.0f ? 1.0f / cnt : 0.0f);
        float m2[NX];
#pragma unroll
        for (int i = 0; i < NX; ++i) {
            m2[i] = 0.0f;
            if (MM != 0 && !((MM >> i) & 1)) continue;
            float s = 0.0f;
#pragma unroll
            for (int p = 0; p < P; ++p) s += (it.uniform || ls + seg * p < it.M) ? x[p][i] : 0.0f;
            mean[i] = s * inv_cnt;
            float q = 0.0f;
            if (i == EY || all_var) {
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const float d = x[p][i] - mean[i];
                    q += (it.uniform || ls + seg * p < it.M) ? d * d : 0.0f;
                }
            }
            m2[i] = q;
        }
        // Chan et al. pairwise merge across the segment; the formulas are symmetric in the two
        // partners, so both ends of every exchange compute bit-identical results.
        if (it.uniform && !all_var) {
            // Equal counts on every lane: merging two halves of n each gives mean = (mean_a +
            // mean_b) / 2 and M2 = M2_a + M2_b + (mean_b - mean_a)^2 n / 2. The lanes carry the sums
            // 2^r mean after r merges instead (scaling by a power of two is exact, so every rounding
            // is the same), which saves a multiply per value and round; the merged means are added
            // two per packed add, and M2 for e_y only. A full warp's five rounds are unrolled, with
            // their scales and counts as constants.
            constexpr int UM = MM != 0 ? MM : (1 << NX) - 1;
            constexpr int NM = mask_count(UM);
            constexpr int JE = mask_count(UM & ((1 << EY) - 1));  // position of e_y among the merged
            float sm[NM];
#pragma unroll
            for (int j = 0; j < NM; ++j) sm[j] = mean[mask_nth(UM, j)];
            float m2e = m2[EY];
            auto merge_round = [&](int off, float scale, float half_n) {
                float sb[NM];
#pragma unroll
                for (int j = 0; j < NM; ++j) sb[j] = __shfl_xor_sync(0xffffffffu, sm[j], off);
                const float d = (sb[JE] - sm[JE]) * scale;
                const float m2b = __shfl_xor_sync(0xffffffffu, m2e, off);
                // d^2 rounded on its own: where half_n is a constant 1 the compiler would
                // otherwise fuse d * d into the sum and change the rounding
                m2e = fmaf(__fmul_rn(d, d), half_n, m2e + m2b);
#pragma unroll
                for (int j = 0; j + 1 < NM; j += 2) {
                    const float2 a = __fadd2_rn(make_float2(sm[j], sm[j + 1]), make_float2(sb[j], sb[j + 1]));
                    sm[j] = a.x;
                    sm[j + 1] = a.y;
                }
                if constexpr (NM % 2 == 1) sm[NM - 1] = __fadd_rn(sm[NM - 1], sb[NM - 1]);
            };
            float scale;
            if (seg == kWarp) {
#pragma unroll
                for (int r = 0; r < 5; ++r) merge_round(16 >> r, 1.0f / (float)(1 << r), 0.5f * (float)(P << r));
                scale = 1.0f / (float)kWarp;
            } else {
                scale = 1.0f;
                for (int off = seg >> 1; off > 0; off >>= 1) {
                    merge_round(off, scale, 0.5f * cnt);
                    scale *= 0.5f;
                    cnt *= 2.0f;
                }
            }
#pragma unroll
            for (int j = 0; j < NM; ++j) mean[mask_nth(UM, j)] = sm[j] * scale;
            m2[EY] = m2e;
        } else if (it.uniform) {
            for (int off = seg >> 1; off > 0; off >>= 1) {
                const float half_n = 0.5f * cnt;
#pragma unroll
                for (int i = 0; i < NX; ++i) {
                    if (!((mmask >> i) & 1)) continue;  // a mean no cost term reads
                    const float mb = __shfl_xor_sync(0xffffffffu, mean[i], off);
                    if (i == EY || all_var) {
                        const float d = mb - mean[i];
                        const float m2b = __shfl_xor_sync(0xffffffffu, m2[i], off);
                        m2[i] = (m2[i] + m2b) + d * d * half_n;
                    }
                    mean[i] = 0.5f * (mean[i] + mb);
                }
                cnt *= 2.0f;
            }
        } else {
            for (int off = seg >> 1; off > 0; off >>= 1) {
                const float cb = __shfl_xor_sync(0xffffffffu, cnt, off);
                const float n = cnt + cb;
                const float inv = n > 0.0f ? 1.0f / n : 0.0f;
                const float fa = cnt * inv, fb = cb * inv, fab = cnt * cb * inv;
#pragma unroll
                for (int i = 0; i < NX; ++i) {
                    if (!((mmask >> i) & 1)) continue;
                    const float mb = __shfl_xor_sync(0xffffffffu, mean[i], off);
                    if (i == EY || all_var) {
                        const float d = mb - mean[i];
                        const float m2b = __shfl_xor_sync(0xffffffffu, m2[i], off);
                        m2[i] = (m2[i] + m2b) + d * d * fab;
                    }
                    mean[i] = __fadd_rn(__fmul_rn(fa, mean[i]), __fmul_rn(fb, mb));
                }
                cnt = n;
            }
        }
#pragma unroll
        for (int i = 0; i < NX; ++i)
            if (MM == 0 || ((MM >> i) & 1)) var[i] = m2[i] * it.invM1;
    } else {
        // Naive one-pass sums: mean = sum x / M, var = (sum x^2 - M mean^2) / (M - 1).
        float s[NX], q[NX];
#pragma unroll
        for (int i = 0; i < NX; ++i) {
            s[i] = 0.0f;
            q[i] = 0.0f;
            if (MM != 0 && !((MM >> i) & 1)) continue;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float xv = (it.uniform || ls + seg * p < it.M) ? x[p][i] : 0.0f;
                s[i] += xv;
                if (i == EY || all_var) q[i] += xv * xv;
            }
        }
        for (int off = seg >> 1; off > 0; off >>= 1) {
#pragma unroll
            for (int i = 0; i < NX; ++i) {
                if (!((mmask >> i) & 1)) continue;
                s[i] += __shfl_xor_sync(0xffffffffu, s[i], off);
                if (i == EY || all_var) q[i] += __shfl_xor_sync(0xffffffffu, q[i], off);
            }
        }
#pragma unroll
        for (int i = 0; i < NX; ++i) {
            if (MM != 0 && !((MM >> i) & 1)) continue;
            mean[i] = s[i] * it.invM;
            var[i] = (q[i] - it.Mf * mean[i] * mean[i]) * it.invM1;
        }
    }
}

// xor-butterfly sum of N values across the segment, two values per packed add (each half rounds as
// the scalar add would, so the sums are those of the one-value butterfly).
template <int N>
__device__ __forceinline__ void butterfly_sum(float (&v)[N], int seg)
{
    for (int off = seg >> 1; off > 0; off >>= 1) {
        float w[N];
#pragma unroll
        for (int e = 0; e < N; ++e) w[e] = __shfl_xor_sync(0xffffffffu, v[e], off);
#pragma unroll
        for (int e = 0; e + 1 < N; e += 2) {
            const float2 a = __fadd2_rn(make_float2(v[e], v[e + 1]), make_float2(w[e], w[e + 1]));
            v[e] = a.x;
            v[e + 1] = a.y;
        }
        if constexpr (N % 2 == 1) v[N - 1] = __fadd_rn(v[N - 1], w[N - 1]);
    }
}

// Full belief of one sample for the re-sampling reading of Algorithm 2: every mean and the unbiased
// covariance (packed lower triangle by rows), in two passes over the segment: the sums give the
// means, then the centred products are summed. xor-butterfly sums are symmetric in the two partners,
// so every lane of the segment ends with bit-identical moments. MM = kPlaneMeanMask: only the means
// of MM and the covariance on kPlaneConMask x kPlaneConMask (a constraint set on the road plane, no
// re-sampling), the same values as the full computation gives for them; other entries untouched.
template <int NX, int P, int MM = 0, typename IT>
__device__ __forceinline__ void belief_moments_full(const IT& dp, const float (&x)[P][NX], int ls, int seg,
                                                    float (&mean)[NX], float (&C)[NX * (NX + 1) / 2])
{
    if constexpr (MM != 0) {
        static_assert(MM == kPlaneMeanMask, "the reduced full belief is built for the road plane");
        constexpr int NM = mask_count(MM), NC = mask_count(kPlaneConMask), NE = NC * (NC + 1) / 2;
        float s[NM];
#pragma unroll
        for (int a = 0; a < NM; ++a) {
            const int i = mask_nth(MM, a);
            s[a] = 0.0f;
#pragma unroll
            for (int p = 0; p < P; ++p) s[a] += (dp.uniform || ls + seg * p < dp.M) ? x[p][i] : 0.0f;
        }
        butterfly_sum<NM>(s, seg);
#pragma unroll
        for (int a = 0; a < NM; ++a) mean[mask_nth(MM, a)] = s[a] * dp.invM;
        float c[NE];
#pragma unroll
        for (int a = 0; a < NC; ++a) {
#pragma unroll
            for (int b = 0; b <= a; ++b) {
                const int i = mask_nth(kPlaneConMask, a), j = mask_nth(kPlaneConMask, b);
                float acc = 0.0f;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const float d = (x[p][i] - mean[i]) * (x[p][j] - mean[j]);
                    acc += (dp.uniform || ls + seg * p < dp.M) ? d : 0.0f;
                }
                c[a * (a + 1) / 2 + b] = acc;
            }
        }
        butterfly_sum<NE>(c, seg);
#pragma unroll
        for (int a = 0; a < NC; ++a)
#pragma unroll
            for (int b = 0; b <= a; ++b) {
                const int i = mask_nth(kPlaneConMask, a), j = mask_nth(kPlaneConMask, b);
                C[i * (i + 1) / 2 + j] = c[a * (a + 1) / 2 + b] * dp.invM1;
            }
    } else {
        float s[NX];
#pragma unroll
        for (int i = 0; i < NX; ++i) {
            s[i] = 0.0f;
#pragma unroll
            for (int p = 0; p < P; ++p) s[i] += (dp.uniform || ls + seg * p < dp.M) ? x[p][i] : 0.0f;
        }
        butterfly_sum<NX>(s, seg);
#pragma unroll
        for (int i = 0; i < NX; ++i) mean[i] = s[i] * dp.invM;
#pragma unroll
        for (int i = 0; i < NX; ++i) {
#pragma unroll
            for (int j = 0; j <= i; ++j) {
                float c = 0.0f;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const float d = (x[p][i] - mean[i]) * (x[p][j] - mean[j]);
                    c += (dp.uniform || ls + seg * p < dp.M) ? d : 0.0f;
                }
                C[i * (i + 1) / 2 + j] = c;
            }
        }
        butterfly_sum<NX * (NX + 1) / 2>(C, seg);
#pragma unroll
        for (int e = 0; e < NX * (NX + 1) / 2; ++e) C[e] *= dp.invM1;
    }
}

// In-place Cholesky factorisation of a packed (lower, by rows) PSD matrix; a pivot that is not
// positive leaves a zero column (a direction without spread).
template <int NX>
__device__ __forceinline__ void cholesky_packed_psd(float (&C)[NX * (NX + 1) / 2])
{
#pragma unroll
    for (int j = 0; j < NX; ++j) {
        float d = C[j * (j + 1) / 2 + j];
#pragma unroll
        for (int k = 0; k < j; ++k) d -= C[j * (j + 1) / 2 + k] * C[j * (j + 1) / 2 + k];
        const bool pos = d > 0.0f;
        const float ljj = pos ? sqrtf(d) : 0.0f;
        const float inv = pos ? 1.0f / ljj : 0.0f;
        C[j * (j + 1) / 2 + j] = ljj;
#pragma unroll
        for (int i = j + 1; i < NX; ++i) {
            float t = C[i * (i + 1) / 2 + j];
#pragma unroll
            for (int k = 0; k < j; ++k) t -= C[i * (i + 1) / 2 + k] * C[j * (j + 1) / 2 + k];
            C[i * (i + 1) / 2 + j] = t * inv;
        }
    }
}

// PSD-tolerant Cholesky factor (lower, row-major) of the caller's initial covariance.
template <int NX>
__device__ __forceinline__ void cholesky_psd(const float* A, float (&L)[NX][NX])
{
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
        for (int j = 0; j < NX; ++j) L[i][j] = 0.0f;
#pragma unroll
    for (int j = 0; j < NX; ++j) {
        float d = A[j * NX + j];
#pragma unroll
        for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
        if (d > 1e-30f) {
            const float ljj = sqrtf(d);
            L[j][j] = ljj;
#pragma unroll
            for (int i = j + 1; i < NX; ++i) {
                float s = A[i * NX + j];
#pragma unroll
                for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
                L[i][j] = s / ljj;
            }
        }
    }
}

// Largest block each model and particle count is compiled for (bounds the registers ptxas may use:
// 65536 / threads per thread). The 8-state wheel-speed model holds 8 states per particle and needs
// more registers per thread, so its blocks are smaller.
template <int MODEL, int P>
__host__ __device__ constexpr int roll_max_threads()
{
    if constexpr (MODEL == 2) return P == 1 ? 640 : (P == 2 ? 512 : 384);
    return P == 1 ? 1024 : (P == 2 ? 896 : (P == 4 ? 768 : 512));
}

// One sample group (the spw samples of one warp): control sequence, rollout, moments, cost.
// Returns the cost S of the lane's own sample (identical on every lane of its segment); my_u keeps
// the segment's clamped control sequence u (T x 2, or T x 4 with UTRIG) until the warp's next group.
// FULL selects the full-belief variant: every mean and the whole covariance each step, which the
// general constraint set (cs->n > 0, Eq. "DCBFchoice") and the literal reading of Algorithm 2
// (dp.resample: particles re-drawn from N(mean, cov) before the next step) need; cs is read only by
// it. PACK: bicycle and
// wheel-speed particles are stepped two at a time with packed FP32 instructions, bit-identical to
// stepping them one at a time. Their constant operands come from the kernel's parameter space; a caller
// whose parameters sit in shared memory turns it off, since there the packed operands would take
// registers of their own. UTRIG: my_u holds (u_0, u_1, sin u_0, cos u_0) per step (T x 4), so the
// steering angle's sine and cosine are taken once per step by the lanes that draw the controls
// instead of by every lane in every step; otherwise T x 2.
// TYRE_POLY: the bicycle's tyre curves from their polynomials where one or two particles share a lane
// (the library route at four and more, measured faster there, and wherever TYRE_POLY is off).
// IT: the object holding the per-solve fields (the sizes K, M, T, seg, spw, uniform, dist_half, M's
// reciprocals, k_off), the Philox round keys and the track's scale and mask. The single-solve kernel
// passes dp itself; the server passes a per-warp item in shared memory while dp, the constants its
// batch's vehicles share, stays in kernel parameter space.
// MM: 0, or the fixed set of states the cost weights (a mask holding e_y; the caller guarantees that
// Q and Qf vanish outside it and that nothing is recorded): only those means are merged and costed.
// With FULL, MM = kPlaneMeanMask: a constraint set on e_y and s only, no re-sampling, nothing recorded;
// the means of MM and the covariance of (e_y, s) are kept.
template <int MODEL, int P, bool COMP, bool FULL = false, typename Tab = float, bool PACK = true, bool UTRIG = false,
          typename IT = DevParams, bool TYRE_POLY = true, int MM = 0>
__device__ __forceinline__ float rollout_group(const DevParams& dp, const IT& it, const RollIO& io,
                                               const Tab* __restrict__ kap_s, const float* __restrict__ v_s,
                                               float* __restrict__ my_u, int group, uint32_t ctr,
                                               const ConSet* cs = nullptr)
{
    constexpr int NX = model_nx(MODEL);
    constexpr int EY = MODEL == 0 ? 4 : (MODEL == 2 ? 6 : 1);
    constexpr int SI = model_s_index(MODEL);  // path coordinate, carried relative to its start (or -1)
    static_assert(MM == 0 || !FULL || MM == kPlaneMeanMask, "the full belief merges every mean, or the plane's");
    constexpr int FCM = (FULL && MM != 0) ? kPlaneConMask : 0;  // the states a constraint set touches
    constexpr bool RECORDS = MM == 0;         // a fixed cost set runs without recording
    const int lane = threadIdx.x & (kWarp - 1);
    const int seg = it.seg;
    const int ls = lane & (seg - 1);
    const int k = group * it.spw + lane / seg;
    const bool active = k < it.K;
    const int kc = active ? k : it.K - 1;  // inactive segments shadow a valid sample, write nothing
    const uint32_t kg = (uint32_t)(kc + it.k_off);  // global sample index: the random streams' key
    const uint32_t kk = dp.crn ? 0u : kg;

    // (a1, a2) control noise eps ~ N(0, Sigma_eps) and clamped samples u = clamp(v + eps); the
    // lanes of the segment split the horizon. eps_eff = u - v feeds the update.
    constexpr bool TRIG = UTRIG && MODEL != 1;
    constexpr int UPS = UTRIG ? 4 : 2;  // floats of my_u per step
    for (int t = ls; t < it.T; t += seg) {
        const uint4 w = draw_words(it, (uint32_t)t, 0u, 0u, kg, kStreamControl, ctr);
        const float2 z = box_muller(w.x, w.y);
        const float e0 = dp.Le00 * z.x;
        const float e1 = fmaf(dp.Le10, z.x, dp.Le11 * z.y);
        const float v0 = v_s[2 * t], v1 = v_s[2 * t + 1];
        const float u0 = fminf(fmaxf(v0 + e0, dp.umin0), dp.umax0);
        const float u1 = fminf(fmaxf(v1 + e1, dp.umin1), dp.umax1);
        my_u[UPS * t] = u0;
        my_u[UPS * t + 1] = u1;
        if constexpr (TRIG) sincosf(u0, &my_u[UPS * t + 2], &my_u[UPS * t + 3]);
        if (active) reinterpret_cast<float2*>(io.eps)[(size_t)k * it.T + t] = make_float2(u0 - v0, u1 - v1);
    }
    __syncwarp();

    // Initial particles: the estimate x_bar_0, spread by Sigma_{x_0} when one is given.
    float x0[NX];
#pragma unroll
    for (int i = 0; i < NX; ++i) x0[i] = io.x0[i];
    const float s0 = (SI >= 0) ? x0[SI] : 0.0f;
    float x[P][NX];
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
        for (int i = 0; i < NX; ++i) x[p][i] = (i == SI) ? 0.0f : x0[i];
    float var0_ey = 0.0f;
    float var0[NX];
#pragma unroll
    for (int i = 0; i < NX; ++i) var0[i] = 0.0f;
    if (io.Sigma0 != nullptr) {
        float L0[NX][NX];
        cholesky_psd<NX>(io.Sigma0, L0);
#pragma unroll
        for (int i = 0; i < NX; ++i) var0[i] = io.Sigma0[i * NX + i];
        var0_ey = var0[EY];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            float xi[NX];
            draw_normals<NX>(it, 0u, (uint32_t)(ls + seg * p), kk, kStreamInitial, ctr, xi);
#pragma unroll
            for (int i = 0; i < NX; ++i) {
                float w = 0.0f;
#pragma unroll
                for (int j = 0; j <= i; ++j) w = fmaf(L0[i][j], xi[j], w);
                x[p][i] += w;
            }
        }
    }

    // Belief z_0 = (z_hat_0, z_hat_{-1} = z_hat_0) from the given estimate (Algorithm 1).
    float mean[NX], var[NX];
#pragma unroll
    for (int i = 0; i < NX; ++i) mean[i] = x0[i];
    bool general = false;
    float h_cur;
    if constexpr (FULL) {
        general = cs->n > 0;
        if (general) {
            float C0[NX * (NX + 1) / 2];
#pragma unroll
            for (int i = 0; i < NX; ++i)
#pragma unroll
                for (int j = 0; j <= i; ++j) C0[i * (i + 1) / 2 + j] = io.Sigma0 ? io.Sigma0[i * NX + j] : 0.0f;
            h_cur = general_barrier<NX, FCM>(*cs, mean, C0);
        } else {
            h_cur = belief_barrier(dp, mean[EY], var0_ey);
        }
    } else {
        h_cur = belief_barrier(dp, mean[EY], var0_ey);
    }
    float h_prev = h_cur;
    const bool writer = active && ls == 0;
    if (RECORDS && dp.record && writer) {
#pragma unroll
        for (int i = 0; i < NX; ++i) {
            io.mean[(size_t)k * (it.T + 1) * NX + i] = mean[i];
            io.var[(size_t)k * (it.T + 1) * NX + i] = var0[i];
        }
    }

    CompSum S;
    float S_naive = 0.0f;
    for (int t = 0; t < it.T; ++t) {
        // (a7) S += q(x_bar_t) + ctrl_w v_t^T Sigma_eps^-1 u_t + C_safe(z_t)
        const float u0 = my_u[UPS * t], u1 = my_u[UPS * t + 1];
        const float v0 = v_s[2 * t], v1 = v_s[2 * t + 1];
        const float ctrl = dp.ctrl_w * (v0 * fmaf(dp.Si00, u0, dp.Si01 * u1) + v1 * fmaf(dp.Si10, u0, dp.Si11 * u1));
        const float csafe = dp.Csafe * fmaxf(fmaf(dp.one_m_gamma, h_prev, -h_cur), 0.0f);
        float q;
        if constexpr (FULL) {
            q = general ? quad_cost<NX, MM>(dp, dp.Q, mean) + (any_constraint_broken<NX, FCM>(*cs, mean) ? dp.Cobs : 0.0f)
                        : state_cost<NX, EY>(dp, dp.Q, mean);
        } else {
            q = state_cost<NX, EY, MM>(dp, dp.Q, mean);
        }
        const float term = q + ctrl + csafe;
        if constexpr (COMP) S.add(term); else S_naive += term;

        // (a3, a4) propagate every particle: x <- f(x, u_t) + L_w z.
        Control c;
        c.steer = u0;
        c.accel = u1;
        if constexpr (TRIG) {
            c.sin_steer = my_u[UPS * t + 2];
            c.cos_steer = my_u[UPS * t + 3];
        } else if constexpr (MODEL != 1) {
            sincosf(u0, &c.sin_steer, &c.cos_steer);
        }
        if constexpr (MODEL != 1) {
            // the heading's sine and cosine: series at the step's start, rotated through the
            // substeps. With PACK, particles 2q and 2q + 1 of the lane share packed FP32 registers.
            constexpr int HI = MODEL == 0 ? 3 : 5;
            constexpr bool PAIRS = PACK && P % 2 == 0;
            using V = typename std::conditional<PAIRS, float2, float>::type;
            constexpr int NV = PAIRS ? P / 2 : P;
            using Ctl = typename std::conditional<MODEL == 0, SubstepCtl<V>, WheelsCtl<V>>::type;
            Ctl sc;
            if constexpr (MODEL == 0) sc = substep_ctl<V>(dp, c);
            else sc = wheels_ctl<V>(dp, c);
            V X[NV][NX], hs[NV], hc[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                if constexpr (PAIRS) {
#pragma unroll
                    for (int i = 0; i < NX; ++i) X[q][i] = make_float2(x[2 * q][i], x[2 * q + 1][i]);
                } else {
#pragma unroll
                    for (int i = 0; i < NX; ++i) X[q][i] = x[q][i];
                }
                sincos_series_v(dp, X[q][HI], hs[q], hc[q]);
            }
            for (int j = 0; j < dp.n_sub; ++j) {
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    if constexpr (MODEL == 0)
                        bicycle_substep<TYRE_POLY && P <= 2>(dp, it, kap_s, s0, sc, X[q], hs[q], hc[q]);
                    else wheels_substep(dp, it, kap_s, s0, sc, X[q], hs[q], hc[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < NV; ++q)
#pragma unroll
                for (int i = 0; i < NX; ++i) {
                    if constexpr (PAIRS) {
                        x[2 * q][i] = X[q][i].x;
                        x[2 * q + 1][i] = X[q][i].y;
                    } else {
                        x[q][i] = X[q][i];
                    }
                }
        } else {
#pragma unroll
            for (int p = 0; p < P; ++p) double_integrator_step(dp, c, x[p]);
        }
        if constexpr (NX == 6 && P >= 2) {
            // particles p and p + P/2 of this lane are n and n + H (H = seg P / 2): one counter
#pragma unroll
            for (int p = 0; p < P / 2; ++p) {
                float zl[NX], zh[NX];
                draw_disturbance_pair(it, (uint32_t)t, (uint32_t)(ls + seg * p), kk, ctr, zl, zh);
                if (dp.lw_diag) {
                    add_diagonal<NX>(dp.Lw, zl, x[p]);
                    add_diagonal<NX>(dp.Lw, zh, x[p + P / 2]);
                } else {
                    add_correlated<NX>(dp.Lw, zl, x[p]);
                    add_correlated<NX>(dp.Lw, zh, x[p + P / 2]);
                }
            }
        } else {
#pragma unroll
            for (int p = 0; p < P; ++p) {
                float z[NX];
                draw_disturbance<NX>(it, (uint32_t)t, (uint32_t)(ls + seg * p), kk, ctr, z);
                if (dp.lw_diag) add_diagonal<NX>(dp.Lw, z, x[p]);
                else add_correlated<NX>(dp.Lw, z, x[p]);
            }
        }

        // (a5) belief moments of step t+1, (a6) barrier.
        float h_next = 0.0f;
        if constexpr (FULL) {
            float C[NX * (NX + 1) / 2];
            belief_moments_full<NX, P, MM>(it, x, ls, seg, mean, C);
            if constexpr (MM == 0) {
#pragma unroll
                for (int i = 0; i < NX; ++i) var[i] = C[i * (i + 1) / 2 + i];
            } else {
                var[EY] = C[EY * (EY + 1) / 2 + EY];
            }
            if (general) {
                float ma[NX];
#pragma unroll
                for (int i = 0; i < NX; ++i) ma[i] = mean[i];
                if constexpr (SI >= 0) ma[SI] += s0;
                h_next = general_barrier<NX, FCM>(*cs, ma, C);
            }
            if (MM == 0 && dp.resample && t + 1 < it.T) {  // re-draw x^n_{t+1} ~ N(mean, cov) for the next step (stream 4)
                cholesky_packed_psd<NX>(C);
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    float xi[NX];
                    draw_normals<NX>(it, (uint32_t)(t + 1), (uint32_t)(ls + seg * p), kk, kStreamResample, ctr, xi);
#pragma unroll
                    for (int i = 0; i < NX; ++i) x[p][i] = mean[i];
                    add_correlated<NX>(C, xi, x[p]);
                }
            }
        } else {
            belief_moments<NX, EY, P, COMP, MM>(dp, it, x, ls, seg, RECORDS && dp.record != 0, mean, var);
        }
        if constexpr (SI >= 0 && (MM == 0 || ((MM >> SI) & 1))) mean[SI] += s0;
        h_prev = h_cur;
        h_cur = general ? h_next : belief_barrier(dp, mean[EY], var[EY]);
        if (RECORDS && dp.record && writer) {
            const size_t base = ((size_t)k * (it.T + 1) + t + 1) * NX;
#pragma unroll
            for (int i = 0; i < NX; ++i) {
                io.mean[base + i] = mean[i];
                io.var[base + i] = var[i];
            }
        }
    }
    // Terminal: phi(x_bar_T) + C_safe(z_T).
    float qT;
    if constexpr (FULL) {
        qT = general ? quad_cost<NX, MM>(dp, dp.Qf, mean) + (any_constraint_broken<NX, FCM>(*cs, mean) ? dp.Cobs : 0.0f)
                     : state_cost<NX, EY>(dp, dp.Qf, mean);
    } else {
        qT = state_cost<NX, EY, MM>(dp, dp.Qf, mean);
    }
    const float term = qT + dp.Csafe * fmaxf(fmaf(dp.one_m_gamma, h_prev, -h_cur), 0.0f);
    float total;
    if constexpr (COMP) {
        S.add(term);
        total = S.value();
    } else {
        total = S_naive + term;
    }
    if (writer) io.S[k] = total;
    return total;
}

}  // namespace bss
