// The persistent rollout kernel and its fused weights/update tail, with its launch planning, as
// templates. Each model's instantiations live in a translation unit of their own
// (rollout_model0/1/2.cu) so that they compile in parallel; rollout.cu dispatches to them.
#pragma once

#include "device.cuh"
#include "internal.h"
#include "rollout_body.cuh"

#include <algorithm>

namespace bss {

// Merge of G log-sum-exp partials {beta_g, eta_g, q_g, N_g[2T]} (stride 3 + 2T from `part`) in
// order: the rollout's last block merges its blocks' partials, the merge kernel those of several
// sample shards. Writes v+ = v + N / eta, u0, the weights of the K local costs S, the diagnostics
// (K_norm samples in all) and the counter, or, with tail.part_out set, only the merged partial and
// the counter. Out of line so that its registers do not weigh on the rollout loop. red: max(2T,
// threads) floats of shared scratch; fac_s, red_e, red_q: G floats each (G <= kTailMaxBlocks).
constexpr int kTailBatch = 8;  // independent L2 loads a thread keeps in flight in the merge

template <bool COMP>
__device__ __noinline__ void tail_merge(const int G, const float* part, const int K, const float K_norm, const int T,
                                        const float lambda, const float inv_lambda, const float* S,
                                        const TailIO tail, const float* v_s, float* red, float* fac_s, float* red_e,
                                        float* red_q, float* bc_s)
{
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int warp = tid / kWarp, lane = tid & (kWarp - 1), wpb = nthr / kWarp;
    const int TN = 2 * T;
    const size_t stride = 3 + TN;
    // beta = min over blocks, then every block's factor exp(-(beta_b - beta)/lambda)
    float b = INFINITY;
    for (int g = tid; g < G; g += nthr) b = fminf(b, __ldcg(part + g * stride));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) b = fminf(b, __shfl_xor_sync(0xffffffffu, b, off));
    if (lane == 0) red[warp] = b;
    __syncthreads();
    if (tid == 0) {
        float x = red[0];
        for (int w = 1; w < wpb; ++w) x = fminf(x, red[w]);
        bc_s[0] = x;
    }
    __syncthreads();
    const float beta = bc_s[0];
    for (int g = tid; g < G; g += nthr) {
        const float bg = __ldcg(part + g * stride);
        const float f = (bg < INFINITY) ? expf((beta - bg) * inv_lambda) : 0.0f;
        fac_s[g] = f;
        red_e[g] = __ldcg(part + g * stride + 1) * f;
        red_q[g] = __ldcg(part + g * stride + 2) * f * f;
    }
    __syncthreads();
    if (warp == 0) {  // eta and sum of squares: lane l adds blocks l, l+32, ... then a fixed tree
        CompSum e, q;
        float e_n = 0.0f, q_n = 0.0f;
        for (int g = lane; g < G; g += kWarp) {
            if constexpr (COMP) {
                e.add(red_e[g]);
                q.add(red_q[g]);
            } else {
                e_n += red_e[g];
                q_n += red_q[g];
            }
        }
        float es = COMP ? e.s : e_n, ec = COMP ? e.c : 0.0f, qs = COMP ? q.s : q_n, qc = COMP ? q.c : 0.0f;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const float es2 = __shfl_xor_sync(0xffffffffu, es, off), ec2 = __shfl_xor_sync(0xffffffffu, ec, off);
            const float qs2 = __shfl_xor_sync(0xffffffffu, qs, off), qc2 = __shfl_xor_sync(0xffffffffu, qc, off);
            comp_merge(es, ec, es2, ec2);
            comp_merge(qs, qc, qs2, qc2);
        }
        if (lane == 0) {
            bc_s[1] = es + ec;
            bc_s[2] = qs + qc;
        }
    }
    // sum_b N_b[i] f_b: thread (group, i) adds blocks group, group + NG, ...; then the NG group sums
    const int NG = max(1, nthr / TN);
    for (int idx = tid; idx < TN * NG; idx += nthr) {
        const int i = idx % TN, grp = idx / TN;
        CompSum n;
        float n_n = 0.0f;
        for (int g0 = grp; g0 < G; g0 += kTailBatch * NG) {  // loads of a batch in flight together
            float x[kTailBatch];
#pragma unroll
            for (int j = 0; j < kTailBatch; ++j) {
                const int g = g0 + j * NG;
                x[j] = g < G ? __ldcg(part + g * stride + 3 + i) * fac_s[g] : 0.0f;
            }
#pragma unroll
            for (int j = 0; j < kTailBatch; ++j) {
                if constexpr (COMP) n.add(x[j]); else n_n += x[j];
            }
        }
        red[grp * TN + i] = COMP ? n.value() : n_n;
    }
    __syncthreads();
    const float eta = bc_s[1], sumsq = bc_s[2];
    for (int i = tid; i < TN; i += nthr) {
        CompSum n;
        float n_n = 0.0f;
        for (int grp = 0; grp < NG; ++grp) {
            if constexpr (COMP) n.add(red[grp * TN + i]); else n_n += red[grp * TN + i];
        }
        const float N = COMP ? n.value() : n_n;
        if (tail.part_out != nullptr) {  // a shard's partial: the update waits for the other shards
            tail.part_out[3 + i] = N;
            continue;
        }
        const float vn = v_s[i] + N / eta;
        if (tail.u0 != nullptr && i < 2) tail.u0[i] = vn;
        if (tail.shift_n == 0) {
            tail.v_out[i] = vn;
        } else {  // the warm-start shift in the same launch: v[t] <- v+[min(t + n, T - 1)]
            const int t = i >> 1, c = i & 1, n = tail.shift_n;
            if (t >= n) tail.v_out[2 * (t - n) + c] = vn;
            if (t == T - 1)
                for (int tt = max(T - n, 0); tt < T; ++tt) tail.v_out[2 * tt + c] = vn;
        }
    }
    if (tail.part_out != nullptr) {
        if (tid == 0) {
            tail.part_out[0] = beta;
            tail.part_out[1] = eta;
            tail.part_out[2] = sumsq;
            if (tail.ctr_out != nullptr) *tail.ctr_out += 1u;
            if (tail.ticket != nullptr) *tail.ticket = 0u;
        }
        return;
    }
    for (int k0 = tid; k0 < K; k0 += kTailBatch * nthr) {
        float s[kTailBatch];
#pragma unroll
        for (int j = 0; j < kTailBatch; ++j) s[j] = k0 + j * nthr < K ? __ldcg(S + k0 + j * nthr) : 0.0f;
#pragma unroll
        for (int j = 0; j < kTailBatch; ++j) {
            if (k0 + j * nthr < K) tail.w[k0 + j * nthr] = expf(-(s[j] - beta) * inv_lambda) / eta;
        }
    }
    if (tid == 0) {
        if (tail.diag != nullptr) {
            tail.diag[0] = beta;
            tail.diag[1] = eta;
            tail.diag[2] = eta * eta / sumsq;
            tail.diag[3] = beta - lambda * logf(eta / K_norm);
        }
        if (tail.ctr_out != nullptr) *tail.ctr_out += 1u;
        if (tail.ticket != nullptr) *tail.ticket = 0u;
    }
}

// A block's partial of the weights/update over the samples it rolled out, read back from S and
// eps (written by the block's own warps, still in L2): beta_b = min S, eta_b = sum exp(-(S - beta_b)/
// lambda), q_b = sum of their squares, N_b[i] = sum exp(-(S - beta_b)/lambda) eps[i]. Samples are taken
// in a fixed order (t -> round j, warp w, slot s), so the result does not depend on timing. red:
// max(2T, threads) floats of shared scratch.
template <bool COMP>
__device__ __noinline__ void block_partial(const int K, const int T, const int spw, const float inv_lambda,
                                           const float* S, const float* eps, float* part, float* red, float* bc_s)
{
    const int tid = threadIdx.x, nthr = blockDim.x, wpb = nthr / kWarp;
    const int warp = tid / kWarp, lane = tid & (kWarp - 1);
    const int TN = 2 * T;
    const int n_groups = (K + spw - 1) / spw;
    const int rounds = (n_groups + gridDim.x * wpb - 1) / (gridDim.x * wpb);
    const int nb = rounds * wpb * spw;  // candidate samples of this block (some past K)
    auto sample = [&](int t) -> int {   // global sample index of block-local t, or -1
        const int s = t % spw, jw = t / spw;
        const int g = blockIdx.x * wpb + (jw % wpb) + (jw / wpb) * gridDim.x * wpb;
        const int k = g * spw + s;
        return (g < n_groups && k < K) ? k : -1;
    };
    // beta_b
    float b = INFINITY;
    for (int t = tid; t < nb; t += nthr) {
        const int k = sample(t);
        if (k >= 0) b = fminf(b, __ldcg(S + k));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) b = fminf(b, __shfl_xor_sync(0xffffffffu, b, off));
    if (lane == 0) red[warp] = b;
    __syncthreads();
    if (tid == 0) {
        float x = red[0];
        for (int w = 1; w < wpb; ++w) x = fminf(x, red[w]);
        bc_s[0] = x;
    }
    __syncthreads();
    const float beta = bc_s[0];
    if (!(beta < INFINITY)) {  // no samples in this block
        for (int i = tid; i < 3 + TN; i += nthr) part[i] = i == 0 ? INFINITY : 0.0f;
        return;
    }
    // eta_b and q_b: thread sums over t = tid, tid + nthr, ...; fixed trees over lanes, then warps
    {
        CompSum e, q;
        float e_n = 0.0f, q_n = 0.0f;
        for (int t = tid; t < nb; t += nthr) {
            const int k = sample(t);
            if (k < 0) continue;
            const float w = expf(-(__ldcg(S + k) - beta) * inv_lambda);
            if constexpr (COMP) {
                e.add(w);
                q.add(w * w);
            } else {
                e_n += w;
                q_n = fmaf(w, w, q_n);
            }
        }
        float es = COMP ? e.s : e_n, ec = COMP ? e.c : 0.0f, qs = COMP ? q.s : q_n, qc = COMP ? q.c : 0.0f;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const float es2 = __shfl_xor_sync(0xffffffffu, es, off), ec2 = __shfl_xor_sync(0xffffffffu, ec, off);
            const float qs2 = __shfl_xor_sync(0xffffffffu, qs, off), qc2 = __shfl_xor_sync(0xffffffffu, qc, off);
            comp_merge(es, ec, es2, ec2);
            comp_merge(qs, qc, qs2, qc2);
        }
        __syncthreads();  // red[] reads of the beta reduction are done
        if (lane == 0) {
            red[4 * warp + 0] = es;
            red[4 * warp + 1] = ec;
            red[4 * warp + 2] = qs;
            red[4 * warp + 3] = qc;
        }
        __syncthreads();
        if (tid == 0) {
            float es0 = red[0], ec0 = red[1], qs0 = red[2], qc0 = red[3];
            for (int w = 1; w < wpb; ++w) {
                comp_merge(es0, ec0, red[4 * w], red[4 * w + 1]);
                comp_merge(qs0, qc0, red[4 * w + 2], red[4 * w + 3]);
            }
            part[0] = beta;
            part[1] = es0 + ec0;
            part[2] = qs0 + qc0;
        }
        __syncthreads();  // red[] is reused below
    }
    // N_b[i]: thread (sub, i) adds t = sub, sub + NG, ... (loads of a batch in flight together);
    // then the NG sub-sums in order
    const int NG = max(1, nthr / TN);
    for (int idx = tid; idx < TN * NG; idx += nthr) {
        const int i = idx % TN, sub = idx / TN;
        CompSum n;
        float n_n = 0.0f;
        for (int t0 = sub; t0 < nb; t0 += kTailBatch * NG) {
            float x[kTailBatch];
#pragma unroll
            for (int j = 0; j < kTailBatch; ++j) {
                const int t = t0 + j * NG;
                const int k = t < nb ? sample(t) : -1;
                x[j] = k >= 0 ? expf(-(__ldcg(S + k) - beta) * inv_lambda) * __ldcg(eps + (size_t)k * TN + i) : 0.0f;
            }
#pragma unroll
            for (int j = 0; j < kTailBatch; ++j) {
                if constexpr (COMP) n.add(x[j]); else n_n += x[j];
            }
        }
        red[sub * TN + i] = COMP ? n.value() : n_n;
    }
    __syncthreads();
    for (int i = tid; i < TN; i += nthr) {
        CompSum n;
        float n_n = 0.0f;
        for (int sub = 0; sub < NG; ++sub) {
            if constexpr (COMP) n.add(red[sub * TN + i]); else n_n += red[sub * TN + i];
        }
        part[3 + i] = COMP ? n.value() : n_n;
    }
}

// Persistent rollout with the weights and update fused into its tail.
//
// The block's warps walk the sample groups with a grid stride; the curvature table and the nominal
// sequence are staged in shared memory once per block. Weights (Eq. "Weights") and update (Eq.
// "MPPI update law") follow the last group without a second launch: every block publishes the
// log-sum-exp partial of its own samples (block_partial), and the last block to arrive (atomic
// ticket) merges the partials in block order and writes v+ = v + N / eta, u0, the normalised weights,
// the diagnostics and the counter (tail_merge). No block waits for another. MM: the cost's states
// when fixed at compile time (rollout_group), else 0.
template <int MODEL, int P, bool COMP, bool FULL, int MM = 0>
__global__ void __launch_bounds__(roll_max_threads<MODEL, P>()) rollout_kernel(const DevParams dp, const RollIO io,
                                                                       const TailIO tail, const ConSet cs)
{
    extern __shared__ float smem[];
    __shared__ float fac_s[kTailMaxBlocks];
    __shared__ float red_e[kTailMaxBlocks], red_q[kTailMaxBlocks];
    __shared__ float bc_s[3];
    __shared__ bool is_last;
    const int ntab = dp.n_track_mask + 1;
    const int TN = 2 * dp.T;
    const int wpb = blockDim.x / kWarp;
    // curvature table as (kappa_i, kappa_{i+1} - kappa_i) pairs: one 8-byte load per lookup
    float2* kap_s = reinterpret_cast<float2*>(smem);
    float* v_s = smem + ((2 * ntab + 3) & ~3);
    float* u_s = v_s + TN;
    float* red = u_s + (size_t)wpb * dp.spw * 2 * TN;  // tail scratch: max(TN, threads) floats

    if constexpr (MODEL != 1) {
        for (int i = threadIdx.x; i < ntab; i += blockDim.x) {
            const float k0 = dp.kappa[i];
            kap_s[i] = make_float2(k0, dp.kappa[i + 1] - k0);
        }
    }
    for (int i = threadIdx.x; i < TN; i += blockDim.x) v_s[i] = io.v[i];
    __syncthreads();

    const uint32_t ctr = *io.ctr;
    const int warp = threadIdx.x / kWarp;
    const int lane = threadIdx.x & (kWarp - 1);
    float* my_u = u_s + (warp * dp.spw + lane / dp.seg) * 2 * TN;  // T x (u_0, u_1, sin u_0, cos u_0)
    const int n_groups = (dp.K + dp.spw - 1) / dp.spw;
    for (int group = blockIdx.x * wpb + warp; group < n_groups; group += gridDim.x * wpb)
        rollout_group<MODEL, P, COMP, FULL, float2, true, true, DevParams, true, MM>(dp, dp, io, kap_s, v_s, my_u,
                                                                                   group, ctr, &cs);
    __syncthreads();

    float* part = tail.part + (size_t)blockIdx.x * (3 + TN);
    block_partial<COMP>(dp.K, dp.T, dp.spw, dp.inv_lambda, io.S, io.eps, part, red, bc_s);

    // The last block to arrive merges the block partials in block order.
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(tail.ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    tail_merge<COMP>(gridDim.x, tail.part, dp.K, (float)dp.K_norm, dp.T, dp.lambda, dp.inv_lambda, io.S, tail, v_s,
                     red, fac_s, red_e, red_q, bc_s);
}

template <int MODEL, int P, bool COMP, bool FULL, int MM>
inline cudaError_t launch_one(const DevParams& dp, const RollIO& io, const TailIO& tail, const ConSet& cs,
                              const RollLaunch& L, cudaStream_t st)
{
    if (L.grid > kTailMaxBlocks) return cudaErrorInvalidValue;
    rollout_kernel<MODEL, P, COMP, FULL, MM><<<L.grid, L.wpb * kWarp, L.smem, st>>>(dp, io, tail, cs);
    return cudaGetLastError();
}

template <int MODEL, bool COMP, bool FULL, int MM = 0>
inline cudaError_t launch_model(const DevParams& dp, const RollIO& io, const TailIO& tail, const ConSet& cs, int P,
                                const RollLaunch& L, cudaStream_t st)
{
    switch (P) {
    case 1: return launch_one<MODEL, 1, COMP, FULL, MM>(dp, io, tail, cs, L, st);
    case 2: return launch_one<MODEL, 2, COMP, FULL, MM>(dp, io, tail, cs, L, st);
    case 4: return launch_one<MODEL, 4, COMP, FULL, MM>(dp, io, tail, cs, L, st);
    case 8:
        if constexpr (MODEL != 2) return launch_one<MODEL, 8, COMP, FULL, MM>(dp, io, tail, cs, L, st);
        else return cudaErrorInvalidValue;  // the wheel-speed model takes M <= 128
    default: return cudaErrorInvalidValue;
    }
}

// Block shape: one block per SM with w warps, w chosen to minimise the makespan of an issue-bound
// kernel, ceil(groups / (SMs w)) rounds of max(w, kSatWarps) warp-times each, among the w that fit
// on an SM (fewer than kSatWarps warps leave issue slots idle on latency).
constexpr int kSatWarps = 16;
template <int MODEL, int P, bool COMP, bool FULL, int MM>
inline cudaError_t plan_one(const DevParams& dp, RollLaunch& L)
{
    auto kern = rollout_kernel<MODEL, P, COMP, FULL, MM>;
    int dev = 0, sms = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes attr{};
    e = cudaFuncGetAttributes(&attr, kern);
    if (e != cudaSuccess) return e;
    sms = std::min(sms, kTailMaxBlocks);
    const int max_w = roll_max_threads<MODEL, P>() / kWarp;
    const size_t optin_dynamic = (size_t)optin > attr.sharedSizeBytes ? (size_t)optin - attr.sharedSizeBytes : 0;
    const size_t smem_cap = std::min(rollout_smem_bytes(dp, max_w), optin_dynamic);
    if (rollout_smem_bytes(dp, 1) > smem_cap) return cudaErrorInvalidValue;  // one warp's share does not fit
    if (smem_cap > 48 * 1024) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cap);
        if (e != cudaSuccess) return e;
    }
    const long groups = (dp.K + dp.spw - 1) / dp.spw;
    long best_cost = -1;
    int best_w = 1;
    for (int w = max_w; w >= 1; --w) {
        if (rollout_smem_bytes(dp, w) > smem_cap) continue;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, w * kWarp, rollout_smem_bytes(dp, w));
        if (e != cudaSuccess) return e;
        if (nb < 1) continue;
        // an SM issues at full rate once about kSatWarps warps hide each other's latency: a round
        // of w warps costs max(w, kSatWarps)
        const long slots = (long)sms * w;
        const long cost = ((groups + slots - 1) / slots) * std::max(w, kSatWarps);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best_w = w;
        }
    }
    L.wpb = best_w;
    L.grid = (int)std::min<long>(sms, (groups + best_w - 1) / best_w);
    L.smem = rollout_smem_bytes(dp, best_w);
    L.cost_mask = MM;
    return cudaSuccess;
}

template <int MODEL, bool COMP, bool FULL, int MM = 0>
inline cudaError_t plan_model(const DevParams& dp, int P, RollLaunch& L)
{
    switch (P) {
    case 1: return plan_one<MODEL, 1, COMP, FULL, MM>(dp, L);
    case 2: return plan_one<MODEL, 2, COMP, FULL, MM>(dp, L);
    case 4: return plan_one<MODEL, 4, COMP, FULL, MM>(dp, L);
    case 8:
        if constexpr (MODEL != 2) return plan_one<MODEL, 8, COMP, FULL, MM>(dp, L);
        else return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

// Per-model entry points (defined in rollout_model<MODEL>.cu): the launch plan and the launch of
// the racing-barrier variants (compensated or naive reductions) and the full-belief variant.
template <int MODEL>
cudaError_t prepare_model(const DevParams& dp, int P, bool comp, bool full, RollLaunch& L, const ConSet* cs);
template <int MODEL>
cudaError_t launch_model_variant(const DevParams& dp, const RollIO& io, const TailIO& tail, const ConSet& cs, int P,
                                 bool comp, bool full, const RollLaunch& L, cudaStream_t st);

}  // namespace bss
