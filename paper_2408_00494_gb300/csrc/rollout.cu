// Per-solve rollout kernel (persistent grid over the sample groups of one controller), its launch
// planning, and the small checking kernels (model step, Philox, Box-Muller). The per-group body
// is in rollout_body.cuh.
#include "device.cuh"
#include "internal.h"
#include "rollout_body.cuh"

#include <algorithm>

namespace bss {

// Persistent rollout: the block's warps walk the sample groups with a grid stride. The curvature
// table and the nominal sequence are staged in shared memory once per block.
template <int MODEL, int P, bool COMP>
__global__ void __launch_bounds__(roll_max_threads<P>()) rollout_kernel(const DevParams dp, const RollIO io)
{
    extern __shared__ float smem[];
    const int ntab = dp.n_track_mask + 1;
    float* kap_s = smem;
    float* v_s = smem + ((ntab + 1 + 3) & ~3);
    float* u_s = v_s + 2 * dp.T;

    if constexpr (MODEL == 0) {
        for (int i = threadIdx.x; i <= ntab; i += blockDim.x) kap_s[i] = dp.kappa[i];
    }
    for (int i = threadIdx.x; i < 2 * dp.T; i += blockDim.x) v_s[i] = io.v[i];
    __syncthreads();

    const uint32_t ctr = *io.ctr;
    const int warp = threadIdx.x / kWarp;
    const int wpb = blockDim.x / kWarp;
    const int lane = threadIdx.x & (kWarp - 1);
    float* my_u = u_s + (warp * dp.spw + lane / dp.seg) * 2 * dp.T;
    const int n_groups = (dp.K + dp.spw - 1) / dp.spw;
    for (int group = blockIdx.x * wpb + warp; group < n_groups; group += gridDim.x * wpb) {
        rollout_group<MODEL, P, COMP>(dp, io, kap_s, v_s, my_u, group, ctr);
        __syncwarp();  // the next group's prologue rewrites my_u
    }
}

size_t rollout_smem_bytes(const DevParams& dp, int wpb)
{
    const int ntab = dp.n_track_mask + 1;
    const size_t floats = (size_t)((ntab + 1 + 3) & ~3) + 2 * (size_t)dp.T + (size_t)wpb * dp.spw * 2 * dp.T;
    return floats * sizeof(float);
}

template <int MODEL, int P, bool COMP>
static cudaError_t launch_one(const DevParams& dp, const RollIO& io, const RollLaunch& L, cudaStream_t st)
{
    rollout_kernel<MODEL, P, COMP><<<L.grid, L.wpb * kWarp, L.smem, st>>>(dp, io);
    return cudaGetLastError();
}

template <int MODEL, bool COMP>
static cudaError_t launch_model(const DevParams& dp, const RollIO& io, int P, const RollLaunch& L, cudaStream_t st)
{
    switch (P) {
    case 1: return launch_one<MODEL, 1, COMP>(dp, io, L, st);
    case 2: return launch_one<MODEL, 2, COMP>(dp, io, L, st);
    case 4: return launch_one<MODEL, 4, COMP>(dp, io, L, st);
    case 8: return launch_one<MODEL, 8, COMP>(dp, io, L, st);
    default: return cudaErrorInvalidValue;
    }
}

// Block shape: one block per SM with w warps, w chosen to minimise the makespan of an issue-bound
// kernel, ceil(groups / (SMs w)) rounds of w warps each, among the w that fit on an SM.
template <int MODEL, int P, bool COMP>
static cudaError_t plan_one(const DevParams& dp, RollLaunch& L)
{
    auto kern = rollout_kernel<MODEL, P, COMP>;
    int dev = 0, sms = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const int max_w = roll_max_threads<P>() / kWarp;
    const size_t smem_cap = std::min(rollout_smem_bytes(dp, max_w), (size_t)optin);
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
        const long slots = (long)sms * w;
        const long cost = ((groups + slots - 1) / slots) * w;
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best_w = w;
        }
    }
    L.wpb = best_w;
    L.grid = (int)std::min<long>(sms, (groups + best_w - 1) / best_w);
    L.smem = rollout_smem_bytes(dp, best_w);
    return cudaSuccess;
}

template <int MODEL, bool COMP>
static cudaError_t plan_model(const DevParams& dp, int P, RollLaunch& L)
{
    switch (P) {
    case 1: return plan_one<MODEL, 1, COMP>(dp, L);
    case 2: return plan_one<MODEL, 2, COMP>(dp, L);
    case 4: return plan_one<MODEL, 4, COMP>(dp, L);
    case 8: return plan_one<MODEL, 8, COMP>(dp, L);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t rollout_prepare(const DevParams& dp, int P, bool comp, RollLaunch& L)
{
    if (dp.nx == 6) return comp ? plan_model<0, true>(dp, P, L) : plan_model<0, false>(dp, P, L);
    return comp ? plan_model<1, true>(dp, P, L) : plan_model<1, false>(dp, P, L);
}

cudaError_t rollout_launch(const DevParams& dp, int P, bool comp, const RollLaunch& L, const float* x0,
                           const float* Sigma0, const float* v, const uint32_t* ctr, float* S, float* eps, float* mean,
                           float* var, cudaStream_t st)
{
    RollIO io{x0, Sigma0, v, ctr, S, eps, mean, var};
    if (dp.nx == 6) return comp ? launch_model<0, true>(dp, io, P, L, st) : launch_model<0, false>(dp, io, P, L, st);
    return comp ? launch_model<1, true>(dp, io, P, L, st) : launch_model<1, false>(dp, io, P, L, st);
}

// Model step for n independent states, plus an optional additive disturbance (model checks and
// simulated plants).
template <int MODEL>
__global__ void model_step_kernel(const DevParams dp, const float* __restrict__ xin, const float* __restrict__ uin,
                                  const float* __restrict__ win, float* __restrict__ xout, int64_t n)
{
    constexpr int NX = MODEL == 0 ? 6 : 4;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x[NX];
#pragma unroll
    for (int j = 0; j < NX; ++j) x[j] = xin[i * NX + j];
    Control c;
    c.steer = uin[2 * i];
    c.accel = uin[2 * i + 1];
    sincosf(c.steer, &c.sin_steer, &c.cos_steer);
    float s0 = 0.0f;
    if constexpr (MODEL == 0) {
        s0 = x[5];
        x[5] = 0.0f;
    }
    model_step<MODEL, NX>(dp, dp.kappa, s0, c, x);
    if constexpr (MODEL == 0) x[5] += s0;
#pragma unroll
    for (int j = 0; j < NX; ++j) xout[i * NX + j] = x[j] + (win != nullptr ? win[i * NX + j] : 0.0f);
}

cudaError_t model_step_launch(const DevParams& dp, const float* x, const float* u, const float* w, float* xn, int64_t n,
                              cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int threads = 128;
    const dim3 grid((unsigned)((n + threads - 1) / threads));
    if (dp.nx == 6) model_step_kernel<0><<<grid, threads, 0, st>>>(dp, x, u, w, xn, n);
    else model_step_kernel<1><<<grid, threads, 0, st>>>(dp, x, u, w, xn, n);
    return cudaGetLastError();
}

__global__ void philox_kernel(const uint4* __restrict__ ctr, uint32_t k0, uint32_t k1, uint4* __restrict__ out, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctr[i], k0, k1);
}

__global__ void box_muller_kernel(const uint2* __restrict__ words, float2* __restrict__ z, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) z[i] = box_muller(words[i].x, words[i].y);
}

cudaError_t philox_launch(const uint32_t* ctr, uint64_t seed, uint32_t* out, int64_t n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    philox_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(
        reinterpret_cast<const uint4*>(ctr), (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32),
        reinterpret_cast<uint4*>(out), n);
    return cudaGetLastError();
}

cudaError_t box_muller_launch(const uint32_t* words, float* z, int64_t n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    box_muller_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(
        reinterpret_cast<const uint2*>(words), reinterpret_cast<float2*>(z), n);
    return cudaGetLastError();
}

}  // namespace bss
