// Launch planning and dispatch of the per-solve rollout kernel (its templates are in
// rollout_kernel.cuh, instantiated per model in rollout_model0/1/2.cu), the merge kernel of a
// sample-sharded solve, and the small checking kernels (model step, Philox, Box-Muller).
#include "rollout_kernel.cuh"

#include <algorithm>

namespace bss {

// One block merges the partials of G sample shards (the exchange of a sample-sharded solve).
template <bool COMP>
__global__ void __launch_bounds__(512) merge_partials_kernel(const int G, const float* parts, const int K,
                                                             const float K_norm, const int T, const float lambda,
                                                             const float inv_lambda, const float* S, const TailIO tail)
{
    extern __shared__ float smem[];
    __shared__ float fac_s[kTailMaxBlocks];
    __shared__ float red_e[kTailMaxBlocks], red_q[kTailMaxBlocks];
    __shared__ float bc_s[3];
    const int TN = 2 * T;
    float* v_s = smem;
    float* red = smem + TN;
    for (int i = threadIdx.x; i < TN; i += blockDim.x) v_s[i] = tail.v_out[i];
    __syncthreads();
    tail_merge<COMP>(G, parts, K, K_norm, T, lambda, inv_lambda, S, tail, v_s, red, fac_s, red_e, red_q, bc_s);
}

cudaError_t merge_partials_launch(const DevParams& dp, int G, const float* parts, bool comp, const float* S,
                                  const TailIO& tail, cudaStream_t st)
{
    if (G < 1 || G > kTailMaxBlocks) return cudaErrorInvalidValue;
    const int threads = 512;
    const size_t smem = sizeof(float) * (2 * (size_t)dp.T + std::max<size_t>(2 * (size_t)dp.T, threads));
    const float Kn = (float)dp.K_norm;
    if (comp)
        merge_partials_kernel<true><<<1, threads, smem, st>>>(G, parts, dp.K, Kn, dp.T, dp.lambda, dp.inv_lambda, S, tail);
    else
        merge_partials_kernel<false><<<1, threads, smem, st>>>(G, parts, dp.K, Kn, dp.T, dp.lambda, dp.inv_lambda, S, tail);
    return cudaGetLastError();
}

// Dynamic shared memory of the rollout kernel at wpb warps per block: the curvature table as
// (value, difference) pairs, the nominal (2T), each segment's controls with the steering angle's
// sine and cosine (4T per segment) and the tail's scratch.
size_t rollout_smem_bytes(const DevParams& dp, int wpb)
{
    const int ntab = dp.n_track_mask + 1;
    const size_t TN = 2 * (size_t)dp.T;
    const size_t floats = (size_t)((2 * ntab + 3) & ~3) + TN + (size_t)wpb * dp.spw * 2 * TN
                        + std::max(TN, (size_t)wpb * kWarp);
    return floats * sizeof(float);
}

// Variants: the racing barrier on persistent particles, with compensated or naive reductions; and
// the full-belief variant (re-sampled particles and/or the general constraint set), always with
// the compensated sums (the host rejects it with naive reductions).
cudaError_t rollout_prepare(const DevParams& dp, int P, bool comp, bool full, RollLaunch& L, const ConSet* cs)
{
    if (full && !comp) return cudaErrorInvalidValue;
    if (dp.nx == 8) return prepare_model<2>(dp, P, comp, full, L, cs);
    if (dp.nx == 6) return prepare_model<0>(dp, P, comp, full, L, cs);
    return prepare_model<1>(dp, P, comp, full, L, cs);
}

cudaError_t rollout_launch(const DevParams& dp, int P, bool comp, const RollLaunch& L, const float* x0,
                           const float* Sigma0, const float* v, const uint32_t* ctr, float* S, float* eps, float* mean,
                           float* var, const TailIO& tail, const ConSet& cs, cudaStream_t st)
{
    RollIO io{x0, Sigma0, v, ctr, S, eps, mean, var};
    const bool full = dp.resample || cs.n > 0;
    if (full && !comp) return cudaErrorInvalidValue;
    if (dp.nx == 8) return launch_model_variant<2>(dp, io, tail, cs, P, comp, full, L, st);
    if (dp.nx == 6) return launch_model_variant<0>(dp, io, tail, cs, P, comp, full, L, st);
    return launch_model_variant<1>(dp, io, tail, cs, P, comp, full, L, st);
}

// Model step for n independent states, plus an optional additive disturbance (model checks and
// simulated plants).
template <int MODEL>
__global__ void model_step_kernel(const DevParams dp, const float* __restrict__ xin, const float* __restrict__ uin,
                                  const float* __restrict__ win, float* __restrict__ xout, int64_t n)
{
    constexpr int NX = model_nx(MODEL);
    constexpr int SI = model_s_index(MODEL);
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
    if constexpr (SI >= 0) {
        s0 = x[SI];
        x[SI] = 0.0f;
    }
    model_step<MODEL, NX>(dp, dp.kappa, s0, c, x);
    if constexpr (SI >= 0) x[SI] += s0;
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
    else if (dp.nx == 8) model_step_kernel<2><<<grid, threads, 0, st>>>(dp, x, u, w, xn, n);
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

__global__ void slip_atan_kernel(const float* __restrict__ t, float* __restrict__ y, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = slip_atan(t[i]);
}

__global__ void tyre_curve_kernel(const DevParams dp, const float* __restrict__ x, float* __restrict__ y, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = tyre_curve(dp, x[i]);
}

cudaError_t tyre_curve_launch(const DevParams& dp, const float* x, float* y, int64_t n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    tyre_curve_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(dp, x, y, n);
    return cudaGetLastError();
}

// Pairs of values through the packed form (the single-solve kernel's two particles per lane); an odd
// last value alone.
__global__ void rear_tyre_kernel(const DevParams dp, const float* __restrict__ t, float* __restrict__ y, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * i + 1 < n) {
        const float2 g = rear_tyre(dp, make_float2(t[2 * i], t[2 * i + 1]));
        y[2 * i] = g.x;
        y[2 * i + 1] = g.y;
    } else if (2 * i < n) {
        y[2 * i] = rear_tyre(dp, t[2 * i]);
    }
}

cudaError_t rear_tyre_launch(const DevParams& dp, const float* t, float* y, int64_t n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    const int64_t pairs = (n + 1) / 2;
    rear_tyre_kernel<<<(unsigned)((pairs + threads - 1) / threads), threads, 0, st>>>(dp, t, y, n);
    return cudaGetLastError();
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

cudaError_t slip_atan_launch(const float* t, float* y, int64_t n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    slip_atan_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(t, y, n);
    return cudaGetLastError();
}

}  // namespace bss
