// Importance weights and control update (Eq. "Weights", Eq. "MPPI update law"):
//   beta = min_k S_k, omega_k = exp(-(S_k - beta) / lambda), eta = sum_k omega_k,
//   v+_t = v_t + sum_k (omega_k / eta) eps_eff_{k,t}   (= sum_k omega_k u_k / eta, since the
//   normalised weights sum to one), then u0 = v+_0 and the solve counter advances.
//
// One launch of G blocks. Every block first reduces beta and eta over all K costs (identical, bit
// for bit, in every block: same data, same order), then block b forms the weighted sum of its
// chunk of samples for all T*2 outputs, reading eps_eff coalesced (thread = output, thread groups
// stride over samples). Partial sums go to scratch; the last block to finish (atomic ticket) adds
// them in block order, writes v+ in place, u0 and the diagnostics, bumps the counter and resets
// the ticket. No block waits on another.
#include "device.cuh"
#include "internal.h"

namespace bss {

static int update_chunk(int K)
{
    const int c = (K + kUpdMaxBlocks - 1) / kUpdMaxBlocks;
    return c < 32 ? 32 : c;
}

int update_blocks(int K)
{
    const int c = update_chunk(K);
    return (K + c - 1) / c;
}

__device__ __forceinline__ float warp_min(float x)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, off));
    return x;
}

template <bool COMP>
__global__ void __launch_bounds__(kUpdThreads) weights_update_kernel(int K, int TN, int chunk, float inv_lambda,
                                                                   float lambda, UpdateIO io)
{
    __shared__ float red_s[kUpdThreads / kWarp];
    __shared__ float red_c[kUpdThreads / kWarp];
    __shared__ float red_q[kUpdThreads / kWarp];
    __shared__ float red_qc[kUpdThreads / kWarp];
    __shared__ float grid_acc[kUpdThreads];
    __shared__ float grid_cmp[kUpdThreads];
    __shared__ float bcast[3];
    __shared__ bool is_last;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    constexpr int NW = kUpdThreads / kWarp;

    // beta = min S
    float m = INFINITY;
    for (int k = tid; k < K; k += kUpdThreads) m = fminf(m, io.S[k]);
    m = warp_min(m);
    if (lane == 0) red_s[wid] = m;
    __syncthreads();
    if (wid == 0) {
        float x = lane < NW ? red_s[lane] : INFINITY;
        x = warp_min(x);
        if (lane == 0) bcast[0] = x;
    }
    __syncthreads();
    const float beta = bcast[0];

    // eta = sum omega (compensated), and sum omega^2 for the effective sample size
    float s = 0.0f, c = 0.0f, q = 0.0f, qc = 0.0f;
    for (int k = tid; k < K; k += kUpdThreads) {
        const float om = expf(-(io.S[k] - beta) * inv_lambda);
        if constexpr (COMP) {
            comp_merge(s, c, om, 0.0f);
            comp_merge(q, qc, om * om, 0.0f);
        } else {
            s += om;
            q += om * om;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, off), c2 = __shfl_xor_sync(0xffffffffu, c, off);
        const float q2 = __shfl_xor_sync(0xffffffffu, q, off), qc2 = __shfl_xor_sync(0xffffffffu, qc, off);
        if constexpr (COMP) {
            comp_merge(s, c, s2, c2);
            comp_merge(q, qc, q2, qc2);
        } else {
            s += s2;
            q += q2;
        }
    }
    if (lane == 0) {
        red_s[wid] = s; red_c[wid] = c; red_q[wid] = q; red_qc[wid] = qc;
    }
    __syncthreads();
    if (wid == 0) {
        s = lane < NW ? red_s[lane] : 0.0f;
        c = lane < NW ? red_c[lane] : 0.0f;
        q = lane < NW ? red_q[lane] : 0.0f;
        qc = lane < NW ? red_qc[lane] : 0.0f;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float s2 = __shfl_xor_sync(0xffffffffu, s, off), c2 = __shfl_xor_sync(0xffffffffu, c, off);
            const float q2 = __shfl_xor_sync(0xffffffffu, q, off), qc2 = __shfl_xor_sync(0xffffffffu, qc, off);
            if constexpr (COMP) {
                comp_merge(s, c, s2, c2);
                comp_merge(q, qc, q2, qc2);
            } else {
                s += s2;
                q += q2;
            }
        }
        if (lane == 0) {
            bcast[1] = COMP ? s + c : s;
            bcast[2] = COMP ? q + qc : q;
        }
    }
    __syncthreads();
    const float eta = bcast[1];
    const float sumsq = bcast[2];

    // Weighted sums of this block's chunk: thread (g, o) accumulates output o over samples
    // k = k0 + g, k0 + g + NG, ...
    const int NG = kUpdThreads / TN;
    const int k0 = blockIdx.x * chunk;
    const int k1 = min(K, k0 + chunk);
    const int g = tid / TN, o = tid - g * TN;
    CompSum acc;
    float acc_naive = 0.0f;
    if (g < NG) {
        for (int k = k0 + g; k < k1; k += NG) {
            const float wk = expf(-(io.S[k] - beta) * inv_lambda) / eta;
            if (o == 0) io.w[k] = wk;
            const float term = wk * io.eps[(size_t)k * TN + o];
            if constexpr (COMP) acc.add(term); else acc_naive += term;
        }
    }
    grid_acc[tid] = COMP ? acc.s : acc_naive;
    grid_cmp[tid] = COMP ? acc.c : 0.0f;
    __syncthreads();
    if (tid < TN) {
        float ps = grid_acc[tid], pc = grid_cmp[tid];
        for (int gg = 1; gg < NG; ++gg) {
            if constexpr (COMP) comp_merge(ps, pc, grid_acc[gg * TN + tid], grid_cmp[gg * TN + tid]);
            else ps += grid_acc[gg * TN + tid];
        }
        io.partial[(size_t)blockIdx.x * TN + tid] = COMP ? ps + pc : ps;
    }

    // The last block to arrive combines the partial sums in block order.
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned int prev = atomicAdd(io.ticket, 1u);
        is_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (tid < TN) {
        float ps = 0.0f, pc = 0.0f;
        for (int b = 0; b < (int)gridDim.x; ++b) {
            const float x = __ldcg(io.partial + (size_t)b * TN + tid);
            if constexpr (COMP) comp_merge(ps, pc, x, 0.0f); else ps += x;
        }
        const float vn = io.v[tid] + (COMP ? ps + pc : ps);
        io.v[tid] = vn;
        if (io.u0 != nullptr && tid < 2) io.u0[tid] = vn;
    }
    if (tid == 0) {
        if (io.diag != nullptr) {
            io.diag[0] = beta;
            io.diag[1] = eta;
            io.diag[2] = eta * eta / sumsq;
            io.diag[3] = beta - lambda * logf(eta / (float)K);
        }
        *io.ctr += 1u;
        *io.ticket = 0u;
    }
}

cudaError_t update_launch(int K, int T, float lambda, bool comp, const UpdateIO& io, cudaStream_t st)
{
    const int G = update_blocks(K);
    const int chunk = update_chunk(K);
    const int TN = 2 * T;
    if (TN > kUpdThreads) return cudaErrorInvalidValue;
    if (comp) weights_update_kernel<true><<<G, kUpdThreads, 0, st>>>(K, TN, chunk, 1.0f / lambda, lambda, io);
    else weights_update_kernel<false><<<G, kUpdThreads, 0, st>>>(K, TN, chunk, 1.0f / lambda, lambda, io);
    return cudaGetLastError();
}

// Receding-horizon shift: v[t] <- v[min(t + n, T - 1)].
__global__ void shift_kernel(float* v, int T, int n)
{
    __shared__ float buf[2 * 256];
    const int i = threadIdx.x;
    if (i < 2 * T) buf[i] = v[i];
    __syncthreads();
    if (i < 2 * T) {
        const int t = i >> 1, j = i & 1;
        const int src = min(t + n, T - 1);
        v[i] = buf[2 * src + j];
    }
}

cudaError_t shift_launch(float* v, int T, int n, cudaStream_t st)
{
    if (T > 256) return cudaErrorInvalidValue;
    shift_kernel<<<1, 512, 0, st>>>(v, T, n);
    return cudaGetLastError();
}

}  // namespace bss
