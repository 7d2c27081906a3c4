// Importance weights and control update (Eq. "Weights", Eq. "MPPI update law"):
//   beta = min_k S_k, omega_k = exp(-(S_k - beta) / lambda), eta = sum_k omega_k,
//   v+_t = v_t + sum_k (omega_k / eta) eps_eff_{k,t}   (= sum_k omega_k u_k / eta, since the
//   normalised weights sum to one), then u0 = v+_0 and the solve counter advances.
//
// The standalone weights/update step behind bssmppi_update_noalloc (a solve computes the same
// quantities in its rollout kernel's tail). One launch of G blocks. Every block first reduces beta
// and eta over all K costs (identical, bit
// for bit, in every block: same data, same order), then block b forms the weighted sum of its
// chunk of samples for all T*2 outputs, reading eps_eff coalesced (thread = output, thread groups
// stride over samples). Partial sums go to scratch; the last block to finish (atomic ticket) adds
// them in block order, writes v+ in place, u0 and the diagnostics, bumps the counter and resets
// the ticket. No block waits on another.
#include "../../include/bssmppi.h"
#include "device.cuh"
#include "internal.h"

#include <cmath>
#include <mutex>
#include <string>

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
    // Thread (g, o) adds the partials of blocks g, g + NG, ... for output o (independent loads in
    // flight across the group), then the NG group sums are added in group order.
    {
        float ps = 0.0f, pc = 0.0f;
        if (g < NG) {
            for (int b = g; b < (int)gridDim.x; b += NG) {
                const float x = __ldcg(io.partial + (size_t)b * TN + o);
                if constexpr (COMP) comp_merge(ps, pc, x, 0.0f); else ps += x;
            }
        }
        grid_acc[tid] = ps;
        grid_cmp[tid] = pc;
    }
    __syncthreads();
    if (tid < TN) {
        float ps = grid_acc[tid], pc = grid_cmp[tid];
        for (int gg = 1; gg < NG; ++gg) {
            if constexpr (COMP) comp_merge(ps, pc, grid_acc[gg * TN + tid], grid_cmp[gg * TN + tid]);
            else ps += grid_acc[gg * TN + tid];
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

// ---------------------------------------------------------------------------------------------
// Weights and update without any allocation (bssmppi_update_noalloc).
//
// Some callers cannot call cudaMalloc once they are running: hard real-time control loops that
// forbid allocation after start-up (an allocation can block and synchronise the device in the
// middle of a control period), and plugins hosted by a process whose own memory manager owns
// the device memory. For them the weights/update step takes its scratch (the per-block partial
// sums, the arrival ticket and a spare counter word) from the fixed array below instead of a
// handle's buffers. Every GPU that loads this library holds the array until the process exits.
// ---------------------------------------------------------------------------------------------
namespace bss {
namespace {

constexpr int kNoallocPartialFloats = kUpdMaxBlocks * 2 * 256;  // 148 blocks x 2T (T <= 256) floats
constexpr int kNoallocFloats = kNoallocPartialFloats + 64;        // + ticket and spare counter word
static __device__ __align__(256) float g_noalloc_scratch[kNoallocFloats];  // 303,360 bytes

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
float* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per device. In host code
// the array's name is only a host-side stand-in; the kernels must receive this address.
cudaError_t noalloc_scratch(float** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_ptr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace bss

extern "C" int bssmppi_update_noalloc(const float* d_S, const float* d_eps, float* d_v, float* d_w, float* d_u0,
                                      float* d_diag, uint32_t* d_counter, int32_t K, int32_t T, float lambda,
                                      int32_t compensated, void* cuda_stream)
{
    using namespace bss;
    if (K < 1 || K > BSSMPPI_K_MAX) {
        set_thread_error("update_noalloc: K out of range [1, 2^20]");
        return BSSMPPI_EINVAL;
    }
    if (T < 1 || T > BSSMPPI_T_MAX) {
        set_thread_error("update_noalloc: T out of range [1, 256]");
        return BSSMPPI_EINVAL;
    }
    if ((size_t)update_blocks(K) * 2 * (size_t)T > (size_t)kNoallocPartialFloats) {
        set_thread_error("update_noalloc: K and T exceed the static scratch (148 x 512 partial sums)");
        return BSSMPPI_EINVAL;
    }
    if (!(lambda > 0.0f) || !std::isfinite(lambda)) {
        set_thread_error("update_noalloc: lambda must be finite and > 0");
        return BSSMPPI_EINVAL;
    }
    if (!d_S || !d_eps || !d_v || !d_w) {
        set_thread_error("update_noalloc: S, eps, v and w must be non-NULL");
        return BSSMPPI_EINVAL;
    }
    float* scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch + kNoallocPartialFloats);
    uint32_t* spare_counter = reinterpret_cast<uint32_t*>(scratch + kNoallocPartialFloats + 32);
    // the arrival ticket must start at zero (the array keeps whatever the last call left)
    if (e == cudaSuccess) e = cudaMemsetAsync(ticket, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) {
        UpdateIO io{d_S, d_eps, d_v, d_w, d_u0, d_diag, d_counter ? d_counter : spare_counter, scratch, ticket};
        e = update_launch(K, T, lambda, compensated != 0, io, st);
    }
    if (e != cudaSuccess) {
        set_thread_error((std::string("update_noalloc: ") + cudaGetErrorString(e)).c_str());
        return BSSMPPI_ECUDA;
    }
    return BSSMPPI_OK;
}
