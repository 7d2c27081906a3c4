// Shield repair by a hand-written adjoint (Shield-MPPI's gradient-based local repair, Sec. II,
// the LocalRepair step of Algorithm 1).
//
// Objective: J_r(v) = sum_{t=1..T} C_safe(z_t), the belief-barrier penalty of Eq. "cbfpenalty"
// along the M-particle rollout of the nominal sequence v itself (no control noise). The
// disturbance draws are those of sample 0 of the current solve counter, fixed across evaluations
// (common random numbers), so J_r is a deterministic, piecewise-smooth function of v.
//
// One block, one thread per particle (M <= 256). Forward: propagate, store every particle's state
// at every Euler substep in scratch (L2-resident), merge count/mean/M2 of e_y across the block
// (Chan's pairwise update), and form h_t, the hinge arguments and J. Reverse: for t = T..1 add
// dJ/dh_t through the mean and the unbiased standard deviation to each particle's e_y cotangent,
// then pull the cotangent back through the n_sub substeps from their stored states (the next
// state is loaded while the current adjoint runs) and sum dJ/du_{t-1} over the particles. The
// kernel is latency-bound (a serial chain per particle); storing the substates removes the
// forward recomputation from the reverse chain. `iters` projected gradient steps
// v <- clamp(v - step dJ/dv) run inside one launch.
#include "device.cuh"
#include "internal.h"

namespace bss {

constexpr int kRepairMaxThreads = 256;
constexpr int kRepairMaxSub = 64;

struct RepairIO {
    const float* x0;
    float* v;             // T*2 nominal; updated in place when iters > 0
    const uint32_t* ctr;
    float* X;             // scratch: (T+1) * NX * M particle states, component-major per step
    float* grad;          // T*2 gradient at the input v (iters == 0) or nullptr
    float* J;             // iters + 1 objective values (before each step, then final) or nullptr
    int iters;
    float step;
};

// Chan merge of (count, mean, M2) of two disjoint sets.
__device__ __forceinline__ void chan_merge(float& n, float& m, float& m2, float nb, float mb, float m2b)
{
    const float nn = n + nb;
    if (nn > 0.0f) {
        const float inv = 1.0f / nn;
        const float d = mb - m;
        m2 = m2 + m2b + d * d * n * nb * inv;
        m = __fadd_rn(__fmul_rn(n * inv, m), __fmul_rn(nb * inv, mb));
    }
    n = nn;
}

template <int MODEL>
__global__ void __launch_bounds__(kRepairMaxThreads) repair_kernel(const DevParams dp, const RepairIO io)
{
    constexpr int NX = MODEL == 0 ? 6 : 4;
    constexpr int EY = MODEL == 0 ? 4 : 1;
    extern __shared__ float smem[];
    const int T = dp.T, M = dp.M;
    const int ntab = dp.n_track_mask + 1;
    float* kap_s = smem;
    float* v_s = smem + ((ntab + 1 + 3) & ~3);   // 2T
    float* mean_s = v_s + 2 * T;                 // T+1
    float* sig_s = mean_s + (T + 1);             // T+1
    float* arg_s = sig_s + (T + 1);              // T+2 (arg_s[T+1] < 0: no successor)
    float* gv_s = arg_s + (T + 2);               // 2T
    float* red = gv_s + 2 * T;                   // 2 buffers x 8 warps x 3

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const int n = tid;
    const bool valid = n < M;
    if constexpr (MODEL == 0) {
        for (int i = tid; i <= ntab; i += blockDim.x) kap_s[i] = dp.kappa[i];
    }
    for (int i = tid; i < 2 * T; i += blockDim.x) v_s[i] = io.v[i];
    __syncthreads();
    const uint32_t ctr = *io.ctr;
    float x0[NX];
#pragma unroll
    for (int i = 0; i < NX; ++i) x0[i] = io.x0[i];
    const float s0 = (MODEL == 0) ? x0[5] : 0.0f;
    // Records of the forward pass, component-major so each field of all particles is contiguous:
    // record (t, j) = the state entering Euler substep j of step t, then (bicycle) that substep's
    // tape. Xat(t, i) = component i of the state at the start of step t.
    const int nsub = (MODEL == 0) ? dp.n_sub : 1;
    constexpr int R = (MODEL == 0) ? NX + kTapeFloats : NX;
    auto Xs = [&](int t, int j, int i) -> float* { return io.X + (((size_t)t * nsub + j) * R + i) * M + n; };
    auto Xat = [&](int t, int i) -> float* { return Xs(t, 0, i); };

    for (int it = 0; it <= io.iters; ++it) {
        const bool last = (it == io.iters);
        if (last && io.grad == nullptr && io.J == nullptr) break;  // nobody reads the final objective
        // ---------------- forward rollout of the nominal sequence
        float x[NX];
#pragma unroll
        for (int i = 0; i < NX; ++i) x[i] = (MODEL == 0 && i == 5) ? 0.0f : x0[i];
        if (valid) {
#pragma unroll
            for (int i = 0; i < NX; ++i) *Xat(0, i) = x[i];
        }
        if (tid == 0) {
            mean_s[0] = x0[EY];
            sig_s[0] = 0.0f;
        }
        for (int t = 0; t < T; ++t) {
            Control c;
            c.steer = v_s[2 * t];
            c.accel = v_s[2 * t + 1];
            if constexpr (MODEL == 0) sincosf(c.steer, &c.sin_steer, &c.cos_steer);
            if constexpr (MODEL == 0) {
                for (int j = 0; j < nsub; ++j) {
                    float tp[kTapeFloats];
                    float xb[6];
#pragma unroll
                    for (int i = 0; i < 6; ++i) xb[i] = x[i];
                    bicycle_substep_taped(dp, kap_s, s0, c, x, tp);
                    if (valid) {  // the state of substep 0 is stored with the previous step's result
                        if (j > 0) {
#pragma unroll
                            for (int i = 0; i < 6; ++i) *Xs(t, j, i) = xb[i];
                        }
#pragma unroll
                        for (int i = 0; i < kTapeFloats; ++i) *Xs(t, j, 6 + i) = tp[i];
                    }
                }
            } else {
                model_step<MODEL, NX>(dp, kap_s, s0, c, x);
            }
            float z[NX];
            draw_disturbance<NX>(dp, (uint32_t)t, (uint32_t)n, 0u, ctr, z);
            add_correlated<NX>(dp.Lw, z, x);
            if (valid) {
#pragma unroll
                for (int i = 0; i < NX; ++i) *Xat(t + 1, i) = x[i];
            }
            float cnt = valid ? 1.0f : 0.0f, mu = valid ? x[EY] : 0.0f, m2 = 0.0f;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const float nb = __shfl_xor_sync(0xffffffffu, cnt, off);
                const float mb = __shfl_xor_sync(0xffffffffu, mu, off);
                const float m2b = __shfl_xor_sync(0xffffffffu, m2, off);
                chan_merge(cnt, mu, m2, nb, mb, m2b);
            }
            float* rb = red + (t & 1) * 24;
            if (lane == 0) {
                rb[3 * wid] = cnt;
                rb[3 * wid + 1] = mu;
                rb[3 * wid + 2] = m2;
            }
            __syncthreads();
            if (tid == 0) {
                float n0 = rb[0], m0 = rb[1], q0 = rb[2];
                for (int w = 1; w < nw; ++w) chan_merge(n0, m0, q0, rb[3 * w], rb[3 * w + 1], rb[3 * w + 2]);
                mean_s[t + 1] = m0;
                sig_s[t + 1] = sqrtf(fmaxf(q0 * dp.invM1, 0.0f));
            }
        }
        __syncthreads();
        if (tid == 0) {
            float h_prev = belief_barrier(dp, mean_s[0], 0.0f);
            float J = 0.0f;
            for (int t = 1; t <= T; ++t) {
                const float b = dp.wT - dp.nu * sig_s[t];
                const float h = b * b - mean_s[t] * mean_s[t];
                const float a = fmaf(dp.one_m_gamma, h_prev, -h);
                arg_s[t] = a;
                J += dp.Csafe * fmaxf(a, 0.0f);
                h_prev = h;
            }
            arg_s[0] = -1.0f;
            arg_s[T + 1] = -1.0f;
            if (io.J) io.J[it] = J;
        }
        __syncthreads();
        if (last && io.grad == nullptr) break;

        // ---------------- reverse sweep
        float g[NX];
#pragma unroll
        for (int i = 0; i < NX; ++i) g[i] = 0.0f;
        for (int t = T; t >= 1; --t) {
            const float gh = (arg_s[t] > 0.0f ? -dp.Csafe : 0.0f) + (arg_s[t + 1] > 0.0f ? dp.Csafe * dp.one_m_gamma : 0.0f);
            if (valid && gh != 0.0f) {
                const float mt = mean_s[t], st = sig_s[t];
                float term = -2.0f * mt * dp.invM;
                if (st > 0.0f) {
                    const float dh_dsig = -2.0f * dp.nu * (dp.wT - dp.nu * st);
                    term += dh_dsig * (*Xat(t, EY) - mt) * dp.invM1 / st;
                }
                g[EY] += gh * term;
            }
            Control c;
            c.steer = v_s[2 * (t - 1)];
            c.accel = v_s[2 * (t - 1) + 1];
            float gs = 0.0f, ga = 0.0f;
            if constexpr (MODEL == 0) {
                sincosf(c.steer, &c.sin_steer, &c.cos_steer);
                // The forward pass stored each substep's state and tape; the next record is loaded
                // while the current substep's adjoint runs, so the loads stay off the chain.
                float cur[R], nxt[R];
#pragma unroll
                for (int i = 0; i < R; ++i) cur[i] = valid ? *Xs(t - 1, nsub - 1, i) : (i < 6 ? x0[i] : 0.0f);
                for (int j = nsub - 1; j >= 0; --j) {
#pragma unroll
                    for (int i = 0; i < R; ++i) nxt[i] = (valid && j > 0) ? *Xs(t - 1, j - 1, i) : cur[i];
                    bicycle_substep_vjp_taped(dp, c, *reinterpret_cast<const float(*)[6]>(cur),
                                              *reinterpret_cast<const float(*)[kTapeFloats]>(cur + 6), g, gs, ga);
#pragma unroll
                    for (int i = 0; i < R; ++i) cur[i] = nxt[i];
                }
            } else {
                double_integrator_step_vjp(dp, g, gs, ga);
            }
            if (!valid) {
                gs = 0.0f;
                ga = 0.0f;
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                gs += __shfl_xor_sync(0xffffffffu, gs, off);
                ga += __shfl_xor_sync(0xffffffffu, ga, off);
            }
            float* rb = red + 48 + (t & 1) * 16;
            if (lane == 0) {
                rb[2 * wid] = gs;
                rb[2 * wid + 1] = ga;
            }
            __syncthreads();
            if (tid == 0) {
                float a0 = 0.0f, a1 = 0.0f;
                for (int w = 0; w < nw; ++w) {
                    a0 += rb[2 * w];
                    a1 += rb[2 * w + 1];
                }
                gv_s[2 * (t - 1)] = a0;
                gv_s[2 * (t - 1) + 1] = a1;
            }
        }
        __syncthreads();
        if (last) {
            for (int i = tid; i < 2 * T; i += blockDim.x) io.grad[i] = gv_s[i];
            break;
        }
        // projected gradient step
        for (int i = tid; i < 2 * T; i += blockDim.x) {
            const float lo = (i & 1) ? dp.umin1 : dp.umin0, hi = (i & 1) ? dp.umax1 : dp.umax0;
            v_s[i] = fminf(fmaxf(v_s[i] - io.step * gv_s[i], lo), hi);
        }
        __syncthreads();
    }
    if (io.iters > 0) {
        for (int i = tid; i < 2 * T; i += blockDim.x) io.v[i] = v_s[i];
    }
}

size_t repair_scratch_floats(const DevParams& dp)
{
    const size_t nsub = dp.nx == 6 ? (size_t)dp.n_sub : 1;
    const size_t record = dp.nx == 6 ? (size_t)dp.nx + kTapeFloats : (size_t)dp.nx;
    return ((size_t)dp.T * nsub + 1) * record * dp.M;
}

static size_t repair_smem_bytes(const DevParams& dp)
{
    const int ntab = dp.n_track_mask + 1;
    const size_t floats = (size_t)((ntab + 1 + 3) & ~3) + 2 * dp.T + 2 * (dp.T + 1) + (dp.T + 2) + 2 * dp.T + 48 + 32;
    return floats * sizeof(float);
}

cudaError_t repair_prepare(const DevParams& dp)
{
    const size_t smem = repair_smem_bytes(dp);
    if (smem <= 48 * 1024) return cudaSuccess;
    if (dp.nx == 6) return cudaFuncSetAttribute(repair_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaFuncSetAttribute(repair_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t repair_launch(const DevParams& dp, const float* x0, float* v, const uint32_t* ctr, float* X, float* grad,
                          float* J, int iters, float step, cudaStream_t st)
{
    if (dp.M > kRepairMaxThreads || dp.n_sub > kRepairMaxSub) return cudaErrorInvalidValue;
    RepairIO io{x0, v, ctr, X, grad, J, iters, step};
    const int threads = ((dp.M + 31) / 32) * 32;
    const size_t smem = repair_smem_bytes(dp);
    if (dp.nx == 6) repair_kernel<0><<<1, threads, smem, st>>>(dp, io);
    else repair_kernel<1><<<1, threads, smem, st>>>(dp, io);
    return cudaGetLastError();
}

}  // namespace bss
