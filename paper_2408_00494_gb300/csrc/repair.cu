// Shield repair by a hand-written adjoint (Shield-MPPI's gradient-based local repair, Sec. II,
// the LocalRepair step of Algorithm 1).
//
// Objective: J_r(v) = sum_{t=1..T} C_safe(z_t), the belief-barrier penalty of Eq. "cbfpenalty"
// along the M-particle rollout of the nominal sequence v itself (no control noise). The
// disturbance draws are those of sample 0 of the current solve counter, fixed across evaluations
// (common random numbers), so J_r is a deterministic, piecewise-smooth function of v.
//
// One block, one thread per particle (M <= 256). Forward: propagate, store every particle's state
// at every Euler substep in scratch (L2-resident); then, in parallel over the steps, merge
// count/mean/M2 of e_y across the particles (Chan's pairwise update) and form h_t, the hinge
// arguments and J. Reverse: for t = T..1 add dJ/dh_t through the mean and the unbiased standard
// deviation to each particle's e_y cotangent, then pull the cotangent back through the n_sub
// substeps from their stored states (the next state is loaded while the current adjoint runs) and
// sum dJ/du_{t-1} over the warp's particles; the sum over warps follows the sweep. Neither pass
// has a barrier inside its loop over the steps, so each warp runs its particles' chains at its own
// pace. The kernel is latency-bound (a serial chain per particle); storing the substates removes
// the forward recomputation from the reverse chain. `iters` projected gradient steps
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

// FS: the stride between the fields of a record (floats), a compile-time bound on M, so that every
// field sits at a fixed offset from the record's base and each load or store needs no address
// arithmetic of its own.
template <int MODEL, int FS>
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
    float* part_s = gv_s + 2 * T;                // 2T x 8: per-warp sums of dJ/du

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
    // Records of the forward pass, component-major so each field of a warp's particles is one
    // contiguous 128-byte line: record s = t n_sub + j holds the state entering Euler substep j of
    // step t, then (bicycle) that substep's tape; field i of particle q at rec(s)[i FS + q].
    // Record t n_sub is the state at the start of step t, record T n_sub the final state.
    const int nsub = (MODEL == 0) ? dp.n_sub : 1;
    constexpr int R = (MODEL == 0) ? NX + kTapeFloats : NX;
    const int nc = valid ? n : M - 1;  // lanes past M read a valid record; their results are masked
    auto rec = [&](int sr) -> float* { return io.X + (size_t)sr * (R * FS); };
    auto Xs = [&](int t, int j, int i) -> float* { return rec(t * nsub + j) + i * FS + n; };
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
            if constexpr (MODEL == 0) sincos_reduced(c.steer, &c.sin_steer, &c.cos_steer);
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
        }
        __syncthreads();  // every particle's states are in X
        // The moments of e_y at every step, in parallel over the steps (the dynamics do not read
        // them, so no particle waits for another during the rollout): warp w takes t = 1 + w,
        // 1 + w + nw, ...; each lane merges particles lane, lane + 32, ... one by one, then Chan's
        // pairwise merge across the lanes.
        for (int t = 1 + wid; t <= T; t += nw) {
            const float* ey = rec(t * nsub) + EY * FS;
            float cnt = 0.0f, mu = 0.0f, m2 = 0.0f;
            for (int q = lane; q < M; q += 32) chan_merge(cnt, mu, m2, 1.0f, ey[q], 0.0f);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const float nb = __shfl_xor_sync(0xffffffffu, cnt, off);
                const float mb = __shfl_xor_sync(0xffffffffu, mu, off);
                const float m2b = __shfl_xor_sync(0xffffffffu, m2, off);
                chan_merge(cnt, mu, m2, nb, mb, m2b);
            }
            if (lane == 0) {
                mean_s[t] = mu;
                sig_s[t] = sqrtf(fmaxf(m2 * dp.invM1, 0.0f));
            }
        }
        __syncthreads();
        if (tid == 0) {
            float h_prev = belief_barrier(dp, mean_s[0], 0.0f);
            float J = 0.0f;
            for (int t = 1; t <= T; ++t) {
                float b = dp.wT - dp.nu * sig_s[t];
                if (dp.clamp_margin) b = fmaxf(b, 0.0f);
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
        // dJ/dh_t into the e_y cotangent (through the mean and the unbiased standard deviation);
        // ey_t is this particle's e_y at step t.
        auto inject = [&](int t, float ey_t) {
            const float gh = (arg_s[t] > 0.0f ? -dp.Csafe : 0.0f) + (arg_s[t + 1] > 0.0f ? dp.Csafe * dp.one_m_gamma : 0.0f);
            if (valid && gh != 0.0f) {
                const float mt = mean_s[t], st = sig_s[t];
                float term = -2.0f * mt * dp.invM;
                if (st > 0.0f) {
                    float margin = dp.wT - dp.nu * st;
                    if (dp.clamp_margin) margin = fmaxf(margin, 0.0f);  // a clamped margin has no slope in sigma
                    const float dh_dsig = -2.0f * dp.nu * margin;
                    term += dh_dsig * (ey_t - mt) * dp.invM1 / st;
                }
                g[EY] += gh * term;
            }
        };
        // the warp's sum of dJ/du_t; the sum over warps waits until the sweep is done (no barrier per step)
        auto store_du = [&](int t, float gs, float ga) {
            if (!valid) {
                gs = 0.0f;
                ga = 0.0f;
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                gs += __shfl_xor_sync(0xffffffffu, gs, off);
                ga += __shfl_xor_sync(0xffffffffu, ga, off);
            }
            if (lane == 0) {
                part_s[(2 * t) * 8 + wid] = gs;
                part_s[(2 * t + 1) * 8 + wid] = ga;
            }
        };
        if constexpr (MODEL == 0) {
            // One pass over the S = T n_sub substep records from the last to the first (record
            // s = t n_sub + j: the state entering substep j of step t and that substep's tape).
            // Records s - 1, s - 2 and s - 3 are in flight while substep s's adjoint runs, across
            // the step boundaries too, so the L2 latency stays off the chain.
            const int S = T * nsub;
            auto load = [&](float (&r)[R], int sr) {
                if (sr >= 0) {
                    const float* p = rec(sr) + nc;
#pragma unroll
                    for (int i = 0; i < R; ++i) r[i] = p[i * FS];
                }
            };
            float r0[R], r1[R], r2[R], r3[R];
            load(r0, S - 1);
            load(r1, S - 2);
            load(r2, S - 3);
            float ey_next = rec(S)[EY * FS + nc];  // e_y at the end of the step being entered
            int t = T - 1, j = nsub - 1;
            Control c;
            float gs = 0.0f, ga = 0.0f;
            for (int sr = S - 1; sr >= 0; --sr) {
                load(r3, sr - 3);
                if (j == nsub - 1) {  // entering step t from its end
                    inject(t + 1, ey_next);
                    c.steer = v_s[2 * t];
                    c.accel = v_s[2 * t + 1];
                    sincos_reduced(c.steer, &c.sin_steer, &c.cos_steer);
                    gs = 0.0f;
                    ga = 0.0f;
                }
                bicycle_substep_vjp_taped(dp, c, *reinterpret_cast<const float(*)[6]>(r0),
                                          *reinterpret_cast<const float(*)[kTapeFloats]>(r0 + 6), g, gs, ga);
                if (j == 0) {  // left step t at its start
                    ey_next = r0[EY];
                    store_du(t, gs, ga);
                    --t;
                    j = nsub - 1;
                } else {
                    --j;
                }
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    r0[i] = r1[i];
                    r1[i] = r2[i];
                    r2[i] = r3[i];
                }
            }
        } else {
            for (int t = T; t >= 1; --t) {
                inject(t, rec(t)[EY * FS + nc]);
                float gs = 0.0f, ga = 0.0f;
                double_integrator_step_vjp(dp, g, gs, ga);
                store_du(t - 1, gs, ga);
            }
        }
        __syncthreads();
        for (int i = tid; i < 2 * T; i += blockDim.x) {
            float a = 0.0f;
            for (int w = 0; w < nw; ++w) a += part_s[i * 8 + w];
            gv_s[i] = a;
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

// The field stride of the records: 64 floats up to 64 particles, else the largest M.
static int repair_field_stride(const DevParams& dp) { return dp.M <= 64 ? 64 : kRepairMaxThreads; }

size_t repair_scratch_floats(const DevParams& dp)
{
    const size_t nsub = dp.nx == 6 ? (size_t)dp.n_sub : 1;
    const size_t record = dp.nx == 6 ? (size_t)dp.nx + kTapeFloats : (size_t)dp.nx;
    return ((size_t)dp.T * nsub + 1) * record * repair_field_stride(dp);
}

static size_t repair_smem_bytes(const DevParams& dp)
{
    const int ntab = dp.n_track_mask + 1;
    const size_t floats = (size_t)((ntab + 1 + 3) & ~3) + 2 * dp.T + 2 * (dp.T + 1) + (dp.T + 2) + 2 * dp.T + 16 * dp.T;
    return floats * sizeof(float);
}

cudaError_t repair_prepare(const DevParams& dp)
{
    const size_t smem = repair_smem_bytes(dp);
    if (smem <= 48 * 1024) return cudaSuccess;
    const int fs = repair_field_stride(dp);
    const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (dp.nx == 6)
        return fs == 64 ? cudaFuncSetAttribute(repair_kernel<0, 64>, attr, (int)smem)
                        : cudaFuncSetAttribute(repair_kernel<0, kRepairMaxThreads>, attr, (int)smem);
    return fs == 64 ? cudaFuncSetAttribute(repair_kernel<1, 64>, attr, (int)smem)
                    : cudaFuncSetAttribute(repair_kernel<1, kRepairMaxThreads>, attr, (int)smem);
}

cudaError_t repair_launch(const DevParams& dp, const float* x0, float* v, const uint32_t* ctr, float* X, float* grad,
                          float* J, int iters, float step, cudaStream_t st)
{
    if (dp.M > kRepairMaxThreads || dp.n_sub > kRepairMaxSub) return cudaErrorInvalidValue;
    RepairIO io{x0, v, ctr, X, grad, J, iters, step};
    const int threads = ((dp.M + 31) / 32) * 32;
    const size_t smem = repair_smem_bytes(dp);
    const bool narrow = repair_field_stride(dp) == 64;
    if (dp.nx == 6) {
        if (narrow) repair_kernel<0, 64><<<1, threads, smem, st>>>(dp, io);
        else repair_kernel<0, kRepairMaxThreads><<<1, threads, smem, st>>>(dp, io);
    } else {
        if (narrow) repair_kernel<1, 64><<<1, threads, smem, st>>>(dp, io);
        else repair_kernel<1, kRepairMaxThreads><<<1, threads, smem, st>>>(dp, io);
    }
    return cudaGetLastError();
}

}  // namespace bss
