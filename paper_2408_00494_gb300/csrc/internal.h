// Host-side declarations shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace bss {

struct DevParams;
struct ConSet;

constexpr int kUpdThreads = 512;    // threads per weights/update block
constexpr int kUpdMaxBlocks = 148;  // upper bound on weights/update blocks (scratch is sized by it)

// Launch shape of the persistent rollout kernel, planned once per handle.
struct RollLaunch {
    int grid = 1;      // blocks (at most one per SM)
    int wpb = 1;       // warps per block
    size_t smem = 0;   // dynamic shared memory per block
    int cost_mask = 0; // states the kernel merges and costs, fixed at compile time (0: set at run time)
};
constexpr int kTailMaxBlocks = 256;  // grid bound of the fused rollout (one block per SM)

// Outputs and scratch of the weights/update fused into the rollout kernel's tail.
struct TailIO {
    float* part;            // scratch: grid x (3 + 2T) block partials
    unsigned int* ticket;   // scratch: zero on entry, left at zero
    float* w;               // K normalised weights (out)
    float* u0;              // 2 (out) or nullptr
    float* diag;            // 4 (out) or nullptr
    uint32_t* ctr_out;      // the solve counter, incremented by the last block (nullptr: left alone)
    float* v_out;           // T*2: v+ (the resident nominal, read by every block first)
    float* part_out;        // nullptr: apply the update; else write the merged log-sum-exp partial
                            // (3 + 2T floats: beta, eta, sum omega^2, N) there and leave v, u0, w, diag
    int shift_n;            // > 0: write v+ shifted left by shift_n steps (last repeated) to v_out
};
size_t rollout_smem_bytes(const DevParams& dp, int wpb);
// full: the full-belief kernel variant (re-sampled particles and/or a general constraint set).
cudaError_t rollout_prepare(const DevParams& dp, int P, bool comp, bool full, RollLaunch& L,
                            const ConSet* cs = nullptr);
cudaError_t rollout_launch(const DevParams& dp, int P, bool comp, const RollLaunch& L, const float* x0,
                           const float* Sigma0, const float* v, const uint32_t* ctr, float* S, float* eps, float* mean,
                           float* var, const TailIO& tail, const ConSet& cs, cudaStream_t st);
// Merge of G log-sum-exp partials (G x (3 + 2T) floats, each {beta, eta, q, N}) into v+ = v + N / eta,
// u0, the diagnostics (K_norm samples in all) and the normalised weights of the K local costs S.
cudaError_t merge_partials_launch(const DevParams& dp, int G, const float* parts, bool comp, const float* S,
                                  const TailIO& tail, cudaStream_t st);
cudaError_t model_step_launch(const DevParams& dp, const float* x, const float* u, const float* w, float* xn, int64_t n,
                              cudaStream_t st);
cudaError_t philox_launch(const uint32_t* ctr, uint64_t seed, uint32_t* out, int64_t n, cudaStream_t st);
cudaError_t box_muller_launch(const uint32_t* words, float* z, int64_t n, cudaStream_t st);
cudaError_t slip_atan_launch(const float* t, float* y, int64_t n, cudaStream_t st);
cudaError_t tyre_curve_launch(const DevParams& dp, const float* x, float* y, int64_t n, cudaStream_t st);
// Coefficients c_0..c_9 of p with sin(C atan x) = x p(x^2) on |x| <= 1 (host, double precision;
// c holds kTyreDeg + 1 = 10 floats).
void tyre_curve_fit(double C, float* c);
// The rear tyre's polynomial in x = t / tau (rear_tyre in device.cuh): tau for B, and c_0..c_9 for B, C.
double rear_tyre_tau(double B);
void rear_tyre_fit(double B, double C, float* c);
cudaError_t rear_tyre_launch(const DevParams& dp, const float* t, float* y, int64_t n, cudaStream_t st);

// Weights + update: the number of blocks for K samples, and the launch.
int update_blocks(int K);
struct UpdateIO {
    const float* S;       // K costs
    const float* eps;     // K*T*2 effective perturbations
    float* v;             // T*2 nominal, updated in place to v+
    float* w;             // K normalised weights (out)
    float* u0;            // 2 (out) or nullptr
    float* diag;          // 4 (out) or nullptr
    uint32_t* ctr;        // solve counter, incremented by one
    float* partial;       // scratch: update_blocks(K) * T*2 partial sums
    unsigned int* ticket; // scratch: one zero-initialised counter, left at zero
};
cudaError_t update_launch(int K, int T, float lambda, bool comp, const UpdateIO& io, cudaStream_t st);
cudaError_t shift_launch(float* v, int T, int n, cudaStream_t st);

// Shield repair (adjoint of the belief-barrier penalty of the nominal rollout).
size_t repair_scratch_floats(const DevParams& dp);
cudaError_t repair_prepare(const DevParams& dp);
cudaError_t repair_launch(const DevParams& dp, const float* x0, float* v, const uint32_t* ctr, float* X, float* grad,
                          float* J, int iters, float step, cudaStream_t st);

// Records the calling thread's error message for entry points without a handle
// (read back through bssmppi_last_error(NULL)).
void set_thread_error(const char* msg);

}  // namespace bss

struct bssmppi_params;
#include <string>

namespace bss {

// Validates a problem and derives the kernels' constants (d) and particles per lane (P); returns
// BSSMPPI_OK or BSSMPPI_EINVAL with the reason in `why`.
int derive_params(const bssmppi_params* p, DevParams& d, int& P, std::string& why);

}  // namespace bss
