// Continuous-batching server for many controllers (serving pattern of the solve).
//
// Each registered controller keeps its problem constants, curvature table, warm-start nominal
// sequence and Philox solve counter resident on the device. Requests (state estimate + K, M, T)
// arrive on any host thread; a newer request of a controller replaces its older pending one
// (latest state wins). A scheduler thread forms batches in arrival order, admitting a request when
// its controller has nothing in flight, the batch has room and the slot's HBM arena can hold its
// buffers (perturbations K*T*2, costs K, weights K). Up to four slots take turns, each with its own
// streams, arena and descriptors, so requests that arrive while a batch runs on the GPU are
// admitted into another slot and overlap with it on the device.
//
// A batch is one fixed sequence, captured once per slot as a CUDA graph and replayed:
//   H2D copy of the batch descriptors (fixed size)
//   -> three persistent rollout kernels in parallel branches, one per particles-per-lane class
//      (P = 1, 2, 4 for M < 8, M <= 64, M <= 128); their warps pull (request, sample-group) items with an
//      atomic counter and run the same per-group body as the single-solve kernel. The constants
//      the batch's vehicles share (a batch holds controllers of one constants class) are a kernel
//      parameter, so the body reads them as instruction operands and steps particle pairs with
//      packed FP32 instructions as the single-solve kernel does; each warp keeps only its item's
//      sizes, the controller's Philox keys and its track's scale in shared memory
//   -> one block per request: weights, update, warm-start shift, counter
//   -> D2H copy of the first controls (fixed size).
// No kernel ever waits on the host or on another kernel.
#include "../../include/bssmppi.h"
#include "device.cuh"
#include "internal.h"
#include "rollout_body.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

namespace bss {

constexpr int kServeClasses = 3;   // P = 1, 2, 4
constexpr int kServeMaxSlots = 8;  // batches in flight at most
constexpr int kServeWarps = 4;     // warps per block of the batched rollout
constexpr int kServeSpwMax = 16;   // samples per warp when M = 2

struct ServeReq {
    int ctrl, K, M, T;
    int seg, spw, uniform, cls;
    int group_begin, n_groups, dist_half, pad1;  // dist_half: particles n and n + H share a counter
    float x0[6];
    float pad2[2];
    unsigned long long off_eps, off_S, off_w;  // float offsets into the slot arena
};

struct ServeHeader {
    int n_req;
    int cls_begin[kServeClasses], cls_count[kServeClasses], cls_groups[kServeClasses];
    unsigned int next[kServeClasses];
};

struct ServeResult {
    float u0[2];
    float beta, eta;
};

// One work item's per-solve fields (the names the per-group body reads from its item object): the
// request's sizes, the controller's Philox round keys and its track's scale and mask.
struct __align__(16) ServeItem {
    uint32_t rk0[10], rk1[10];
    int K, M, T, seg, spw, uniform, dist_half, k_off;
    float Mf, invM, invM1, track_scale;
    int n_track_mask, pad[3];
};

// Largest sample count per warp of a particle class: 32 / seg for its smallest segment (class 0:
// M = 2 on 2 lanes; class 1: M = 8 on 4 lanes, two particles per lane; class 2: a whole warp).
__host__ __device__ constexpr int serve_spw_max(int cls) { return cls == 0 ? kServeSpwMax : (cls == 1 ? 8 : 1); }

// Blocks of kServeWarps warps per SM for the register bound: 6, 5 and 4 for 1, 2 and 4 particles
// per lane (80, 102 and 128 registers), the tightest bounds at which the loop over work items
// spills at most 8 bytes. (Two blocks more, the single-solve kernel's threads per SM, spilled 60-116
// bytes and served 4 % fewer particle-steps per second at saturation.)
template <int P>
__host__ __device__ constexpr int serve_min_blocks() { return P == 1 ? 6 : (P == 2 ? 5 : 4); }

template <int P>
__global__ void __launch_bounds__(kServeWarps * kWarp, serve_min_blocks<P>())
    serve_rollout_kernel(const __grid_constant__ DevParams fleet, ServeHeader* hdr, const ServeReq* reqs,
                         const DevParams* ctrl_dp, float* arena, const float* ctrl_v, const uint32_t* ctrl_ctr,
                         int cls, int T_max)
{
    extern __shared__ __align__(16) unsigned char serve_smem[];
    const int warp = threadIdx.x / kWarp, lane = threadIdx.x & (kWarp - 1);
    ServeItem* it = reinterpret_cast<ServeItem*>(serve_smem) + warp;
    float* ubuf = reinterpret_cast<float*>(reinterpret_cast<ServeItem*>(serve_smem) + kServeWarps)
                + (size_t)warp * serve_spw_max(cls) * 2 * T_max;
    const int total = hdr->cls_groups[cls];
    const int rb = hdr->cls_begin[cls], rc = hdr->cls_count[cls];
    while (true) {
        unsigned int item = 0;
        if (lane == 0) item = atomicAdd(&hdr->next[cls], 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= (unsigned int)total) break;
        int lo = rb, hi = rb + rc - 1;  // the request whose groups contain this item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (reqs[mid].group_begin <= (int)item) lo = mid; else hi = mid - 1;
        }
        const ServeReq& rq = reqs[lo];
        const DevParams& cd = ctrl_dp[rq.ctrl];
        if (lane < 10) {
            it->rk0[lane] = cd.rk0[lane];
            it->rk1[lane] = cd.rk1[lane];
        }
        if (lane == 0) {
            it->K = rq.K; it->M = rq.M; it->T = rq.T;
            it->seg = rq.seg; it->spw = rq.spw; it->uniform = rq.uniform; it->dist_half = rq.dist_half;
            it->k_off = 0;
            it->Mf = (float)rq.M; it->invM = 1.0f / (float)rq.M; it->invM1 = 1.0f / (float)(rq.M - 1);
            it->track_scale = cd.track_scale;
            it->n_track_mask = cd.n_track_mask;
        }
        __syncwarp();
        const float* v = ctrl_v + (size_t)rq.ctrl * 2 * T_max;
        RollIO io{rq.x0, nullptr, v, ctrl_ctr + rq.ctrl, arena + rq.off_S, arena + rq.off_eps, nullptr, nullptr};
        float* my_u = ubuf + (lane / rq.seg) * 2 * rq.T;
        // a class whose cost weights only v_x, e_psi and e_y merges and costs those means only
        if ((fleet.mean_mask & ~kRacingCostMask) == 0)
            rollout_group<0, P, true, false, float, true, false, ServeItem, true, kRacingCostMask>(
                fleet, *it, io, cd.kappa, v, my_u, (int)item - rq.group_begin, ctrl_ctr[rq.ctrl]);
        else
            rollout_group<0, P, true, false, float, true, false, ServeItem, true>(
                fleet, *it, io, cd.kappa, v, my_u, (int)item - rq.group_begin, ctrl_ctr[rq.ctrl]);
        __syncwarp();
    }
}

// Weights (Eq. "Weights"), update (Eq. "MPPI update law"), warm-start shift and counter of one
// request per block, with compensated sums.
__global__ void __launch_bounds__(kUpdThreads) serve_update_kernel(const ServeHeader* hdr, const ServeReq* reqs,
                                                                 const DevParams* ctrl_dp, float* arena, float* ctrl_v,
                                                                 uint32_t* ctrl_ctr, ServeResult* res, int T_max)
{
    __shared__ float red[4][kUpdThreads / kWarp];
    __shared__ float acc_s[kUpdThreads], cmp_s[kUpdThreads];
    __shared__ float vn_s[2 * BSSMPPI_T_MAX];
    __shared__ float bc[3];
    const int r = blockIdx.x;
    if (r >= hdr->n_req) return;
    const ServeReq rq = reqs[r];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    constexpr int NW = kUpdThreads / kWarp;
    const float inv_lambda = ctrl_dp[rq.ctrl].inv_lambda;
    const float* S = arena + rq.off_S;
    const float* eps = arena + rq.off_eps;
    float* w = arena + rq.off_w;
    float* v = ctrl_v + (size_t)rq.ctrl * 2 * T_max;
    const int K = rq.K, TN = 2 * rq.T;

    float m = INFINITY;
    for (int k = tid; k < K; k += kUpdThreads) m = fminf(m, S[k]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (lane == 0) red[0][wid] = m;
    __syncthreads();
    if (tid == 0) {
        float x = red[0][0];
        for (int i = 1; i < NW; ++i) x = fminf(x, red[0][i]);
        bc[0] = x;
    }
    __syncthreads();
    const float beta = bc[0];
    float s = 0.0f, c = 0.0f;
    for (int k = tid; k < K; k += kUpdThreads) comp_merge(s, c, expf(-(S[k] - beta) * inv_lambda), 0.0f);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, off), c2 = __shfl_xor_sync(0xffffffffu, c, off);
        comp_merge(s, c, s2, c2);
    }
    if (lane == 0) {
        red[1][wid] = s;
        red[2][wid] = c;
    }
    __syncthreads();
    if (tid == 0) {
        float a = red[1][0], b = red[2][0];
        for (int i = 1; i < NW; ++i) comp_merge(a, b, red[1][i], red[2][i]);
        bc[1] = a + b;
    }
    __syncthreads();
    const float eta = bc[1];

    const int NG = kUpdThreads / TN;
    const int g = tid / TN, o = tid - g * TN;
    CompSum acc;
    if (g < NG) {
        for (int k = g; k < K; k += NG) {
            const float wk = expf(-(S[k] - beta) * inv_lambda) / eta;
            if (o == 0) w[k] = wk;
            acc.add(wk * eps[(size_t)k * TN + o]);
        }
    }
    acc_s[tid] = acc.s;
    cmp_s[tid] = acc.c;
    __syncthreads();
    if (tid < TN) {
        float ps = acc_s[tid], pc = cmp_s[tid];
        for (int gg = 1; gg < NG; ++gg) comp_merge(ps, pc, acc_s[gg * TN + tid], cmp_s[gg * TN + tid]);
        vn_s[tid] = v[tid] + (ps + pc);
    }
    __syncthreads();
    if (tid < TN) {
        const int t = tid >> 1, j = tid & 1;
        v[tid] = vn_s[2 * min(t + 1, rq.T - 1) + j];  // warm start: v+ shifted by one step
    }
    if (tid == 0) {
        res[r].u0[0] = vn_s[0];
        res[r].u0[1] = vn_s[1];
        res[r].beta = beta;
        res[r].eta = eta;
        ctrl_ctr[rq.ctrl] += 1u;
    }
}

}  // namespace bss

using namespace bss;

namespace {

double now_us(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
}

struct Pending {
    uint64_t id = 0;
    int ctrl = 0, K = 0, M = 0, T = 0, fleet = 0;
    float x0[6] = {};
    double t_submit = 0.0;
    uint64_t seq = 0;
};

struct Slot {
    cudaStream_t s[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t fork = nullptr, join1 = nullptr, join2 = nullptr, done = nullptr;
    ServeHeader* d_hdr = nullptr;   // header followed by the request table (one allocation)
    ServeReq* d_reqs = nullptr;
    ServeResult* d_res = nullptr;
    unsigned char* h_desc = nullptr; // pinned: header + requests
    ServeResult* h_res = nullptr;    // pinned
    float* d_arena = nullptr;
    size_t arena_floats = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t roll_node[kServeClasses] = {nullptr, nullptr, nullptr};  // the rollout kernels' nodes
    cudaKernelNodeParams roll_kp[kServeClasses] = {};
    int fleet = -1;        // constants class of the batch in the slot
    DevParams fleet_params{};  // its constants, copied under the lock when the batch is formed
    int graph_fleet = -1;  // constants class the graph's rollout nodes were last given
    bool busy = false;
    std::vector<Pending> batch;
    double t_launch = 0.0;
};

}  // namespace

// A one-shot request to copy a controller's next completed solve out of the slot's arena.
struct Capture {
    float* h_out = nullptr;
    int64_t cap_floats = 0;
    int64_t* h_written = nullptr;
    bool armed = false;
};

struct bssmppi_server {
    bssmppi_server_config cfg{};
    int device = 0, sms = 0;
    size_t desc_bytes = 0, res_bytes = 0;
    int roll_grid[kServeClasses] = {1, 1, 1};
    size_t roll_smem[kServeClasses] = {0, 0, 0};
    // constants classes: controllers whose problem constants agree in everything but their Philox
    // keys and track share a class; a batch holds one class, whose constants are the rollout
    // kernels' parameter
    std::vector<DevParams> fleets;
    std::vector<int> fleet_of;
    // controller table
    std::vector<DevParams> h_dp;
    std::vector<float*> d_tracks;
    DevParams* d_dp = nullptr;
    float* d_v = nullptr;
    uint32_t* d_ctr = nullptr;
    int n_ctrl = 0;
    // host state (under mu)
    std::mutex mu;
    std::condition_variable cv;
    std::vector<Pending> pending;
    std::vector<char> has_pending, in_flight;
    std::vector<Capture> capture;
    std::vector<bssmppi_result> done;
    uint64_t seq = 0;
    bssmppi_server_stats stats{};
    Slot slots[kServeMaxSlots];
    int n_slots = 2;
    std::thread worker;
    std::atomic<bool> stop{false};
    std::atomic<int> worker_error{0};
    std::string err;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
};

namespace {

int srv_fail(bssmppi_server* s, int code, const std::string& msg)
{
    if (s) {
        std::lock_guard<std::mutex> lock(s->mu);
        s->err = msg;
    } else {
        set_thread_error(msg.c_str());
    }
    return code;
}

size_t request_floats(int K, int T)
{
    auto round = [](size_t n) { return (n + 63) & ~(size_t)63; };
    return round((size_t)K * T * 2) + round(K) + round(K);
}

// Particle classes by particles per lane: M < 8 one (segments of the next power of two >= M lanes),
// 8 <= M <= 64 two (segments of the next power of two >= M / 2 lanes: packed pairs, and half the
// per-step merge and cost work per particle; a batch has warps enough to hide latency), M > 64 four.
int class_of(int M) { return M < 8 ? 0 : (M <= 64 ? 1 : 2); }

// Issue one batch on the slot's streams (also used, once, under capture to build the graph).
cudaError_t issue_batch(bssmppi_server* s, Slot& sl)
{
    cudaError_t e = cudaMemcpyAsync(sl.d_hdr, sl.h_desc, s->desc_bytes, cudaMemcpyHostToDevice, sl.s[0]);
    if (e == cudaSuccess) e = cudaEventRecord(sl.fork, sl.s[0]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sl.s[1], sl.fork, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sl.s[2], sl.fork, 0);
    if (e != cudaSuccess) return e;
    const int T_max = s->cfg.T_max;
    const DevParams fleet = sl.fleet_params;
    serve_rollout_kernel<1><<<s->roll_grid[0], kServeWarps * kWarp, s->roll_smem[0], sl.s[0]>>>(
        fleet, sl.d_hdr, sl.d_reqs, s->d_dp, sl.d_arena, s->d_v, s->d_ctr, 0, T_max);
    serve_rollout_kernel<2><<<s->roll_grid[1], kServeWarps * kWarp, s->roll_smem[1], sl.s[1]>>>(
        fleet, sl.d_hdr, sl.d_reqs, s->d_dp, sl.d_arena, s->d_v, s->d_ctr, 1, T_max);
    serve_rollout_kernel<4><<<s->roll_grid[2], kServeWarps * kWarp, s->roll_smem[2], sl.s[2]>>>(
        fleet, sl.d_hdr, sl.d_reqs, s->d_dp, sl.d_arena, s->d_v, s->d_ctr, 2, T_max);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(sl.join1, sl.s[1]);
    if (e == cudaSuccess) e = cudaEventRecord(sl.join2, sl.s[2]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sl.s[0], sl.join1, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sl.s[0], sl.join2, 0);
    if (e != cudaSuccess) return e;
    serve_update_kernel<<<s->cfg.max_batch, kUpdThreads, 0, sl.s[0]>>>(sl.d_hdr, sl.d_reqs, s->d_dp, sl.d_arena, s->d_v,
                                                                     s->d_ctr, sl.d_res, T_max);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.h_res, sl.d_res, s->res_bytes, cudaMemcpyDeviceToHost, sl.s[0]);
    return e;
}

// After capture: the graph's three rollout kernel nodes and their launch parameters.
cudaError_t find_rollout_nodes(Slot& sl)
{
    size_t n = 0;
    cudaError_t e = cudaGraphGetNodes(sl.graph, nullptr, &n);
    if (e != cudaSuccess) return e;
    std::vector<cudaGraphNode_t> nodes(n);
    e = cudaGraphGetNodes(sl.graph, nodes.data(), &n);
    const void* fn[kServeClasses] = {reinterpret_cast<const void*>(serve_rollout_kernel<1>),
                                     reinterpret_cast<const void*>(serve_rollout_kernel<2>),
                                     reinterpret_cast<const void*>(serve_rollout_kernel<4>)};
    for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
        cudaGraphNodeType type;
        e = cudaGraphNodeGetType(nodes[i], &type);
        if (e != cudaSuccess || type != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp{};
        e = cudaGraphKernelNodeGetParams(nodes[i], &kp);
        for (int c = 0; c < kServeClasses && e == cudaSuccess; ++c)
            if (kp.func == fn[c]) {
                sl.roll_node[c] = nodes[i];
                sl.roll_kp[c] = kp;
            }
    }
    for (int c = 0; c < kServeClasses && e == cudaSuccess; ++c)
        if (!sl.roll_node[c]) e = cudaErrorInvalidValue;
    return e;
}

// Give the instantiated graph's rollout kernels the constants of the slot's batch class (applies
// to this and later launches of the graph; launches already queued keep theirs).
cudaError_t set_graph_fleet(bssmppi_server* s, Slot& sl)
{
    DevParams fleet = sl.fleet_params;
    const DevParams* d_dp = s->d_dp;
    float* arena = sl.d_arena;
    const float* v = s->d_v;
    const uint32_t* ctr = s->d_ctr;
    int T_max = s->cfg.T_max;
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < kServeClasses && e == cudaSuccess; ++c) {
        int cls = c;
        void* args[] = {&fleet, &sl.d_hdr, &sl.d_reqs, &d_dp, &arena, &v, &ctr, &cls, &T_max};
        cudaKernelNodeParams kp = sl.roll_kp[c];
        kp.kernelParams = args;
        kp.extra = nullptr;
        e = cudaGraphExecKernelNodeSetParams(sl.exec, sl.roll_node[c], &kp);
    }
    if (e == cudaSuccess) sl.graph_fleet = sl.fleet;
    return e;
}

// Fill the slot's descriptors from its admitted requests (sorted by particle class).
void fill_descriptors(Slot& sl)
{
    std::stable_sort(sl.batch.begin(), sl.batch.end(),
                     [](const Pending& a, const Pending& b) { return class_of(a.M) < class_of(b.M); });
    auto* hdr = reinterpret_cast<ServeHeader*>(sl.h_desc);
    auto* reqs = reinterpret_cast<ServeReq*>(sl.h_desc + ((sizeof(ServeHeader) + 255) & ~(size_t)255));
    std::memset(hdr, 0, sizeof(ServeHeader));
    hdr->n_req = (int)sl.batch.size();
    size_t off = 0;
    for (int i = 0; i < (int)sl.batch.size(); ++i) {
        const Pending& p = sl.batch[i];
        ServeReq& q = reqs[i];
        std::memset(&q, 0, sizeof(q));
        q.ctrl = p.ctrl; q.K = p.K; q.M = p.M; q.T = p.T;
        int seg = 1, P = 1;
        if (class_of(p.M) == 1) {
            while (2 * seg < p.M) seg <<= 1;
            P = 2;
        } else {
            while (seg < p.M && seg < 32) seg <<= 1;
            const int ppl = (p.M + seg - 1) / seg;
            while (P < ppl) P <<= 1;
        }
        q.seg = seg; q.spw = 32 / seg; q.uniform = (p.M == seg * P) ? 1 : 0;
        q.dist_half = seg * P / 2;
        q.cls = class_of(p.M);
        q.n_groups = (p.K + q.spw - 1) / q.spw;
        if (hdr->cls_count[q.cls] == 0) hdr->cls_begin[q.cls] = i;
        q.group_begin = hdr->cls_groups[q.cls];
        hdr->cls_count[q.cls] += 1;
        hdr->cls_groups[q.cls] += q.n_groups;
        std::memcpy(q.x0, p.x0, sizeof(q.x0));
        auto round = [](size_t n) { return (n + 63) & ~(size_t)63; };
        q.off_eps = off; off += round((size_t)p.K * p.T * 2);
        q.off_S = off; off += round(p.K);
        q.off_w = off; off += round(p.K);
    }
}

// Copy the costs, weights and perturbations of every completed request with an armed capture to
// its host buffer. Runs before harvest releases the slot, so the arena still holds them.
void copy_captures(bssmppi_server* s, Slot& sl)
{
    std::vector<std::pair<int, Capture>> todo;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        for (int i = 0; i < (int)sl.batch.size(); ++i) {
            Capture& c = s->capture[sl.batch[i].ctrl];
            if (!c.armed) continue;
            todo.emplace_back(i, c);
            c.armed = false;
        }
    }
    if (todo.empty()) return;
    const auto* reqs = reinterpret_cast<const ServeReq*>(sl.h_desc + ((sizeof(ServeHeader) + 255) & ~(size_t)255));
    for (auto& [i, c] : todo) {
        const ServeReq& q = reqs[i];
        const int64_t need = (int64_t)q.K * (2 + 2 * q.T);
        int64_t written = -1;
        if (need <= c.cap_floats) {
            cudaError_t e = cudaMemcpyAsync(c.h_out, sl.d_arena + q.off_S, sizeof(float) * q.K, cudaMemcpyDeviceToHost,
                                            sl.s[0]);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c.h_out + q.K, sl.d_arena + q.off_w, sizeof(float) * q.K, cudaMemcpyDeviceToHost,
                                    sl.s[0]);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c.h_out + 2 * (size_t)q.K, sl.d_arena + q.off_eps, sizeof(float) * q.K * 2 * q.T,
                                    cudaMemcpyDeviceToHost, sl.s[0]);
            if (e == cudaSuccess) e = cudaStreamSynchronize(sl.s[0]);
            written = e == cudaSuccess ? need : -2;
        }
        *c.h_written = written;
    }
}

void harvest(bssmppi_server* s, Slot& sl)
{
    copy_captures(s, sl);
    const double t = now_us(s->t0);
    std::lock_guard<std::mutex> lock(s->mu);
    for (int i = 0; i < (int)sl.batch.size(); ++i) {
        const Pending& p = sl.batch[i];
        bssmppi_result r{};
        r.req_id = p.id;
        r.ctrl_id = p.ctrl;
        r.status = BSSMPPI_OK;
        r.u0[0] = sl.h_res[i].u0[0];
        r.u0[1] = sl.h_res[i].u0[1];
        r.beta = sl.h_res[i].beta;
        r.K = p.K; r.M = p.M; r.T = p.T;
        r.t_submit_us = p.t_submit;
        r.t_start_us = sl.t_launch;
        r.t_done_us = t;
        s->done.push_back(r);
        s->in_flight[p.ctrl] = 0;
        s->stats.completed += 1;
    }
    sl.batch.clear();
    sl.busy = false;
    s->cv.notify_all();
}

// Admit pending requests in arrival order into the slot; returns true if any was admitted.
bool form_batch(bssmppi_server* s, Slot& sl)
{
    std::lock_guard<std::mutex> lock(s->mu);
    std::vector<int> order;
    for (int c = 0; c < s->n_ctrl; ++c)
        if (s->has_pending[c] && !s->in_flight[c]) order.push_back(c);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return s->pending[a].seq < s->pending[b].seq; });
    size_t used = 0;
    int64_t work = 0;
    sl.fleet = order.empty() ? -1 : s->pending[order.front()].fleet;  // the oldest request's class
    if (sl.fleet >= 0) sl.fleet_params = s->fleets[sl.fleet];
    for (int c : order) {
        if ((int)sl.batch.size() >= s->cfg.max_batch) break;
        const Pending& p = s->pending[c];
        if (p.fleet != sl.fleet) continue;  // another constants class: waits for a batch of its own
        const size_t need = request_floats(p.K, p.T);
        if (used + need > sl.arena_floats) break;  // strict arrival order: the oldest waits for room
        const int64_t w = (int64_t)p.K * p.M * p.T;
        if (!sl.batch.empty() && s->cfg.max_batch_work > 0 && work + w > s->cfg.max_batch_work) break;
        used += need;
        work += w;
        sl.batch.push_back(p);
        s->has_pending[c] = 0;
        s->in_flight[c] = 1;
    }
    if (!sl.batch.empty()) {
        s->stats.batches += 1;
        s->stats.admitted += sl.batch.size();
        if ((int64_t)sl.batch.size() > s->stats.max_batch_seen) s->stats.max_batch_seen = (int64_t)sl.batch.size();
    }
    return !sl.batch.empty();
}

void worker_loop(bssmppi_server* s)
{
    cudaSetDevice(s->device);
    while (!s->stop.load()) {
        bool progress = false;
        for (int i = 0; i < s->n_slots; ++i) {
            Slot& sl = s->slots[i];
            if (sl.busy) {
                const cudaError_t q = cudaEventQuery(sl.done);
                if (q == cudaSuccess) {
                    harvest(s, sl);
                    progress = true;
                } else if (q != cudaErrorNotReady) {
                    s->worker_error.store((int)q);
                    s->stop.store(true);
                    break;
                }
            }
        }
        for (int i = 0; i < s->n_slots && !s->stop.load(); ++i) {
            Slot& sl = s->slots[i];
            if (sl.busy || !form_batch(s, sl)) continue;
            fill_descriptors(sl);
            sl.t_launch = now_us(s->t0);
            cudaError_t e = cudaSuccess;
            if (s->cfg.use_graphs && sl.graph_fleet != sl.fleet) e = set_graph_fleet(s, sl);
            if (e == cudaSuccess) e = s->cfg.use_graphs ? cudaGraphLaunch(sl.exec, sl.s[0]) : issue_batch(s, sl);
            if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.s[0]);
            if (e != cudaSuccess) {
                s->worker_error.store((int)e);
                s->stop.store(true);
                break;
            }
            sl.busy = true;
            progress = true;
        }
        if (!progress) {
            std::unique_lock<std::mutex> lock(s->mu);
            s->cv.wait_for(lock, std::chrono::microseconds(20));
        }
    }
}

void destroy_slot(Slot& sl)
{
    if (sl.exec) cudaGraphExecDestroy(sl.exec);
    if (sl.graph) cudaGraphDestroy(sl.graph);
    for (cudaStream_t st : sl.s)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : {sl.fork, sl.join1, sl.join2, sl.done})
        if (ev) cudaEventDestroy(ev);
    if (sl.d_hdr) cudaFree(sl.d_hdr);
    if (sl.d_res) cudaFree(sl.d_res);
    if (sl.d_arena) cudaFree(sl.d_arena);
    if (sl.h_desc) cudaFreeHost(sl.h_desc);
    if (sl.h_res) cudaFreeHost(sl.h_res);
}

void destroy_server(bssmppi_server* s)
{
    if (s->worker.joinable()) {
        s->stop.store(true);
        s->cv.notify_all();
        s->worker.join();
    }
    cudaDeviceSynchronize();
    for (Slot& sl : s->slots) destroy_slot(sl);
    for (float* t : s->d_tracks)
        if (t) cudaFree(t);
    if (s->d_dp) cudaFree(s->d_dp);
    if (s->d_v) cudaFree(s->d_v);
    if (s->d_ctr) cudaFree(s->d_ctr);
    delete s;
}

}  // namespace

extern "C" {

int bssmppi_server_create(const bssmppi_server_config* cfg, bssmppi_server_t* out)
{
    if (!out) return srv_fail(nullptr, BSSMPPI_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg) return srv_fail(nullptr, BSSMPPI_EINVAL, "config is NULL");
    if (cfg->max_controllers < 1 || cfg->max_controllers > 65536) return srv_fail(nullptr, BSSMPPI_EINVAL, "max_controllers out of range [1, 65536]");
    if (cfg->max_batch < 1 || cfg->max_batch > 4096) return srv_fail(nullptr, BSSMPPI_EINVAL, "max_batch out of range [1, 4096]");
    if (cfg->T_max < 1 || cfg->T_max > BSSMPPI_T_MAX) return srv_fail(nullptr, BSSMPPI_EINVAL, "T_max out of range [1, 256]");
    if (cfg->slots < 1 || cfg->slots > kServeMaxSlots) return srv_fail(nullptr, BSSMPPI_EINVAL, "slots out of range [1, 8]");
    if (cfg->hbm_budget_bytes < (size_t)(1 << 20)) return srv_fail(nullptr, BSSMPPI_EINVAL, "hbm_budget_bytes must be >= 1 MiB");
    auto* s = new bssmppi_server();
    s->cfg = *cfg;
    s->n_slots = cfg->slots;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
    const int C = cfg->max_controllers;
    s->h_dp.resize(C);
    s->d_tracks.assign(C, nullptr);
    s->pending.resize(C);
    s->has_pending.assign(C, 0);
    s->in_flight.assign(C, 0);
    s->capture.resize(C);
    s->fleet_of.assign(C, 0);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_dp, sizeof(DevParams) * C);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_v, sizeof(float) * 2 * cfg->T_max * C);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_ctr, sizeof(uint32_t) * C);
    if (e == cudaSuccess) e = cudaMemset(s->d_v, 0, sizeof(float) * 2 * cfg->T_max * C);
    if (e == cudaSuccess) e = cudaMemset(s->d_ctr, 0, sizeof(uint32_t) * C);
    const size_t hdr_bytes = (sizeof(ServeHeader) + 255) & ~(size_t)255;
    s->desc_bytes = hdr_bytes + sizeof(ServeReq) * cfg->max_batch;
    s->res_bytes = sizeof(ServeResult) * cfg->max_batch;
    for (int c = 0; c < kServeClasses; ++c)
        s->roll_smem[c] = sizeof(ServeItem) * kServeWarps
                        + sizeof(float) * kServeWarps * serve_spw_max(c) * 2 * cfg->T_max;
    const auto smem_attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(serve_rollout_kernel<1>, smem_attr, (int)s->roll_smem[0]);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(serve_rollout_kernel<2>, smem_attr, (int)s->roll_smem[1]);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(serve_rollout_kernel<4>, smem_attr, (int)s->roll_smem[2]);
    if (e == cudaSuccess) {
        int nb[3] = {0, 0, 0};
        const int tb = kServeWarps * kWarp;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb[0], serve_rollout_kernel<1>, tb, s->roll_smem[0]);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb[1], serve_rollout_kernel<2>, tb, s->roll_smem[1]);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb[2], serve_rollout_kernel<4>, tb, s->roll_smem[2]);
        for (int i = 0; i < 3; ++i) s->roll_grid[i] = std::max(1, nb[i]) * s->sms;
    }
    const size_t arena_bytes = cfg->hbm_budget_bytes / cfg->slots;
    for (int i = 0; i < s->n_slots && e == cudaSuccess; ++i) {
        Slot& sl = s->slots[i];
        sl.arena_floats = arena_bytes / sizeof(float);
        for (int j = 0; j < 3 && e == cudaSuccess; ++j) e = cudaStreamCreateWithFlags(&sl.s[j], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.join1, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.join2, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&sl.d_hdr), s->desc_bytes);
        if (e == cudaSuccess) sl.d_reqs = reinterpret_cast<ServeReq*>(reinterpret_cast<unsigned char*>(sl.d_hdr) + hdr_bytes);
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&sl.d_res), s->res_bytes);
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&sl.d_arena), arena_bytes);
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&sl.h_desc), s->desc_bytes);
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&sl.h_res), s->res_bytes);
        if (e == cudaSuccess) {
            std::memset(sl.h_desc, 0, s->desc_bytes);  // an empty batch: n_req = 0
            std::memset(sl.h_res, 0, s->res_bytes);
        }
        if (e == cudaSuccess && cfg->use_graphs) {
            e = cudaStreamBeginCapture(sl.s[0], cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const cudaError_t e_issue = issue_batch(s, sl);
                e = cudaStreamEndCapture(sl.s[0], &sl.graph);
                if (e == cudaSuccess) e = e_issue;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&sl.exec, sl.graph, 0);
            if (e == cudaSuccess) e = find_rollout_nodes(sl);
        }
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        const std::string msg = std::string("server create: ") + cudaGetErrorString(e);
        destroy_server(s);
        return srv_fail(nullptr, e == cudaErrorMemoryAllocation ? BSSMPPI_ENOMEM : BSSMPPI_ECUDA, msg);
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return BSSMPPI_OK;
}

int bssmppi_server_add_controller(bssmppi_server_t s, const bssmppi_params* p, int32_t* ctrl_id)
{
    if (!s || !p || !ctrl_id) return srv_fail(s, BSSMPPI_EINVAL, "NULL argument");
    if (p->model != BSSMPPI_MODEL_BICYCLE6) return srv_fail(s, BSSMPPI_ENOTSUP, "the server runs the bicycle model");
    if (p->record_moments || !p->compensated) return srv_fail(s, BSSMPPI_ENOTSUP, "the server runs compensated solves without recorded moments");
    if (p->resample) return srv_fail(s, BSSMPPI_ENOTSUP, "the server runs persistent particles (resample = 0)");
    DevParams d{};
    int P = 1;
    std::string why;
    const int rc = derive_params(p, d, P, why);
    if (rc != BSSMPPI_OK) return srv_fail(s, rc, why);
    int id;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->n_ctrl >= s->cfg.max_controllers) {
            s->err = "controller table full";
            return BSSMPPI_EBUSY;
        }
        id = s->n_ctrl;
    }
    const int ntab = d.n_track_mask + 1;
    std::vector<float> tab(ntab + 1);
    std::memcpy(tab.data(), p->track_kappa, sizeof(float) * ntab);
    tab[ntab] = tab[0];
    float* d_track = nullptr;
    cudaError_t e = cudaMalloc(&d_track, sizeof(float) * (ntab + 1));
    if (e == cudaSuccess) e = cudaMemcpy(d_track, tab.data(), sizeof(float) * (ntab + 1), cudaMemcpyHostToDevice);
    d.kappa = d_track;
    if (e == cudaSuccess) e = cudaMemcpy(s->d_dp + id, &d, sizeof(DevParams), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (d_track) cudaFree(d_track);
        return srv_fail(s, BSSMPPI_ECUDA, std::string("add_controller: ") + cudaGetErrorString(e));
    }
    // its constants class: everything but the Philox keys, the track and the per-request sizes
    DevParams key = d;
    key.key0 = key.key1 = 0u;
    std::memset(key.rk0, 0, sizeof(key.rk0));
    std::memset(key.rk1, 0, sizeof(key.rk1));
    key.kappa = nullptr;
    key.track_scale = 0.0f;
    key.n_track_mask = 0;
    key.K = key.M = key.T = key.seg = key.spw = key.uniform = key.dist_half = key.k_off = key.K_norm = 0;
    key.Mf = key.invM = key.invM1 = 0.0f;
    std::lock_guard<std::mutex> lock(s->mu);
    int fleet = -1;
    for (int f = 0; f < (int)s->fleets.size() && fleet < 0; ++f)
        if (std::memcmp(&s->fleets[f], &key, sizeof(DevParams)) == 0) fleet = f;
    if (fleet < 0) {
        fleet = (int)s->fleets.size();
        s->fleets.push_back(key);
    }
    s->fleet_of[id] = fleet;
    s->h_dp[id] = d;
    s->d_tracks[id] = d_track;
    s->n_ctrl = id + 1;
    *ctrl_id = id;
    return BSSMPPI_OK;
}

int bssmppi_server_submit(bssmppi_server_t s, int32_t ctrl_id, const float* h_x0, int32_t K, int32_t M, int32_t T,
                          uint64_t req_id)
{
    if (!s || !h_x0) return srv_fail(s, BSSMPPI_EINVAL, "NULL argument");
    if (K < 1 || K > BSSMPPI_K_MAX) return srv_fail(s, BSSMPPI_EINVAL, "K out of range [1, 2^20]");
    if (M < 2 || M > 128) return srv_fail(s, BSSMPPI_EINVAL, "M out of range [2, 128] for serving");
    if (T < 1 || T > s->cfg.T_max) return srv_fail(s, BSSMPPI_EINVAL, "T out of range [1, T_max]");
    if (request_floats(K, T) > s->slots[0].arena_floats) return srv_fail(s, BSSMPPI_ENOMEM, "request larger than a slot's HBM arena");
    if (s->worker_error.load() != 0) return srv_fail(s, BSSMPPI_ECUDA, "server stopped after a CUDA error");
    std::lock_guard<std::mutex> lock(s->mu);
    if (ctrl_id < 0 || ctrl_id >= s->n_ctrl) {
        s->err = "unknown controller";
        return BSSMPPI_EINVAL;
    }
    Pending p;
    p.id = req_id; p.ctrl = ctrl_id; p.K = K; p.M = M; p.T = T; p.fleet = s->fleet_of[ctrl_id];
    std::memcpy(p.x0, h_x0, sizeof(p.x0));
    p.t_submit = now_us(s->t0);
    p.seq = s->seq++;
    s->stats.submitted += 1;
    if (s->has_pending[ctrl_id]) {  // superseded by the newer state estimate
        const Pending& old = s->pending[ctrl_id];
        bssmppi_result r{};
        r.req_id = old.id;
        r.ctrl_id = ctrl_id;
        r.status = BSSMPPI_EBUSY;
        r.K = old.K; r.M = old.M; r.T = old.T;
        r.t_submit_us = old.t_submit;
        r.t_start_us = -1.0;
        r.t_done_us = p.t_submit;
        s->done.push_back(r);
        s->stats.superseded += 1;
    }
    s->pending[ctrl_id] = p;
    s->has_pending[ctrl_id] = 1;
    s->cv.notify_all();
    return BSSMPPI_OK;
}

int bssmppi_server_poll(bssmppi_server_t s, bssmppi_result* out, int32_t max, int32_t* n)
{
    if (!s || !n || (max > 0 && !out)) return srv_fail(s, BSSMPPI_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    const int k = (int)std::min<size_t>(s->done.size(), (size_t)std::max(0, max));
    std::copy(s->done.begin(), s->done.begin() + k, out);
    s->done.erase(s->done.begin(), s->done.begin() + k);
    *n = k;
    return s->worker_error.load() ? BSSMPPI_ECUDA : BSSMPPI_OK;
}

int bssmppi_server_drain(bssmppi_server_t s, int32_t timeout_ms)
{
    if (!s) return srv_fail(nullptr, BSSMPPI_EINVAL, "NULL server");
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    std::unique_lock<std::mutex> lock(s->mu);
    while (true) {
        bool idle = true;
        for (int c = 0; c < s->n_ctrl && idle; ++c) idle = !s->has_pending[c] && !s->in_flight[c];
        if (idle) return BSSMPPI_OK;
        if (s->worker_error.load() != 0) {
            s->err = "server stopped after a CUDA error";
            return BSSMPPI_ECUDA;
        }
        if (s->cv.wait_until(lock, deadline) == std::cv_status::timeout) {
            s->err = "drain timed out";
            return BSSMPPI_ETIMEOUT;
        }
    }
}

int bssmppi_server_get_state(bssmppi_server_t s, int32_t ctrl_id, float* h_v, uint32_t* counter)
{
    if (!s || !h_v || !counter) return srv_fail(s, BSSMPPI_EINVAL, "NULL argument");
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (ctrl_id < 0 || ctrl_id >= s->n_ctrl) {
            s->err = "unknown controller";
            return BSSMPPI_EINVAL;
        }
        if (s->has_pending[ctrl_id] || s->in_flight[ctrl_id]) {
            s->err = "controller has work queued or in flight";
            return BSSMPPI_EBUSY;
        }
    }
    cudaError_t e = cudaMemcpy(h_v, s->d_v + (size_t)ctrl_id * 2 * s->cfg.T_max, sizeof(float) * 2 * s->cfg.T_max,
                               cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(counter, s->d_ctr + ctrl_id, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? BSSMPPI_OK : srv_fail(s, BSSMPPI_ECUDA, cudaGetErrorString(e));
}

int bssmppi_server_set_state(bssmppi_server_t s, int32_t ctrl_id, const float* h_v, uint32_t counter)
{
    if (!s || !h_v) return srv_fail(s, BSSMPPI_EINVAL, "NULL argument");
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (ctrl_id < 0 || ctrl_id >= s->n_ctrl) {
            s->err = "unknown controller";
            return BSSMPPI_EINVAL;
        }
        if (s->has_pending[ctrl_id] || s->in_flight[ctrl_id]) {
            s->err = "controller has work queued or in flight";
            return BSSMPPI_EBUSY;
        }
    }
    cudaError_t e = cudaMemcpy(s->d_v + (size_t)ctrl_id * 2 * s->cfg.T_max, h_v, sizeof(float) * 2 * s->cfg.T_max,
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->d_ctr + ctrl_id, &counter, sizeof(uint32_t), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? BSSMPPI_OK : srv_fail(s, BSSMPPI_ECUDA, cudaGetErrorString(e));
}

int bssmppi_server_capture(bssmppi_server_t s, int32_t ctrl_id, float* h_out, int64_t cap_floats, int64_t* h_written)
{
    if (!s || !h_out || !h_written) return srv_fail(s, BSSMPPI_EINVAL, "NULL argument");
    if (cap_floats < 3) return srv_fail(s, BSSMPPI_EINVAL, "cap_floats must hold at least one sample");
    std::lock_guard<std::mutex> lock(s->mu);
    if (ctrl_id < 0 || ctrl_id >= s->n_ctrl) {
        s->err = "unknown controller";
        return BSSMPPI_EINVAL;
    }
    if (s->has_pending[ctrl_id] || s->in_flight[ctrl_id]) {
        s->err = "controller has work queued or in flight";
        return BSSMPPI_EBUSY;
    }
    *h_written = 0;
    s->capture[ctrl_id] = Capture{h_out, cap_floats, h_written, true};
    return BSSMPPI_OK;
}

int bssmppi_server_get_stats(bssmppi_server_t s, bssmppi_server_stats* out)
{
    if (!s || !out) return srv_fail(s, BSSMPPI_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    *out = s->stats;
    int64_t q = 0;
    for (int c = 0; c < s->n_ctrl; ++c) q += s->has_pending[c] ? 1 : 0;
    out->queued = q;
    out->now_us = now_us(s->t0);
    return BSSMPPI_OK;
}

const char* bssmppi_server_last_error(bssmppi_server_t s)
{
    if (!s) return bssmppi_last_error(nullptr);
    std::lock_guard<std::mutex> lock(s->mu);
    thread_local std::string copy;
    copy = s->err;
    return copy.c_str();
}

int bssmppi_server_destroy(bssmppi_server_t s)
{
    if (!s) return BSSMPPI_OK;
    destroy_server(s);
    return BSSMPPI_OK;
}

}  // extern "C"
