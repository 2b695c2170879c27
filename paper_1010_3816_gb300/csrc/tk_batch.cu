// tk_batch.cu -- many independent solvers advanced by one kernel launch per
// inner Lax-Wendroff tick, replayed from a captured CUDA graph, with the
// segment length chosen by timing candidates on the batch itself.
//
// Members may differ in every grid parameter (Nr, Ntheta, the angular packing
// K, a, m, ...) and in their number of inner steps per outer step k_i; they
// share the outer step dt.  One outer step is kmax = lcm(k_i) ticks; member i
// steps on ticks t with (t + 1) % (kmax / k_i) == 0 and writes its waveform
// sample on the last tick.  Each tick is one launch of a persistent kernel:
// warps take work items (member, column range) from a queue in device memory
// until it is empty; items are ordered by decreasing cost (columns x rows),
// so the longest ones start first.  A warp recomputes the half-step value at
// the left edge of its item, so items are independent; the arithmetic of
// every half node and node is the same code as the single-solver kernel, and
// the results are bit-identical to stepping each solver alone.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "tk_solver_impl.h"
#include "tk_stencil.cuh"

namespace tk {
namespace {

constexpr int kBatchThreads = 128;

struct BatchMember {
    void *u0, *u1;            // the member's two time levels
    const void *half, *node;  // folded coefficient tables
    int Nr, K;
    int substeps, ratio;      // k_i and kmax / k_i
    int level0;               // level holding the state when the call started
    double eh, en;            // dt_i / 4, dt_i / 2
    double *wave;
    long long cap;
    long long *sample;        // the member's device sample counter
    const double *w_row;
    ObsDev obs;
};

struct BatchItem {
    int member, i0, i1;
};

// Columns [i0, i1) of one member: the single-solver sweep with the left half
// node recomputed.
template <typename T, int K>
__device__ void sweep(const BatchMember &m, const T *__restrict__ u_in, T *__restrict__ u_out,
                      int i0, int i1, bool observe_now, int lane)
{
    constexpr int NP = 32 * K;
    constexpr size_t SP = 4 * NP, HP = (size_t)kNCH * NP, NQ = (size_t)kNCN * NP;
    const T *half = (const T *)m.half;
    const T *node = (const T *)m.node;
    const T eh = (T)m.eh, en = (T)m.en;
    const int Nr = m.Nr;
    const int row = lane * K;
    T ua[4][K], hm[4][K];
    load_col<T, K>(u_in + (size_t)i0 * SP + row, ua);
    if (i0 > 0) {
        T ul[4][K];
        load_col<T, K>(u_in + (size_t)(i0 - 1) * SP + row, ul);
        half_node<T, K>(ul, ua, half + (size_t)(i0 - 1) * HP + row, hm);
    } else {
        zero_col<T, K>(hm);
    }
    for (int i = i0; i < i1; ++i) {
        T uc[4][K], hp[4][K], o[4][K];
        if (i + 1 < Nr) {
            load_col<T, K>(u_in + (size_t)(i + 1) * SP + row, uc);
            half_node<T, K>(ua, uc, half + (size_t)i * HP + row, hp);
        } else {
            zero_col<T, K>(uc);
            zero_col<T, K>(hp);
        }
        full_node<T, K>(hm, hp, ua, node + (size_t)i * NQ + row, en, o);
        if (i == 0 || i == Nr - 1) zero_col<T, K>(o);
        store_col<T, K>(u_out + (size_t)i * SP + row, o);
        if (observe_now) observe<T, K>(i, lane, o, m.obs, m.wave, m.cap, m.sample, m.w_row);
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int t = 0; t < K; ++t) {
                hm[c][t] = hp[c][t];
                ua[c][t] = uc[c][t];
            }
    }
}

// One tick for every participating member.  ctr[0]: next work item, ctr[1]:
// blocks finished.  The last block to finish empties the queue for the next
// launch and, after the last tick of an outer step, moves every member's
// sample counter on (every block has read them by then).
template <typename T>
__global__ void __launch_bounds__(kBatchThreads)
batch_step_kernel(const BatchMember *__restrict__ mem, int nmem, const BatchItem *__restrict__ items,
                  int nitems, int tick, int kmax, int outer, unsigned int *ctr)
{
    chain_start();   // the queue counters and the members' levels are the previous tick's
    const int lane = threadIdx.x & 31;
    const bool last_tick = (tick == kmax - 1);
    for (;;) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(&ctr[0], 1u);
        it = __shfl_sync(kFull, it, 0);
        if (it >= nitems) break;
        const BatchItem w = items[it];
        const BatchMember &m = mem[w.member];
        const int before = outer * m.substeps + tick / m.ratio;
        const int lev = m.level0 ^ (before & 1);
        const T *u_in = (const T *)(lev ? m.u1 : m.u0);
        T *u_out = (T *)(lev ? m.u0 : m.u1);
        const bool obs_now = last_tick && m.obs.n > 0;
        switch (m.K) {
        case 1: sweep<T, 1>(m, u_in, u_out, w.i0, w.i1, obs_now, lane); break;
        case 2: sweep<T, 2>(m, u_in, u_out, w.i0, w.i1, obs_now, lane); break;
        default: sweep<T, 4>(m, u_in, u_out, w.i0, w.i1, obs_now, lane); break;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int prev = atomicAdd(&ctr[1], 1u);
        if (prev == gridDim.x - 1) {
            atomicExch(&ctr[0], 0u);
            if (last_tick)
                for (int k = 0; k < nmem; ++k)
                    if (mem[k].obs.n > 0) atomicAdd((unsigned long long *)mem[k].sample, 1ull);
            atomicExch(&ctr[1], 0u);
            __threadfence();
        }
    }
}

}  // namespace

static int batch_resident_blocks(int precision)
{
    int n = 0;
    cudaError_t e = precision == 0
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<double>, kBatchThreads, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<float>, kBatchThreads, 0);
    return (e != cudaSuccess || n < 1) ? 1 : n;
}

static cudaError_t launch_batch_tick(int precision, int blocks, const BatchMember *mem, int nmem,
                                     const BatchItem *items, int nitems, int tick, int kmax,
                                     int outer, unsigned int *ctr, cudaStream_t st)
{
    if (precision == 0)
        return launch_chained(batch_step_kernel<double>, (unsigned)blocks, kBatchThreads, 0, st, mem,
                              nmem, items, nitems, tick, kmax, outer, ctr);
    return launch_chained(batch_step_kernel<float>, (unsigned)blocks, kBatchThreads, 0, st, mem, nmem,
                          items, nitems, tick, kmax, outer, ctr);
}

}  // namespace tk

struct tk_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    int precision = 0;
    int n = 0;
    std::vector<tk_solver *> mem;
    int kmax = 1;
    int blocks = 1;
    int seg = 32;
    // step the members one after another, each as tk_step would (segment
    // length 0), instead of the work queue
    bool per_member = false;
    tk::BatchMember *d_mem = nullptr;
    tk::BatchItem *d_items = nullptr;
    size_t items_cap = 0;
    std::vector<int> tick_off, tick_n;
    unsigned int *d_ctr = nullptr;
    // graph of `graph_outer` outer steps
    int graph_chunk = -1;
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_outer = 0;
    std::vector<long long> graph_key;
    char err[512] = {0};
};

namespace {

tk_status bfail(tk_batch *B, tk_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    if (B) vsnprintf(B->err, sizeof B->err, fmt, ap);
    va_end(ap);
    return st;
}

#define TKB_CUDA(B, call)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return bfail((B), e_ == cudaErrorMemoryAllocation ? TK_ERR_OOM : TK_ERR_CUDA,   \
                         "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

int gcd(int a, int b) { return b ? gcd(b, a % b) : a; }

// Work items of every tick for segment length `seg`, longest first.
tk_status build_items(tk_batch *B, int seg)
{
    std::vector<tk::BatchItem> all;
    B->tick_off.assign(B->kmax, 0);
    B->tick_n.assign(B->kmax, 0);
    for (int t = 0; t < B->kmax; ++t) {
        std::vector<std::pair<long long, tk::BatchItem>> v;
        for (int k = 0; k < B->n; ++k) {
            const tk_solver *S = B->mem[k];
            const int ratio = B->kmax / S->substeps;
            if ((t + 1) % ratio) continue;
            const int pieces = (S->Nr + seg - 1) / seg;
            for (int p = 0; p < pieces; ++p) {
                tk::BatchItem it;
                it.member = k;
                it.i0 = (int)((long long)p * S->Nr / pieces);
                it.i1 = (int)((long long)(p + 1) * S->Nr / pieces);
                v.push_back({(long long)(it.i1 - it.i0) * S->K, it});
            }
        }
        std::stable_sort(v.begin(), v.end(),
                         [](const auto &a, const auto &b) { return a.first > b.first; });
        B->tick_off[t] = (int)all.size();
        B->tick_n[t] = (int)v.size();
        for (auto &x : v) all.push_back(x.second);
    }
    // a replay still in flight may read the current items
    TKB_CUDA(B, cudaStreamSynchronize(B->stream));
    if (all.size() > B->items_cap) {
        if (B->d_items) cudaFree(B->d_items);
        B->d_items = nullptr;
        B->items_cap = 0;
        TKB_CUDA(B, cudaMalloc(&B->d_items, all.size() * sizeof(tk::BatchItem)));
        B->items_cap = all.size();
    }
    TKB_CUDA(B, cudaMemcpy(B->d_items, all.data(), all.size() * sizeof(tk::BatchItem),
                           cudaMemcpyHostToDevice));
    B->graph_key.clear();
    B->seg = seg;
    return TK_OK;
}

// Upload the member table for a call that starts now.
tk_status upload_members(tk_batch *B)
{
    std::vector<tk::BatchMember> h(B->n);
    for (int k = 0; k < B->n; ++k) {
        tk_solver *S = B->mem[k];
        tk::BatchMember &m = h[k];
        memset(&m, 0, sizeof m);
        m.u0 = S->u[0];
        m.u1 = S->u[1];
        m.half = S->half;
        m.node = S->node;
        m.Nr = S->Nr;
        m.K = S->K;
        m.substeps = S->substeps;
        m.ratio = B->kmax / S->substeps;
        m.level0 = S->cur;
        m.eh = 0.25 * (S->dt / S->substeps);
        m.en = 0.5 * (S->dt / S->substeps);
        m.wave = S->wave;
        m.cap = S->wave_cap;
        m.sample = S->ctr;
        m.w_row = S->w_row;
        tk::StepLaunch L;
        tkh::fill_launch(S, L);
        m.obs = L.obs;
    }
    TKB_CUDA(B, cudaMemcpyAsync(B->d_mem, h.data(), B->n * sizeof(tk::BatchMember),
                                cudaMemcpyHostToDevice, B->stream));
    // pageable source: the copy is staged before cudaMemcpyAsync returns
    return TK_OK;
}

tk_status enqueue(tk_batch *B, int outer_steps, cudaStream_t st)
{
    for (int o = 0; o < outer_steps; ++o)
        for (int t = 0; t < B->kmax; ++t) {
            if (B->tick_n[t] == 0) continue;
            TKB_CUDA(B, tk::launch_batch_tick(B->precision, B->blocks, B->d_mem, B->n,
                                              B->d_items + B->tick_off[t], B->tick_n[t], t, B->kmax,
                                              o, B->d_ctr, st));
        }
    return TK_OK;
}

// Outer steps per replay: every member must take an even number of steps so
// that each replay starts from the same levels.
int chunk_of(const tk_batch *B)
{
    int unit = 1;
    for (tk_solver *S : B->mem)
        if (S->substeps % 2) unit = 2;
    if (B->graph_chunk == 0) return 0;
    int want = B->graph_chunk > 0 ? B->graph_chunk : std::max(1, 64 / B->kmax);
    return ((want + unit - 1) / unit) * unit;
}

// The graph bakes the item list and its per-tick ranges, the grid and the
// chunk; member pointers, levels and waveform buffers are read from the
// member table at run time.
std::vector<long long> graph_key_of(const tk_batch *B)
{
    std::vector<long long> key = {B->seg, B->blocks, chunk_of(B), (long long)(uintptr_t)B->d_items};
    return key;
}

tk_status advance_members(tk_batch *B, int n)
{
    for (tk_solver *S : B->mem) {
        if ((long long)n * S->substeps % 2) S->cur ^= 1;
        S->count += n;
        S->steps_done += n;
    }
    return TK_OK;
}

tk_status check_members(tk_batch *B)
{
    for (tk_solver *S : B->mem)
        if (!S->have_state || !S->state_valid)
            return bfail(B, TK_ERR_STATE, "tk_batch: a member has no valid state");
    return TK_OK;
}

}  // namespace

extern "C" {

tk_status tk_batch_create(tk_batch **out, tk_solver *const *members, int n)
{
    if (!out || !members || n < 1) return TK_ERR_ARG;
    *out = nullptr;
    tk_batch *B = new (std::nothrow) tk_batch();
    if (!B) return TK_ERR_OOM;
    B->n = n;
    B->mem.assign(members, members + n);
    tk_solver *S0 = members[0];
    if (!S0) {
        delete B;
        return TK_ERR_ARG;
    }
    B->device = S0->device;
    B->stream = S0->stream;
    B->precision = S0->precision;
    long long lcm = 1;
    for (tk_solver *S : B->mem) {
        if (!S || S->device != B->device || S->precision != B->precision || S->dt != S0->dt) {
            delete B;
            return TK_ERR_ARG;
        }
        lcm = lcm / gcd((int)lcm, S->substeps) * S->substeps;
        if (lcm > 64) {
            delete B;
            return TK_ERR_ARG;
        }
    }
    B->kmax = (int)lcm;
    tk_status st = TK_OK;
    if (cudaSetDevice(B->device) != cudaSuccess) st = TK_ERR_CUDA;
    if (st == TK_OK && cudaMalloc(&B->d_mem, n * sizeof(tk::BatchMember)) != cudaSuccess) st = TK_ERR_OOM;
    if (st == TK_OK && cudaMalloc(&B->d_ctr, 2 * sizeof(unsigned int)) != cudaSuccess) st = TK_ERR_OOM;
    if (st == TK_OK && cudaMemset(B->d_ctr, 0, 2 * sizeof(unsigned int)) != cudaSuccess) st = TK_ERR_CUDA;
    if (st == TK_OK) {
        B->blocks = S0->num_sms * tk::batch_resident_blocks(B->precision);
        long long cols = 0;
        for (tk_solver *S : B->mem) cols += S->Nr;
        // default: about four items per warp of the resident grid
        const long long warps = (long long)B->blocks * (tk::kBatchThreads / 32);
        int seg = (int)std::max(8LL, cols / std::max(1LL, 4 * warps));
        st = build_items(B, seg);
    }
    if (st != TK_OK) {
        cudaGetLastError();
        if (B->d_mem) cudaFree(B->d_mem);
        if (B->d_ctr) cudaFree(B->d_ctr);
        if (B->d_items) cudaFree(B->d_items);
        delete B;
        return st;
    }
    *out = B;
    return TK_OK;
}

tk_status tk_batch_set_segment(tk_batch *B, int seg)
{
    if (!B || seg == 1 || seg < 0)
        return bfail(B, TK_ERR_ARG, "tk_batch_set_segment: seg must be 0 or >= 2");
    TKB_CUDA(B, cudaSetDevice(B->device));
    B->per_member = (seg == 0);
    if (B->per_member) return TK_OK;
    return build_items(B, seg);
}

tk_status tk_batch_set_graph_chunk(tk_batch *B, int outer_steps)
{
    if (!B || outer_steps < -1) return bfail(B, TK_ERR_ARG, "tk_batch_set_graph_chunk: bad value");
    B->graph_chunk = outer_steps;
    return TK_OK;
}

tk_status tk_batch_step(tk_batch *B, int n)
{
    if (!B) return TK_ERR_ARG;
    if (n < 0) return bfail(B, TK_ERR_ARG, "tk_batch_step: n < 0");
    TKB_CUDA(B, cudaSetDevice(B->device));
    tk_status st = check_members(B);
    if (st != TK_OK || n == 0) return st;
    if (B->per_member) {
        for (tk_solver *S : B->mem) {
            st = tk_step(S, n);
            if (st != TK_OK) return bfail(B, st, "tk_batch_step: %s", S->err);
        }
        return TK_OK;
    }
    for (tk_solver *S : B->mem) {
        st = tkh::ensure_wave(S, S->count + n);
        if (st != TK_OK) return bfail(B, st, "tk_batch_step: %s", S->err);
    }
    st = upload_members(B);
    if (st != TK_OK) return st;
    const int chunk = chunk_of(B);
    int done = 0;
    if (chunk > 0 && n >= chunk) {
        const std::vector<long long> key = graph_key_of(B);
        if (!B->graph || key != B->graph_key) {
            if (B->graph) cudaGraphExecDestroy(B->graph);
            B->graph = nullptr;
            if (!B->capture_stream)
                TKB_CUDA(B, cudaStreamCreateWithFlags(&B->capture_stream, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            TKB_CUDA(B, cudaStreamBeginCapture(B->capture_stream, cudaStreamCaptureModeThreadLocal));
            tk_status es = enqueue(B, chunk, B->capture_stream);
            cudaError_t e = cudaStreamEndCapture(B->capture_stream, &g);
            if (es != TK_OK) {
                if (g) cudaGraphDestroy(g);
                return es;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&B->graph, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                B->graph = nullptr;
                return bfail(B, TK_ERR_CUDA, "tk_batch_step: graph capture: %s", cudaGetErrorString(e));
            }
            B->graph_key = key;
        }
        for (; done + chunk <= n; done += chunk) TKB_CUDA(B, cudaGraphLaunch(B->graph, B->stream));
    }
    // the levels are back to level0 after whole replays, so the rest restarts at outer = 0
    st = enqueue(B, n - done, B->stream);
    if (st != TK_OK) return st;
    return advance_members(B, n);
}

tk_status tk_batch_tune(tk_batch *B, int trial_steps, int *best_seg, double *best_ms)
{
    if (!B || trial_steps < 1) return bfail(B, TK_ERR_ARG, "tk_batch_tune: trial_steps < 1");
    TKB_CUDA(B, cudaSetDevice(B->device));
    tk_status st = check_members(B);
    if (st != TK_OK) return st;
    for (tk_solver *S : B->mem) {
        st = tkh::ensure_wave(S, S->count + 2 * trial_steps);
        if (st != TK_OK) return bfail(B, st, "tk_batch_tune: %s", S->err);
    }
    // keep every member's state and sample counter, restore them after each trial
    std::vector<void *> keep(B->n, nullptr);
    std::vector<long long> keep_ctr(B->n);
    size_t bytes_total = 0;
    for (int k = 0; k < B->n; ++k) {
        tk_solver *S = B->mem[k];
        const size_t bytes = (size_t)S->Nr * 4 * S->NP * S->esz;
        bytes_total += bytes;
        if (cudaMalloc(&keep[k], bytes) != cudaSuccess) {
            for (void *p : keep)
                if (p) cudaFree(p);
            cudaGetLastError();
            return bfail(B, TK_ERR_OOM, "tk_batch_tune: no room to save the states (%zu bytes)", bytes_total);
        }
        TKB_CUDA(B, cudaMemcpyAsync(keep[k], S->u[S->cur], bytes, cudaMemcpyDeviceToDevice, B->stream));
        TKB_CUDA(B, cudaMemcpyAsync(&keep_ctr[k], S->ctr, sizeof(long long), cudaMemcpyDeviceToHost, B->stream));
    }
    TKB_CUDA(B, cudaStreamSynchronize(B->stream));
    const int old_chunk = B->graph_chunk;
    B->graph_chunk = 0;   // trials launch directly
    // the search space: segment length (columns per work item) x grid size
    // (blocks per SM, up to the resident maximum; fewer blocks leave each
    // warp more items of the queue)
    const int candidates[] = {4, 8, 12, 16, 24, 32, 48, 64, 96, 128};
    const int sms = B->mem[0]->num_sms, max_per_sm = tk::batch_resident_blocks(B->precision);
    int best = B->seg, best_blocks = B->blocks;
    double best_t = 1e300;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int per_sm = max_per_sm; per_sm >= 1 && st == TK_OK; --per_sm)
    for (int seg : candidates) {
        B->blocks = sms * per_sm;
        st = build_items(B, seg);
        if (st != TK_OK) break;
        st = upload_members(B);
        if (st != TK_OK) break;
        cudaEventRecord(e0, B->stream);
        st = enqueue(B, trial_steps, B->stream);
        cudaEventRecord(e1, B->stream);
        if (st != TK_OK) break;
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_t) {
            best_t = ms;
            best = seg;
            best_blocks = B->blocks;
        }
        for (int k = 0; k < B->n; ++k) {   // undo the trial
            tk_solver *S = B->mem[k];
            cudaMemcpyAsync(S->u[S->cur], keep[k], (size_t)S->Nr * 4 * S->NP * S->esz,
                            cudaMemcpyDeviceToDevice, B->stream);
            cudaMemcpyAsync(S->ctr, &keep_ctr[k], sizeof(long long), cudaMemcpyHostToDevice, B->stream);
        }
        cudaStreamSynchronize(B->stream);
    }
    // The best work-queue pair against the other strategy, the members one
    // after another through tk_step: each timed on the device at trial_steps
    // and 2 trial_steps outer steps, and compared by the difference, so that
    // fixed start-up costs (of each launch sequence, of each member's
    // cooperative launch and host synchronization), which a long
    // tk_batch_step amortizes, count for neither.
    double queue_ms = 1e300;
    if (st == TK_OK) {
        B->blocks = best_blocks;
        st = build_items(B, best);
        if (st == TK_OK) st = upload_members(B);
        double t[2] = {0.0, 0.0};
        for (int r = 0; r < 2 && st == TK_OK; ++r) {
            cudaEventRecord(e0, B->stream);
            st = enqueue(B, (r + 1) * trial_steps, B->stream);
            cudaEventRecord(e1, B->stream);
            if (st != TK_OK) break;
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            t[r] = ms;
            for (int k = 0; k < B->n; ++k) {   // undo the trial
                tk_solver *S = B->mem[k];
                cudaMemcpyAsync(S->u[S->cur], keep[k], (size_t)S->Nr * 4 * S->NP * S->esz,
                                cudaMemcpyDeviceToDevice, B->stream);
                cudaMemcpyAsync(S->ctr, &keep_ctr[k], sizeof(long long), cudaMemcpyHostToDevice, B->stream);
            }
            cudaStreamSynchronize(B->stream);
        }
        queue_ms = t[1] - t[0];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // Only members that each fill the GPU alone (one block per SM in their own
    // persistent launch) are candidates for the other strategy: smaller ones
    // are what the work queue is for (24 members of 1601 x 32 run 1.18x
    // faster through it), and short trials of direct launches understate it.
    bool all_fill = true;
    for (tk_solver *S : B->mem) all_fill = all_fill && S->persist && S->warps != tk::kNarrowWarps;
    bool per_member = false;
    if (st == TK_OK && all_fill) {
        std::vector<int> cur0(B->n);
        std::vector<long long> count0(B->n), done0(B->n);
        for (int k = 0; k < B->n; ++k) {
            cur0[k] = B->mem[k]->cur;
            count0[k] = B->mem[k]->count;
            done0[k] = B->mem[k]->steps_done;
        }
        for (tk_solver *S : B->mem) {
            st = tkh::ensure_wave(S, S->count + 2 * trial_steps);
            if (st != TK_OK) {
                bfail(B, st, "tk_batch_tune: %s", S->err);
                break;
            }
        }
        cudaEvent_t a0, a1;
        cudaEventCreate(&a0);
        cudaEventCreate(&a1);
        double ms_n[2] = {0.0, 0.0};
        for (int r = 0; r < 2 && st == TK_OK; ++r) {
            cudaDeviceSynchronize();
            for (tk_solver *S : B->mem) {
                cudaEventRecord(a0, S->stream);
                st = tk_step(S, (r + 1) * trial_steps);
                cudaEventRecord(a1, S->stream);
                if (st != TK_OK) {
                    bfail(B, st, "tk_batch_tune: %s", S->err);
                    break;
                }
                cudaEventSynchronize(a1);
                float m = 0.f;
                cudaEventElapsedTime(&m, a0, a1);
                ms_n[r] += m;
            }
            cudaDeviceSynchronize();
            for (int k = 0; k < B->n; ++k) {   // undo the trial
                tk_solver *S = B->mem[k];
                S->cur = cur0[k];
                S->count = count0[k];
                S->steps_done = done0[k];
                cudaMemcpyAsync(S->u[S->cur], keep[k], (size_t)S->Nr * 4 * S->NP * S->esz,
                                cudaMemcpyDeviceToDevice, B->stream);
                cudaMemcpyAsync(S->ctr, &keep_ctr[k], sizeof(long long), cudaMemcpyHostToDevice, B->stream);
            }
            cudaStreamSynchronize(B->stream);
        }
        cudaEventDestroy(a0);
        cudaEventDestroy(a1);
        const double ms = ms_n[1] - ms_n[0];   // trial_steps outer steps without the fixed costs
        if (st == TK_OK && ms > 0.0 && ms < queue_ms) per_member = true;
        best_t = per_member ? ms : (queue_ms > 0.0 && queue_ms < 1e300 ? queue_ms : best_t);
    }
    for (void *p : keep) cudaFree(p);
    B->graph_chunk = old_chunk;
    B->blocks = best_blocks;
    if (st != TK_OK) return st;
    st = build_items(B, best);
    if (st != TK_OK) return st;
    B->per_member = per_member;
    if (best_seg) *best_seg = per_member ? 0 : best;
    if (best_ms) *best_ms = best_t / trial_steps;
    TKB_CUDA(B, cudaGetLastError());
    return TK_OK;
}

tk_status tk_batch_info(const tk_batch *B, int *kmax, int *seg, int *blocks)
{
    if (!B) return TK_ERR_ARG;
    if (kmax) *kmax = B->kmax;
    if (seg) *seg = B->per_member ? 0 : B->seg;
    if (blocks) *blocks = B->per_member ? 0 : B->blocks;
    return TK_OK;
}

const char *tk_batch_last_error(const tk_batch *B) { return B ? B->err : "null batch"; }

void tk_batch_destroy(tk_batch *B)
{
    if (!B) return;
    cudaSetDevice(B->device);
    cudaStreamSynchronize(B->stream);
    if (B->graph) cudaGraphExecDestroy(B->graph);
    if (B->capture_stream) cudaStreamDestroy(B->capture_stream);
    if (B->d_mem) cudaFree(B->d_mem);
    if (B->d_items) cudaFree(B->d_items);
    if (B->d_ctr) cudaFree(B->d_ctr);
    delete B;
}

}  // extern "C"
