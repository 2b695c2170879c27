// tk_step.cu -- the fused two-step Lax-Wendroff time step, Eqs. (lw1) and (lw2).
//
// One warp owns all theta rows of a range of r* columns ("segment") and walks
// it from left to right.  Per column i it
//   1. loads u^n_{i+1} (one coalesced vector load per plane),
//   2. forms the half-step value u^{n+1/2}_{i+1/2} (Eq. lw1: the averaging of
//      the paper's kernel_average1 plus the bracketed right-hand side), with
//      the theta neighbours of the averaged Phi taken from the adjacent lanes
//      by warp shuffles,
//   3. forms u^{n+1}_i from u^{n+1/2}_{i-1/2} (kept in registers from the
//      previous column), u^{n+1/2}_{i+1/2} and u^n_i (Eq. lw2),
//   4. stores u^{n+1}_i, zero on the two radial edges (Sec. 3.2), and
//   5. on the last inner step of an outer step, writes the observer's partial
//      bilinear sample when i is one of its two interpolation columns.
// The half-step planes of the paper's OpenCL code never exist in memory.  The
// theta-pole boundary conditions are folded into the coefficient tables, so
// the arithmetic is branch-free: 28 FP64 (or FP32) operations per half node
// and 28 per node.
#include "tk_stencil.cuh"

namespace tk {
namespace {

struct WaveArgs {
    int write;
    int64_t cap;
    const long long *sample;   // device counter: index of the sample this outer step writes
    unsigned int *done;        // device counter: blocks finished in this launch
    double *wave;
    const double *w_row;
    ObsDev obs;
};

// Programmatic dependent launch of consecutive one-step launches: the next
// launch is set up while the current one runs.
constexpr bool kUsePDL = true;

// After the last inner step of an outer step the last block to finish moves
// the sample counter on.  Every block reads the counter before it arrives
// here, so the increment cannot race with a read of the same launch; the next
// launch on the stream sees it.  Keeping the index on the device lets a
// captured chunk of launches be replayed unchanged.
__device__ __forceinline__ void advance_sample(const WaveArgs &wa, int samples = 1)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int prev = atomicAdd(wa.done, 1u);
        if (prev == gridDim.x - 1) {
            atomicAdd((unsigned long long *)wa.sample, (unsigned long long)samples);
            atomicExch(wa.done, 0u);
            __threadfence();
        }
    }
}

// Warps per block.  A "wide" launch runs one block per SM with the most warps
// (a multiple of four) whose registers fit in the SM's register file at the
// register count the kernel compiles to for that element type and K; a
// "narrow" launch runs blocks of four warps, several per SM, for grids too
// small to give every warp of a wide launch a column.
template <typename T, int K>
constexpr int wide_warps()
{
    return sizeof(T) == 8 ? (K == 1 ? 24 : K == 2 ? 16 : 8) : (K == 1 ? 32 : K == 2 ? 24 : 16);
}

// State loads of the one-step sweep: through L1 when the state is read-only
// for the launch, from L2 (ld.global.cg) when other blocks of the same launch
// have written it (the persistent kernel), so that no stale L1 line is read.
template <typename T, int K, bool CG>
__device__ __forceinline__ void load_state(const T *p, T (&u)[4][K])
{
    if constexpr (!CG) {
        load_col<T, K>(p, u);
    } else {
        constexpr int NP = 32 * K;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const T *q = p + c * NP;
            if constexpr (sizeof(T) == 8 && K == 1) {
                u[c][0] = __ldcg(q);
            } else if constexpr (sizeof(T) == 8) {
#pragma unroll
                for (int t = 0; t < K; t += 2) {
                    const double2 x = __ldcg(reinterpret_cast<const double2 *>(q + t));
                    u[c][t] = x.x;
                    u[c][t + 1] = x.y;
                }
            } else if constexpr (K == 1) {
                u[c][0] = __ldcg(q);
            } else if constexpr (K == 2) {
                const float2 x = __ldcg(reinterpret_cast<const float2 *>(q));
                u[c][0] = x.x;
                u[c][1] = x.y;
            } else {
                const float4 x = __ldcg(reinterpret_cast<const float4 *>(q));
                u[c][0] = x.x;
                u[c][1] = x.y;
                u[c][2] = x.z;
                u[c][3] = x.w;
            }
        }
    }
}

// One Lax-Wendroff step over the block's columns (the body of lw_step_kernel):
// every warp walks its range, the first warp of the block recomputes its left
// half node, the others receive it through shared memory after a block
// barrier.  write: observe this step; sample_offset: samples after the
// counter's value.
template <typename T, int K, int W>
__device__ __forceinline__ void step_sweep(unsigned char *sh_raw, const T *__restrict__ u_in,
                                           T *__restrict__ u_out,
                                           const T *__restrict__ half, const T *__restrict__ node,
                                           int Nr, T eh, T en, const WaveArgs &wa, int write,
                                           int sample_offset)
{
    constexpr int NP = 32 * K;
    constexpr size_t SP = 4 * NP, HP = (size_t)kNCH * NP, NQ = (size_t)kNCN * NP;
    // per warp: [0] its last half node (read by the right neighbour),
    //           [1] u^n at its first column, [2] u^{n+1/2} right of its first column
    T(*sh)[3][4][NP] = reinterpret_cast<T(*)[3][4][NP]>(sh_raw);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int i0, i1, left;
    warp_range<W>(Nr, wib, &i0, &i1, &left);
    const int row = lane * K;
    const bool lead = (left < 0);

    T ua[4][K], hm[4][K];
    if (i1 > i0) {
        load_state<T, K, false>(u_in + (size_t)i0 * SP + row, ua);
        if (lead && i0 > 0) {
            T ul[4][K];
            load_state<T, K, false>(u_in + (size_t)(i0 - 1) * SP + row, ul);
            half_node<T, K>(ul, ua, half + (size_t)(i0 - 1) * HP + row, hm);
        } else {
            zero_col<T, K>(hm);
        }
        for (int i = i0; i < i1; ++i) {
            T uc[4][K], hp[4][K], o[4][K];
            if (i + 1 < Nr) {
                load_state<T, K, false>(u_in + (size_t)(i + 1) * SP + row, uc);
                half_node<T, K>(ua, uc, half + (size_t)i * HP + row, hp);
            } else {
                zero_col<T, K>(uc);
                zero_col<T, K>(hp);
            }
            if (i == i0 && !lead) {
#pragma unroll
                for (int c = 0; c < 4; ++c)
#pragma unroll
                    for (int t = 0; t < K; ++t) {
                        sh[wib][1][c][row + t] = ua[c][t];
                        sh[wib][2][c][row + t] = hp[c][t];
                    }
            } else {
                full_node<T, K>(hm, hp, ua, node + (size_t)i * NQ + row, en, o);
                if (i == 0 || i == Nr - 1) zero_col<T, K>(o);
                store_col<T, K>(u_out + (size_t)i * SP + row, o);
                if (write)
                    observe<T, K>(i, lane, o, wa.obs, wa.wave, wa.cap, wa.sample, wa.w_row, sample_offset);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int t = 0; t < K; ++t) {
                    hm[c][t] = hp[c][t];
                    ua[c][t] = uc[c][t];
                }
        }
    } else {
        zero_col<T, K>(hm);
    }
    // hm now holds u^{n+1/2} at i1 - 1/2: the right neighbour's left half node
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int t = 0; t < K; ++t) sh[wib][0][c][row + t] = hm[c][t];
    __syncthreads();
    if (!lead && i1 > i0) {
        T hl[4][K], hp[4][K], o[4][K];
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int t = 0; t < K; ++t) {
                hl[c][t] = sh[left][0][c][row + t];
                ua[c][t] = sh[wib][1][c][row + t];
                hp[c][t] = sh[wib][2][c][row + t];
            }
        full_node<T, K>(hl, hp, ua, node + (size_t)i0 * NQ + row, en, o);
        if (i0 == 0 || i0 == Nr - 1) zero_col<T, K>(o);
        store_col<T, K>(u_out + (size_t)i0 * SP + row, o);
        if (write) observe<T, K>(i0, lane, o, wa.obs, wa.wave, wa.cap, wa.sample, wa.w_row, sample_offset);
    }
}

template <typename T, int K, int W>
__global__ void __launch_bounds__(W * 32, wide_warps<T, K>() / W)
lw_step_kernel(const T *__restrict__ u_in, T *__restrict__ u_out, const T *__restrict__ half,
               const T *__restrict__ node, int Nr, T eh, T en, const WaveArgs wa)
{
    extern __shared__ __align__(16) unsigned char sh_raw[];
    if (kUsePDL) chain_start();
    step_sweep<T, K, W>(sh_raw, u_in, u_out, half, node, Nr, eh, en, wa, wa.write, 0);
    if (wa.write) advance_sample(wa);
}

// The blocks' neighbour barrier of the ring and four-step sweeps: the block
// publishes epoch and waits (bounded, by thread 0) until both neighbouring
// blocks have published it; false if a wait ran out.
__device__ __forceinline__ bool neighbour_barrier(unsigned int *flags, unsigned int epoch, int *err,
                                                  long long max_spins = kMaxSpins)
{
    __shared__ int ok;
    __syncthreads();                       // the block's stores of this step are issued
    if (threadIdx.x == 0) {
        __threadfence();                   // and visible to the other blocks
        atomicExch(&flags[blockIdx.x], epoch);
        int good = 1;
        for (int side = -1; side <= 1 && good; side += 2) {
            const int nb = (int)blockIdx.x + side;
            if (nb < 0 || nb >= (int)gridDim.x) continue;
            long long spins = 0;
            while (load_acquire(&flags[nb]) < epoch) {
                if (++spins > max_spins || *(volatile int *)err) {
                    good = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        if (!good) atomicExch(err, 1);
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}


// One step of the persistent sweep with no block barrier: every warp waits
// only for what it uses.  Counters (number of finished steps, or of steps
// whose first phase is finished) per warp in shared memory, and per block
// for its first and last warp in global memory (flags[b] and
// flags[blocks + b]).  Step s of warp w:
//   - first phase (every half node and node that involves only the block's
//     columns, as in step_sweep): it reads the right sibling's first column
//     and overwrites its own last half node, which the right sibling read in
//     the last step, so it waits until that sibling has finished step s - 1;
//     then it publishes that its first phase of step s is done;
//   - the block's last warp waits until the right neighbouring block's first
//     warp has finished step s - 1 (it reads that warp's column, and
//     overwrites its own last column, which that warp read), then forms it;
//   - the deferred first node: the block's first warp waits until the left
//     neighbouring block's last warp has finished step s - 1 and forms its
//     left half node from that warp's column; every other warp waits until
//     its left sibling's first phase of step s is done and takes that
//     sibling's last half node;
//   - it publishes that it has finished step s.
// Every wait is bounded; after one ran out every later wait returns at once.
// Same arithmetic on the same operands as step_sweep.
template <typename T, int K, int W>
__device__ __forceinline__ void step_sweep_async(unsigned char *sh_raw, const T *__restrict__ u_in,
                                                 T *__restrict__ u_out, const T *__restrict__ half,
                                                 const T *__restrict__ node, int Nr, T en,
                                                 const WaveArgs &wa, int write, int sample_offset,
                                                 unsigned int *flags, unsigned int *first_done,
                                                 unsigned int *step_done, unsigned int s, int *err)
{
    constexpr int NP = 32 * K;
    constexpr size_t SP = 4 * NP, HP = (size_t)kNCH * NP, NQ = (size_t)kNCN * NP;
    T(*sh)[3][4][NP] = reinterpret_cast<T(*)[3][4][NP]>(sh_raw);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int i0, i1, left;
    warp_range<W>(Nr, wib, &i0, &i1, &left);
    // The launch has at most Nr / W blocks, so every block has at least W
    // columns and warp_range gives every warp at least one; a warp without
    // one would never publish, and its left sibling's wait would run out.
    if (i1 <= i0) return;
    const int row = lane * K;
    const bool lead = (left < 0);
    const int b1 = (int)(((long long)(blockIdx.x + 1) * Nr) / gridDim.x);
    const bool last = (i1 == b1);
    const int iend = last ? i1 - 1 : i1;
    const unsigned int nb = gridDim.x;
    if (s > 0 && !last) warp_wait_cta(&step_done[wib + 1], s, err);
    T ua[4][K], hm[4][K];
    zero_col<T, K>(hm);
    load_state<T, K, true>(u_in + (size_t)i0 * SP + row, ua);
    for (int i = i0; i < iend; ++i) {
        T uc[4][K], hp[4][K], o[4][K];
        if (i + 1 < Nr) {
            load_state<T, K, true>(u_in + (size_t)(i + 1) * SP + row, uc);
            half_node<T, K>(ua, uc, half + (size_t)i * HP + row, hp);
        } else {
            zero_col<T, K>(uc);
            zero_col<T, K>(hp);
        }
        if (i == i0) {
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int t = 0; t < K; ++t) {
                    sh[wib][1][c][row + t] = ua[c][t];
                    sh[wib][2][c][row + t] = hp[c][t];
                }
        } else {
            full_node<T, K>(hm, hp, ua, node + (size_t)i * NQ + row, en, o);
            if (i == 0 || i == Nr - 1) zero_col<T, K>(o);
            store_col<T, K>(u_out + (size_t)i * SP + row, o);
            if (write) observe<T, K>(i, lane, o, wa.obs, wa.wave, wa.cap, wa.sample, wa.w_row, sample_offset);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int t = 0; t < K; ++t) {
                hm[c][t] = hp[c][t];
                ua[c][t] = uc[c][t];
            }
    }
    if (!last)
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int t = 0; t < K; ++t) sh[wib][0][c][row + t] = hm[c][t];
    warp_publish_cta(&first_done[wib], s + 1);
    if (last) {
        if (s > 0 && blockIdx.x + 1 < nb) warp_wait_flag(flags + blockIdx.x + 1, s, err);
        const int i = i1 - 1;
        T uc[4][K], hp[4][K];
        if (i + 1 < Nr) {
            load_state<T, K, true>(u_in + (size_t)(i + 1) * SP + row, uc);
            half_node<T, K>(ua, uc, half + (size_t)i * HP + row, hp);
        } else {
            zero_col<T, K>(uc);
            zero_col<T, K>(hp);
        }
        if (i == i0) {
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int t = 0; t < K; ++t) {
                    sh[wib][1][c][row + t] = ua[c][t];
                    sh[wib][2][c][row + t] = hp[c][t];
                }
        } else {
            T o[4][K];
            full_node<T, K>(hm, hp, ua, node + (size_t)i * NQ + row, en, o);
            if (i == 0 || i == Nr - 1) zero_col<T, K>(o);
            store_col<T, K>(u_out + (size_t)i * SP + row, o);
            if (write) observe<T, K>(i, lane, o, wa.obs, wa.wave, wa.cap, wa.sample, wa.w_row, sample_offset);
        }
        __syncwarp();
    }
    {
        T hl[4][K], uf[4][K], hf[4][K], o[4][K];
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int t = 0; t < K; ++t) {
                uf[c][t] = sh[wib][1][c][row + t];
                hf[c][t] = sh[wib][2][c][row + t];
            }
        if (lead) {
            if (s > 0 && blockIdx.x > 0) warp_wait_flag(flags + nb + blockIdx.x - 1, s, err);
            if (i0 > 0) {
                T ul[4][K];
                load_state<T, K, true>(u_in + (size_t)(i0 - 1) * SP + row, ul);
                half_node<T, K>(ul, uf, half + (size_t)(i0 - 1) * HP + row, hl);
            } else {
                zero_col<T, K>(hl);
            }
        } else {
            warp_wait_cta(&first_done[left], s + 1, err);
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int t = 0; t < K; ++t) hl[c][t] = sh[left][0][c][row + t];
        }
        full_node<T, K>(hl, hf, uf, node + (size_t)i0 * NQ + row, en, o);
        if (i0 == 0 || i0 == Nr - 1) zero_col<T, K>(o);
        store_col<T, K>(u_out + (size_t)i0 * SP + row, o);
        if (write) observe<T, K>(i0, lane, o, wa.obs, wa.wave, wa.cap, wa.sample, wa.w_row, sample_offset);
    }
    if (lead) warp_publish_gpu(flags + blockIdx.x, s + 1);
    if (last) warp_publish_gpu(flags + nb + blockIdx.x, s + 1);
    warp_publish_cta(&step_done[wib], s + 1);
}

// Every Lax-Wendroff step of a call in one launch (the FP64 default).  All
// blocks are resident at once (cooperative launch).  There is no barrier between steps:
// each warp waits only for the warps whose data it reads or overwrites -- its
// two siblings in the block, and for a block's first and last warp the edge
// warp of the neighbouring block -- through counters of finished steps
// (step_sweep_async).  Every wait is bounded: after kMaxSpins polls the warp
// sets *err, and from then on every wait returns at once, so this kernel runs
// its remaining steps without waiting and the persistent kernels below leave
// their loops (the state is then invalid and the host reports the error).
// State loads go through L2 (other blocks write them).  u0 holds u^n at the start; the result
// is in u0 or u1 by the parity of n_inner.
template <typename T, int K, int W>
__global__ void __launch_bounds__(W * 32, wide_warps<T, K>() / W)
lw_persistent_kernel(T *u0, T *u1, const T *__restrict__ half, const T *__restrict__ node, int Nr,
                     T en, const WaveArgs wa, int n_inner, int substeps, unsigned int *flags, int *err)
{
    extern __shared__ __align__(16) unsigned char sh_raw[];
    __shared__ unsigned int first_done[W], step_done[W];
    if (threadIdx.x < W) {
        first_done[threadIdx.x] = 0;
        step_done[threadIdx.x] = 0;
    }
    __syncthreads();
    for (int s = 0; s < n_inner; ++s) {
        const T *in = (s & 1) ? u1 : u0;
        T *out = (s & 1) ? u0 : u1;
        const int write = wa.write && ((s + 1) % substeps == 0);
        step_sweep_async<T, K, W>(sh_raw, in, out, half, node, Nr, en, wa, write, (s + 1) / substeps - 1, flags,
                                  first_done, step_done, (unsigned)s, err);
    }
    if (wa.write) advance_sample(wa, n_inner / substeps);
}

// Diagnostic of the bounded waits: every block but `silent` publishes epoch 1
// and waits for its neighbours as the persistent kernels do between steps
// (the block-level wait, error word err[0]), then waits for each neighbour
// as the edge warps of the one-step sweep do (the warp-level wait on a global
// flag, err[1]).  `silent` instead waits on a shared-memory counter that
// nothing sets, as the one-step sweep's warps wait for their siblings (err[2]),
// and returns without publishing; so all three kinds of wait run out after
// max_spins polls and set their error words.
__global__ void wait_check_kernel(unsigned int *flags, int *err, int silent, long long max_spins)
{
    __shared__ unsigned int never;
    if ((int)blockIdx.x == silent) {
        if (threadIdx.x == 0) never = 0;
        __syncwarp();
        warp_wait_cta(&never, 1u, err + 2, max_spins);
        return;
    }
    neighbour_barrier(flags, 1u, err, max_spins);
    if (blockIdx.x > 0) warp_wait_flag(flags + blockIdx.x - 1, 1u, err + 1, max_spins);
    if (blockIdx.x + 1 < gridDim.x) warp_wait_flag(flags + blockIdx.x + 1, 1u, err + 1, max_spins);
}

// Two Lax-Wendroff steps per launch, u^n -> u^{n+2}, for the HBM-bound
// precision: state and tables cross DRAM once per two steps.  A warp owns the
// output columns [i0, i1) of the same split as the one-step kernel and
// recomputes the intermediate level u^{n+1} on [i0 - 1, i1], one column
// beyond each end, so warps need nothing from each other.  It loads u^n_p for
// p = i0 - 2 .. i1 + 1 and runs four lagged stages per p: the level-1 half
// node p - 1/2, the level-1 node p - 1, the level-2 half node p - 3/2 and the
// level-2 node p - 2.  The tables of a column are read twice, one column
// apart, the second time from cache.  Every node and half node does the
// arithmetic of the one-step kernel on the same operands, so two fused steps
// are bit-identical to two one-step launches.  obs_mask bit 0: an outer step
// ends after the first of the two steps; bit 1: after the second.
template <typename T, int K>
constexpr int fused_warps()
{
    return sizeof(T) == 8 ? (K == 1 ? 20 : K == 2 ? 8 : 4) : (K == 1 ? 32 : K == 2 ? 16 : 8);
}

template <typename T, int K, int W>
__global__ void __launch_bounds__(W * 32, fused_warps<T, K>() / W)
lw_step2_kernel(const T *__restrict__ u_in, T *__restrict__ u_out, const T *__restrict__ half,
                const T *__restrict__ node, int Nr, T eh, T en, const WaveArgs wa, int obs_mask)
{
    constexpr int NP = 32 * K;
    constexpr size_t SP = 4 * NP, HP = (size_t)kNCH * NP, NQ = (size_t)kNCN * NP;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int i0, i1, left;
    warp_range<W>(Nr, wib, &i0, &i1, &left);
    const int row = lane * K;
    const int second = obs_mask & 1;   // sample offset of the level-2 observation
    if (i1 > i0) {
        T a0[4][K], h1m[4][K], u1m[4][K], h2m[4][K];
        zero_col<T, K>(a0);
        zero_col<T, K>(h1m);
        zero_col<T, K>(u1m);
        zero_col<T, K>(h2m);
        for (int p = i0 - 2; p <= i1 + 1; ++p) {
            T c0[4][K], h1p[4][K], u1c[4][K], h2p[4][K];
            if (p >= 0 && p < Nr) load_col<T, K>(u_in + (size_t)p * SP + row, c0);
            else zero_col<T, K>(c0);
            // level 1, half node between p - 1 and p
            if (p >= i0 - 1 && p >= 1 && p < Nr)
                half_node<T, K>(a0, c0, half + (size_t)(p - 1) * HP + row, h1p);
            else
                zero_col<T, K>(h1p);
            // level 1, node q = p - 1 (zero on the radial edges and outside the grid)
            const int q = p - 1;
            if (p >= i0 && q >= 1 && q <= Nr - 2)
                full_node<T, K>(h1m, h1p, a0, node + (size_t)q * NQ + row, en, u1c);
            else
                zero_col<T, K>(u1c);
            if ((obs_mask & 1) && q >= i0 && q < i1)
                observe<T, K>(q, lane, u1c, wa.obs, wa.wave, wa.cap, wa.sample, wa.w_row, 0);
            // level 2, half node between r = p - 2 and p - 1
            const int r = p - 2;
            if (p >= i0 + 1 && r >= 0 && r + 1 < Nr)
                half_node<T, K>(u1m, u1c, half + (size_t)r * HP + row, h2p);
            else
                zero_col<T, K>(h2p);
            // level 2, node r
            if (p >= i0 + 2) {
                T o[4][K];
                if (r >= 1 && r <= Nr - 2)
                    full_node<T, K>(h2m, h2p, u1m, node + (size_t)r * NQ + row, en, o);
                else
                    zero_col<T, K>(o);
                store_col<T, K>(u_out + (size_t)r * SP + row, o);
                if (obs_mask & 2)
                    observe<T, K>(r, lane, o, wa.obs, wa.wave, wa.cap, wa.sample, wa.w_row, second);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int t = 0; t < K; ++t) {
                    a0[c][t] = c0[c][t];
                    h1m[c][t] = h1p[c][t];
                    u1m[c][t] = u1c[c][t];
                    h2m[c][t] = h2p[c][t];
                }
        }
    }
    if (obs_mask) advance_sample(wa, (obs_mask & 1) + ((obs_mask >> 1) & 1));
}

// The two-step sweep with its loads staged through shared memory.  Per warp
// a ring of three slots, each one column's state (4 planes) and tables (11 +
// 10 entries): while the warp computes column p from slot p % 3 (level 1)
// and slot (p - 1) % 3 (level 2, the same tables one column later), the
// copies of column p + 1 into the third slot are in flight (cp.async, one
// group per column; a lane copies and reads only its own rows, so
// cp.async.wait_group is the only synchronisation).  DRAM is read once per
// column and the load latency of column p + 1 overlaps the arithmetic of
// column p.  The arithmetic is that of lw_step2_kernel.
constexpr int kRingSlots = 3;
constexpr int kSlotCols = kNCH + kNCN;   // half-node table, node table
constexpr int kSlotNode = kNCH;          // offset of the node table in a slot

template <typename T, int K>
constexpr int ring_warps()
{
    return K == 1 ? 24 : K == 2 ? 12 : 4;
}

template <typename T, int K>
constexpr size_t ring_smem_bytes()
{
    return (size_t)ring_warps<T, K>() * kRingSlots * kSlotCols * 32 * K * sizeof(T);
}

template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(gmem), "n"(BYTES)
                     : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Bulk copies (the TMA unit's cp.async.bulk) of a column's tables into a
// warp's shared-memory ring: one thread issues the two copies of a column
// (half-node and node tables, contiguous in global memory), which complete on
// the mbarrier of their ring slot; the warp waits on that mbarrier's phase
// before reading the slot.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_fetch(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Polls of a ring slot's mbarrier before the wait gives up (each try_wait
// itself suspends the warp for a while); a copy of valid memory completes
// long before.
constexpr long long kMaxMbarPolls = 1ll << 22;

__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity)
{
    for (long long i = 0; i < kMaxMbarPolls; ++i)
        if (mbar_test(bar, parity)) return true;
    return false;
}

// The ring's per-warp state across sweeps: the slot of the next copy (also
// the slot the next wait is for), and per slot the parity of the next phase
// to wait for and of the copies issued.
struct RingState {
    int cur;
    unsigned wait_ph, issue_ph;
};

// Issue the copies of the first-level tables of sweep step p (half_{p-1},
// node_{p-1}) into `slot`, then commit a group (empty where the column is
// outside the grid).
template <typename T, int K>
__device__ __forceinline__ void ring_fetch(T *slot, const T *__restrict__ half,
                                           const T *__restrict__ node, int p, int Nr, int row)
{
    constexpr int NP = 32 * K, B = K * (int)sizeof(T);
    if (p >= 1 && p < Nr) {
#pragma unroll
        for (int q = 0; q < kNCH; ++q)
            cp_async<B>(slot + q * NP + row, half + ((size_t)(p - 1) * kNCH + q) * NP + row);
#pragma unroll
        for (int q = 0; q < kNCN; ++q)
            cp_async<B>(slot + (kSlotNode + q) * NP + row, node + ((size_t)(p - 1) * kNCN + q) * NP + row);
    }
    cp_async_commit();
}

// The two-step sweep over the block's columns (the body of the ring kernel).
// mask: bit 0, an outer step ends after the first step, bit 1 after the
// second; off1, off2: their samples after the counter's value.  CG: the state
// is loaded from L2 (other blocks of the same launch wrote it).
template <typename T, int K, int W, bool CG>
__device__ __forceinline__ void ring_sweep(unsigned char *sh_raw, const T *__restrict__ u_in,
                                           T *__restrict__ u_out, const T *__restrict__ half,
                                           const T *__restrict__ node, int Nr, T en,
                                           const WaveArgs &wa, int mask, int off1, int off2)
{
    constexpr int NP = 32 * K;
    constexpr size_t SP = 4 * NP;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    T *ring = reinterpret_cast<T *>(sh_raw) + (size_t)wib * kRingSlots * kSlotCols * NP;
    int i0, i1, left;
    warp_range<W>(Nr, wib, &i0, &i1, &left);
    const int row = lane * K;
    if (i1 > i0) {
        T a0[4][K], h1m[4][K], u1m[4][K], h2m[4][K];
        zero_col<T, K>(a0);
        zero_col<T, K>(h1m);
        zero_col<T, K>(u1m);
        zero_col<T, K>(h2m);
        ring_fetch<T, K>(ring, half, node, i0 - 2, Nr, row);
        T cn[4][K];   // the state column p + 1, loaded one column ahead
        if (i0 - 2 >= 0) load_state<T, K, CG>(u_in + (size_t)(i0 - 2) * SP + row, cn);
        else zero_col<T, K>(cn);
        int cur = 0;
        for (int p = i0 - 2; p <= i1 + 1; ++p) {
            const int nxt = cur == kRingSlots - 1 ? 0 : cur + 1;
            const int prv = cur == 0 ? kRingSlots - 1 : cur - 1;
            if (p + 1 <= i1 + 1)
                ring_fetch<T, K>(ring + nxt * kSlotCols * NP, half, node, p + 1, Nr, row);
            else
                cp_async_commit();
            cp_async_wait_one();
            const T *sc = ring + cur * kSlotCols * NP;    // tables of step p: half_{p-1}, node_{p-1}
            const T *sp = ring + prv * kSlotCols * NP;    // of step p - 1: half_{p-2}, node_{p-2}
            T c0[4][K], h1p[4][K], u1c[4][K], h2p[4][K];
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int t = 0; t < K; ++t) c0[c][t] = cn[c][t];
            if (p + 1 >= 0 && p + 1 < Nr && p + 1 <= i1 + 1)
                load_state<T, K, CG>(u_in + (size_t)(p + 1) * SP + row, cn);
            else
                zero_col<T, K>(cn);
            if (p >= i0 - 1 && p >= 1 && p < Nr)
                half_node<T, K>(a0, c0, sc + row, h1p);
            else
                zero_col<T, K>(h1p);
            const int q = p - 1;
            if (p >= i0 && q >= 1 && q <= Nr - 2)
                full_node<T, K>(h1m, h1p, a0, sc + kSlotNode * NP + row, en, u1c);
            else
                zero_col<T, K>(u1c);
            if ((mask & 1) && q >= i0 && q < i1)
                observe<T, K>(q, lane, u1c, wa.obs, wa.wave, wa.cap, wa.sample, wa.w_row, off1);
            const int r = p - 2;
            if (p >= i0 + 1 && r >= 0 && r + 1 < Nr)
                half_node<T, K>(u1m, u1c, sp + row, h2p);
            else
                zero_col<T, K>(h2p);
            if (p >= i0 + 2) {
                T o[4][K];
                if (r >= 1 && r <= Nr - 2)
                    full_node<T, K>(h2m, h2p, u1m, sp + kSlotNode * NP + row, en, o);
                else
                    zero_col<T, K>(o);
                store_col<T, K>(u_out + (size_t)r * SP + row, o);
                if (mask & 2)
                    observe<T, K>(r, lane, o, wa.obs, wa.wave, wa.cap, wa.sample, wa.w_row, off2);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int t = 0; t < K; ++t) {
                    a0[c][t] = c0[c][t];
                    h1m[c][t] = h1p[c][t];
                    u1m[c][t] = u1c[c][t];
                    h2m[c][t] = h2p[c][t];
                }
            cur = nxt;
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    }
}

template <typename T, int K, int W>
__global__ void __launch_bounds__(W * 32, 1)
lw_step2_ring_kernel(const T *__restrict__ u_in, T *__restrict__ u_out, const T *__restrict__ half,
                     const T *__restrict__ node, int Nr, T eh, T en, const WaveArgs wa, int obs_mask)
{
    extern __shared__ __align__(16) unsigned char sh_raw[];
    ring_sweep<T, K, W, false>(sh_raw, u_in, u_out, half, node, Nr, en, wa, obs_mask, 0, obs_mask & 1);
    if (obs_mask) advance_sample(wa, (obs_mask & 1) + ((obs_mask >> 1) & 1));
}

// The two-step sweep for many pairs of steps in one cooperative launch, the
// blocks waiting only for their two neighbours between pairs (as in
// lw_persistent_kernel): a block's columns need the two columns on each side
// from its neighbours, and a block overwrites the level its neighbours read
// in the previous pair.  Pair p takes inner steps 2p and 2p + 1 of the call;
// an outer step of k inner steps that ends inside it is observed there.
template <typename T, int K, int W>
__global__ void __launch_bounds__(W * 32, 1)
lw_ring_persistent_kernel(T *u0, T *u1, const T *__restrict__ half, const T *__restrict__ node,
                          int Nr, T en, const WaveArgs wa, int n_pairs, int k, unsigned int *flags,
                          int *err)
{
    extern __shared__ __align__(16) unsigned char sh_raw[];
    for (int p = 0; p < n_pairs; ++p) {
        const T *in = (p & 1) ? u1 : u0;
        T *out = (p & 1) ? u0 : u1;
        const int t = 2 * p;
        const int mask = wa.write ? (((t + 1) % k == 0) | (((t + 2) % k == 0) << 1)) : 0;
        ring_sweep<T, K, W, true>(sh_raw, in, out, half, node, Nr, en, wa, mask, (t + 1) / k - 1,
                                  (t + 2) / k - 1);
        if (p + 1 < n_pairs && !neighbour_barrier(flags, (unsigned)(p + 1), err)) break;
    }
    if (wa.write) advance_sample(wa, (2 * n_pairs) / k);
}

// LV Lax-Wendroff steps per sweep, u^n -> u^{n+LV} (the FP32 default on
// large grids with every step of a call in one launch): the state and the
// tables cross DRAM once per LV steps.  The ring sweep above generalised: a
// warp owns the output columns [i0, i1) and computes level l (1..LV) on
// [i0 - (LV - l), i1 + (LV - l)), recomputing the halo; at sweep position p
// (the newest level-0 column) level l forms the half node between columns
// p - l and p - l + 1 and the node p - l, from level l - 1's values at those
// columns (the one formed at this position and the one kept from the last).
// Column c's tables (the compact FP32 copy: 16 entries, one bulk copy per
// column) are used by level 1 at position c + 1 and by level LV at c + LV,
// and are copied kRingAhead positions before level 1 needs them, so the ring
// holds LV + kRingAhead columns.  Every node and half node does the one-step
// kernel's arithmetic on the same operands (the compact tables give the same
// 21 entries bit for bit), so LV steps are bit-identical to LV single steps.
// mask bit l - 1: an outer step ends after level l; off[l - 1]: its sample
// after the counter's value.
constexpr int kSweepLevels = 4;
constexpr int kRingAhead = 2;

template <typename T, int K>
constexpr int multi_warps()
{
    return K == 1 ? 16 : K == 2 ? 8 : 4;
}

template <int LV>
__host__ __device__ constexpr int multi_slots()
{
    return LV + kRingAhead;
}

template <int K, int W, int LV>
__host__ __device__ constexpr size_t multi_ring_bytes()
{
    return (size_t)W * multi_slots<LV>() * kNCC * 32 * K * sizeof(float);
}

// the rings, then one mbarrier per ring slot
template <int K, int W, int LV>
constexpr size_t multi_smem_bytes()
{
    return multi_ring_bytes<K, W, LV>() + (size_t)W * multi_slots<LV>() * sizeof(unsigned long long);
}

// Bulk copy of the compact tables of sweep position p (column p - 1, clamped
// into the grid where the values are not used) into the ring slot st.cur, by
// lane 0.  The slot's previous column was last read at an earlier position:
// the warp's reads are ordered before the copy by the warp barrier and the
// proxy fence.
template <int K, int S>
__device__ __forceinline__ void ring_issue(float *ring, unsigned long long *bars, RingState &st,
                                           const float *__restrict__ cmp, int p, int Nr, int lane)
{
    constexpr int NP = 32 * K;
    constexpr unsigned CB = kNCC * NP * sizeof(float);
    const int s = st.cur;
    __syncwarp();
    if (lane == 0) {
        int c = p - 1;
        c = c < 0 ? 0 : (c > Nr - 1 ? Nr - 1 : c);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect(bars + s, CB);
        bulk_fetch(ring + (size_t)s * kNCC * NP, cmp + (size_t)c * kNCC * NP, CB, bars + s);
    }
    st.issue_ph ^= 1u << s;
    st.cur = s == S - 1 ? 0 : s + 1;
}

// Wait for the copy into slot s (the oldest one not yet waited for).
template <int S>
__device__ __forceinline__ void ring_wait(unsigned long long *bars, RingState &st, int s, int *err)
{
    if (!mbar_wait(bars + s, (st.wait_ph >> s) & 1u)) atomicExch(err, 1);
    st.wait_ph ^= 1u << s;
}

// The four-step sweep copies the Phi values of up to kObsCols observer
// columns per warp (held in registers; -1: none) to a scratch area at the
// levels where an outer step ends, and forms the waveform samples from there
// after its loop.  Sampling inside the loop, at every column checked for an
// observer, cost a fifth of the sweep's time, and the warps holding an
// observer set the pace of the persistent launch.  A call whose observers put
// more than kObsCols columns in one warp's range runs in pairs of steps
// instead (multi_obs_fit).
constexpr int kObsCols = 4;

// Scratch per block: per warp, column slot and level, Phi_R and Phi_I (2 NP).
template <int K, int LV>
constexpr size_t multi_obs_scratch_elems_per_warp()
{
    return (size_t)kObsCols * LV * 2 * 32 * K;
}

template <typename T, int K, int LV>
__device__ __forceinline__ void multi_body(float *ring, unsigned long long *bars, RingState &rs, int *err,
                                           int i0, int i1, int lane, const T *__restrict__ u_in,
                                           T *__restrict__ u_out, const float *__restrict__ cmp,
                                           const float (&gp)[K], const float (&gm)[K],
                                           const F32Derive &fd, int Nr, T en, int mask,
                                           const int (&oc)[kObsCols], T *__restrict__ scr)
{
    static_assert(sizeof(T) == 4, "the four-step sweep is the FP32 path");
    constexpr int NP = 32 * K;
    constexpr int S = multi_slots<LV>();
    constexpr size_t SP = 4 * NP;
    const int row = lane * K;
    T hm[LV][4][K];   // level l + 1: the half node formed at the last position
    T um[LV][4][K];   // level l: the value formed at the last position
#pragma unroll
    for (int l = 0; l < LV; ++l) {
        zero_col<T, K>(hm[l]);
        zero_col<T, K>(um[l]);
    }
    const int pa = i0 - LV, pb = i1 + LV - 1;
    int cur = rs.cur;   // the slot of position pa
#pragma unroll
    for (int a = 0; a < kRingAhead; ++a)
        if (pa + a <= pb) ring_issue<K, S>(ring, bars, rs, cmp, pa + a, Nr, lane);
    T cn[4][K];
    if (pa >= 0) load_state<T, K, true>(u_in + (size_t)pa * SP + row, cn);
    else zero_col<T, K>(cn);
    // the warp's observer columns span [olo, ohi] (olo > ohi: none)
    int olo = 0x7fffffff, ohi = -1;
#pragma unroll
    for (int h = 0; h < kObsCols; ++h)
        if (oc[h] >= 0) {
            olo = oc[h] < olo ? oc[h] : olo;
            ohi = oc[h] > ohi ? oc[h] : ohi;
        }
    if (!mask) ohi = -1;
    for (int p = pa; p <= pb; ++p) {
        const int nxt = cur == S - 1 ? 0 : cur + 1;
        if (p + kRingAhead <= pb) ring_issue<K, S>(ring, bars, rs, cmp, p + kRingAhead, Nr, lane);
        ring_wait<S>(bars, rs, cur, err);
        T cu[4][K];   // level l - 1 at column p - l + 1
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int t = 0; t < K; ++t) cu[c][t] = cn[c][t];
        if (p + 1 <= pb && p + 1 >= 0 && p + 1 < Nr)
            load_state<T, K, true>(u_in + (size_t)(p + 1) * SP + row, cn);
        else
            zero_col<T, K>(cn);
        // Every node and half node is formed, also outside a level's valid
        // columns [i0 - (LV - l), i1 + LV - l): the values there are finite
        // (formed from finite tables of a column clamped into the grid, and
        // from zeros beyond its edges) and feed only other values outside, so
        // they need no masking.  The node values on the radial edges c = 0
        // and c = Nr - 1 are set to zero (Sec. 3.2), at every level.
#pragma unroll
        for (int l = 1; l <= LV; ++l) {
            const int c = p - l;
            int sl = cur - (l - 1);
            if (sl < 0) sl += S;
            const float *tab = ring + sl * kNCC * NP;   // compact tables of column c
            T hp[4][K], uc[4][K];
            {
                float q[kNCH][K];
                derive_half<K>(tab + row, gp, gm, fd, q);
                half_node_q<T, K>(um[l - 1], cu, q, hp);
            }
            {
                float q[kNCN][K];
                derive_node<K>(tab + C_B * NP + row, gp, gm, fd, q);
                full_node_q<T, K>(hm[l - 1], hp, um[l - 1], q, en, uc);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int t = 0; t < K; ++t) {
                    um[l - 1][q][t] = cu[q][t];
                    hm[l - 1][q][t] = hp[q][t];
                    cu[q][t] = uc[q][t];
                }
            if (c == 0 || c == Nr - 1) zero_col<T, K>(cu);
            // the Phi values of an observer column at a level where an outer
            // step ends, for the samples formed after the loop
            if (c >= olo && c <= ohi && ((mask >> (l - 1)) & 1))
#pragma unroll
                for (int h = 0; h < kObsCols; ++h)
                    if (c == oc[h]) {
                        T *d = scr + ((size_t)h * LV + (l - 1)) * 2 * NP + row;
                        stk<T, K>(d, cu[0]);
                        stk<T, K>(d + NP, cu[1]);
                    }
        }
        if (p - LV >= i0) store_col<T, K>(u_out + (size_t)(p - LV) * SP + row, cu);
        cur = nxt;
    }
}

// The sweep, with the waveform samples formed after its loop (see kObsCols).
template <typename T, int K, int W, int LV>
__device__ __forceinline__ void multi_sweep(unsigned char *sh_raw, RingState &rs, int *err,
                                            const T *__restrict__ u_in,
                                            T *__restrict__ u_out, const float *__restrict__ cmp,
                                            const float (&gp)[K], const float (&gm)[K],
                                            const F32Derive &fd, int Nr, T en,
                                            const WaveArgs &wa, int mask, const int (&off)[LV],
                                            T *__restrict__ scr)
{
    constexpr int NP = 32 * K;
    constexpr int S = multi_slots<LV>();
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    float *ring = reinterpret_cast<float *>(sh_raw) + (size_t)wib * S * kNCC * NP;
    unsigned long long *bars =
        reinterpret_cast<unsigned long long *>(sh_raw + multi_ring_bytes<K, W, LV>()) + wib * S;
    int i0, i1, left;
    warp_range<W>(Nr, wib, &i0, &i1, &left);
    if (i1 <= i0) return;
    // this warp's distinct observer columns (the host made sure there are at
    // most kObsCols)
    int oc[kObsCols];
#pragma unroll
    for (int h = 0; h < kObsCols; ++h) oc[h] = -1;
    int n = 0;
    if (mask && wa.write)
        for (int k = 0; k < wa.obs.n; ++k)
            for (int sl = 0; sl < 2; ++sl) {
                const int col = wa.obs.i0[k] + sl;
                if (col < i0 || col >= i1) continue;
                bool seen = false;
#pragma unroll
                for (int h = 0; h < kObsCols; ++h) seen |= (oc[h] == col);
                if (!seen && n < kObsCols) {
#pragma unroll
                    for (int h = 0; h < kObsCols; ++h)
                        if (h == n) oc[h] = col;
                    ++n;
                }
            }
    constexpr size_t kWarpScr = (size_t)kObsCols * LV * 2 * NP;   // per warp
    T *wscr = scr + (size_t)(blockIdx.x * W + wib) * kWarpScr;
    multi_body<T, K, LV>(ring, bars, rs, err, i0, i1, lane, u_in, u_out, cmp, gp, gm, fd, Nr, en, mask, oc,
                         wscr);
    if (n == 0) return;
    const int row = lane * K;
    // The sample counter does not move during the launch (advance_sample at
    // its end): read it once.  All the stored values are loaded before any
    // sample is formed, so that their loads overlap instead of forming a
    // chain of round trips through L2 on the warp that sets the launch's pace.
    const long long base = *(volatile const long long *)wa.sample;
    T v[kObsCols][LV][2][K];
#pragma unroll
    for (int h = 0; h < kObsCols; ++h)
#pragma unroll
        for (int l = 0; l < LV; ++l)
            if (oc[h] >= 0 && ((mask >> l) & 1)) {
                const T *d = wscr + ((size_t)h * LV + l) * 2 * NP + row;
                ldk<T, K>(d, v[h][l][0]);
                ldk<T, K>(d + NP, v[h][l][1]);
            }
#pragma unroll
    for (int h = 0; h < kObsCols; ++h)
#pragma unroll
        for (int l = 0; l < LV; ++l)
            if (oc[h] >= 0 && ((mask >> l) & 1))
                observe_at<T, K>(oc[h], lane, v[h][l][0], v[h][l][1], wa.obs, wa.wave, wa.cap, wa.w_row,
                                 base + off[l]);
}

// Groups of LV steps in one cooperative launch, the blocks waiting for their
// two neighbours between groups (each block owns at least LV columns, so the
// columns a group reads beyond a block's range belong to its neighbours).
// Group g takes inner steps LV g .. LV g + LV - 1 of the call, which starts on
// an outer step's boundary (k inner steps per outer step).
template <typename T, int K, int W, int LV>
__global__ void __launch_bounds__(W * 32, 1)
lw_multi_persistent_kernel(T *u0, T *u1, const float *__restrict__ cmp, const float *__restrict__ gpm,
                           F32Derive fd, int Nr, T en, const WaveArgs wa, int n_groups, int k,
                           unsigned int *flags, int *err, T *scr)
{
    extern __shared__ __align__(16) unsigned char sh_raw[];
    constexpr int S = multi_slots<LV>();
    constexpr int NP = 32 * K;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned long long *bars =
        reinterpret_cast<unsigned long long *>(sh_raw + multi_ring_bytes<K, W, LV>()) + wib * S;
    if (lane == 0) {
        for (int q = 0; q < S; ++q) mbar_init(bars + q);
        mbar_init_fence();
    }
    __syncwarp();
    float gp[K], gm[K];   // the lane's rows' theta factors of the compact tables
    ldk<float, K>(gpm + lane * K, gp);
    ldk<float, K>(gpm + NP + lane * K, gm);
    RingState rs{0, 0u, 0u};
    for (int g = 0; g < n_groups; ++g) {
        const T *in = (g & 1) ? u1 : u0;
        T *out = (g & 1) ? u0 : u1;
        const int t = LV * g;
        int mask = 0;
        int off[LV];
#pragma unroll
        for (int l = 0; l < LV; ++l) {
            if (wa.write && (t + l + 1) % k == 0) mask |= 1 << l;
            off[l] = (t + l + 1) / k - 1;
        }
        multi_sweep<T, K, W, LV>(sh_raw, rs, err, in, out, cmp, gp, gm, fd, Nr, en, wa, mask, off, scr);
        if (g + 1 < n_groups && !neighbour_barrier(flags, (unsigned)(g + 1), err)) break;
    }
    // every copy issued has been waited for, unless a wait gave up: then wait
    // (bounded) for the last copy into each slot before the block exits
    if (rs.wait_ph != rs.issue_ph && lane == 0)
        for (int q = 0; q < S; ++q)
            if (((rs.wait_ph ^ rs.issue_ph) >> q) & 1u) mbar_wait(bars + q, ((rs.issue_ph >> q) & 1u) ^ 1u);
    if (wa.write) advance_sample(wa, (LV * n_groups) / k);
}

template <typename T, int K, int W>
constexpr size_t step_smem_bytes()
{
    return (size_t)W * 3 * 4 * 32 * K * sizeof(T);
}

// Opt the kernel in to its dynamic shared memory once (above 48 KB).
template <typename T, int K, int W>
cudaError_t step_smem_setup()
{
    static cudaError_t e = cudaFuncSetAttribute(lw_step_kernel<T, K, W>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)step_smem_bytes<T, K, W>());
    return e;
}

template <typename T, int K, int W>
cudaError_t launch_shape(const StepLaunch &L, const WaveArgs &wa, cudaStream_t st)
{
    cudaError_t e = step_smem_setup<T, K, W>();
    if (e != cudaSuccess) return e;
    if (!kUsePDL) {
        lw_step_kernel<T, K, W><<<L.blocks, W * 32, step_smem_bytes<T, K, W>(), st>>>(
            (const T *)L.u_in, (T *)L.u_out, (const T *)L.half, (const T *)L.node, L.Nr,
            (T)(0.25 * L.dt_inner), (T)(0.5 * L.dt_inner), wa);
        return cudaGetLastError();
    }
    return launch_chained(lw_step_kernel<T, K, W>, (unsigned)L.blocks, W * 32, step_smem_bytes<T, K, W>(),
                          st, (const T *)L.u_in, (T *)L.u_out, (const T *)L.half, (const T *)L.node,
                          L.Nr, (T)(0.25 * L.dt_inner), (T)(0.5 * L.dt_inner), wa);
}

template <typename T, int K, int W>
cudaError_t ring_smem_setup()
{
    static cudaError_t e = cudaFuncSetAttribute(
        lw_step2_ring_kernel<T, K, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)(ring_smem_bytes<T, K>() / ring_warps<T, K>() * W));
    return e;
}

template <typename T, int K, int W>
cudaError_t launch_ring(const StepLaunch &L, const WaveArgs &wa, T eh, T en, int mask, cudaStream_t st)
{
    cudaError_t e = ring_smem_setup<T, K, W>();
    if (e != cudaSuccess) return e;
    const size_t smem = ring_smem_bytes<T, K>() / ring_warps<T, K>() * W;
    lw_step2_ring_kernel<T, K, W><<<L.blocks, W * 32, smem, st>>>(
        (const T *)L.u_in, (T *)L.u_out, (const T *)L.half, (const T *)L.node, L.Nr, eh, en, wa, mask);
    return cudaGetLastError();
}

// Two-step launch: the shared-memory ring kernel for FP32 (memory-bound), the
// register-only kernel for FP64.
template <typename T, int K>
cudaError_t launch_fused(const StepLaunch &L, const WaveArgs &wa, cudaStream_t st)
{
    const T eh = (T)(0.25 * L.dt_inner), en = (T)(0.5 * L.dt_inner);
    const int mask = L.write_wave ? L.obs_mask : 0;
    if constexpr (sizeof(T) == 4) {
        constexpr int WR = ring_warps<T, K>();
        if (L.warps == WR) return launch_ring<T, K, WR>(L, wa, eh, en, mask, st);
        if (L.warps == kNarrowWarps) return launch_ring<T, K, kNarrowWarps>(L, wa, eh, en, mask, st);
        return cudaErrorInvalidValue;
    } else {
        constexpr int WF = fused_warps<T, K>();
        if (L.warps == WF)
            lw_step2_kernel<T, K, WF><<<L.blocks, WF * 32, 0, st>>>(
                (const T *)L.u_in, (T *)L.u_out, (const T *)L.half, (const T *)L.node, L.Nr, eh, en,
                wa, mask);
        else if (L.warps == kNarrowWarps)
            lw_step2_kernel<T, K, kNarrowWarps><<<L.blocks, kNarrowWarps * 32, 0, st>>>(
                (const T *)L.u_in, (T *)L.u_out, (const T *)L.half, (const T *)L.node, L.Nr, eh, en,
                wa, mask);
        else
            return cudaErrorInvalidValue;
        return cudaGetLastError();
    }
}

template <typename T, int K>
cudaError_t launch_typed(const StepLaunch &L, cudaStream_t st)
{
    WaveArgs wa;
    wa.write = L.write_wave;
    wa.sample = L.sample_ctr;
    wa.done = L.done_ctr;
    wa.cap = L.wave_cap;
    wa.wave = L.wave;
    wa.w_row = L.w_row;
    wa.obs = L.obs;
    if (L.fused) return launch_fused<T, K>(L, wa, st);
    if (L.warps == wide_warps<T, K>()) return launch_shape<T, K, wide_warps<T, K>()>(L, wa, st);
    if (L.warps == kNarrowWarps) return launch_shape<T, K, kNarrowWarps>(L, wa, st);
    return cudaErrorInvalidValue;
}

template <typename T, int K, int W>
int resident_blocks()
{
    int n = 0;
    if (step_smem_setup<T, K, W>() != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, lw_step_kernel<T, K, W>, W * 32,
                                                      step_smem_bytes<T, K, W>()) != cudaSuccess)
        n = 0;
    return n;
}

template <typename T, int K>
int grid_shape(int Nr, int num_sms, int *warps)
{
    // Wide when every warp of one block per SM gets a column and the block
    // fits; otherwise narrow blocks, one wave of them at most and at least
    // one column per warp (on a small grid every warp's sweep is
    // latency-bound, and shorter sweeps finish sooner).
    constexpr int WW = wide_warps<T, K>();
    if ((long long)Nr >= (long long)num_sms * WW && resident_blocks<T, K, WW>() >= 1) {
        *warps = WW;
        return num_sms;
    }
    *warps = kNarrowWarps;
    int per_sm = resident_blocks<T, K, kNarrowWarps>();
    if (per_sm < 1) per_sm = 1;
    int blocks = num_sms * per_sm;
    if (blocks > Nr / kNarrowWarps) blocks = Nr / kNarrowWarps;
    return blocks < 1 ? 1 : blocks;
}

template <typename T, int K>
int fused_shape(int Nr, int num_sms, int *warps)
{
    constexpr int WF = sizeof(T) == 4 ? ring_warps<T, K>() : fused_warps<T, K>();
    if ((long long)Nr >= (long long)num_sms * WF) {
        *warps = WF;
        return num_sms;
    }
    *warps = kNarrowWarps;
    int n = 0;
    cudaError_t e;
    if constexpr (sizeof(T) == 4) {
        e = ring_smem_setup<T, K, kNarrowWarps>();
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &n, lw_step2_ring_kernel<T, K, kNarrowWarps>, kNarrowWarps * 32,
                ring_smem_bytes<T, K>() / ring_warps<T, K>() * kNarrowWarps);
    } else {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, lw_step2_kernel<T, K, kNarrowWarps>,
                                                          kNarrowWarps * 32, 0);
    }
    if (e != cudaSuccess || n < 1) n = 1;
    int blocks = num_sms * n;
    if (blocks > Nr / kNarrowWarps) blocks = Nr / kNarrowWarps;
    return blocks < 1 ? 1 : blocks;
}

template <typename T, int K, int W>
int persistent_blocks_w(int Nr, int num_sms)
{
    int n = 0;
    if (step_smem_setup<T, K, W>() != cudaSuccess) return 0;
    static cudaError_t e0 = cudaFuncSetAttribute(lw_persistent_kernel<T, K, W>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)step_smem_bytes<T, K, W>());
    if (e0 != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, lw_persistent_kernel<T, K, W>, W * 32,
                                                      step_smem_bytes<T, K, W>()) != cudaSuccess ||
        n < 1)
        return 0;
    int blocks = num_sms * n;
    if (blocks > Nr / W) blocks = Nr / W;
    return blocks < 1 ? 0 : blocks;
}

template <typename T, int K>
int persistent_blocks(int Nr, int num_sms, int warps)
{
    constexpr int WW = wide_warps<T, K>();
    if (warps == WW) return persistent_blocks_w<T, K, WW>(Nr, num_sms);
    if (warps == kNarrowWarps) return persistent_blocks_w<T, K, kNarrowWarps>(Nr, num_sms);
    return 0;
}

template <typename T, int K, int W>
cudaError_t launch_persistent_w(const StepLaunch &L, void *u_other, int n_inner, int substeps,
                                unsigned int *flags, int *err, cudaStream_t st)
{
    WaveArgs wa;
    wa.write = L.write_wave;
    wa.sample = L.sample_ctr;
    wa.done = L.done_ctr;
    wa.cap = L.wave_cap;
    wa.wave = L.wave;
    wa.w_row = L.w_row;
    wa.obs = L.obs;
    T *u0 = (T *)L.u_in, *u1 = (T *)u_other;
    const T *half = (const T *)L.half, *node = (const T *)L.node;
    int Nr = L.Nr;
    T en = (T)(0.5 * L.dt_inner);
    void *args[] = {&u0, &u1, &half, &node, &Nr, &en, &wa, &n_inner, &substeps, &flags, &err};
    return cudaLaunchCooperativeKernel((const void *)lw_persistent_kernel<T, K, W>, dim3(L.blocks),
                                       dim3(W * 32), args, step_smem_bytes<T, K, W>(), st);
}

template <typename T, int K>
cudaError_t launch_persistent_typed(const StepLaunch &L, void *u_other, int n_inner, int substeps,
                                    unsigned int *flags, int *err, cudaStream_t st)
{
    constexpr int WW = wide_warps<T, K>();
    if (L.warps == WW)
        return launch_persistent_w<T, K, WW>(L, u_other, n_inner, substeps, flags, err, st);
    if (L.warps == kNarrowWarps)
        return launch_persistent_w<T, K, kNarrowWarps>(L, u_other, n_inner, substeps, flags, err, st);
    return cudaErrorInvalidValue;
}

template <typename T, int K, int W>
cudaError_t launch_ring_persistent_w(const StepLaunch &L, void *u_other, int n_pairs, int k,
                                     unsigned int *flags, int *err, cudaStream_t st)
{
    cudaError_t e = ring_smem_setup<T, K, W>();
    if (e != cudaSuccess) return e;
    static cudaError_t e0 = cudaFuncSetAttribute(lw_ring_persistent_kernel<T, K, W>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)(ring_smem_bytes<T, K>() / ring_warps<T, K>() * W));
    if (e0 != cudaSuccess) return e0;
    WaveArgs wa;
    wa.write = L.write_wave;
    wa.sample = L.sample_ctr;
    wa.done = L.done_ctr;
    wa.cap = L.wave_cap;
    wa.wave = L.wave;
    wa.w_row = L.w_row;
    wa.obs = L.obs;
    T *u0 = (T *)L.u_in, *u1 = (T *)u_other;
    const T *half = (const T *)L.half, *node = (const T *)L.node;
    int Nr = L.Nr;
    T en = (T)(0.5 * L.dt_inner);
    void *args[] = {&u0, &u1, &half, &node, &Nr, &en, &wa, &n_pairs, &k, &flags, &err};
    return cudaLaunchCooperativeKernel((const void *)lw_ring_persistent_kernel<T, K, W>, dim3(L.blocks),
                                       dim3(W * 32), args,
                                       ring_smem_bytes<T, K>() / ring_warps<T, K>() * W, st);
}

template <typename T, int K>
cudaError_t launch_ring_persistent_typed(const StepLaunch &L, void *u_other, int n_pairs, int k,
                                         unsigned int *flags, int *err, cudaStream_t st)
{
    constexpr int WR = ring_warps<T, K>();
    if (L.warps == WR) return launch_ring_persistent_w<T, K, WR>(L, u_other, n_pairs, k, flags, err, st);
    if (L.warps == kNarrowWarps)
        return launch_ring_persistent_w<T, K, kNarrowWarps>(L, u_other, n_pairs, k, flags, err, st);
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_ring_persistent(const StepLaunch &L, void *u_other, int n_pairs, int k,
                                   unsigned int *flags, int *err, cudaStream_t st)
{
    if (L.precision != 1) return cudaErrorInvalidValue;
    if (L.K == 1) return launch_ring_persistent_typed<float, 1>(L, u_other, n_pairs, k, flags, err, st);
    if (L.K == 2) return launch_ring_persistent_typed<float, 2>(L, u_other, n_pairs, k, flags, err, st);
    return launch_ring_persistent_typed<float, 4>(L, u_other, n_pairs, k, flags, err, st);
}

namespace {

template <typename T, int K, int W>
cudaError_t launch_multi_persistent_w(const StepLaunch &L, void *u_other, int n_groups, int k,
                                      unsigned int *flags, int *err, void *scratch, cudaStream_t st)
{
    constexpr size_t smem = multi_smem_bytes<K, W, kSweepLevels>();
    static cudaError_t e0 = cudaFuncSetAttribute(lw_multi_persistent_kernel<T, K, W, kSweepLevels>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e0 != cudaSuccess) return e0;
    if (!L.cmp || !L.gpm) return cudaErrorInvalidValue;
    WaveArgs wa;
    wa.write = L.write_wave;
    wa.sample = L.sample_ctr;
    wa.done = L.done_ctr;
    wa.cap = L.wave_cap;
    wa.wave = L.wave;
    wa.w_row = L.w_row;
    wa.obs = L.obs;
    T *u0 = (T *)L.u_in, *u1 = (T *)u_other;
    const float *cmp = L.cmp, *gpm = L.gpm;
    F32Derive fd = f32_derive(L.dt_inner);
    int Nr = L.Nr;
    T en = (T)(0.5 * L.dt_inner);
    T *scr = (T *)scratch;
    void *args[] = {&u0, &u1, &cmp, &gpm, &fd, &Nr, &en, &wa, &n_groups, &k, &flags, &err, &scr};
    return cudaLaunchCooperativeKernel((const void *)lw_multi_persistent_kernel<T, K, W, kSweepLevels>,
                                       dim3(L.blocks), dim3(W * 32), args, smem, st);
}

}  // namespace

int multi_grid_shape(int precision, int K, int Nr, int num_sms, int *warps)
{
    const int W = K == 1 ? multi_warps<float, 1>() : K == 2 ? multi_warps<float, 2>() : multi_warps<float, 4>();
    *warps = W;
    if (precision != 1 || (long long)Nr < (long long)num_sms * W * kSweepLevels) return 0;
    return num_sms;
}

int multi_levels() { return kSweepLevels; }

size_t multi_obs_scratch_bytes(int K, int blocks, int warps)
{
    return multi_obs_scratch_elems_per_warp<kMaxK, kSweepLevels>() / kMaxK * K * sizeof(float) *
           (size_t)blocks * warps;
}

// Whether no warp of the four-step sweep's grid (blocks x warps, the column
// split of warp_range) holds more than kObsCols distinct observer columns.
bool multi_obs_fit(int Nr, int blocks, int warps, const int *obs_i0, int nobs)
{
    const int G = warps / 4;
    for (int b = 0; b < blocks; ++b) {
        const int b0 = (int)(((long long)b * Nr) / blocks), b1 = (int)(((long long)(b + 1) * Nr) / blocks);
        const int C = b1 - b0;
        int start = b0;
        for (int w = 0; w < warps; ++w) {
            const int p = w % 4, q = w / 4;
            const int cp = ((p + 1) * C) / 4 - (p * C) / 4;
            const int c = ((q + 1) * cp) / G - (q * cp) / G;
            int cols[2 * kMaxObservers], n = 0;
            for (int k = 0; k < nobs; ++k)
                for (int sl = 0; sl < 2; ++sl) {
                    const int col = obs_i0[k] + sl;
                    if (col < start || col >= start + c) continue;
                    bool seen = false;
                    for (int h = 0; h < n; ++h) seen |= cols[h] == col;
                    if (!seen) cols[n++] = col;
                }
            if (n > kObsCols) return false;
            start += c;
        }
    }
    return true;
}

cudaError_t launch_multi_persistent(const StepLaunch &L, void *u_other, int n_groups, int k,
                                    unsigned int *flags, int *err, void *scratch, cudaStream_t st)
{
    if (L.precision != 1) return cudaErrorInvalidValue;
    if (L.K == 1 && L.warps == multi_warps<float, 1>())
        return launch_multi_persistent_w<float, 1, multi_warps<float, 1>()>(L, u_other, n_groups, k, flags, err,
                                                                            scratch, st);
    if (L.K == 2 && L.warps == multi_warps<float, 2>())
        return launch_multi_persistent_w<float, 2, multi_warps<float, 2>()>(L, u_other, n_groups, k, flags, err,
                                                                            scratch, st);
    if (L.K == 4 && L.warps == multi_warps<float, 4>())
        return launch_multi_persistent_w<float, 4, multi_warps<float, 4>()>(L, u_other, n_groups, k, flags, err,
                                                                            scratch, st);
    return cudaErrorInvalidValue;
}

int persistent_grid_blocks(int precision, int K, int Nr, int num_sms, int warps)
{
    if (precision == 0)
        return K == 1 ? persistent_blocks<double, 1>(Nr, num_sms, warps)
             : K == 2 ? persistent_blocks<double, 2>(Nr, num_sms, warps)
                      : persistent_blocks<double, 4>(Nr, num_sms, warps);
    return K == 1 ? persistent_blocks<float, 1>(Nr, num_sms, warps)
         : K == 2 ? persistent_blocks<float, 2>(Nr, num_sms, warps)
                  : persistent_blocks<float, 4>(Nr, num_sms, warps);
}

cudaError_t launch_wait_check(int n_blocks, int silent, long long max_spins, unsigned int *flags,
                              int *err, cudaStream_t st)
{
    void *args[] = {&flags, &err, &silent, &max_spins};
    return cudaLaunchCooperativeKernel((const void *)wait_check_kernel, dim3(n_blocks), dim3(32), args,
                                       0, st);
}

cudaError_t launch_lw_persistent(const StepLaunch &L, void *u_other, int n_inner, int substeps,
                                 unsigned int *flags, int *err, cudaStream_t st)
{
    if (L.precision == 0) {
        if (L.K == 1) return launch_persistent_typed<double, 1>(L, u_other, n_inner, substeps, flags, err, st);
        if (L.K == 2) return launch_persistent_typed<double, 2>(L, u_other, n_inner, substeps, flags, err, st);
        return launch_persistent_typed<double, 4>(L, u_other, n_inner, substeps, flags, err, st);
    }
    if (L.K == 1) return launch_persistent_typed<float, 1>(L, u_other, n_inner, substeps, flags, err, st);
    if (L.K == 2) return launch_persistent_typed<float, 2>(L, u_other, n_inner, substeps, flags, err, st);
    return launch_persistent_typed<float, 4>(L, u_other, n_inner, substeps, flags, err, st);
}

int fused_grid_shape(int precision, int K, int Nr, int num_sms, int *warps)
{
    if (precision == 0)
        return K == 1 ? fused_shape<double, 1>(Nr, num_sms, warps)
             : K == 2 ? fused_shape<double, 2>(Nr, num_sms, warps)
                      : fused_shape<double, 4>(Nr, num_sms, warps);
    return K == 1 ? fused_shape<float, 1>(Nr, num_sms, warps)
         : K == 2 ? fused_shape<float, 2>(Nr, num_sms, warps)
                  : fused_shape<float, 4>(Nr, num_sms, warps);
}

int step_grid_shape(int precision, int K, int Nr, int num_sms, int *warps)
{
    if (precision == 0)
        return K == 1 ? grid_shape<double, 1>(Nr, num_sms, warps)
             : K == 2 ? grid_shape<double, 2>(Nr, num_sms, warps)
                      : grid_shape<double, 4>(Nr, num_sms, warps);
    return K == 1 ? grid_shape<float, 1>(Nr, num_sms, warps)
         : K == 2 ? grid_shape<float, 2>(Nr, num_sms, warps)
                  : grid_shape<float, 4>(Nr, num_sms, warps);
}

cudaError_t launch_lw_step(const StepLaunch &L, cudaStream_t st)
{
    if (L.precision == 0) {
        switch (L.K) {
        case 1: return launch_typed<double, 1>(L, st);
        case 2: return launch_typed<double, 2>(L, st);
        case 4: return launch_typed<double, 4>(L, st);
        }
    } else {
        switch (L.K) {
        case 1: return launch_typed<float, 1>(L, st);
        case 2: return launch_typed<float, 2>(L, st);
        case 4: return launch_typed<float, 4>(L, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace tk
