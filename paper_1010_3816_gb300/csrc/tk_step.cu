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

// After the last inner step of an outer step the last block to finish moves
// the sample counter on.  Every block reads the counter before it arrives
// here, so the increment cannot race with a read of the same launch; the next
// launch on the stream sees it.  Keeping the index on the device lets a
// captured chunk of launches be replayed unchanged.
__device__ __forceinline__ void advance_sample(const WaveArgs &wa)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int prev = atomicAdd(wa.done, 1u);
        if (prev == gridDim.x - 1) {
            atomicAdd((unsigned long long *)wa.sample, 1ull);
            atomicExch(wa.done, 0u);
            __threadfence();
        }
    }
}

// Work split: the grid is one wave of resident blocks (SMs x blocks per SM),
// or fewer on a small grid (at least one column per warp).  Block b owns
// columns [b Nr / B, (b+1) Nr / B), within which its warps take contiguous
// ranges.  Warps w and w + 4 run on the same SM sub-partition, so the four
// quarters of the block's columns go to the four pairs and each pair splits
// its quarter in two: every sub-partition gets the same number of columns to
// within one, and the extra column of a pair costs no idle pipe.  A warp
// needs the half-step value at the left edge of its range; the first warp of
// a block recomputes it, every other warp receives it from its left
// neighbour through shared memory once both have finished their sweep (the
// warp's first node is deferred until then).
// Also returns the nearest warp to the left in the block that owns columns
// (-1 if none: this warp then recomputes its left half-step value itself).
__device__ __forceinline__ void warp_range(int Nr, int wib, int *i0, int *i1, int *left)
{
    constexpr int W = kStepThreads / 32;
    const long long B = gridDim.x, b = blockIdx.x;
    const int b0 = (int)((b * Nr) / B), b1 = (int)(((b + 1) * Nr) / B);
    const int C = b1 - b0;
    int start = b0, cnt = 0, prev = -1;
    for (int w = 0; w <= wib; ++w) {
        const int p = w % (W / 2);
        const int cp = (int)(((long long)(p + 1) * C) / (W / 2) - ((long long)p * C) / (W / 2));
        const int c = (w < W / 2) ? (cp + 1) / 2 : cp / 2;
        if (w < wib) {
            start += c;
            if (c > 0) prev = w;
        } else {
            cnt = c;
        }
    }
    *i0 = start;
    *i1 = start + cnt;
    *left = prev;
}

template <typename T, int K>
__global__ void __launch_bounds__(kStepThreads)
lw_step_kernel(const T *__restrict__ u_in, T *__restrict__ u_out, const T *__restrict__ half,
               const T *__restrict__ node, int Nr, T eh, T en, const WaveArgs wa)
{
    constexpr int NP = 32 * K;
    constexpr size_t SP = 4 * NP, HP = (size_t)kNCH * NP, NQ = (size_t)kNCN * NP;
    // per warp: [0] its last half node (read by the right neighbour),
    //           [1] u^n at its first column, [2] u^{n+1/2} right of its first column
    extern __shared__ __align__(16) unsigned char sh_raw[];
    T(*sh)[3][4][NP] = reinterpret_cast<T(*)[3][4][NP]>(sh_raw);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int i0, i1, left;
    warp_range(Nr, wib, &i0, &i1, &left);
    const int row = lane * K;
    const bool lead = (left < 0);

    T ua[4][K], hm[4][K];
    if (i1 > i0) {
        load_col<T, K>(u_in + (size_t)i0 * SP + row, ua);
        if (lead && i0 > 0) {
            T ul[4][K];
            load_col<T, K>(u_in + (size_t)(i0 - 1) * SP + row, ul);
            half_node<T, K>(ul, ua, half + (size_t)(i0 - 1) * HP + row, eh, hm);
        } else {
            zero_col<T, K>(hm);
        }
        for (int i = i0; i < i1; ++i) {
            T uc[4][K], hp[4][K], o[4][K];
            if (i + 1 < Nr) {
                load_col<T, K>(u_in + (size_t)(i + 1) * SP + row, uc);
                half_node<T, K>(ua, uc, half + (size_t)i * HP + row, eh, hp);
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
                if (wa.write) observe<T, K>(i, lane, o, wa.obs, wa.wave, wa.cap, wa.sample, wa.w_row);
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
        if (wa.write) observe<T, K>(i0, lane, o, wa.obs, wa.wave, wa.cap, wa.sample, wa.w_row);
    }
    if (wa.write) advance_sample(wa);
}

template <typename T, int K>
constexpr size_t step_smem_bytes()
{
    return (size_t)(kStepThreads / 32) * 3 * 4 * 32 * K * sizeof(T);
}

// Opt the kernel in to its dynamic shared memory once (above 48 KB for K = 4).
template <typename T, int K>
cudaError_t step_smem_setup()
{
    static cudaError_t e = cudaFuncSetAttribute(lw_step_kernel<T, K>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)step_smem_bytes<T, K>());
    return e;
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
    cudaError_t e = step_smem_setup<T, K>();
    if (e != cudaSuccess) return e;
    lw_step_kernel<T, K><<<L.blocks, kStepThreads, step_smem_bytes<T, K>(), st>>>(
        (const T *)L.u_in, (T *)L.u_out, (const T *)L.half, (const T *)L.node, L.Nr,
        (T)(0.25 * L.dt_inner), (T)(0.5 * L.dt_inner), wa);
    return cudaGetLastError();
}

template <typename T, int K>
int resident_blocks()
{
    int n = 0;
    if (step_smem_setup<T, K>() != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, lw_step_kernel<T, K>, kStepThreads,
                                                      step_smem_bytes<T, K>()) != cudaSuccess)
        n = 1;
    return n < 1 ? 1 : n;
}

}  // namespace

int step_grid_blocks(int precision, int K, int Nr, int num_sms)
{
    int per_sm = 1;
    if (precision == 0)
        per_sm = K == 1 ? resident_blocks<double, 1>() : K == 2 ? resident_blocks<double, 2>()
                                                                : resident_blocks<double, 4>();
    else
        per_sm = K == 1 ? resident_blocks<float, 1>() : K == 2 ? resident_blocks<float, 2>()
                                                               : resident_blocks<float, 4>();
    // One wave of resident blocks (a multiple of the SM count) when the grid
    // is large; for a small grid, as many warps as columns, since there every
    // warp's sweep is latency-bound and shorter sweeps finish sooner.
    const int W = kStepThreads / 32;
    int blocks = num_sms * per_sm;
    const int max_blocks = Nr / W;   // every warp keeps at least one column
    if (blocks > max_blocks) blocks = max_blocks;
    return blocks < 1 ? 1 : blocks;
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
