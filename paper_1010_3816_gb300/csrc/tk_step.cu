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
// and 28 per node.  A segment recomputes one half node at its left end.
#include "tk_internal.h"

namespace tk {
namespace {

constexpr unsigned kFull = 0xffffffffu;

template <typename T, int K>
__device__ __forceinline__ void ldk(const T *__restrict__ p, T (&v)[K])
{
    if constexpr (sizeof(T) == 8 && K == 1) {
        v[0] = p[0];
    } else if constexpr (sizeof(T) == 8) {
#pragma unroll
        for (int t = 0; t < K; t += 2) {
            const double2 x = *reinterpret_cast<const double2 *>(p + t);
            v[t] = x.x;
            v[t + 1] = x.y;
        }
    } else if constexpr (K == 1) {
        v[0] = p[0];
    } else if constexpr (K == 2) {
        const float2 x = *reinterpret_cast<const float2 *>(p);
        v[0] = x.x;
        v[1] = x.y;
    } else {
        const float4 x = *reinterpret_cast<const float4 *>(p);
        v[0] = x.x;
        v[1] = x.y;
        v[2] = x.z;
        v[3] = x.w;
    }
}

template <typename T, int K>
__device__ __forceinline__ void stk(T *__restrict__ p, const T (&v)[K])
{
    if constexpr (sizeof(T) == 8 && K == 1) {
        p[0] = v[0];
    } else if constexpr (sizeof(T) == 8) {
#pragma unroll
        for (int t = 0; t < K; t += 2) *reinterpret_cast<double2 *>(p + t) = make_double2(v[t], v[t + 1]);
    } else if constexpr (K == 1) {
        p[0] = v[0];
    } else if constexpr (K == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    } else {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
}

template <typename T, int K>
__device__ __forceinline__ void load_col(const T *__restrict__ p, T (&u)[4][K])
{
    constexpr int NP = 32 * K;
#pragma unroll
    for (int c = 0; c < 4; ++c) ldk<T, K>(p + c * NP, u[c]);
}

template <typename T, int K>
__device__ __forceinline__ void store_col(T *__restrict__ p, const T (&u)[4][K])
{
    constexpr int NP = 32 * K;
#pragma unroll
    for (int c = 0; c < 4; ++c) stk<T, K>(p + c * NP, u[c]);
}

template <typename T, int K>
__device__ __forceinline__ void zero_col(T (&u)[4][K])
{
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int t = 0; t < K; ++t) u[c][t] = T(0);
}

// Neighbouring-row values of s (row j+1 -> up, row j-1 -> dn) for every row
// a lane holds.  Lane 0's j-1 and lane 31's j+1 read their own values; the
// folded tables give those terms a zero coefficient.
template <typename T, int K>
__device__ __forceinline__ void theta_neighbours(const T (&s)[K], T (&up)[K], T (&dn)[K])
{
    const T nxt = __shfl_down_sync(kFull, s[0], 1);
    const T prv = __shfl_up_sync(kFull, s[K - 1], 1);
#pragma unroll
    for (int t = 0; t < K; ++t) {
        up[t] = (t + 1 < K) ? s[t + 1] : nxt;
        dn[t] = (t > 0) ? s[t - 1] : prv;
    }
}

// Eq. (lw1): u^{n+1/2}_{i+1/2} from a = u^n_i and c = u^n_{i+1}.
template <typename T, int K>
__device__ __forceinline__ void half_node(const T (&a)[4][K], const T (&c)[4][K],
                                          const T *__restrict__ tab, const T e, T (&h)[4][K])
{
    constexpr int NP = 32 * K;
    T sR[K], sI[K], upR[K], upI[K], dnR[K], dnI[K];
#pragma unroll
    for (int t = 0; t < K; ++t) {
        sR[t] = a[0][t] + c[0][t];
        sI[t] = a[1][t] + c[1][t];
    }
    theta_neighbours<T, K>(sR, upR, dnR);
    theta_neighbours<T, K>(sI, upI, dnI);
    T q[kNCH][K];
#pragma unroll
    for (int k = 0; k < kNCH; ++k) ldk<T, K>(tab + k * NP, q[k]);
#pragma unroll
    for (int t = 0; t < K; ++t) {
        const T sPR = a[2][t] + c[2][t];
        const T sPI = a[3][t] + c[3][t];
        h[0][t] = fma(q[H_HQ][t], c[0][t], fma(q[H_HP][t], a[0][t], e * sPR));
        h[1][t] = fma(q[H_HQ][t], c[1][t], fma(q[H_HP][t], a[1][t], e * sPI));
        T x = q[H_PAR][t] * a[2][t];
        x = fma(q[H_PCR][t], c[2][t], x);
        x = fma(-q[H_PI][t], sPI, x);
        x = fma(q[H_FAR][t], a[0][t], x);
        x = fma(-q[H_FAI][t], a[1][t], x);
        x = fma(q[H_FCR][t], c[0][t], x);
        x = fma(-q[H_FCI][t], c[1][t], x);
        x = fma(q[H_KP][t], upR[t], x);
        x = fma(q[H_KM][t], dnR[t], x);
        h[2][t] = x;
        T y = q[H_PAR][t] * a[3][t];
        y = fma(q[H_PCR][t], c[3][t], y);
        y = fma(q[H_PI][t], sPR, y);
        y = fma(q[H_FAR][t], a[1][t], y);
        y = fma(q[H_FAI][t], a[0][t], y);
        y = fma(q[H_FCR][t], c[1][t], y);
        y = fma(q[H_FCI][t], c[0][t], y);
        y = fma(q[H_KP][t], upI[t], y);
        y = fma(q[H_KM][t], dnI[t], y);
        h[3][t] = y;
    }
}

// Eq. (lw2): u^{n+1}_i from hm = u^{n+1/2}_{i-1/2}, hp = u^{n+1/2}_{i+1/2}, u = u^n_i.
template <typename T, int K>
__device__ __forceinline__ void full_node(const T (&hm)[4][K], const T (&hp)[4][K],
                                          const T (&u)[4][K], const T *__restrict__ tab,
                                          const T e, T (&o)[4][K])
{
    constexpr int NP = 32 * K;
    T sR[K], sI[K], upR[K], upI[K], dnR[K], dnI[K];
#pragma unroll
    for (int t = 0; t < K; ++t) {
        sR[t] = hp[0][t] + hm[0][t];
        sI[t] = hp[1][t] + hm[1][t];
    }
    theta_neighbours<T, K>(sR, upR, dnR);
    theta_neighbours<T, K>(sI, upI, dnI);
    T q[kNCN][K];
#pragma unroll
    for (int k = 0; k < kNCN; ++k) ldk<T, K>(tab + k * NP, q[k]);
#pragma unroll
    for (int t = 0; t < K; ++t) {
        const T sPR = hp[2][t] + hm[2][t];
        const T sPI = hp[3][t] + hm[3][t];
        o[0][t] = fma(e, sPR, fma(q[N_B][t], hm[0][t], fma(-q[N_B][t], hp[0][t], u[0][t])));
        o[1][t] = fma(e, sPI, fma(q[N_B][t], hm[1][t], fma(-q[N_B][t], hp[1][t], u[1][t])));
        T x = fma(q[N_PPR][t], hp[2][t], u[2][t]);
        x = fma(q[N_PMR][t], hm[2][t], x);
        x = fma(-q[N_C2I][t], sPI, x);
        x = fma(q[N_FPR][t], hp[0][t], x);
        x = fma(-q[N_FPI][t], hp[1][t], x);
        x = fma(q[N_FMR][t], hm[0][t], x);
        x = fma(-q[N_FMI][t], hm[1][t], x);
        x = fma(q[N_KP][t], upR[t], x);
        x = fma(q[N_KM][t], dnR[t], x);
        o[2][t] = x;
        T y = fma(q[N_PPR][t], hp[3][t], u[3][t]);
        y = fma(q[N_PMR][t], hm[3][t], y);
        y = fma(q[N_C2I][t], sPR, y);
        y = fma(q[N_FPR][t], hp[1][t], y);
        y = fma(q[N_FPI][t], hp[0][t], y);
        y = fma(q[N_FMR][t], hm[1][t], y);
        y = fma(q[N_FMI][t], hm[0][t], y);
        y = fma(q[N_KP][t], upI[t], y);
        y = fma(q[N_KM][t], dnI[t], y);
        o[3][t] = y;
    }
}

struct WaveArgs {
    int write;
    int64_t sample, cap;
    double *wave;
    const double *w_row;
    ObsDev obs;
};

// Partial bilinear sample (Sec. "waveform extraction" of the design notes):
// slot 0 holds (1 - fr) * [(1-fth) w_j0 Phi_{i0,j0} + fth w_j0+1 Phi_{i0,j0+1}],
// slot 1 the same at column i0 + 1 times fr; the sample is slot 0 + slot 1.
template <typename T, int K>
__device__ __forceinline__ void observe(int i, int lane, const T (&o)[4][K], const WaveArgs &wa)
{
    for (int k = 0; k < wa.obs.n; ++k) {
        const int slot = (i == wa.obs.i0[k]) ? 0 : ((i == wa.obs.i0[k] + 1) ? 1 : -1);
        if (slot < 0) continue;
        const int j0 = wa.obs.j0[k];
        const double w0 = (1.0 - wa.obs.ft[k]) * wa.w_row[j0];
        const double w1 = wa.obs.ft[k] * wa.w_row[j0 + 1];
        double cr = 0.0, ci = 0.0;
#pragma unroll
        for (int t = 0; t < K; ++t) {
            const int r = lane * K + t;
            if (r == j0) {
                cr += w0 * (double)o[0][t];
                ci += w0 * (double)o[1][t];
            } else if (r == j0 + 1) {
                cr += w1 * (double)o[0][t];
                ci += w1 * (double)o[1][t];
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            cr += __shfl_xor_sync(kFull, cr, off);
            ci += __shfl_xor_sync(kFull, ci, off);
        }
        if (lane == 0) {
            const double wr = slot ? wa.obs.wr1[k] : wa.obs.wr0[k];
            double *dst = wa.wave + ((size_t)k * wa.cap + wa.sample) * 4 + 2 * slot;
            dst[0] = wr * cr;
            dst[1] = wr * ci;
        }
    }
}

// Work split: the grid has exactly (SMs x resident blocks) blocks of
// kStepWarps warps; global warp g owns columns [g Nr / G, (g+1) Nr / G), so
// every SM gets the same number of columns to within one per warp.  A warp
// needs the half-step value at the left edge of its range; the first warp of
// a block recomputes it, every other warp receives it from its left
// neighbour through shared memory once both have finished their sweep (the
// warp's first node is deferred until then).
template <typename T, int K>
__global__ void __launch_bounds__(kStepThreads)
lw_step_kernel(const T *__restrict__ u_in, T *__restrict__ u_out, const T *__restrict__ half,
               const T *__restrict__ node, int Nr, T eh, T en, const WaveArgs wa)
{
    constexpr int NP = 32 * K;
    constexpr size_t SP = 4 * NP, HP = (size_t)kNCH * NP, NQ = (size_t)kNCN * NP;
    constexpr int W = kStepThreads / 32;
    // per warp: [0] its last half node (read by the right neighbour),
    //           [1] u^n at its first column, [2] u^{n+1/2} right of its first column
    __shared__ T sh[W][3][4][NP];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const long long G = (long long)gridDim.x * W;
    const long long g = (long long)blockIdx.x * W + wib;
    const int i0 = (int)((g * Nr) / G);
    const int i1 = (int)(((g + 1) * Nr) / G);
    const int row = lane * K;
    const bool lead = (wib == 0);

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
                if (wa.write) observe<T, K>(i, lane, o, wa);
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
                hl[c][t] = sh[wib - 1][0][c][row + t];
                ua[c][t] = sh[wib][1][c][row + t];
                hp[c][t] = sh[wib][2][c][row + t];
            }
        full_node<T, K>(hl, hp, ua, node + (size_t)i0 * NQ + row, en, o);
        if (i0 == 0 || i0 == Nr - 1) zero_col<T, K>(o);
        store_col<T, K>(u_out + (size_t)i0 * SP + row, o);
        if (wa.write) observe<T, K>(i0, lane, o, wa);
    }
}

template <typename T, int K>
cudaError_t launch_typed(const StepLaunch &L, cudaStream_t st)
{
    WaveArgs wa;
    wa.write = L.write_wave;
    wa.sample = L.sample;
    wa.cap = L.wave_cap;
    wa.wave = L.wave;
    wa.w_row = L.w_row;
    wa.obs = L.obs;
    lw_step_kernel<T, K><<<L.blocks, kStepThreads, 0, st>>>(
        (const T *)L.u_in, (T *)L.u_out, (const T *)L.half, (const T *)L.node, L.Nr,
        (T)(0.25 * L.dt_inner), (T)(0.5 * L.dt_inner), wa);
    return cudaGetLastError();
}

template <typename T, int K>
int resident_blocks()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, lw_step_kernel<T, K>, kStepThreads, 0) !=
        cudaSuccess)
        n = 1;
    return n < 1 ? 1 : n;
}

}  // namespace

int step_grid_blocks(int precision, int K, int Nr, int num_sms)
{
    // one wave of resident blocks, each warp at least two columns wide
    int per_sm = 1;
    if (precision == 0)
        per_sm = K == 1 ? resident_blocks<double, 1>() : K == 2 ? resident_blocks<double, 2>()
                                                                : resident_blocks<double, 4>();
    else
        per_sm = K == 1 ? resident_blocks<float, 1>() : K == 2 ? resident_blocks<float, 2>()
                                                               : resident_blocks<float, 4>();
    const int W = kStepThreads / 32;
    int blocks = num_sms * per_sm;
    const int max_blocks = Nr / (2 * W);
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
