// tk_stencil.cuh -- per-column device routines of the fused Lax-Wendroff step,
// shared by the single-solver kernel (tk_step.cu) and the batched kernel
// (tk_batch.cu).  One warp owns all theta rows of a column: lane l holds rows
// K*l .. K*l+K-1; u[c][t] is component c (Phi_R, Phi_I, Pi_R, Pi_I) of row K*l+t.
#pragma once

#include "tk_internal.h"

namespace tk {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// GB300's FP64 pipe issues DADD and DMUL at a lower rate than DFMA (the
// one-step kernel runs 2.4 % faster with the sums and products below as
// FMAs).  x + y is formed as fma(x, 1, y) and a * b as fma(a, b, -0), which
// round exactly like the add and the multiply; in FP64 the constants 1 and -0
// are read from device memory (through the read-only cache) at run time, so
// the compiler cannot fold the FMAs back into adds and multiplies.  FP32 has
// no such gap and takes them as literals (the compiler then issues the add
// and the multiply).
__device__ double g_fma_one = 1.0;
__device__ double g_fma_nzero = -0.0;

template <typename T>
struct FmaK {
    T one, nz;
};

template <typename T>
__device__ __forceinline__ FmaK<T> fma_k()
{
    if constexpr (sizeof(T) == 8) return {__ldg(&g_fma_one), __ldg(&g_fma_nzero)};
    else return {T(1), T(-0.0)};
}

// Chained launches (programmatic dependent launch).  A kernel launched by
// launch_chained may be scheduled while the previous kernel on the stream is
// still running; it calls chain_start() first, which lets the next kernel be
// scheduled in turn and then waits until the previous kernel has completed
// and its writes are visible.  Both instructions are no-ops for a kernel
// launched without the programmatic edge.
__device__ __forceinline__ void chain_start()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_chained(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem,
                           cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

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

// Work split.  Block b owns columns [b Nr / B, (b+1) Nr / B), within which
// its warps take contiguous ranges, in warp order.  Warps w, w + 4, w + 8,
// ... run on the same SM sub-partition, so the four quarters of the block's
// columns go to the four sub-partitions, and each sub-partition's warps split
// their quarter evenly: with one block per SM every sub-partition gets the
// same number of columns to within one.  A warp needs the half-step value at
// the left edge of its range; the first warp of a block recomputes it, every
// other warp receives it from its left neighbour through shared memory once
// both have finished their sweep (the warp's first node is deferred until
// then).  Also returns the nearest warp to the left in the block that owns
// columns (-1 if none: this warp then recomputes its left half-step value).
template <int W>
__device__ __forceinline__ void warp_range(int Nr, int wib, int *i0, int *i1, int *left)
{
    constexpr int G = W / 4;   // warps per sub-partition
    const long long B = gridDim.x, b = blockIdx.x;
    const int b0 = (int)((b * Nr) / B), b1 = (int)(((b + 1) * Nr) / B);
    const int C = b1 - b0;
    int start = b0, cnt = 0, prev = -1;
    for (int w = 0; w <= wib; ++w) {
        const int p = w % 4, q = w / 4;
        const int cp = ((p + 1) * C) / 4 - (p * C) / 4;
        const int c = ((q + 1) * cp) / G - (q * cp) / G;
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

// FP32 with two rows per lane: the rows go in pairs through GB300's packed
// FP32 instructions (__ffma2_rn, __fadd2_rn, __fmul2_rn: two single-precision
// operations per instruction, each rounded exactly like the scalar one), so
// the node routines below are bit-identical to their scalar form with half as
// many FP32 arithmetic instructions.  With four rows per lane the scalar form
// is the faster one (the four-step sweep on 25601 x 128: 20.3 against 22.2 us
// per step; on 25601 x 64, two rows, the pairs win, 10.3 against 11.0 us), so
// only K = 2 pairs its rows.
template <int K>
constexpr bool kPairRows = (K == 2);
__device__ __forceinline__ float2 pr2(const float *v, int t) { return make_float2(v[t], v[t + 1]); }
__device__ __forceinline__ float2 ng2(float2 v) { return make_float2(-v.x, -v.y); }
__device__ __forceinline__ void st2(float *v, int t, float2 x)
{
    v[t] = x.x;
    v[t + 1] = x.y;
}

// Eq. (lw1): u^{n+1/2}_{i+1/2} from a = u^n_i and c = u^n_{i+1}.  The Phi
// components come out divided by eh = dt/4: the table entries HP, HQ carry the
// factor 1/eh and the node tables multiply the half-node Phi values back by
// eh, so the term eh (Pi_a + Pi_c) is added without a multiplication.
// PI_TERM = false leaves that term out (the derivative of the step with
// respect to the tables, where it is constant).
template <typename T, int K, bool PI_TERM = true>
__device__ __forceinline__ void half_node_q(const T (&a)[4][K], const T (&c)[4][K],
                                            const T (&q)[kNCH][K], T (&h)[4][K])
{
    const FmaK<T> k1 = fma_k<T>();
    T sR[K], sI[K], upR[K], upI[K], dnR[K], dnI[K];
    if constexpr (sizeof(T) == 4 && kPairRows<K>) {
#pragma unroll
        for (int t = 0; t < K; t += 2) {
            st2(sR, t, __fadd2_rn(pr2(a[0], t), pr2(c[0], t)));
            st2(sI, t, __fadd2_rn(pr2(a[1], t), pr2(c[1], t)));
        }
    } else {
#pragma unroll
        for (int t = 0; t < K; ++t) {
            sR[t] = fma(a[0][t], k1.one, c[0][t]);
            sI[t] = fma(a[1][t], k1.one, c[1][t]);
        }
    }
    theta_neighbours<T, K>(sR, upR, dnR);
    theta_neighbours<T, K>(sI, upI, dnI);
    if constexpr (sizeof(T) == 4 && kPairRows<K>) {
#pragma unroll
        for (int t = 0; t < K; t += 2) {
            const float2 a0 = pr2(a[0], t), a1 = pr2(a[1], t), a2 = pr2(a[2], t), a3 = pr2(a[3], t);
            const float2 c0 = pr2(c[0], t), c1 = pr2(c[1], t), c2 = pr2(c[2], t), c3 = pr2(c[3], t);
            const float2 sPR = __fadd2_rn(a2, c2);
            const float2 sPI = __fadd2_rn(a3, c3);
            const float2 HP = pr2(q[H_HP], t), HQ = pr2(q[H_HQ], t), PAR = pr2(q[H_PAR], t);
            const float2 PCR = pr2(q[H_PCR], t), PI = pr2(q[H_PI], t), FAR = pr2(q[H_FAR], t);
            const float2 FAI = pr2(q[H_FAI], t), FCR = pr2(q[H_FCR], t), FCI = pr2(q[H_FCI], t);
            const float2 KP = pr2(q[H_KP], t), KM = pr2(q[H_KM], t);
            if constexpr (PI_TERM) {
                st2(h[0], t, __ffma2_rn(HQ, c0, __ffma2_rn(HP, a0, sPR)));
                st2(h[1], t, __ffma2_rn(HQ, c1, __ffma2_rn(HP, a1, sPI)));
            } else {
                st2(h[0], t, __ffma2_rn(HQ, c0, __fmul2_rn(HP, a0)));
                st2(h[1], t, __ffma2_rn(HQ, c1, __fmul2_rn(HP, a1)));
            }
            float2 x = __fmul2_rn(PAR, a2);
            x = __ffma2_rn(PCR, c2, x);
            x = __ffma2_rn(ng2(PI), sPI, x);
            x = __ffma2_rn(FAR, a0, x);
            x = __ffma2_rn(ng2(FAI), a1, x);
            x = __ffma2_rn(FCR, c0, x);
            x = __ffma2_rn(ng2(FCI), c1, x);
            x = __ffma2_rn(KP, pr2(upR, t), x);
            x = __ffma2_rn(KM, pr2(dnR, t), x);
            st2(h[2], t, x);
            float2 y = __fmul2_rn(PAR, a3);
            y = __ffma2_rn(PCR, c3, y);
            y = __ffma2_rn(PI, sPR, y);
            y = __ffma2_rn(FAR, a1, y);
            y = __ffma2_rn(FAI, a0, y);
            y = __ffma2_rn(FCR, c1, y);
            y = __ffma2_rn(FCI, c0, y);
            y = __ffma2_rn(KP, pr2(upI, t), y);
            y = __ffma2_rn(KM, pr2(dnI, t), y);
            st2(h[3], t, y);
        }
        return;
    }
#pragma unroll
    for (int t = 0; t < K; ++t) {
        const T sPR = fma(a[2][t], k1.one, c[2][t]);
        const T sPI = fma(a[3][t], k1.one, c[3][t]);
        if constexpr (PI_TERM) {
            h[0][t] = fma(q[H_HQ][t], c[0][t], fma(q[H_HP][t], a[0][t], sPR));
            h[1][t] = fma(q[H_HQ][t], c[1][t], fma(q[H_HP][t], a[1][t], sPI));
        } else {
            h[0][t] = fma(q[H_HQ][t], c[0][t], fma(q[H_HP][t], a[0][t], k1.nz));
            h[1][t] = fma(q[H_HQ][t], c[1][t], fma(q[H_HP][t], a[1][t], k1.nz));
        }
        T x = fma(q[H_PAR][t], a[2][t], k1.nz);
        x = fma(q[H_PCR][t], c[2][t], x);
        x = fma(-q[H_PI][t], sPI, x);
        x = fma(q[H_FAR][t], a[0][t], x);
        x = fma(-q[H_FAI][t], a[1][t], x);
        x = fma(q[H_FCR][t], c[0][t], x);
        x = fma(-q[H_FCI][t], c[1][t], x);
        x = fma(q[H_KP][t], upR[t], x);
        x = fma(q[H_KM][t], dnR[t], x);
        h[2][t] = x;
        T y = fma(q[H_PAR][t], a[3][t], k1.nz);
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
__device__ __forceinline__ void full_node_q(const T (&hm)[4][K], const T (&hp)[4][K],
                                            const T (&u)[4][K], const T (&q)[kNCN][K],
                                            const T e, T (&o)[4][K])
{
    const FmaK<T> k1 = fma_k<T>();
    T sR[K], sI[K], upR[K], upI[K], dnR[K], dnI[K];
    if constexpr (sizeof(T) == 4 && kPairRows<K>) {
#pragma unroll
        for (int t = 0; t < K; t += 2) {
            st2(sR, t, __fadd2_rn(pr2(hp[0], t), pr2(hm[0], t)));
            st2(sI, t, __fadd2_rn(pr2(hp[1], t), pr2(hm[1], t)));
        }
    } else {
#pragma unroll
        for (int t = 0; t < K; ++t) {
            sR[t] = fma(hp[0][t], k1.one, hm[0][t]);
            sI[t] = fma(hp[1][t], k1.one, hm[1][t]);
        }
    }
    theta_neighbours<T, K>(sR, upR, dnR);
    theta_neighbours<T, K>(sI, upI, dnI);
    if constexpr (sizeof(T) == 4 && kPairRows<K>) {
        const float2 e2 = make_float2(e, e);
#pragma unroll
        for (int t = 0; t < K; t += 2) {
            const float2 m0 = pr2(hm[0], t), m1 = pr2(hm[1], t), m2 = pr2(hm[2], t), m3 = pr2(hm[3], t);
            const float2 p0 = pr2(hp[0], t), p1 = pr2(hp[1], t), p2 = pr2(hp[2], t), p3 = pr2(hp[3], t);
            const float2 sPR = __fadd2_rn(p2, m2);
            const float2 sPI = __fadd2_rn(p3, m3);
            const float2 B = pr2(q[N_B], t), PPR = pr2(q[N_PPR], t), PMR = pr2(q[N_PMR], t);
            const float2 C2I = pr2(q[N_C2I], t), FPR = pr2(q[N_FPR], t), FPI = pr2(q[N_FPI], t);
            const float2 FMR = pr2(q[N_FMR], t), FMI = pr2(q[N_FMI], t);
            const float2 KP = pr2(q[N_KP], t), KM = pr2(q[N_KM], t);
            st2(o[0], t, __ffma2_rn(e2, sPR, __ffma2_rn(B, m0, __ffma2_rn(ng2(B), p0, pr2(u[0], t)))));
            st2(o[1], t, __ffma2_rn(e2, sPI, __ffma2_rn(B, m1, __ffma2_rn(ng2(B), p1, pr2(u[1], t)))));
            float2 x = __ffma2_rn(PPR, p2, pr2(u[2], t));
            x = __ffma2_rn(PMR, m2, x);
            x = __ffma2_rn(ng2(C2I), sPI, x);
            x = __ffma2_rn(FPR, p0, x);
            x = __ffma2_rn(ng2(FPI), p1, x);
            x = __ffma2_rn(FMR, m0, x);
            x = __ffma2_rn(ng2(FMI), m1, x);
            x = __ffma2_rn(KP, pr2(upR, t), x);
            x = __ffma2_rn(KM, pr2(dnR, t), x);
            st2(o[2], t, x);
            float2 y = __ffma2_rn(PPR, p3, pr2(u[3], t));
            y = __ffma2_rn(PMR, m3, y);
            y = __ffma2_rn(C2I, sPR, y);
            y = __ffma2_rn(FPR, p1, y);
            y = __ffma2_rn(FPI, p0, y);
            y = __ffma2_rn(FMR, m1, y);
            y = __ffma2_rn(FMI, m0, y);
            y = __ffma2_rn(KP, pr2(upI, t), y);
            y = __ffma2_rn(KM, pr2(dnI, t), y);
            st2(o[3], t, y);
        }
        return;
    }
#pragma unroll
    for (int t = 0; t < K; ++t) {
        const T sPR = fma(hp[2][t], k1.one, hm[2][t]);
        const T sPI = fma(hp[3][t], k1.one, hm[3][t]);
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

// The node routines with their tables read from a table column (the 21-entry
// layout of both precisions).
template <typename T, int K, bool PI_TERM = true>
__device__ __forceinline__ void half_node(const T (&a)[4][K], const T (&c)[4][K],
                                          const T *__restrict__ tab, T (&h)[4][K])
{
    constexpr int NP = 32 * K;
    T q[kNCH][K];
#pragma unroll
    for (int k = 0; k < kNCH; ++k) ldk<T, K>(tab + k * NP, q[k]);
    half_node_q<T, K, PI_TERM>(a, c, q, h);
}

template <typename T, int K>
__device__ __forceinline__ void full_node(const T (&hm)[4][K], const T (&hp)[4][K],
                                          const T (&u)[4][K], const T *__restrict__ tab,
                                          const T e, T (&o)[4][K])
{
    constexpr int NP = 32 * K;
    T q[kNCN][K];
#pragma unroll
    for (int k = 0; k < kNCN; ++k) ldk<T, K>(tab + k * NP, q[k]);
    full_node_q<T, K>(hm, hp, u, q, e, o);
}

// FP32 compact tables (kNCC entries per column): the 21 entries of a column
// from its 16 stored ones, the lane's theta factors gp, gm and the constants
// of F32Derive, by the FP32 operations with which the table builder formed
// the full tables (so both layouts give the same bits).  Scalar even with two
// rows per lane: the four-step sweep on 25601 x 64 runs 10.1 us per step with
// these in scalar form against 10.4 with them paired too.
template <int K>
__device__ __forceinline__ void derive_half(const float *__restrict__ tab, const float (&gp)[K],
                                            const float (&gm)[K], const F32Derive &fd,
                                            float (&q)[kNCH][K])
{
    constexpr int NP = 32 * K;
    float C4[K];
    ldk<float, K>(tab + C_HP * NP, q[H_HP]);
    ldk<float, K>(tab + C_PAR * NP, q[H_PAR]);
    ldk<float, K>(tab + C_PI * NP, q[H_PI]);
    ldk<float, K>(tab + C_FAR * NP, q[H_FAR]);
    ldk<float, K>(tab + C_FAI * NP, q[H_FAI]);
    ldk<float, K>(tab + C_FCR * NP, q[H_FCR]);
    ldk<float, K>(tab + C_FCI * NP, q[H_FCI]);
    ldk<float, K>(tab + C_C4H * NP, C4);
#pragma unroll
    for (int t = 0; t < K; ++t) {
        q[H_HQ][t] = __fadd_rn(fd.ih, -q[H_HP][t]);
        q[H_PCR][t] = __fadd_rn(q[H_PAR][t], __fmaf_rn(fd.t2, q[H_HP][t], -1.0f));
        q[H_KP][t] = __fmul_rn(C4[t], gp[t]);
        q[H_KM][t] = __fmul_rn(C4[t], gm[t]);
    }
}

template <int K>
__device__ __forceinline__ void derive_node(const float *__restrict__ tab, const float (&gp)[K],
                                            const float (&gm)[K], const F32Derive &fd,
                                            float (&q)[kNCN][K])
{
    constexpr int NP = 32 * K;
    float C4[K];
    ldk<float, K>(tab + (C_B - C_B) * NP, q[N_B]);
    ldk<float, K>(tab + (C_PMR - C_B) * NP, q[N_PMR]);
    ldk<float, K>(tab + (C_C2I - C_B) * NP, q[N_C2I]);
    ldk<float, K>(tab + (C_FPR - C_B) * NP, q[N_FPR]);
    ldk<float, K>(tab + (C_FPI - C_B) * NP, q[N_FPI]);
    ldk<float, K>(tab + (C_FMR - C_B) * NP, q[N_FMR]);
    ldk<float, K>(tab + (C_FMI - C_B) * NP, q[N_FMI]);
    ldk<float, K>(tab + (C_C4N - C_B) * NP, C4);
#pragma unroll
    for (int t = 0; t < K; ++t) {
        q[N_PPR][t] = __fmaf_rn(fd.bn2, q[N_B][t], q[N_PMR][t]);
        q[N_KP][t] = __fmul_rn(C4[t], gp[t]);
        q[N_KM][t] = __fmul_rn(C4[t], gm[t]);
    }
}

// Partial bilinear sample (the paper prints no extraction rule; the sample
// is the bilinear interpolant in (r*, theta) of the physical Phi = w Phi^):
// in FP64, slot 0 holds (1 - fr) * [(1-fth) w_j0 Phi_{i0,j0} + fth w_j0+1 Phi_{i0,j0+1}],
// slot 1 the same at column i0 + 1 times fr; the sample is slot 0 + slot 1.
// In FP32 a slot holds the four FP32 values Phi_{R,I} at rows j0, j0 + 1, and
// the read-out forms the same sample from them in FP64 (WaveRead).
// observe_one_at: observer k's slot of sample `sample` from the column's
// Phi_R, Phi_I (K rows per lane); all 32 lanes take part, lane 0 writes.
template <typename T, int K>
__device__ __forceinline__ void observe_one_at(int lane, int k, int slot, const T (&re)[K], const T (&im)[K],
                                               const ObsDev &obs, double *wave, int64_t cap,
                                               const double *w_row, long long sample)
{
    // only rows j0 and j0 + 1 contribute: fetch them from the lanes that hold
    // them (two shuffles) and let lane 0 do the few operations, instead of a
    // reduction over the warp, whose FP64 adds hold GB300's FP64 pipe for
    // microseconds
    const int j0 = obs.j0[k];
    const int t0 = j0 % K, t1 = (j0 + 1) % K;
    T ar = re[0], ai = im[0], br = re[0], bi = im[0];
#pragma unroll
    for (int t = 1; t < K; ++t) {
        if (t == t0) {
            ar = re[t];
            ai = im[t];
        }
        if (t == t1) {
            br = re[t];
            bi = im[t];
        }
    }
    ar = __shfl_sync(kFull, ar, j0 / K);
    ai = __shfl_sync(kFull, ai, j0 / K);
    br = __shfl_sync(kFull, br, (j0 + 1) / K);
    bi = __shfl_sync(kFull, bi, (j0 + 1) / K);
    if (lane == 0) {
        double *dst = wave + ((size_t)k * cap + sample) * 4 + 2 * slot;
        if constexpr (sizeof(T) == 4) {
            // FP32: the values themselves, one 16-byte store, no arithmetic
            // (the entry is 16-byte aligned: 4 doubles per sample, 2 per slot)
            *reinterpret_cast<float4 *>(dst) = make_float4(ar, ai, br, bi);
        } else {
            const double w0 = (1.0 - obs.ft[k]) * w_row[j0];
            const double w1 = obs.ft[k] * w_row[j0 + 1];
            const double cr = w0 * (double)ar + w1 * (double)br;
            const double ci = w0 * (double)ai + w1 * (double)bi;
            const double wr = slot ? obs.wr1[k] : obs.wr0[k];
            dst[0] = wr * cr;
            dst[1] = wr * ci;
        }
    }
}

// Every observer slot at column i, for sample `sample`.
template <typename T, int K>
__device__ __forceinline__ void observe_at(int i, int lane, const T (&re)[K], const T (&im)[K], const ObsDev &obs,
                                           double *wave, int64_t cap, const double *w_row, long long sample)
{
    for (int k = 0; k < obs.n; ++k) {
        const int slot = (i == obs.i0[k]) ? 0 : ((i == obs.i0[k] + 1) ? 1 : -1);
        if (slot < 0) continue;
        observe_one_at<T, K>(lane, k, slot, re, im, obs, wave, cap, w_row, sample);
    }
}

// The same with the sample index read from the device counter (which a
// replayed graph of launches moves on between outer steps) plus an offset.
template <typename T, int K>
__device__ __forceinline__ void observe(int i, int lane, const T (&o)[4][K], const ObsDev &obs,
                                        double *wave, int64_t cap, const long long *sample_ctr,
                                        const double *w_row, int sample_offset = 0)
{
    for (int k = 0; k < obs.n; ++k) {
        const int slot = (i == obs.i0[k]) ? 0 : ((i == obs.i0[k] + 1) ? 1 : -1);
        if (slot < 0) continue;
        long long sample = 0;
        if (lane == 0) sample = *(volatile const long long *)sample_ctr + sample_offset;
        observe_one_at<T, K>(lane, k, slot, o[0], o[1], obs, wave, cap, w_row, sample);
    }
}

// Bounded waits of the persistent kernels.  A wait gives up after kMaxSpins
// polls (about 8.6 s on GB300), or at once when *err is already set, and
// sets *err; the launch then ends and the host reports the error.
constexpr long long kMaxSpins = 1ll << 24;

__device__ __forceinline__ unsigned int load_acquire(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// A whole warp waits (bounded) until *flag >= epoch; every lane reads the
// flag with acquire semantics, and the lanes leave together.
__device__ __forceinline__ void warp_wait_flag(const unsigned int *flag, unsigned int epoch, int *err,
                                               long long max_spins = kMaxSpins)
{
    long long spins = 0;
    while (!__all_sync(0xffffffffu, load_acquire(flag) >= epoch)) {
        if (__any_sync(0xffffffffu, ++spins > max_spins || *(volatile int *)err != 0)) {
            if ((threadIdx.x & 31) == 0) atomicExch(err, 1);
            return;
        }
        __nanosleep(64);
    }
}

// Progress counters between the warps of a block, in shared memory: a
// release store after the warp's writes, acquire loads by the waiting warp.
__device__ __forceinline__ void cta_release(unsigned int *p, unsigned int v)
{
    asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)),
                 "r"(v)
                 : "memory");
}

__device__ __forceinline__ unsigned int cta_acquire(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];"
                 : "=r"(v)
                 : "r"((unsigned)__cvta_generic_to_shared(p))
                 : "memory");
    return v;
}

// A whole warp waits (bounded) until the shared counter *c >= v.
__device__ __forceinline__ void warp_wait_cta(const unsigned int *c, unsigned int v, int *err,
                                              long long max_spins = kMaxSpins)
{
    long long spins = 0;
    while (!__all_sync(0xffffffffu, cta_acquire(c) >= v)) {
        if (__any_sync(0xffffffffu, ++spins > max_spins || *(volatile int *)err != 0)) {
            if ((threadIdx.x & 31) == 0) atomicExch(err, 1);
            return;
        }
        __nanosleep(32);
    }
}

// The warp's writes so far are visible to the block (cta) or to the GPU
// before the counter or flag says so.
__device__ __forceinline__ void warp_publish_cta(unsigned int *c, unsigned int v)
{
    __syncwarp();
    if ((threadIdx.x & 31) == 0) cta_release(c, v);
}

__device__ __forceinline__ void warp_publish_gpu(unsigned int *f, unsigned int v)
{
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        __threadfence();
        atomicExch(f, v);
    }
}

}  // namespace
}  // namespace tk
