// tk_adjoint.cu -- the transpose of the fused Lax-Wendroff step, for
// gradients of waveform losses with respect to the initial data.
//
// One inner step is linear and time-invariant: u^{n+1} = A u^n, with
//   h_{i+1/2} = H(u_i, u_{i+1})                        (Eq. lw1, folded tables "half")
//   u^{n+1}_i = u^n_i + N(h_{i-1/2}, h_{i+1/2})        (Eq. lw2, folded tables "node")
// and u^{n+1} = 0 on the two radial edges.  Its transpose maps an adjoint
// state lam (dL/du^{n+1}) to mu = A^T lam (dL/du^n):
//   lam~ = lam with the edge columns set to 0,
//   eta_{i+1/2} = (dN_i/dh_{i+1/2})^T lam~_i + (dN_{i+1}/dh_{i+1/2})^T lam~_{i+1},
//   mu_i = lam~_i + (dH_{i+1/2}/du_i)^T eta_{i+1/2} + (dH_{i-1/2}/du_i)^T eta_{i-1/2},
// where every (.)^T is the transposed 4x4 block of the same folded table
// entries the forward kernel uses, and the theta-neighbour couplings (KP to
// row j+1, KM to row j-1) become KP of row j-1 and KM of row j+1.  The
// waveform sample of an outer step is linear in the state, so its loss
// gradient enters as a source on the adjoint state of that step.
//
// A warp owns all theta rows of a range of output columns and walks it left
// to right; the work split and the hand-off of the left-edge eta between the
// warps of a block are those of the forward step kernel.
#include <math.h>
#include <string.h>

#include <vector>

#include "tk_solver_impl.h"
#include "tk_stencil.cuh"

namespace tk {
namespace {

struct InjectArgs {
    int on;                  // add the observation gradient of sample `sample`
    long long sample, count; // sample index; samples per observer in dwave
    const double *dwave;     // [obs][count][2]: dL/dRe W, dL/dIm W
    const double *w_row;
    ObsDev obs;
};

// Load the adjoint state of column i, add the gradient of the waveform sample
// `sample` taken at this column (if `on` and the column holds an observer),
// and zero it on the radial edges.
template <typename T, int K>
__device__ __forceinline__ void load_lam(const T *__restrict__ lam, int i, int Nr, int lane,
                                         const InjectArgs &inj, int on, long long sample, T (&l)[4][K])
{
    constexpr int NP = 32 * K;
    load_col<T, K>(lam + (size_t)i * 4 * NP + lane * K, l);
    if (on) {
        for (int k = 0; k < inj.obs.n; ++k) {
            const int slot = (i == inj.obs.i0[k]) ? 0 : ((i == inj.obs.i0[k] + 1) ? 1 : -1);
            if (slot < 0) continue;
            const int j0 = inj.obs.j0[k];
            const double wr = slot ? inj.obs.wr1[k] : inj.obs.wr0[k];
            const double *g = inj.dwave + ((size_t)k * inj.count + sample) * 2;
            const double gr = g[0], gi = g[1];
#pragma unroll
            for (int t = 0; t < K; ++t) {
                const int r = lane * K + t;
                double wt = 0.0;
                if (r == j0) wt = wr * (1.0 - inj.obs.ft[k]) * inj.w_row[j0];
                else if (r == j0 + 1) wt = wr * inj.obs.ft[k] * inj.w_row[j0 + 1];
                if (wt != 0.0) {
                    l[0][t] += (T)(wt * gr);
                    l[1][t] += (T)(wt * gi);
                }
            }
        }
    }
    if (i == 0 || i == Nr - 1) zero_col<T, K>(l);
}

// Transposed theta coupling: with the forward coupling sending KP_j x_j to
// row j+1 and KM_j x_j to row j-1, row j receives
//   KP_{j-1} x_{j-1} + KM_{j+1} x_{j+1}
// for both components xr, xi.  The coefficients and the values are shuffled
// separately, which costs two FP64 operations per component.  Row 0 has no
// row -1 and the last padded row no row below: the shuffles return the lane's
// own values there, so those coefficients are masked to zero.
template <typename T, int K>
__device__ __forceinline__ void neighbour_in(const T (&kp)[K], const T (&km)[K], const T (&xr)[K],
                                             const T (&xi)[K], T (&outr)[K], T (&outi)[K])
{
    const FmaK<T> k1 = fma_k<T>();
    const int lane = threadIdx.x & 31;
    const T kp_prv = __shfl_up_sync(kFull, kp[K - 1], 1);
    const T km_nxt = __shfl_down_sync(kFull, km[0], 1);
    T xru[K], xrd[K], xiu[K], xid[K];
    theta_neighbours<T, K>(xr, xru, xrd);
    theta_neighbours<T, K>(xi, xiu, xid);
#pragma unroll
    for (int t = 0; t < K; ++t) {
        T kpd = (t > 0) ? kp[t - 1] : kp_prv;
        T kmu = (t + 1 < K) ? km[t + 1] : km_nxt;
        if (t == 0 && lane == 0) kpd = T(0);
        if (t == K - 1 && lane == 31) kmu = T(0);
        outr[t] = fma(kpd, xrd[t], fma(kmu, xru[t], k1.nz));
        outi[t] = fma(kpd, xid[t], fma(kmu, xiu[t], k1.nz));
    }
}

// Node n's theta-neighbour sources Z_n = (KP_n lamPi_n)(j-1) + (KM_n lamPi_n)(j+1).
template <typename T, int K>
__device__ __forceinline__ void node_z(const T *__restrict__ ntab, const T (&l)[4][K],
                                       T (&zr)[K], T (&zi)[K])
{
    constexpr int NP = 32 * K;
    T kp[K], km[K];
    ldk<T, K>(ntab + N_KP * NP, kp);
    ldk<T, K>(ntab + N_KM * NP, km);
    neighbour_in<T, K>(kp, km, l[2], l[3], zr, zi);
}

// eta at the half node between nodes a (left) and c (right).
template <typename T, int K>
__device__ __forceinline__ void eta_half(const T (&la)[4][K], const T (&lc)[4][K],
                                         const T (&zar)[K], const T (&zai)[K], const T (&zcr)[K],
                                         const T (&zci)[K], const T *__restrict__ ta,
                                         const T *__restrict__ tc, const T E, T (&h)[4][K])
{
    const FmaK<T> k1 = fma_k<T>();
    constexpr int NP = 32 * K;
    T B[K], FR[K], FI[K], PR[K], CI[K];
    // left node: the half node is its h+ (coefficients -B, FP, PPR, C2I)
    ldk<T, K>(ta + N_B * NP, B);
    ldk<T, K>(ta + N_FPR * NP, FR);
    ldk<T, K>(ta + N_FPI * NP, FI);
    ldk<T, K>(ta + N_PPR * NP, PR);
    ldk<T, K>(ta + N_C2I * NP, CI);
#pragma unroll
    for (int t = 0; t < K; ++t) {
        h[0][t] = fma(FI[t], la[3][t], fma(FR[t], la[2][t], fma(-B[t], la[0][t], fma(zar[t], k1.one, zcr[t]))));
        h[1][t] = fma(FR[t], la[3][t], fma(-FI[t], la[2][t], fma(-B[t], la[1][t], fma(zai[t], k1.one, zci[t]))));
        h[2][t] = fma(CI[t], la[3][t], fma(PR[t], la[2][t], fma(E, la[0][t], k1.nz)));
        h[3][t] = fma(PR[t], la[3][t], fma(-CI[t], la[2][t], fma(E, la[1][t], k1.nz)));
    }
    // right node: the half node is its h- (coefficients +B, FM, PMR, C2I)
    ldk<T, K>(tc + N_B * NP, B);
    ldk<T, K>(tc + N_FMR * NP, FR);
    ldk<T, K>(tc + N_FMI * NP, FI);
    ldk<T, K>(tc + N_PMR * NP, PR);
    ldk<T, K>(tc + N_C2I * NP, CI);
#pragma unroll
    for (int t = 0; t < K; ++t) {
        h[0][t] = fma(FI[t], lc[3][t], fma(FR[t], lc[2][t], fma(B[t], lc[0][t], h[0][t])));
        h[1][t] = fma(FR[t], lc[3][t], fma(-FI[t], lc[2][t], fma(B[t], lc[1][t], h[1][t])));
        h[2][t] = fma(CI[t], lc[3][t], fma(PR[t], lc[2][t], fma(E, lc[0][t], h[2][t])));
        h[3][t] = fma(PR[t], lc[3][t], fma(-CI[t], lc[2][t], fma(E, lc[1][t], h[3][t])));
    }
}

// Half node's theta-neighbour sources Y_h = (KP_h etaPi)(j-1) + (KM_h etaPi)(j+1).
template <typename T, int K>
__device__ __forceinline__ void half_y(const T *__restrict__ htab, const T (&h)[4][K],
                                       T (&yr)[K], T (&yi)[K])
{
    constexpr int NP = 32 * K;
    T kp[K], km[K];
    ldk<T, K>(htab + H_KP * NP, kp);
    ldk<T, K>(htab + H_KM * NP, km);
    neighbour_in<T, K>(kp, km, h[2], h[3], yr, yi);
}

// mu at node i from lam~_i, eta+ (half node i+1/2: u_i is its "a") and eta-
// (half node i-1/2: u_i is its "c").
template <typename T, int K>
__device__ __forceinline__ void mu_node(const T (&l)[4][K], const T (&ep)[4][K],
                                        const T (&em)[4][K], const T (&ypr)[K], const T (&ypi)[K],
                                        const T (&ymr)[K], const T (&ymi)[K],
                                        const T *__restrict__ hp_tab, const T *__restrict__ hm_tab,
                                        T (&mu)[4][K])
{
    const FmaK<T> k1 = fma_k<T>();
    constexpr int NP = 32 * K;
    T S[K], FR[K], FI[K], PR[K], PI[K];
    // eta+ with the "a" entries of half node i+1/2
    ldk<T, K>(hp_tab + H_HP * NP, S);
    ldk<T, K>(hp_tab + H_FAR * NP, FR);
    ldk<T, K>(hp_tab + H_FAI * NP, FI);
    ldk<T, K>(hp_tab + H_PAR * NP, PR);
    ldk<T, K>(hp_tab + H_PI * NP, PI);
#pragma unroll
    for (int t = 0; t < K; ++t) {
        mu[0][t] = fma(FI[t], ep[3][t], fma(FR[t], ep[2][t], fma(S[t], ep[0][t],
                       fma(l[0][t], k1.one, fma(ypr[t], k1.one, ymr[t])))));
        mu[1][t] = fma(FR[t], ep[3][t], fma(-FI[t], ep[2][t], fma(S[t], ep[1][t],
                       fma(l[1][t], k1.one, fma(ypi[t], k1.one, ymi[t])))));
        mu[2][t] = fma(PI[t], ep[3][t], fma(PR[t], ep[2][t], fma(ep[0][t], k1.one, l[2][t])));
        mu[3][t] = fma(PR[t], ep[3][t], fma(-PI[t], ep[2][t], fma(ep[1][t], k1.one, l[3][t])));
    }
    // eta- with the "c" entries of half node i-1/2
    ldk<T, K>(hm_tab + H_HQ * NP, S);
    ldk<T, K>(hm_tab + H_FCR * NP, FR);
    ldk<T, K>(hm_tab + H_FCI * NP, FI);
    ldk<T, K>(hm_tab + H_PCR * NP, PR);
    ldk<T, K>(hm_tab + H_PI * NP, PI);
#pragma unroll
    for (int t = 0; t < K; ++t) {
        mu[0][t] = fma(FI[t], em[3][t], fma(FR[t], em[2][t], fma(S[t], em[0][t], mu[0][t])));
        mu[1][t] = fma(FR[t], em[3][t], fma(-FI[t], em[2][t], fma(S[t], em[1][t], mu[1][t])));
        mu[2][t] = fma(PI[t], em[3][t], fma(PR[t], em[2][t], fma(em[0][t], k1.one, mu[2][t])));
        mu[3][t] = fma(PR[t], em[3][t], fma(-PI[t], em[2][t], fma(em[1][t], k1.one, mu[3][t])));
    }
}

// Warps per block of the wide launch (one block per SM): the most warps, in
// multiples of four, whose registers fit in the register file at the count
// the kernel compiles to for this element type and K.
template <typename T, int K>
constexpr int adj_wide_warps()
{
    return sizeof(T) == 8 ? (K == 1 ? 24 : K == 2 ? 16 : 8) : (K == 1 ? 32 : K == 2 ? 24 : 12);
}

// Shared memory per warp, in theta-columns of NP values: [0, 6) eta at the
// warp's last half node with its neighbour sources (read by the right
// neighbour), [6, 16) lam~, eta+ and its sources at the warp's first column
// (its deferred node).
constexpr int kAdjShared = 16;

template <typename T, int K, int W>
__global__ void __launch_bounds__(W * 32, adj_wide_warps<T, K>() / W)
lw_adjoint_kernel(const T *__restrict__ lam, T *__restrict__ mu_out, const T *__restrict__ half,
                  const T *__restrict__ node, int Nr, T eh, T en, const InjectArgs inj)
{
    constexpr int NP = 32 * K;
    constexpr size_t SP = 4 * NP, HP = (size_t)kNCH * NP, NQ = (size_t)kNCN * NP;
    extern __shared__ __align__(16) unsigned char sh_raw[];
    T(*sh)[kAdjShared][NP] = reinterpret_cast<T(*)[kAdjShared][NP]>(sh_raw);
    chain_start();   // lam is the previous launch's output
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int i0, i1, left;
    warp_range<W>(Nr, wib, &i0, &i1, &left);
    const int row = lane * K;
    const bool lead = (left < 0);

    T la[4][K], zar[K], zai[K];        // node i: lam~ and its neighbour sources
    T em[4][K], ymr[K], ymi[K];        // half node i-1/2: eta and its neighbour sources
    zero_col<T, K>(em);
#pragma unroll
    for (int t = 0; t < K; ++t) ymr[t] = ymi[t] = T(0);
    if (i1 > i0) {
        load_lam<T, K>(lam, i0, Nr, lane, inj, inj.on, inj.sample, la);
        node_z<T, K>(node + (size_t)i0 * NQ + row, la, zar, zai);
        if (lead && i0 > 0) {
            T ll[4][K], zlr[K], zli[K];
            load_lam<T, K>(lam, i0 - 1, Nr, lane, inj, inj.on, inj.sample, ll);
            node_z<T, K>(node + (size_t)(i0 - 1) * NQ + row, ll, zlr, zli);
            eta_half<T, K>(ll, la, zlr, zli, zar, zai, node + (size_t)(i0 - 1) * NQ + row,
                           node + (size_t)i0 * NQ + row, en, em);
            half_y<T, K>(half + (size_t)(i0 - 1) * HP + row, em, ymr, ymi);
        }
        for (int i = i0; i < i1; ++i) {
            T lc[4][K], zcr[K], zci[K], ep[4][K], ypr[K], ypi[K];
            if (i + 1 < Nr) {
                load_lam<T, K>(lam, i + 1, Nr, lane, inj, inj.on, inj.sample, lc);
                node_z<T, K>(node + (size_t)(i + 1) * NQ + row, lc, zcr, zci);
                eta_half<T, K>(la, lc, zar, zai, zcr, zci, node + (size_t)i * NQ + row,
                               node + (size_t)(i + 1) * NQ + row, en, ep);
                half_y<T, K>(half + (size_t)i * HP + row, ep, ypr, ypi);
            } else {
                zero_col<T, K>(lc);
                zero_col<T, K>(ep);
#pragma unroll
                for (int t = 0; t < K; ++t) zcr[t] = zci[t] = ypr[t] = ypi[t] = T(0);
            }
            if (i == i0 && !lead) {
#pragma unroll
                for (int t = 0; t < K; ++t) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        sh[wib][6 + c][row + t] = la[c][t];
                        sh[wib][10 + c][row + t] = ep[c][t];
                    }
                    sh[wib][14][row + t] = ypr[t];
                    sh[wib][15][row + t] = ypi[t];
                }
            } else {
                T mu[4][K];
                const T *hm_tab = half + (size_t)(i > 0 ? i - 1 : 0) * HP + row;
                mu_node<T, K>(la, ep, em, ypr, ypi, ymr, ymi, half + (size_t)i * HP + row, hm_tab, mu);
                store_col<T, K>(mu_out + (size_t)i * SP + row, mu);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int t = 0; t < K; ++t) {
                    la[c][t] = lc[c][t];
                    em[c][t] = ep[c][t];
                }
#pragma unroll
            for (int t = 0; t < K; ++t) {
                zar[t] = zcr[t];
                zai[t] = zci[t];
                ymr[t] = ypr[t];
                ymi[t] = ypi[t];
            }
        }
    }
    // em, ymr, ymi now belong to the half node i1 - 1/2: the right neighbour's left edge
#pragma unroll
    for (int t = 0; t < K; ++t) {
#pragma unroll
        for (int c = 0; c < 4; ++c) sh[wib][c][row + t] = em[c][t];
        sh[wib][4][row + t] = ymr[t];
        sh[wib][5][row + t] = ymi[t];
    }
    __syncthreads();
    if (!lead && i1 > i0) {
        T l0[4][K], ep[4][K], el[4][K], ypr[K], ypi[K], yml[K], ymli[K], mu[4][K];
#pragma unroll
        for (int t = 0; t < K; ++t) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                el[c][t] = sh[left][c][row + t];
                l0[c][t] = sh[wib][6 + c][row + t];
                ep[c][t] = sh[wib][10 + c][row + t];
            }
            yml[t] = sh[left][4][row + t];
            ymli[t] = sh[left][5][row + t];
            ypr[t] = sh[wib][14][row + t];
            ypi[t] = sh[wib][15][row + t];
        }
        mu_node<T, K>(l0, ep, el, ypr, ypi, yml, ymli, half + (size_t)i0 * HP + row,
                      half + (size_t)(i0 - 1) * HP + row, mu);
        store_col<T, K>(mu_out + (size_t)i0 * SP + row, mu);
    }
}

// Every adjoint step of a tk_adjoint call in one cooperative launch, with the
// dataflow of the forward persistent sweep (step_sweep_async): no barrier
// between steps; each warp waits (bounded) only for its two siblings and, at
// a block's edges, the neighbouring block's edge warp.  Step s:
//   - first phase (every half node and node that involves only the block's
//     columns): it reads the right sibling's first column and overwrites its
//     own last half node, which that sibling read in the last step, so it
//     waits until that sibling has finished step s - 1;
//   - the block's last warp waits until the right neighbouring block's first
//     warp has finished step s - 1, then forms its last column;
//   - the deferred first node: the block's first warp waits until the left
//     neighbouring block's last warp has finished step s - 1 and forms its
//     left half node from that warp's column; every other warp takes its left
//     sibling's last half node once that sibling's first phase is done.
// Same arithmetic on the same operands as lw_adjoint_kernel.
template <typename T, int K, int W>
__device__ __forceinline__ void adj_sweep_async(unsigned char *sh_raw, const T *__restrict__ lam,
                                                T *__restrict__ mu_out, const T *__restrict__ half,
                                                const T *__restrict__ node, int Nr, T en, const InjectArgs &inj,
                                                int on, long long sample, unsigned int *flags,
                                                unsigned int *first_done, unsigned int *step_done, unsigned int s,
                                                int *err)
{
    constexpr int NP = 32 * K;
    constexpr size_t SP = 4 * NP, HP = (size_t)kNCH * NP, NQ = (size_t)kNCN * NP;
    T(*sh)[kAdjShared][NP] = reinterpret_cast<T(*)[kAdjShared][NP]>(sh_raw);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int i0, i1, left;
    warp_range<W>(Nr, wib, &i0, &i1, &left);
    // at most Nr / W blocks: every warp has a column (as in step_sweep_async)
    if (i1 <= i0) return;
    const int row = lane * K;
    const bool lead = (left < 0);
    const int b1 = (int)(((long long)(blockIdx.x + 1) * Nr) / gridDim.x);
    const bool last = (i1 == b1);
    const int iend = last ? i1 - 1 : i1;
    const unsigned int nb = gridDim.x;
    if (s > 0 && !last) warp_wait_cta(&step_done[wib + 1], s, err);

    T la[4][K], zar[K], zai[K];        // node i: lam~ and its neighbour sources
    T em[4][K], ymr[K], ymi[K];        // half node i-1/2: eta and its neighbour sources
    zero_col<T, K>(em);
#pragma unroll
    for (int t = 0; t < K; ++t) ymr[t] = ymi[t] = T(0);
    load_lam<T, K>(lam, i0, Nr, lane, inj, on, sample, la);
    node_z<T, K>(node + (size_t)i0 * NQ + row, la, zar, zai);
    // the right half node of column i (from column i + 1) and, for i > i0, its node
    auto column = [&](int i) {
        T lc[4][K], zcr[K], zci[K], ep[4][K], ypr[K], ypi[K];
        if (i + 1 < Nr) {
            load_lam<T, K>(lam, i + 1, Nr, lane, inj, on, sample, lc);
            node_z<T, K>(node + (size_t)(i + 1) * NQ + row, lc, zcr, zci);
            eta_half<T, K>(la, lc, zar, zai, zcr, zci, node + (size_t)i * NQ + row,
                           node + (size_t)(i + 1) * NQ + row, en, ep);
            half_y<T, K>(half + (size_t)i * HP + row, ep, ypr, ypi);
        } else {
            zero_col<T, K>(lc);
            zero_col<T, K>(ep);
#pragma unroll
            for (int t = 0; t < K; ++t) zcr[t] = zci[t] = ypr[t] = ypi[t] = T(0);
        }
        if (i == i0) {
#pragma unroll
            for (int t = 0; t < K; ++t) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    sh[wib][6 + c][row + t] = la[c][t];
                    sh[wib][10 + c][row + t] = ep[c][t];
                }
                sh[wib][14][row + t] = ypr[t];
                sh[wib][15][row + t] = ypi[t];
            }
        } else {
            T mu[4][K];
            mu_node<T, K>(la, ep, em, ypr, ypi, ymr, ymi, half + (size_t)i * HP + row,
                          half + (size_t)(i - 1) * HP + row, mu);
            store_col<T, K>(mu_out + (size_t)i * SP + row, mu);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int t = 0; t < K; ++t) {
                la[c][t] = lc[c][t];
                em[c][t] = ep[c][t];
            }
#pragma unroll
        for (int t = 0; t < K; ++t) {
            zar[t] = zcr[t];
            zai[t] = zci[t];
            ymr[t] = ypr[t];
            ymi[t] = ypi[t];
        }
    };
    for (int i = i0; i < iend; ++i) column(i);
    if (!last)   // eta at i1 - 1/2 with its sources: the right sibling's left edge
#pragma unroll
        for (int t = 0; t < K; ++t) {
#pragma unroll
            for (int c = 0; c < 4; ++c) sh[wib][c][row + t] = em[c][t];
            sh[wib][4][row + t] = ymr[t];
            sh[wib][5][row + t] = ymi[t];
        }
    warp_publish_cta(&first_done[wib], s + 1);
    if (last) {
        if (s > 0 && blockIdx.x + 1 < nb) warp_wait_flag(flags + blockIdx.x + 1, s, err);
        column(i1 - 1);
        __syncwarp();
    }
    {   // the deferred first node
        T l0[4][K], ep[4][K], el[4][K], ypr[K], ypi[K], yml[K], ymli[K], mu[4][K];
#pragma unroll
        for (int t = 0; t < K; ++t) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                l0[c][t] = sh[wib][6 + c][row + t];
                ep[c][t] = sh[wib][10 + c][row + t];
            }
            ypr[t] = sh[wib][14][row + t];
            ypi[t] = sh[wib][15][row + t];
        }
        if (lead) {
            if (s > 0 && blockIdx.x > 0) warp_wait_flag(flags + nb + blockIdx.x - 1, s, err);
            if (i0 > 0) {
                T ll[4][K], zlr[K], zli[K], z0r[K], z0i[K];
                load_lam<T, K>(lam, i0 - 1, Nr, lane, inj, on, sample, ll);
                node_z<T, K>(node + (size_t)(i0 - 1) * NQ + row, ll, zlr, zli);
                node_z<T, K>(node + (size_t)i0 * NQ + row, l0, z0r, z0i);
                eta_half<T, K>(ll, l0, zlr, zli, z0r, z0i, node + (size_t)(i0 - 1) * NQ + row,
                               node + (size_t)i0 * NQ + row, en, el);
                half_y<T, K>(half + (size_t)(i0 - 1) * HP + row, el, yml, ymli);
            } else {
                zero_col<T, K>(el);
#pragma unroll
                for (int t = 0; t < K; ++t) yml[t] = ymli[t] = T(0);
            }
        } else {
            warp_wait_cta(&first_done[left], s + 1, err);
#pragma unroll
            for (int t = 0; t < K; ++t) {
#pragma unroll
                for (int c = 0; c < 4; ++c) el[c][t] = sh[left][c][row + t];
                yml[t] = sh[left][4][row + t];
                ymli[t] = sh[left][5][row + t];
            }
        }
        mu_node<T, K>(l0, ep, el, ypr, ypi, yml, ymli, half + (size_t)i0 * HP + row,
                      half + (size_t)(i0 > 0 ? i0 - 1 : 0) * HP + row, mu);
        store_col<T, K>(mu_out + (size_t)i0 * SP + row, mu);
    }
    if (lead) warp_publish_gpu(flags + blockIdx.x, s + 1);
    if (last) warp_publish_gpu(flags + nb + blockIdx.x, s + 1);
    warp_publish_cta(&step_done[wib], s + 1);
}

// Launch step s is the transpose of inner step n_inner - 1 - s: the gradient
// of sample count - 1 - s / substeps is injected at its first sub-step.  The
// adjoint state starts in a0; the result is in a0 or a1 by the parity of
// n_inner.
template <typename T, int K, int W>
__global__ void __launch_bounds__(W * 32, adj_wide_warps<T, K>() / W)
lw_adjoint_persistent_kernel(T *a0, T *a1, const T *__restrict__ half, const T *__restrict__ node, int Nr,
                             T en, const InjectArgs inj, int inject, long long n_inner, int substeps,
                             unsigned int *flags, int *err)
{
    extern __shared__ __align__(16) unsigned char sh_raw[];
    __shared__ unsigned int first_done[W], step_done[W];
    if (threadIdx.x < W) {
        first_done[threadIdx.x] = 0;
        step_done[threadIdx.x] = 0;
    }
    __syncthreads();
    for (long long s = 0; s < n_inner; ++s) {
        const T *lam = (s & 1) ? a1 : a0;
        T *mu = (s & 1) ? a0 : a1;
        adj_sweep_async<T, K, W>(sh_raw, lam, mu, half, node, Nr, en, inj, inject && (s % substeps == 0),
                                 inj.count - 1 - s / substeps, flags, first_done, step_done, (unsigned)s, err);
    }
}

// Transpose of the initial-data map of tk_set_initial_data: the adjoint state
// lam0 = dL/du^0 (device layout) to dL/d(input planes) in [Ntheta][Nr].
// independent_pi: the momentum planes were given (4 output planes); else
// Pi_m = b_m (Phi_{m+1} - Phi_{m-1}) / (2 dr*) at interior m (2 output planes).
template <typename T>
__global__ void initial_transpose_kernel(int Nr, int Nth, int NP, double drs,
                                         const T *__restrict__ lam0, const double *__restrict__ b_node,
                                         int independent_pi, double *__restrict__ out)
{
    const int jp = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (jp >= Nth || i >= Nr) return;
    const size_t plane = (size_t)Nth * Nr, k = (size_t)jp * Nr + i;
    auto L = [&](int ii, int c) { return (double)lam0[((size_t)ii * 4 + c) * NP + jp]; };
    double g[4] = {0.0, 0.0, 0.0, 0.0};
    if (i > 0 && i < Nr - 1) {
        for (int c = 0; c < 4; ++c) g[c] = L(i, c);
        if (!independent_pi) {
            for (int c = 0; c < 2; ++c) {
                if (i - 1 >= 1) g[c] += b_node[(size_t)(i - 1) * NP + jp] * L(i - 1, 2 + c) / (2.0 * drs);
                if (i + 1 <= Nr - 2) g[c] -= b_node[(size_t)(i + 1) * NP + jp] * L(i + 1, 2 + c) / (2.0 * drs);
            }
        }
    }
    const int nout = independent_pi ? 4 : 2;
    for (int c = 0; c < nout; ++c) out[c * plane + k] = g[c];
}

// ---- gradients with respect to the black-hole parameters (a or M) ----
//
// With the tables T(p) of one inner step u^{j+1} = A(p) u^j, the loss
// gradient is dL/dp = sum_j lam~^{j+1} . (dA/dp) u^j (+ the initial-data
// term below), lam~^{j+1} the adjoint state the adjoint kernel loads (with
// the waveform gradient of the step added and the radial edges zeroed).  By
// the product rule through the half nodes h = H u,
//   (dA/dp) u at node i = N'(h_{i-1/2}, h_{i+1/2}) + N(h'_{i-1/2}, h'_{i+1/2}),
// where N' is the node update with the derivative tables and no constant
// terms, h' = H' u the half nodes with the derivative tables, and N applies
// the ordinary node tables to h'.  One warp per column range, recomputing
// its left edge; every block adds its partial sum to its own slot of acc, so
// the sum is in a fixed order.
template <int K>
__global__ void __launch_bounds__(128)
param_tangent_kernel(const double *__restrict__ u, const double *__restrict__ lam,
                     const double *__restrict__ half, const double *__restrict__ node,
                     const double *__restrict__ dhalf, const double *__restrict__ dnode, int Nr,
                     double eh, double en, const InjectArgs inj, double *__restrict__ acc)
{
    constexpr int NP = 32 * K;
    constexpr size_t SP = 4 * NP, HP = (size_t)kNCH * NP, NQ = (size_t)kNCN * NP;
    __shared__ double part[4];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    int i0, i1, left;
    warp_range<4>(Nr, wib, &i0, &i1, &left);
    const int row = lane * K;
    double sum = 0.0;
    if (i1 > i0) {
        double ua[4][K], hm[4][K], dm[4][K], zero[4][K];
        zero_col<double, K>(zero);
        load_col<double, K>(u + (size_t)i0 * SP + row, ua);
        if (i0 > 0) {
            double ul[4][K];
            load_col<double, K>(u + (size_t)(i0 - 1) * SP + row, ul);
            half_node<double, K>(ul, ua, half + (size_t)(i0 - 1) * HP + row, hm);
            half_node<double, K, false>(ul, ua, dhalf + (size_t)(i0 - 1) * HP + row, dm);
        } else {
            zero_col<double, K>(hm);
            zero_col<double, K>(dm);
        }
        for (int i = i0; i < i1; ++i) {
            double uc[4][K], hp[4][K], dp[4][K];
            if (i + 1 < Nr) {
                load_col<double, K>(u + (size_t)(i + 1) * SP + row, uc);
                half_node<double, K>(ua, uc, half + (size_t)i * HP + row, hp);
                half_node<double, K, false>(ua, uc, dhalf + (size_t)i * HP + row, dp);
            } else {
                zero_col<double, K>(uc);
                zero_col<double, K>(hp);
                zero_col<double, K>(dp);
            }
            if (i >= 1 && i <= Nr - 2) {
                double d1[4][K], d2[4][K], l[4][K];
                full_node<double, K>(hm, hp, zero, dnode + (size_t)i * NQ + row, 0.0, d1);
                full_node<double, K>(dm, dp, zero, node + (size_t)i * NQ + row, en, d2);
                load_lam<double, K>(lam, i, Nr, lane, inj, inj.on, inj.sample, l);
#pragma unroll
                for (int c = 0; c < 4; ++c)
#pragma unroll
                    for (int t = 0; t < K; ++t) sum = fma(l[c][t], d1[c][t] + d2[c][t], sum);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int t = 0; t < K; ++t) {
                    ua[c][t] = uc[c][t];
                    hm[c][t] = hp[c][t];
                    dm[c][t] = dp[c][t];
                }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
    if (lane == 0) part[wib] = sum;
    __syncthreads();
    if (threadIdx.x == 0) acc[blockIdx.x] += (part[0] + part[1]) + (part[2] + part[3]);
}

// Initial-data term for a momentum derived from Phi^0: Pi^0 = b d_* Phi^0
// depends on the parameter through b, d Pi^0 / dp = (db/dp / b) Pi^0.
// lam0 = dL/du^0.  Partial sums per block into part[blockIdx] (fixed order).
__global__ void param_initial_kernel(int Nr, int Nth, int NP, const double *__restrict__ u0,
                                     const double *__restrict__ lam0, const double *__restrict__ b_node,
                                     const double *__restrict__ db_node, double *__restrict__ part)
{
    __shared__ double ws[8];
    double sum = 0.0;
    const long long n = (long long)Nr * NP;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(k / NP), jp = (int)(k - (long long)i * NP);
        if (jp >= Nth || i == 0 || i == Nr - 1) continue;
        const double f = db_node[k] / b_node[k];
        const size_t col = (size_t)i * 4 * NP + jp;
        sum = fma(lam0[col + 2 * NP], f * u0[col + 2 * NP], sum);
        sum = fma(lam0[col + 3 * NP], f * u0[col + 3 * NP], sum);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
    if (lane == 0) ws[w] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += ws[k];
        part[blockIdx.x] = t;
    }
}

// dst += w * src over n doubles.
__global__ void axpy_kernel(size_t n, double w, const double *__restrict__ src, double *__restrict__ dst)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        dst[k] = fma(w, src[k], dst[k]);
}

cudaError_t launch_axpy(size_t n, double w, const double *src, double *dst, cudaStream_t st)
{
    size_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    axpy_kernel<<<(unsigned)blocks, 256, 0, st>>>(n, w, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_param_tangent(int K, int blocks, const double *u, const double *lam,
                                 const double *half, const double *node, const double *dhalf,
                                 const double *dnode, int Nr, double dt_in, const InjectArgs &inj,
                                 double *acc, cudaStream_t st)
{
    const double eh = 0.25 * dt_in, en = 0.5 * dt_in;
    if (K == 1)
        param_tangent_kernel<1><<<blocks, 128, 0, st>>>(u, lam, half, node, dhalf, dnode, Nr, eh, en, inj, acc);
    else if (K == 2)
        param_tangent_kernel<2><<<blocks, 128, 0, st>>>(u, lam, half, node, dhalf, dnode, Nr, eh, en, inj, acc);
    else
        param_tangent_kernel<4><<<blocks, 128, 0, st>>>(u, lam, half, node, dhalf, dnode, Nr, eh, en, inj, acc);
    return cudaGetLastError();
}

template <typename T, int K, int W>
constexpr size_t adj_smem_bytes()
{
    return (size_t)W * kAdjShared * 32 * K * sizeof(T);
}

template <typename T, int K, int W>
cudaError_t adj_smem_setup()
{
    static cudaError_t e = cudaFuncSetAttribute(lw_adjoint_kernel<T, K, W>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)adj_smem_bytes<T, K, W>());
    return e;
}

template <typename T, int K, int W>
cudaError_t launch_adj_shape(const void *lam, void *mu, const void *half, const void *node,
                             int Nr, int blocks, double dt_in, const InjectArgs &inj,
                             cudaStream_t st)
{
    cudaError_t e = adj_smem_setup<T, K, W>();
    if (e != cudaSuccess) return e;
    return launch_chained(lw_adjoint_kernel<T, K, W>, (unsigned)blocks, W * 32, adj_smem_bytes<T, K, W>(),
                          st, (const T *)lam, (T *)mu, (const T *)half, (const T *)node, Nr,
                          (T)(0.25 * dt_in), (T)(0.5 * dt_in), inj);
}

template <typename T, int K>
cudaError_t launch_adj(const void *lam, void *mu, const void *half, const void *node, int Nr,
                       int blocks, int warps, double dt_in, const InjectArgs &inj, cudaStream_t st)
{
    constexpr int WW = adj_wide_warps<T, K>();
    if (warps == WW)
        return launch_adj_shape<T, K, WW>(lam, mu, half, node, Nr, blocks, dt_in, inj, st);
    if (warps == kNarrowWarps)
        return launch_adj_shape<T, K, kNarrowWarps>(lam, mu, half, node, Nr, blocks, dt_in, inj, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_adjoint_step(int precision, int K, const void *lam, void *mu, const void *half,
                                const void *node, int Nr, int blocks, int warps, double dt_in,
                                const InjectArgs &inj, cudaStream_t st)
{
    if (precision == 0) {
        if (K == 1) return launch_adj<double, 1>(lam, mu, half, node, Nr, blocks, warps, dt_in, inj, st);
        if (K == 2) return launch_adj<double, 2>(lam, mu, half, node, Nr, blocks, warps, dt_in, inj, st);
        return launch_adj<double, 4>(lam, mu, half, node, Nr, blocks, warps, dt_in, inj, st);
    }
    if (K == 1) return launch_adj<float, 1>(lam, mu, half, node, Nr, blocks, warps, dt_in, inj, st);
    if (K == 2) return launch_adj<float, 2>(lam, mu, half, node, Nr, blocks, warps, dt_in, inj, st);
    return launch_adj<float, 4>(lam, mu, half, node, Nr, blocks, warps, dt_in, inj, st);
}

template <typename T, int K, int W>
int adj_persistent_blocks_w(int Nr, int num_sms)
{
    static cudaError_t e0 = cudaFuncSetAttribute(lw_adjoint_persistent_kernel<T, K, W>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)adj_smem_bytes<T, K, W>());
    int n = 0;
    if (e0 != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, lw_adjoint_persistent_kernel<T, K, W>, W * 32,
                                                      adj_smem_bytes<T, K, W>()) != cudaSuccess ||
        n < 1)
        return 0;
    long long blocks = (long long)num_sms * n;
    if (blocks > Nr / W) blocks = Nr / W;
    return blocks < 1 ? 0 : (int)blocks;
}

template <typename T, int K>
int adj_persistent_blocks_t(int Nr, int num_sms, int warps)
{
    constexpr int WW = adj_wide_warps<T, K>();
    if (warps == WW) return adj_persistent_blocks_w<T, K, WW>(Nr, num_sms);
    if (warps == kNarrowWarps) return adj_persistent_blocks_w<T, K, kNarrowWarps>(Nr, num_sms);
    return 0;
}

template <typename T, int K, int W>
cudaError_t launch_adj_persistent_w(void *a0, void *a1, const void *half, const void *node, int Nr, int blocks,
                                    double dt_in, const InjectArgs &inj, int inject, long long n_inner,
                                    int substeps, unsigned int *flags, int *err, cudaStream_t st)
{
    T *p0 = (T *)a0, *p1 = (T *)a1;
    const T *h = (const T *)half, *nd = (const T *)node;
    T en = (T)(0.5 * dt_in);
    InjectArgs in = inj;
    void *args[] = {&p0, &p1, &h, &nd, &Nr, &en, &in, &inject, &n_inner, &substeps, &flags, &err};
    return cudaLaunchCooperativeKernel((const void *)lw_adjoint_persistent_kernel<T, K, W>, dim3(blocks),
                                       dim3(W * 32), args, adj_smem_bytes<T, K, W>(), st);
}

template <typename T, int K>
cudaError_t launch_adj_persistent_t(void *a0, void *a1, const void *half, const void *node, int Nr, int blocks,
                                    int warps, double dt_in, const InjectArgs &inj, int inject,
                                    long long n_inner, int substeps, unsigned int *flags, int *err,
                                    cudaStream_t st)
{
    constexpr int WW = adj_wide_warps<T, K>();
    if (warps == WW)
        return launch_adj_persistent_w<T, K, WW>(a0, a1, half, node, Nr, blocks, dt_in, inj, inject, n_inner,
                                                 substeps, flags, err, st);
    if (warps == kNarrowWarps)
        return launch_adj_persistent_w<T, K, kNarrowWarps>(a0, a1, half, node, Nr, blocks, dt_in, inj, inject,
                                                           n_inner, substeps, flags, err, st);
    return cudaErrorInvalidValue;
}

// Blocks of the persistent adjoint launch for this grid (all resident at
// once, at most Nr / warps), or 0 if it cannot run.
int adjoint_persistent_blocks(int precision, int K, int Nr, int num_sms, int warps)
{
    if (precision == 0)
        return K == 1 ? adj_persistent_blocks_t<double, 1>(Nr, num_sms, warps)
             : K == 2 ? adj_persistent_blocks_t<double, 2>(Nr, num_sms, warps)
                      : adj_persistent_blocks_t<double, 4>(Nr, num_sms, warps);
    return K == 1 ? adj_persistent_blocks_t<float, 1>(Nr, num_sms, warps)
         : K == 2 ? adj_persistent_blocks_t<float, 2>(Nr, num_sms, warps)
                  : adj_persistent_blocks_t<float, 4>(Nr, num_sms, warps);
}

cudaError_t launch_adjoint_persistent(int precision, int K, void *a0, void *a1, const void *half,
                                      const void *node, int Nr, int blocks, int warps, double dt_in,
                                      const InjectArgs &inj, int inject, long long n_inner, int substeps,
                                      unsigned int *flags, int *err, cudaStream_t st)
{
    if (precision == 0) {
        if (K == 1)
            return launch_adj_persistent_t<double, 1>(a0, a1, half, node, Nr, blocks, warps, dt_in, inj, inject,
                                                      n_inner, substeps, flags, err, st);
        if (K == 2)
            return launch_adj_persistent_t<double, 2>(a0, a1, half, node, Nr, blocks, warps, dt_in, inj, inject,
                                                      n_inner, substeps, flags, err, st);
        return launch_adj_persistent_t<double, 4>(a0, a1, half, node, Nr, blocks, warps, dt_in, inj, inject,
                                                  n_inner, substeps, flags, err, st);
    }
    if (K == 1)
        return launch_adj_persistent_t<float, 1>(a0, a1, half, node, Nr, blocks, warps, dt_in, inj, inject,
                                                 n_inner, substeps, flags, err, st);
    if (K == 2)
        return launch_adj_persistent_t<float, 2>(a0, a1, half, node, Nr, blocks, warps, dt_in, inj, inject,
                                                 n_inner, substeps, flags, err, st);
    return launch_adj_persistent_t<float, 4>(a0, a1, half, node, Nr, blocks, warps, dt_in, inj, inject,
                                             n_inner, substeps, flags, err, st);
}

template <typename T, int K, int W>
int adj_resident()
{
    int n = 0;
    if (adj_smem_setup<T, K, W>() != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, lw_adjoint_kernel<T, K, W>, W * 32,
                                                      adj_smem_bytes<T, K, W>()) != cudaSuccess)
        n = 0;
    return n;
}

template <typename T, int K>
int adj_shape(int Nr, int num_sms, int *warps)
{
    constexpr int WW = adj_wide_warps<T, K>();
    if ((long long)Nr >= (long long)num_sms * WW && adj_resident<T, K, WW>() >= 1) {
        *warps = WW;
        return num_sms;
    }
    *warps = kNarrowWarps;
    int per_sm = adj_resident<T, K, kNarrowWarps>();
    if (per_sm < 1) per_sm = 1;
    int blocks = num_sms * per_sm;
    if (blocks > Nr / kNarrowWarps) blocks = Nr / kNarrowWarps;
    return blocks < 1 ? 1 : blocks;
}

}  // namespace

int adjoint_grid_shape(int precision, int K, int Nr, int num_sms, int *warps)
{
    if (precision == 0)
        return K == 1 ? adj_shape<double, 1>(Nr, num_sms, warps)
             : K == 2 ? adj_shape<double, 2>(Nr, num_sms, warps)
                      : adj_shape<double, 4>(Nr, num_sms, warps);
    return K == 1 ? adj_shape<float, 1>(Nr, num_sms, warps)
         : K == 2 ? adj_shape<float, 2>(Nr, num_sms, warps)
                  : adj_shape<float, 4>(Nr, num_sms, warps);
}

}  // namespace tk

extern "C" tk_status tk_adjoint(tk_solver *S, const double *dL_dwave, const double *dL_dfinal,
                                int on_device, double *grad, int grad_on_device, int independent_pi)
{
    tk_status st = tkh::enter(S);
    if (st != TK_OK) return st;
    st = tkh::need_state(S, "tk_adjoint");
    if (st != TK_OK) return st;
    if (!grad) return tkh::fail(S, TK_ERR_ARG, "tk_adjoint: grad is NULL");
    if (!dL_dwave && !dL_dfinal)
        return tkh::fail(S, TK_ERR_ARG, "tk_adjoint: give dL_dwave, dL_dfinal or both");
    if (dL_dwave && S->nobs == 0) return tkh::fail(S, TK_ERR_ARG, "tk_adjoint: no observers");
    const size_t se = (size_t)S->Nr * 4 * S->NP;
    const size_t plane = (size_t)S->Nth * S->Nr;
    // adjoint levels and staging (allocated on first use, kept)
    for (int k = 0; k < 2; ++k)
        if (!S->adj[k]) {
            st = tkh::alloc(S, &S->adj[k], se * S->esz);
            if (st != TK_OK) return st;
        }
    const long long count = S->count;
    double *dwave = nullptr;
    double *dfin = nullptr;
    double *gdev = nullptr;
    auto cleanup = [&]() {
        if (dwave && !on_device) cudaFree(dwave);
        if (dfin) cudaFree(dfin);
        if (gdev && !grad_on_device) cudaFree(gdev);
    };
    if (dL_dwave) {
        if (on_device) {
            dwave = const_cast<double *>(dL_dwave);
        } else {
            st = tkh::alloc(S, (void **)&dwave, (size_t)S->nobs * count * 2 * sizeof(double));
            if (st != TK_OK) return st;
            cudaError_t e = cudaMemcpyAsync(dwave, dL_dwave, (size_t)S->nobs * count * 2 * sizeof(double),
                                            cudaMemcpyHostToDevice, S->stream);
            if (e != cudaSuccess) {
                cleanup();
                return tkh::fail(S, TK_ERR_CUDA, "tk_adjoint: %s", cudaGetErrorString(e));
            }
        }
    }
    // lam = dL/du(T): the final-state gradient (or 0)
    cudaError_t e = cudaSuccess;
    if (dL_dfinal) {
        const double *src = dL_dfinal;
        if (!on_device) {
            st = tkh::alloc(S, (void **)&dfin, 4 * plane * sizeof(double));
            if (st != TK_OK) {
                cleanup();
                return st;
            }
            e = cudaMemcpyAsync(dfin, dL_dfinal, 4 * plane * sizeof(double), cudaMemcpyHostToDevice, S->stream);
            src = dfin;
        }
        if (e == cudaSuccess)
            e = tk::launch_import_state(S->precision, S->Nr, S->Nth, S->NP, S->drs, src, src + plane,
                                        src + 2 * plane, src + 3 * plane, S->b_node, S->adj[0], S->stream);
    } else {
        e = cudaMemsetAsync(S->adj[0], 0, se * S->esz, S->stream);
    }
    tk::InjectArgs inj;
    memset(&inj, 0, sizeof inj);
    inj.count = count;
    inj.dwave = dwave;
    inj.w_row = S->w_row;
    {
        tk::StepLaunch L;
        tkh::fill_launch(S, L);
        inj.obs = L.obs;
    }
    int cur = 0;
    const double dt_in = S->dt / S->substeps;
    const long long n_inner = count * S->substeps;
    // the solver's launch structure: every step in one persistent launch, or
    // one launch per step
    const int pblocks = (S->persist && n_inner > 0)
                            ? tk::adjoint_persistent_blocks(S->precision, S->K, S->Nr, S->num_sms, S->adj_warps)
                            : 0;
    if (pblocks > 0 && e == cudaSuccess) {
        unsigned int *flags = nullptr;
        const size_t fbytes = (size_t)2 * pblocks * sizeof(unsigned int) + sizeof(int);
        st = tkh::alloc(S, (void **)&flags, fbytes);
        if (st != TK_OK) {
            cleanup();
            return st;
        }
        int *derr = (int *)(flags + 2 * pblocks);
        int herr = 0;
        e = cudaMemsetAsync(flags, 0, fbytes, S->stream);
        if (e == cudaSuccess)
            e = tk::launch_adjoint_persistent(S->precision, S->K, S->adj[0], S->adj[1], S->half, S->node, S->Nr,
                                              pblocks, S->adj_warps, dt_in, inj, dwave != nullptr, n_inner,
                                              S->substeps, flags, derr, S->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, S->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
        cudaFree(flags);
        if (e == cudaSuccess && herr) {
            cleanup();
            return tkh::fail(S, TK_ERR_INTERNAL, "tk_adjoint: a block of the persistent launch waited too "
                                                 "long for a neighbour; the gradient is invalid");
        }
        cur = (int)(n_inner & 1);
    } else {
        for (long long t = count - 1; t >= 0 && e == cudaSuccess; --t)
            for (int k = 0; k < S->substeps && e == cudaSuccess; ++k) {
                inj.on = (k == 0) && dwave != nullptr;
                inj.sample = t;
                e = tk::launch_adjoint_step(S->precision, S->K, S->adj[cur], S->adj[cur ^ 1], S->half,
                                            S->node, S->Nr, S->adj_blocks, S->adj_warps, dt_in, inj, S->stream);
                cur ^= 1;
            }
    }
    if (e != cudaSuccess) {
        cleanup();
        return tkh::fail(S, TK_ERR_CUDA, "tk_adjoint: %s", cudaGetErrorString(e));
    }
    // the initial-data map
    const int nout = independent_pi ? 4 : 2;
    if (grad_on_device) {
        gdev = grad;
    } else {
        st = tkh::alloc(S, (void **)&gdev, nout * plane * sizeof(double));
        if (st != TK_OK) {
            cleanup();
            return st;
        }
    }
    dim3 block(32, 8), gridd((S->NP + 31) / 32, (S->Nr + 7) / 8);
    if (S->precision == 0)
        tk::initial_transpose_kernel<double><<<gridd, block, 0, S->stream>>>(
            S->Nr, S->Nth, S->NP, S->drs, (const double *)S->adj[cur], S->b_node, independent_pi, gdev);
    else
        tk::initial_transpose_kernel<float><<<gridd, block, 0, S->stream>>>(
            S->Nr, S->Nth, S->NP, S->drs, (const float *)S->adj[cur], S->b_node, independent_pi, gdev);
    e = cudaGetLastError();
    if (e == cudaSuccess && !grad_on_device)
        e = cudaMemcpyAsync(grad, gdev, nout * plane * sizeof(double), cudaMemcpyDeviceToHost, S->stream);
    if (e == cudaSuccess && (!grad_on_device || !on_device)) e = cudaStreamSynchronize(S->stream);
    cleanup();
    if (e != cudaSuccess) return tkh::fail(S, TK_ERR_CUDA, "tk_adjoint: %s", cudaGetErrorString(e));
    return TK_OK;
}

// Gradient of a waveform loss with respect to the spin a (param 0) or the mass
// M (param 1), through checkpointed recomputation of the trajectory.
extern "C" tk_status tk_param_gradient(tk_solver *S, int param, const double *dL_dwave, int on_device,
                                       int checkpoint_every, double *grad)
{
    tk_status st = tkh::enter(S);
    if (st != TK_OK) return st;
    if (!grad || !dL_dwave) return tkh::fail(S, TK_ERR_ARG, "tk_param_gradient: NULL argument");
    if (param != 0 && param != 1) return tkh::fail(S, TK_ERR_ARG, "tk_param_gradient: param %d is not 0 (a) or 1 (M)", param);
    if (S->precision != TK_PREC_F64)
        return tkh::fail(S, TK_ERR_ARG, "tk_param_gradient: FP64 solvers only");
    if (!S->have_state || !S->state_valid || !S->init_valid)
        return tkh::fail(S, TK_ERR_STATE, "tk_param_gradient: needs a trajectory from tk_set_initial_data "
                                          "(not restarted with tk_set_state)");
    if (S->nobs == 0) return tkh::fail(S, TK_ERR_ARG, "tk_param_gradient: no observers");
    const long long count = S->count;
    if (count <= 0) return tkh::fail(S, TK_ERR_STATE, "tk_param_gradient: no steps taken");
    const int k = S->substeps;
    long long C = checkpoint_every;
    if (C <= 0) {
        C = (long long)sqrt((double)count / k);
        if (C < 1) C = 1;
    }
    if (C > count) C = count;
    const long long nck = (count + C - 1) / C;
    const size_t se = (size_t)S->Nr * 4 * S->NP, sb = se * sizeof(double);
    const size_t nh = (size_t)S->Nr * tk::kNCH * S->NP, nn = (size_t)S->Nr * tk::kNCN * S->NP;
    const size_t nb = (size_t)S->Nr * S->NP;

    // scratch, freed on every exit
    double *dwave = nullptr, *thalf = nullptr, *tnode = nullptr, *tb = nullptr, *tw = nullptr;
    double *tx = nullptr, *tang = nullptr, *ck = nullptr, *seg = nullptr, *acc = nullptr;
    auto cleanup = [&]() {
        void *p[] = {thalf, tnode, tb, tw, tx, tang, ck, seg, acc};
        for (void *q : p)
            if (q) cudaFree(q);
        if (dwave && !on_device) cudaFree(dwave);
    };
    auto bail = [&](tk_status s2) {
        cleanup();
        return s2;
    };
    for (int q = 0; q < 2; ++q)
        if (!S->adj[q] && (st = tkh::alloc(S, &S->adj[q], sb)) != TK_OK) return bail(st);
    if (!S->dhalf && (st = tkh::alloc(S, (void **)&S->dhalf, nh * sizeof(double))) != TK_OK) return bail(st);
    if (!S->dnode && (st = tkh::alloc(S, (void **)&S->dnode, nn * sizeof(double))) != TK_OK) return bail(st);
    if (!S->db_node && (st = tkh::alloc(S, (void **)&S->db_node, nb * sizeof(double))) != TK_OK) return bail(st);
    if ((st = tkh::alloc(S, (void **)&thalf, nh * sizeof(double))) != TK_OK ||
        (st = tkh::alloc(S, (void **)&tnode, nn * sizeof(double))) != TK_OK ||
        (st = tkh::alloc(S, (void **)&tb, nb * sizeof(double))) != TK_OK ||
        (st = tkh::alloc(S, (void **)&tw, (size_t)S->NP * sizeof(double))) != TK_OK ||
        (st = tkh::alloc(S, (void **)&tx, (size_t)2 * S->Nr * sizeof(double))) != TK_OK ||
        (st = tkh::alloc(S, (void **)&tang, (size_t)2 * S->NP * sizeof(double))) != TK_OK)
        return bail(st);
    if (on_device) {
        dwave = const_cast<double *>(dL_dwave);
    } else {
        if ((st = tkh::alloc(S, (void **)&dwave, (size_t)S->nobs * count * 2 * sizeof(double))) != TK_OK)
            return bail(st);
        cudaError_t e = cudaMemcpyAsync(dwave, dL_dwave, (size_t)S->nobs * count * 2 * sizeof(double),
                                        cudaMemcpyHostToDevice, S->stream);
        if (e != cudaSuccess) return bail(tkh::fail(S, TK_ERR_CUDA, "tk_param_gradient: %s", cudaGetErrorString(e)));
    }
    cudaError_t e = cudaSuccess;
    const double dt_in = S->dt / k;
    // 1. derivative tables, 4-point central differences in the parameter:
    //    dT/dp = [8 (T(p+d) - T(p-d)) - (T(p+2d) - T(p-2d))] / (12 d)
    {
        const double M = S->kerr.M, a = S->kerr.a;
        double d = 1e-3 * M;
        if (d > 0.25 * (M - fabs(a))) d = 0.25 * (M - fabs(a));
        const double off[4] = {d, -d, 2 * d, -2 * d};
        const double wgt[4] = {8.0 / (12 * d), -8.0 / (12 * d), -1.0 / (12 * d), 1.0 / (12 * d)};
        e = cudaMemsetAsync(S->dhalf, 0, nh * sizeof(double), S->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(S->dnode, 0, nn * sizeof(double), S->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(S->db_node, 0, nb * sizeof(double), S->stream);
        for (int q = 0; q < 4 && e == cudaSuccess; ++q) {
            tk::Kerr P = S->kerr;
            if (param == 0) P.a += off[q];
            else P.M += off[q];
            e = tk::launch_invert_tortoise(P, S->rs_min, S->drs, S->Nr, tx, tx + S->Nr, S->stream);
            if (e == cudaSuccess)
                e = tk::launch_coeff_tables(P, S->variable, S->Nr, S->Nth, S->NP, S->drs, dt_in, tx,
                                            tx + S->Nr, tang, 0, thalf, tnode, tb, tw, nullptr,
                                            nullptr, S->stream);
            if (e == cudaSuccess) e = tk::launch_axpy(nh, wgt[q], thalf, S->dhalf, S->stream);
            if (e == cudaSuccess) e = tk::launch_axpy(nn, wgt[q], tnode, S->dnode, S->stream);
            if (e == cudaSuccess) e = tk::launch_axpy(nb, wgt[q], tb, S->db_node, S->stream);
        }
    }
    if (e != cudaSuccess) return bail(tkh::fail(S, TK_ERR_CUDA, "tk_param_gradient: %s", cudaGetErrorString(e)));
    // 2. checkpoints of the trajectory every C outer steps, from u^0
    if ((st = tkh::alloc(S, (void **)&ck, (size_t)nck * sb)) != TK_OK) return bail(st);
    if ((st = tkh::alloc(S, (void **)&seg, (size_t)(C * k) * sb)) != TK_OK) return bail(st);
    tk::StepLaunch L;
    tkh::fill_launch(S, L);
    L.write_wave = 0;
    e = cudaMemcpyAsync(ck, S->u_init, sb, cudaMemcpyDeviceToDevice, S->stream);
    for (long long c = 0; c + 1 < nck && e == cudaSuccess; ++c) {
        const double *src = ck + (size_t)c * se;
        double *dst = ck + (size_t)(c + 1) * se;
        // C outer steps: ping-pong through the first two segment slots
        const void *in = src;
        for (long long j = 0; j < C * k && e == cudaSuccess; ++j) {
            void *out = (j == C * k - 1) ? (void *)dst : (void *)(seg + (size_t)(j & 1) * se);
            L.u_in = in;
            L.u_out = out;
            e = tk::launch_lw_step(L, S->stream);
            in = out;
        }
    }
    // 3. backward over the segments: recompute the segment's inner states,
    //    then the tangent contraction and the adjoint step for each of them
    int blocks = 0;
    if (e == cudaSuccess) {
        const int K = S->K;
        int per = 0;
        if (K == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tk::param_tangent_kernel<1>, 128, 0);
        else if (K == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tk::param_tangent_kernel<2>, 128, 0);
        else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tk::param_tangent_kernel<4>, 128, 0);
        if (per < 1) per = 1;
        blocks = S->num_sms * per;
        if (blocks > S->Nr / 4) blocks = S->Nr / 4;
        if (blocks < 1) blocks = 1;
    }
    const int pblocks = 1024;
    if (e == cudaSuccess && (st = tkh::alloc(S, (void **)&acc, (size_t)(blocks + pblocks) * sizeof(double))) != TK_OK)
        return bail(st);
    if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, (size_t)(blocks + pblocks) * sizeof(double), S->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->adj[0], 0, sb, S->stream);
    tk::InjectArgs inj;
    memset(&inj, 0, sizeof inj);
    inj.count = count;
    inj.dwave = dwave;
    inj.w_row = S->w_row;
    inj.obs = L.obs;
    int cur = 0;
    for (long long c = nck - 1; c >= 0 && e == cudaSuccess; --c) {
        const long long t0 = c * C, len = (c == nck - 1) ? count - t0 : C;
        // seg[j] = u^{t0 k + j}, j < len k
        e = cudaMemcpyAsync(seg, ck + (size_t)c * se, sb, cudaMemcpyDeviceToDevice, S->stream);
        for (long long j = 0; j + 1 < len * k && e == cudaSuccess; ++j) {
            L.u_in = seg + (size_t)j * se;
            L.u_out = seg + (size_t)(j + 1) * se;
            e = tk::launch_lw_step(L, S->stream);
        }
        for (long long t = t0 + len - 1; t >= t0 && e == cudaSuccess; --t)
            for (int kk = 0; kk < k && e == cudaSuccess; ++kk) {
                inj.on = (kk == 0);
                inj.sample = t;
                const long long j = (t - t0) * k + (k - 1 - kk);     // u^j is the step's input
                e = tk::launch_param_tangent(S->K, blocks, seg + (size_t)j * se, (const double *)S->adj[cur],
                                             (const double *)S->half, (const double *)S->node, S->dhalf,
                                             S->dnode, S->Nr, dt_in, inj, acc, S->stream);
                if (e == cudaSuccess)
                    e = tk::launch_adjoint_step(0, S->K, S->adj[cur], S->adj[cur ^ 1], S->half, S->node,
                                                S->Nr, S->adj_blocks, S->adj_warps, dt_in, inj, S->stream);
                cur ^= 1;
            }
    }
    // 4. the initial-data term (momentum derived from Phi^0 through b)
    if (e == cudaSuccess && S->init_pi_derived) {
        tk::param_initial_kernel<<<pblocks, 256, 0, S->stream>>>(S->Nr, S->Nth, S->NP,
                                                                  (const double *)S->u_init,
                                                                  (const double *)S->adj[cur], S->b_node,
                                                                  S->db_node, acc + blocks);
        e = cudaGetLastError();
    }
    std::vector<double> h((size_t)blocks + pblocks, 0.0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), acc, h.size() * sizeof(double), cudaMemcpyDeviceToHost, S->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
    if (e != cudaSuccess)
        return bail(tkh::fail(S, e == cudaErrorMemoryAllocation ? TK_ERR_OOM : TK_ERR_CUDA,
                              "tk_param_gradient: %s", cudaGetErrorString(e)));
    double g = 0.0;
    for (size_t q = 0; q < h.size(); ++q) g += h[q];
    *grad = g;
    cleanup();
    return TK_OK;
}
