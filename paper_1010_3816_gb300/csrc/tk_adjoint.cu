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
// to right, recomputing eta at the left edge of its range.
#include "tk_solver_impl.h"
#include "tk_stencil.cuh"

namespace tk {
namespace {

constexpr int kAdjThreads = 128;

struct InjectArgs {
    int on;                  // add the observation gradient of sample `sample`
    long long sample, count; // sample index; samples per observer in dwave
    const double *dwave;     // [obs][count][2]: dL/dRe W, dL/dIm W
    const double *w_row;
    ObsDev obs;
};

// Load the adjoint state of column i, add the gradient of the waveform sample
// taken at this column (if any), and zero it on the radial edges.
template <typename T, int K>
__device__ __forceinline__ void load_lam(const T *__restrict__ lam, int i, int Nr, int lane,
                                         const InjectArgs &inj, T (&l)[4][K])
{
    constexpr int NP = 32 * K;
    load_col<T, K>(lam + (size_t)i * 4 * NP + lane * K, l);
    if (inj.on) {
        for (int k = 0; k < inj.obs.n; ++k) {
            const int slot = (i == inj.obs.i0[k]) ? 0 : ((i == inj.obs.i0[k] + 1) ? 1 : -1);
            if (slot < 0) continue;
            const int j0 = inj.obs.j0[k];
            const double wr = slot ? inj.obs.wr1[k] : inj.obs.wr0[k];
            const double *g = inj.dwave + ((size_t)k * inj.count + inj.sample) * 2;
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

// Theta-neighbour part of a transposed coupling: for z+ = KP * x (sent to
// row j+1) and z- = KM * x (sent to row j-1), the amount row j receives.
template <typename T, int K>
__device__ __forceinline__ void neighbour_in(const T (&kp)[K], const T (&km)[K], const T (&x)[K],
                                             T (&out)[K])
{
    T zp[K], zm[K], dn[K], up[K];
#pragma unroll
    for (int t = 0; t < K; ++t) {
        zp[t] = kp[t] * x[t];
        zm[t] = km[t] * x[t];
    }
    // row j receives zp from row j-1 (the "dn" neighbour) and zm from row j+1 ("up")
    T tmp_up[K], tmp_dn[K];
    theta_neighbours<T, K>(zp, tmp_up, dn);
    theta_neighbours<T, K>(zm, up, tmp_dn);
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int t = 0; t < K; ++t) {
        // lane 0's row 0 has no row -1 and lane 31's last row no row N: the
        // shuffles return the lane's own values there, whose coefficients are 0
        // only on the sending side, so mask them explicitly
        const T a = (lane == 0 && t == 0) ? T(0) : dn[t];
        const T b = (lane == 31 && t == K - 1) ? T(0) : up[t];
        out[t] = a + b;
    }
    (void)tmp_up;
    (void)tmp_dn;
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
    neighbour_in<T, K>(kp, km, l[2], zr);
    neighbour_in<T, K>(kp, km, l[3], zi);
}

// eta at the half node between nodes a (left) and c (right).
template <typename T, int K>
__device__ __forceinline__ void eta_half(const T (&la)[4][K], const T (&lc)[4][K],
                                         const T (&zar)[K], const T (&zai)[K], const T (&zcr)[K],
                                         const T (&zci)[K], const T *__restrict__ ta,
                                         const T *__restrict__ tc, const T E, T (&h)[4][K])
{
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
        h[0][t] = fma(FI[t], la[3][t], fma(FR[t], la[2][t], fma(-B[t], la[0][t], zar[t] + zcr[t])));
        h[1][t] = fma(FR[t], la[3][t], fma(-FI[t], la[2][t], fma(-B[t], la[1][t], zai[t] + zci[t])));
        h[2][t] = fma(CI[t], la[3][t], fma(PR[t], la[2][t], E * la[0][t]));
        h[3][t] = fma(PR[t], la[3][t], fma(-CI[t], la[2][t], E * la[1][t]));
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
    neighbour_in<T, K>(kp, km, h[2], yr);
    neighbour_in<T, K>(kp, km, h[3], yi);
}

// mu at node i from lam~_i, eta+ (half node i+1/2: u_i is its "a") and eta-
// (half node i-1/2: u_i is its "c").
template <typename T, int K>
__device__ __forceinline__ void mu_node(const T (&l)[4][K], const T (&ep)[4][K],
                                        const T (&em)[4][K], const T (&ypr)[K], const T (&ypi)[K],
                                        const T (&ymr)[K], const T (&ymi)[K],
                                        const T *__restrict__ hp_tab, const T *__restrict__ hm_tab,
                                        const T e, T (&mu)[4][K])
{
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
        mu[0][t] = fma(FI[t], ep[3][t], fma(FR[t], ep[2][t], fma(S[t], ep[0][t], l[0][t] + (ypr[t] + ymr[t]))));
        mu[1][t] = fma(FR[t], ep[3][t], fma(-FI[t], ep[2][t], fma(S[t], ep[1][t], l[1][t] + (ypi[t] + ymi[t]))));
        mu[2][t] = fma(PI[t], ep[3][t], fma(PR[t], ep[2][t], fma(e, ep[0][t], l[2][t])));
        mu[3][t] = fma(PR[t], ep[3][t], fma(-PI[t], ep[2][t], fma(e, ep[1][t], l[3][t])));
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
        mu[2][t] = fma(PI[t], em[3][t], fma(PR[t], em[2][t], fma(e, em[0][t], mu[2][t])));
        mu[3][t] = fma(PR[t], em[3][t], fma(-PI[t], em[2][t], fma(e, em[1][t], mu[3][t])));
    }
}

template <typename T, int K>
__global__ void __launch_bounds__(kAdjThreads)
lw_adjoint_kernel(const T *__restrict__ lam, T *__restrict__ mu_out, const T *__restrict__ half,
                  const T *__restrict__ node, int Nr, T eh, T en, const InjectArgs inj)
{
    constexpr int NP = 32 * K;
    constexpr size_t SP = 4 * NP, HP = (size_t)kNCH * NP, NQ = (size_t)kNCN * NP;
    const int lane = threadIdx.x & 31;
    const long long G = (long long)gridDim.x * (kAdjThreads / 32);
    const long long g = (long long)blockIdx.x * (kAdjThreads / 32) + (threadIdx.x >> 5);
    const int i0 = (int)((g * Nr) / G);
    const int i1 = (int)(((g + 1) * Nr) / G);
    if (i1 <= i0) return;
    const int row = lane * K;

    T la[4][K], zar[K], zai[K];        // node i: lam~ and its neighbour sources
    T em[4][K], ymr[K], ymi[K];        // half node i-1/2: eta and its neighbour sources
    load_lam<T, K>(lam, i0, Nr, lane, inj, la);
    node_z<T, K>(node + (size_t)i0 * NQ + row, la, zar, zai);
    if (i0 > 0) {
        T ll[4][K], zlr[K], zli[K];
        load_lam<T, K>(lam, i0 - 1, Nr, lane, inj, ll);
        node_z<T, K>(node + (size_t)(i0 - 1) * NQ + row, ll, zlr, zli);
        eta_half<T, K>(ll, la, zlr, zli, zar, zai, node + (size_t)(i0 - 1) * NQ + row,
                       node + (size_t)i0 * NQ + row, en, em);
        half_y<T, K>(half + (size_t)(i0 - 1) * HP + row, em, ymr, ymi);
    } else {
        zero_col<T, K>(em);
#pragma unroll
        for (int t = 0; t < K; ++t) ymr[t] = ymi[t] = T(0);
    }
    for (int i = i0; i < i1; ++i) {
        T lc[4][K], zcr[K], zci[K], ep[4][K], ypr[K], ypi[K], mu[4][K];
        if (i + 1 < Nr) {
            load_lam<T, K>(lam, i + 1, Nr, lane, inj, lc);
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
        const T *hm_tab = half + (size_t)(i > 0 ? i - 1 : 0) * HP + row;
        mu_node<T, K>(la, ep, em, ypr, ypi, ymr, ymi, half + (size_t)i * HP + row, hm_tab, eh, mu);
        store_col<T, K>(mu_out + (size_t)i * SP + row, mu);
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

template <typename T, int K>
cudaError_t launch_adj(const void *lam, void *mu, const void *half, const void *node, int Nr,
                       int blocks, double dt_in, const InjectArgs &inj, cudaStream_t st)
{
    lw_adjoint_kernel<T, K><<<blocks, kAdjThreads, 0, st>>>((const T *)lam, (T *)mu, (const T *)half,
                                                            (const T *)node, Nr, (T)(0.25 * dt_in),
                                                            (T)(0.5 * dt_in), inj);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_step(int precision, int K, const void *lam, void *mu, const void *half,
                                const void *node, int Nr, int blocks, double dt_in,
                                const InjectArgs &inj, cudaStream_t st)
{
    if (precision == 0) {
        if (K == 1) return launch_adj<double, 1>(lam, mu, half, node, Nr, blocks, dt_in, inj, st);
        if (K == 2) return launch_adj<double, 2>(lam, mu, half, node, Nr, blocks, dt_in, inj, st);
        return launch_adj<double, 4>(lam, mu, half, node, Nr, blocks, dt_in, inj, st);
    }
    if (K == 1) return launch_adj<float, 1>(lam, mu, half, node, Nr, blocks, dt_in, inj, st);
    if (K == 2) return launch_adj<float, 2>(lam, mu, half, node, Nr, blocks, dt_in, inj, st);
    return launch_adj<float, 4>(lam, mu, half, node, Nr, blocks, dt_in, inj, st);
}

template <typename T, int K>
int adj_resident()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, lw_adjoint_kernel<T, K>, kAdjThreads, 0) !=
        cudaSuccess)
        n = 1;
    return n < 1 ? 1 : n;
}

}  // namespace

int adjoint_grid_blocks(int precision, int K, int Nr, int num_sms)
{
    int per_sm;
    if (precision == 0)
        per_sm = K == 1 ? adj_resident<double, 1>() : K == 2 ? adj_resident<double, 2>()
                                                             : adj_resident<double, 4>();
    else
        per_sm = K == 1 ? adj_resident<float, 1>() : K == 2 ? adj_resident<float, 2>()
                                                            : adj_resident<float, 4>();
    int blocks = num_sms * per_sm;
    const int max_blocks = Nr / (kAdjThreads / 32);
    if (blocks > max_blocks) blocks = max_blocks;
    return blocks < 1 ? 1 : blocks;
}

}  // namespace tk

extern "C" tk_status tk_adjoint(tk_solver *S, const double *dL_dwave, const double *dL_dfinal,
                                int on_device, double *grad, int grad_on_device, int independent_pi)
{
    tk_status st = tkh::enter(S);
    if (st != TK_OK) return st;
    if (!S->have_state) return tkh::fail(S, TK_ERR_STATE, "tk_adjoint before tk_set_initial_data");
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
    for (long long t = count - 1; t >= 0 && e == cudaSuccess; --t)
        for (int k = 0; k < S->substeps && e == cudaSuccess; ++k) {
            inj.on = (k == 0) && dwave != nullptr;
            inj.sample = t;
            e = tk::launch_adjoint_step(S->precision, S->K, S->adj[cur], S->adj[cur ^ 1], S->half,
                                        S->node, S->Nr, S->adj_blocks, dt_in, inj, S->stream);
            cur ^= 1;
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
