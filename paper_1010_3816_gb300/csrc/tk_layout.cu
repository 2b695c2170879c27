// tk_layout.cu -- moves the state between the ABI's planes [Ntheta][Nr] (the
// paper's idx(b,a) = N*b + a layout) and the device-resident column layout
// u[i][c][jp]; sets the initial momentum; finite check; waveform sums.
#include <math.h>

#include "tk_internal.h"

namespace tk {
namespace {

// Initial data (Sec. 3.2).  Pi is either given or, for zero time derivative,
// Pi = b d_* Phi with the centred difference (Phi_{i+1} - Phi_{i-1})/(2 dr*).
// Both fields vanish on the radial edges; padding rows are zero.
template <typename T>
__global__ void import_kernel(int Nr, int Nth, int NP, double drs, const double *__restrict__ phr,
                              const double *__restrict__ phi, const double *__restrict__ pir,
                              const double *__restrict__ pii, const double *__restrict__ b_node,
                              T *__restrict__ u)
{
    const int jp = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (jp >= NP || i >= Nr) return;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (jp < Nth && i > 0 && i < Nr - 1) {
        const size_t k = (size_t)jp * Nr + i;
        v[0] = phr[k];
        v[1] = phi[k];
        if (pir) {
            v[2] = pir[k];
            v[3] = pii[k];
        } else {
            const double b = b_node[(size_t)i * NP + jp];
            v[2] = b * (phr[k + 1] - phr[k - 1]) / (2.0 * drs);
            v[3] = b * (phi[k + 1] - phi[k - 1]) / (2.0 * drs);
        }
    }
    T *col = u + (size_t)i * 4 * NP + jp;
#pragma unroll
    for (int c = 0; c < 4; ++c) col[(size_t)c * NP] = (T)v[c];
}

template <typename T>
__global__ void export_kernel(int Nr, int Nth, int NP, const T *__restrict__ u,
                              double *__restrict__ out)
{
    const int jp = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (jp >= Nth || i >= Nr) return;
    const T *col = u + (size_t)i * 4 * NP + jp;
    const size_t plane = (size_t)Nth * Nr;
#pragma unroll
    for (int c = 0; c < 4; ++c) out[c * plane + (size_t)jp * Nr + i] = (double)col[(size_t)c * NP];
}

template <typename T>
__global__ void finite_kernel(size_t n, const T *__restrict__ u, int *flag)
{
    int bad = 0;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        bad |= !isfinite((double)u[k]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

__global__ void wave_sum_kernel(const double *__restrict__ w, int64_t count, double *__restrict__ re,
                                double *__restrict__ im)
{
    const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n >= count) return;
    re[n] = w[4 * n + 0] + w[4 * n + 2];
    im[n] = w[4 * n + 1] + w[4 * n + 3];
}

}  // namespace

cudaError_t launch_import_state(int precision, int Nr, int Ntheta, int NP, double drs,
                                const double *phi_re, const double *phi_im, const double *pi_re,
                                const double *pi_im, const double *b_node, void *u,
                                cudaStream_t st)
{
    dim3 block(32, 8), grid((NP + 31) / 32, (Nr + 7) / 8);
    if (precision == 0)
        import_kernel<double><<<grid, block, 0, st>>>(Nr, Ntheta, NP, drs, phi_re, phi_im, pi_re, pi_im,
                                                      b_node, (double *)u);
    else
        import_kernel<float><<<grid, block, 0, st>>>(Nr, Ntheta, NP, drs, phi_re, phi_im, pi_re, pi_im,
                                                     b_node, (float *)u);
    return cudaGetLastError();
}

cudaError_t launch_export_state(int precision, int Nr, int Ntheta, int NP, const void *u,
                                double *planes4, cudaStream_t st)
{
    dim3 block(32, 8), grid((NP + 31) / 32, (Nr + 7) / 8);
    if (precision == 0)
        export_kernel<double><<<grid, block, 0, st>>>(Nr, Ntheta, NP, (const double *)u, planes4);
    else
        export_kernel<float><<<grid, block, 0, st>>>(Nr, Ntheta, NP, (const float *)u, planes4);
    return cudaGetLastError();
}

cudaError_t launch_finite_check(int precision, size_t n, const void *u, int *flag, cudaStream_t st)
{
    const int blocks = 304, threads = 256;
    if (precision == 0)
        finite_kernel<double><<<blocks, threads, 0, st>>>(n, (const double *)u, flag);
    else
        finite_kernel<float><<<blocks, threads, 0, st>>>(n, (const float *)u, flag);
    return cudaGetLastError();
}

cudaError_t launch_wave_sum(const double *wave_obs, int64_t count, double *re, double *im,
                            cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = (count + threads - 1) / threads;
    wave_sum_kernel<<<(unsigned)blocks, threads, 0, st>>>(wave_obs, count, re, im);
    return cudaGetLastError();
}

}  // namespace tk
