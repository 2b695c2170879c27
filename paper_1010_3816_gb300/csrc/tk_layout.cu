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

// Waveform read-out (the bilinear sample of Phi = w Phi^ in r* and theta).
// FP64 entries are two weighted partial sums: the sample is their sum.  FP32
// entries are the state values of the interpolation cell (WaveRead): the
// sample is formed here in FP64 by the FP64 path's own expression,
//   slot s = wr_s [(1 - fth) w_j0 Phi_{s,j0} + fth w_j0+1 Phi_{s,j0+1}],
// on the exactly converted values.
__global__ void wave_sum_kernel(const double *__restrict__ w, int64_t first, int64_t count,
                                const WaveRead r, double *__restrict__ re, double *__restrict__ im)
{
    const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n >= count) return;
    const double *p = w + 4 * (first + n);
    if (r.precision == 0) {
        re[n] = p[0] + p[2];
        im[n] = p[1] + p[3];
        return;
    }
    const float4 *f = reinterpret_cast<const float4 *>(p);
    const double w0 = (1.0 - r.ft) * r.w_row[r.j0];
    const double w1 = r.ft * r.w_row[r.j0 + 1];
    double sr[2], si[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const float4 v = f[s];   // Phi_R, Phi_I at row j0, then at row j0 + 1
        const double cr = w0 * (double)v.x + w1 * (double)v.z;
        const double ci = w0 * (double)v.y + w1 * (double)v.w;
        const double wr = s ? r.wr1 : r.wr0;
        sr[s] = wr * cr;
        si[s] = wr * ci;
    }
    re[n] = sr[0] + sr[1];
    im[n] = si[0] + si[1];
}

// SplitMix64 (G. L. Steele, D. Lea, C. H. Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014) in its counter form: output k
// (k = 0, 1, ...) of seed S is the 64-bit finaliser applied to
// S + (k + 1) * 0x9E3779B97F4A7C15; a uniform double in [0, 1) is the top 53
// bits times 2^-53.
__device__ __forceinline__ double splitmix64_uniform(unsigned long long seed, unsigned long long k)
{
    unsigned long long z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1.0p-53;
}

// Gaussian pulse with the sin^2(theta) profile plus uniform noise, planes
// [Ntheta][Nr]: re = sin^2(theta_j) * amp * exp(-(r*_i - c)^2 / (2 w^2))
// + noise * (2 u - 1), im = noise * (2 u' - 1), with u the SplitMix64 output
// j Nr + i and u' the output Nr Ntheta + j Nr + i.  Every operation is rounded
// on its own (no contraction), so the planes agree with the same formula
// evaluated one IEEE operation at a time up to the last bits of exp and sin.
__global__ void gaussian_kernel(int Nr, int Nth, double rs_min, double drs, double dth, double amp,
                                double center, double two_w2, double noise,
                                unsigned long long seed, double *__restrict__ re,
                                double *__restrict__ im)
{
    const long long P = (long long)Nr * Nth;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < P;
         k += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(k / Nr), i = (int)(k - (long long)j * Nr);
        const double rs = __dadd_rn(rs_min, __dmul_rn((double)i, drs));
        const double th = __dmul_rn(__dadd_rn((double)j, 0.5), dth);
        const double d = __dsub_rn(rs, center);
        const double g = __dmul_rn(amp, exp(-__ddiv_rn(__dmul_rn(d, d), two_w2)));
        const double sn = sin(th);
        double vr = __dmul_rn(__dmul_rn(sn, sn), g), vi = 0.0;
        if (noise > 0.0) {
            const double ur = splitmix64_uniform(seed, (unsigned long long)k);
            const double ui = splitmix64_uniform(seed, (unsigned long long)(P + k));
            vr = __dadd_rn(vr, __dmul_rn(noise, __dsub_rn(__dmul_rn(2.0, ur), 1.0)));
            vi = __dmul_rn(noise, __dsub_rn(__dmul_rn(2.0, ui), 1.0));
        }
        re[k] = vr;
        im[k] = vi;
    }
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

cudaError_t launch_wave_sum(const double *wave_obs, int64_t first, int64_t count, const WaveRead &r,
                            double *re, double *im, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = (count + threads - 1) / threads;
    wave_sum_kernel<<<(unsigned)blocks, threads, 0, st>>>(wave_obs, first, count, r, re, im);
    return cudaGetLastError();
}

cudaError_t launch_gaussian(int Nr, int Ntheta, double rs_min, double drs, double amp,
                            double center, double width, double noise, unsigned long long seed,
                            double *re, double *im, cudaStream_t st)
{
    const long long P = (long long)Nr * Ntheta;
    long long blocks = (P + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    gaussian_kernel<<<(unsigned)blocks, 256, 0, st>>>(Nr, Ntheta, rs_min, drs, M_PI / Ntheta, amp,
                                                      center, 2.0 * (width * width), noise, seed,
                                                      re, im);
    return cudaGetLastError();
}

}  // namespace tk
