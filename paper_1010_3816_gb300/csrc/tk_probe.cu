// tk_probe.cu -- measured rate of the FP64 fused multiply-add pipe.
//
// The FP64 step is bound by the FP64 pipe, not by memory (54 FP64 FMA
// instructions per update against 64 bytes of state), so its roofline is the
// pipe's FMA rate.  This microbenchmark measures that rate on the device the
// library runs on: every thread advances kChains independent FMA chains
// (enough to cover the pipe's latency), blocks fill every SM, and CUDA events
// time the launch.
#include "tk_solver_impl.h"

namespace {

constexpr int kChains = 8;

__global__ void fp64_fma_kernel(int iters, const double *__restrict__ ab, double *__restrict__ out)
{
    const double a = ab[0], b = ab[1];
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    // a = 1, b = 0 at run time: s stays finite; written only if it is not, so
    // the chains cannot be removed and nothing is stored
    if (s == -1.0) out[blockIdx.x] = s;
}

}  // namespace

extern "C" tk_status tk_probe_fp64_fma(int blocks_per_sm, int threads, int iters, double *seconds,
                                       double *flop)
{
    if (blocks_per_sm < 1 || blocks_per_sm > 32 || threads < 32 || threads > 1024 || threads % 32 ||
        iters < 1 || !seconds || !flop)
        return tkh::fail(nullptr, TK_ERR_ARG, "tk_probe_fp64_fma: bad arguments");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double *buf = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (e == cudaSuccess) e = cudaMalloc((void **)&buf, 2 * sizeof(double) + (size_t)sms * blocks_per_sm * sizeof(double));
    const double ab[2] = {1.0, 0.0};
    if (e == cudaSuccess) e = cudaMemcpy(buf, ab, sizeof ab, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    const int grid = sms * blocks_per_sm;
    if (e == cudaSuccess) {
        fp64_fma_kernel<<<grid, threads>>>(iters / 8 + 1, buf, buf + 2);   // warm-up
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[0]);
    if (e == cudaSuccess) {
        fp64_fma_kernel<<<grid, threads>>>(iters, buf, buf + 2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[1]);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (buf) cudaFree(buf);
    if (e != cudaSuccess) return tkh::fail(nullptr, TK_ERR_CUDA, "tk_probe_fp64_fma: %s", cudaGetErrorString(e));
    *seconds = ms * 1e-3;
    *flop = 2.0 * kChains * (double)iters * threads * grid;
    return TK_OK;
}
