// tk_static.cu -- tk_extract_noalloc: reading a waveform into host memory
// without any device allocation.
//
// tk_extract with a host destination sums the two partial samples of every
// step into a temporary device buffer that it allocates with cudaMalloc on
// each call.  Callers that must not allocate device memory -- code running
// while another thread captures a CUDA graph, real-time loops whose memory
// budget is fixed up front, or hosts that route all device memory through
// their own pool -- use this variant instead: the same summing kernel writes
// into a fixed array compiled into the library, and the result is copied from
// there to the caller's host buffers.
#include <mutex>

#include "tk_solver_impl.h"

namespace {

// Samples one call can return (per real and per imaginary part).
constexpr int kMaxNoallocSamples = 65536;

// The scratch: real parts in [0, count), imaginary parts in [count, 2 count).
// 1 MiB, held by every GPU that loads the library until the process exits.
// Every call reuses it and it keeps the last call's contents; each call
// writes every element it then reads, so nothing has to start at zero.
static __device__ __align__(256) double g_noalloc_scratch[2 * kMaxNoallocSamples];

// Device address of g_noalloc_scratch, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

__global__ void wave_sum_into_kernel(const double *__restrict__ w, long long first, int count,
                                     double *__restrict__ out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= count) return;
    const double *p = w + 4 * (first + n);
    out[n] = p[0] + p[2];
    out[count + n] = p[1] + p[3];
}

// With the solver's device current: the scratch's device address on it.
tk_status scratch_for(tk_solver *S, double **ptr)
{
    if (S->device < 0 || S->device >= kMaxDevices)
        return tkh::fail(S, TK_ERR_ARG, "tk_extract_noalloc: device %d not supported", S->device);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[S->device]) {
        double *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return tkh::fail(S, TK_ERR_CUDA, "tk_extract_noalloc: cudaGetSymbolAddress: %s",
                             cudaGetErrorString(e));
        g_scratch_ptr[S->device] = p;
    }
    *ptr = g_scratch_ptr[S->device];
    return TK_OK;
}

}  // namespace

extern "C" tk_status tk_extract_noalloc(tk_solver *S, int obs_id, int first, int count, double *re,
                                        double *im)
{
    tk_status st = tkh::enter(S);
    if (st != TK_OK) return st;
    if (obs_id < 0 || obs_id >= S->nobs)
        return tkh::fail(S, TK_ERR_ARG, "tk_extract_noalloc: bad observer id %d", obs_id);
    if (count < 0 || count > kMaxNoallocSamples)
        return tkh::fail(S, TK_ERR_ARG,
                         "tk_extract_noalloc: count %d outside [0, %d]; read longer waveforms "
                         "in pieces with `first`", count, kMaxNoallocSamples);
    if (first < 0 || (long long)first + count > S->count)
        return tkh::fail(S, TK_ERR_ARG,
                         "tk_extract_noalloc: samples [%d, %lld) requested, %lld taken", first,
                         (long long)first + count, (long long)S->count);
    if (count == 0) return TK_OK;
    if (!re || !im) return tkh::fail(S, TK_ERR_ARG, "tk_extract_noalloc: re/im NULL");
    double *scratch = nullptr;
    st = scratch_for(S, &scratch);
    if (st != TK_OK) return st;
    const double *src = S->wave + (size_t)obs_id * S->wave_cap * 4;
    const int threads = 256;
    wave_sum_into_kernel<<<(count + threads - 1) / threads, threads, 0, S->stream>>>(src, first, count,
                                                                                   scratch);
    TK_CUDA(S, cudaGetLastError());
    TK_CUDA(S, cudaMemcpyAsync(re, scratch, (size_t)count * sizeof(double), cudaMemcpyDeviceToHost,
                               S->stream));
    TK_CUDA(S, cudaMemcpyAsync(im, scratch + count, (size_t)count * sizeof(double),
                               cudaMemcpyDeviceToHost, S->stream));
    TK_CUDA(S, cudaStreamSynchronize(S->stream));
    return TK_OK;
}
