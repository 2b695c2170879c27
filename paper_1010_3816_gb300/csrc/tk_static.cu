// tk_static.cu -- tk_extract_noalloc: reading a waveform into host memory
// without any device allocation.
//
// tk_extract with a host destination forms the samples in a device buffer
// that the solver allocates on first use and again whenever the waveform
// buffer grows.  Some callers must not allocate device memory at all once
// they are set up: hosts that hand all device memory to their own pool and
// treat any other cudaMalloc as a failure, and loops whose device-memory
// budget is fixed up front (a cudaMalloc there can also synchronize the
// device and stall other streams).  They use this variant instead: the same
// read-out kernel writes into a fixed array compiled into the library, and
// the result is copied from there to the caller's host buffers.
#include "tk_solver_impl.h"

namespace {

// Samples one call can return (per real and per imaginary part).
constexpr int kMaxNoallocSamples = 65536;

// The scratch: real parts in [0, count), imaginary parts in [count, 2 count).
// 1 MiB, held by every GPU that loads the library until the process exits.
// Every call reuses it and it keeps the last call's contents; each call
// writes every element it then reads, so nothing has to start at zero.
static __device__ __align__(256) double g_noalloc_scratch[2 * kMaxNoallocSamples];

// With the solver's device current: the scratch's device address on it.  The
// address is looked up on every call (after the first call on a device this
// is a table lookup): a cached pointer would go stale if the program reset
// the device and the module were loaded again at another address.
tk_status scratch_for(tk_solver *S, double **ptr)
{
    double *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return tkh::fail(S, TK_ERR_CUDA, "tk_extract_noalloc: cudaGetSymbolAddress: %s",
                         cudaGetErrorString(e));
    *ptr = p;
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
    TK_CUDA(S, tk::launch_wave_sum(src, first, count, tkh::wave_read(S, obs_id), scratch,
                                   scratch + count, S->stream));
    TK_CUDA(S, cudaMemcpyAsync(re, scratch, (size_t)count * sizeof(double), cudaMemcpyDeviceToHost,
                               S->stream));
    TK_CUDA(S, cudaMemcpyAsync(im, scratch + count, (size_t)count * sizeof(double),
                               cudaMemcpyDeviceToHost, S->stream));
    TK_CUDA(S, cudaStreamSynchronize(S->stream));
    return TK_OK;
}
