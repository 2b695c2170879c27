// tk_solver_impl.h -- the solver object behind the opaque tk_solver handle,
// and the host helpers shared by tk_api.cu and tk_batch.cu.
#pragma once

#include <stdint.h>

#include "tk.h"
#include "tk_internal.h"

struct tk_solver {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    // grid
    int Nr = 0, Nth = 0, K = 1, NP = 32, substeps = 1, variable = 1, precision = 0;
    double rs_min = 0, rs_max = 0, drs = 0, dt = 0;
    size_t esz = 8;
    // device buffers
    void *u[2] = {nullptr, nullptr};
    int cur = 0;
    void *half = nullptr, *node = nullptr;
    float *cmp = nullptr, *gpm = nullptr;   // FP32: compact tables, theta factors (tk_internal.h)
    double *b_node = nullptr, *w_row = nullptr, *x_node = nullptr, *x_half = nullptr;
    double *ang = nullptr;      // regularised angular stencil [2][NP]
    double *staging = nullptr;  // 4 * Nth * Nr doubles, for host transfers
    int *flag = nullptr;
    unsigned long long *stiff = nullptr;  // [max omega^2, max b] as double bit patterns
    long long *ctr = nullptr;   // [0]: sample index of the next outer step, [1]: blocks done
    void *adj[2] = {nullptr, nullptr};  // adjoint state levels (tk_adjoint), allocated on use
    // parameter gradients (tk_param_gradient): u^0 and the derivative tables
    void *u_init = nullptr;             // copy of u^0 (FP64 solvers)
    bool init_valid = false;            // u_init starts the current trajectory
    bool init_pi_derived = false;       // Pi^0 = b d_* Phi^0 (depends on the parameters through b)
    double *dhalf = nullptr, *dnode = nullptr, *db_node = nullptr;   // d(tables)/d(parameter)
    // physics
    tk::Kerr kerr{};
    bool have_coeffs = false, have_state = false;
    // false after a persistent launch's bounded wait ran out: the state is
    // then invalid until tk_set_initial_data or tk_set_state replaces it
    bool state_valid = true;
    bool inject_wait_timeout = false;   // tk_inject_wait_timeout (host-side test hook)
    // observers and waveform samples
    struct Obs {
        double rs, th;
        int i0, j0;
        double fr, ft;
    } obs[tk::kMaxObservers];
    int nobs = 0;
    double *wave = nullptr;  // [obs][cap][2 slots][re, im]
    int64_t wave_cap = 0;
    double *xbuf = nullptr;  // tk_extract's device buffer for host read-outs (2 * xbuf_cap)
    int64_t xbuf_cap = 0;
    int64_t count = 0;
    int64_t steps_done = 0;
    // launch shape
    bool auto_k = false;        // substeps from the stability bound at each precompute
    int blocks = 1;             // step kernel launch shape
    int warps = 4;
    int persist = 0;            // 1: all inner steps of a tk_step call in one persistent launch
    int persist_blocks = 0;     // its grid (0: the grid is too large for it)
    unsigned int *pflags = nullptr;     // its per-block step flags, then the error flag
    void *obs_scr = nullptr;    // the four-step sweep's waveform-sample scratch
    int multi_blocks = 0;       // FP32: groups of tk::multi_levels() steps per sweep (0: not used)
    int multi_warps = 4;
    int fuse = 0;               // 1: inner steps in pairs, one two-step launch per pair
    int fuse_mode = 0;          // as set by tk_set_steps_per_launch (0: automatic)
    int fused_blocks = 1;       // two-step kernel launch shape
    int fused_warps = 4;
    int adj_blocks = 1;         // adjoint kernel launch shape
    int adj_warps = 4;
    // CUDA-graph replay of chunks of outer steps (0 = launch every step directly)
    int graph_chunk = -1;            // -1: choose automatically
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};   // by parity of the current level
    int graph_outer[2] = {0, 0};
    long long graph_epoch[2] = {-1, -1};
    long long epoch = 0;             // bumped whenever captured parameters change
    char err[512] = {0};
};

namespace tkh {

// Record a one-line message on the solver (or thread-locally if S is NULL).
tk_status fail(tk_solver *S, tk_status st, const char *fmt, ...);
tk_status alloc(tk_solver *S, void **p, size_t bytes);
tk_status ensure_wave(tk_solver *S, int64_t need);
tk_status enter(tk_solver *S);
void fill_launch(const tk_solver *S, tk::StepLaunch &L);
// How observer k's samples are read out of the waveform buffer.
tk::WaveRead wave_read(const tk_solver *S, int k);
// TK_ERR_STATE unless the solver holds a valid state (initial data set, and
// no persistent launch failed since); `what` names the call.
tk_status need_state(tk_solver *S, const char *what);

}  // namespace tkh

#define TK_CUDA(S, call)                                                                  \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return tkh::fail((S), e_ == cudaErrorMemoryAllocation ? TK_ERR_OOM : TK_ERR_CUDA, \
                             "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)
