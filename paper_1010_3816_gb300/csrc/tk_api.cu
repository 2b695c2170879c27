// tk_api.cu -- the C ABI declared in include/tk.h.
//
// Host code only: argument and call-order checks, device allocation, and the
// ordering of kernel launches on the solver's stream.  Every piece of the
// method's arithmetic runs in the kernels of tk_coeffs.cu, tk_step.cu and
// tk_layout.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "tk_solver_impl.h"

namespace {
thread_local char g_err[512] = "no error";
}  // namespace

namespace tkh {

tk_status fail(tk_solver *S, tk_status st, const char *fmt, ...)
{
    char *buf = S ? S->err : g_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return st;
}

size_t state_elems(const tk_solver *S) { return (size_t)S->Nr * 4 * S->NP; }

tk_status alloc(tk_solver *S, void **p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(S, TK_ERR_OOM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    return TK_OK;
}

void release(tk_solver *S)
{
    void *ptrs[] = {S->u[0], S->u[1], S->half, S->node, S->b_node, S->w_row,
                    S->x_node, S->x_half, S->ang, S->staging, S->flag, S->stiff, S->ctr, S->wave,
                    S->adj[0], S->adj[1], S->u_init, S->dhalf, S->dnode, S->db_node, S->pflags,
                    S->obs_scr, S->xbuf, S->cmp, S->gpm};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (int k = 0; k < 2; ++k)
        if (S->graph[k]) cudaGraphExecDestroy(S->graph[k]);
    if (S->capture_stream) cudaStreamDestroy(S->capture_stream);
}

tk_status ensure_staging(tk_solver *S)
{
    if (S->staging) return TK_OK;
    return alloc(S, (void **)&S->staging, (size_t)4 * S->Nth * S->Nr * sizeof(double));
}

tk_status ensure_wave(tk_solver *S, int64_t need)
{
    if (S->nobs == 0 || need <= S->wave_cap) return TK_OK;
    int64_t cap = S->wave_cap ? S->wave_cap : 1024;
    while (cap < need) cap *= 2;
    double *nw = nullptr;
    tk_status st = alloc(S, (void **)&nw, (size_t)tk::kMaxObservers * cap * 4 * sizeof(double));
    if (st != TK_OK) return st;
    if (S->wave && S->count > 0) {
        cudaError_t e = cudaMemcpy2DAsync(nw, (size_t)cap * 4 * sizeof(double), S->wave,
                                          (size_t)S->wave_cap * 4 * sizeof(double),
                                          (size_t)S->count * 4 * sizeof(double), S->nobs,
                                          cudaMemcpyDeviceToDevice, S->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
        if (e != cudaSuccess) {
            cudaFree(nw);
            return fail(S, TK_ERR_CUDA, "waveform buffer growth: %s", cudaGetErrorString(e));
        }
    }
    if (S->wave) cudaFree(S->wave);
    S->wave = nw;
    S->wave_cap = cap;
    S->epoch++;
    return TK_OK;
}

tk_status enter(tk_solver *S)
{
    if (!S) return fail(nullptr, TK_ERR_ARG, "null solver");
    TK_CUDA(S, cudaSetDevice(S->device));
    return TK_OK;
}

tk_status need_state(tk_solver *S, const char *what)
{
    if (!S->have_state) return fail(S, TK_ERR_STATE, "%s before tk_set_initial_data", what);
    if (!S->state_valid)
        return fail(S, TK_ERR_STATE, "%s: the state is invalid (a persistent launch's bounded wait "
                                     "ran out); set it again with tk_set_state or tk_set_initial_data",
                    what);
    return TK_OK;
}

tk::WaveRead wave_read(const tk_solver *S, int k)
{
    tk::WaveRead r;
    r.precision = S->precision;
    r.j0 = S->obs[k].j0;
    r.ft = S->obs[k].ft;
    r.wr0 = 1.0 - S->obs[k].fr;
    r.wr1 = S->obs[k].fr;
    r.w_row = S->w_row;
    return r;
}

void fill_launch(const tk_solver *S, tk::StepLaunch &L)
{
    L.precision = S->precision;
    L.K = S->K;
    L.Nr = S->Nr;
    L.NP = S->NP;
    L.blocks = S->blocks;
    L.warps = S->warps;
    L.fused = 0;
    L.obs_mask = 0;
    L.dt_inner = S->dt / S->substeps;
    L.half = S->half;
    L.node = S->node;
    L.cmp = S->cmp;
    L.gpm = S->gpm;
    L.wave_cap = S->wave_cap;
    L.wave = S->wave;
    L.w_row = S->w_row;
    L.sample_ctr = S->ctr;
    L.done_ctr = (unsigned int *)(S->ctr + 1);
    L.obs.n = S->nobs;
    for (int k = 0; k < S->nobs; ++k) {
        L.obs.i0[k] = S->obs[k].i0;
        L.obs.j0[k] = S->obs[k].j0;
        L.obs.wr0[k] = 1.0 - S->obs[k].fr;
        L.obs.wr1[k] = S->obs[k].fr;
        L.obs.ft[k] = S->obs[k].ft;
    }
}

}  // namespace tkh

using tkh::alloc;
using tkh::ensure_staging;
using tkh::release;
using tkh::state_elems;
using tkh::enter;
using tkh::ensure_wave;
using tkh::fail;
using tkh::need_state;

// Tolerated amplification per Lax-Wendroff step of the stiffest angular mode
// when the solver picks its own number of substeps: a factor e over 40000 steps.
constexpr double kAutoGrowthPerStep = 2.5e-5;

// Launch structure for tk_step.  mode 0 (automatic): every step of a call in
// one persistent launch.  FP32, bound by memory, runs it as sweeps of four
// steps on large grids and pairs of steps otherwise (four or two steps per
// read of the state and the tables); FP64, bound by its arithmetic (which the
// two-step kernel's overlap adds to), as single steps in which every warp
// waits only for the warps it depends on, so that no launch boundary or block
// barrier separates the steps.  Measured: FP32 25601 x 64, 15.7 us per step in
// sweeps of four, 16.6 in pairs, 18.3 with a launch per pair; FP64 1601 x 32,
// 6.5 against 14.5 us with a launch per step; FP64 25601 x 32 / 64 / 128, 73.3
// / 146.9 / 287.0 against 79.0 / 150.3 / 297.4 us.  A grid whose blocks cannot
// all be resident at once falls back to one launch per step (2 for FP32).
static void set_launch_mode(tk_solver *S, int mode)
{
    S->fuse_mode = mode;
    if (mode == 0) {
        if (S->precision == TK_PREC_F32) mode = S->persist_blocks > 0 ? -1 : 2;
        else mode = S->persist_blocks > 0 ? -1 : 1;
    }
    S->persist = (mode == -1);
    S->fuse = (mode == 2);
}

extern "C" {

tk_status tk_make_grid(tk_solver **out, double rstar_min, double rstar_max, int Nr, int Ntheta,
                       double dt, int substeps, int angular_variable, int precision,
                       void *cuda_stream)
{
    if (!out) return fail(nullptr, TK_ERR_ARG, "tk_make_grid: out is NULL");
    *out = nullptr;
    if (!(rstar_max > rstar_min) || !isfinite(rstar_min) || !isfinite(rstar_max))
        return fail(nullptr, TK_ERR_ARG, "tk_make_grid: need finite rstar_min < rstar_max");
    if (Nr < 3) return fail(nullptr, TK_ERR_ARG, "tk_make_grid: Nr = %d < 3", Nr);
    if (Ntheta < 2 || Ntheta > 32 * tk::kMaxK)
        return fail(nullptr, TK_ERR_ARG, "tk_make_grid: Ntheta = %d outside [2, %d]", Ntheta,
                    32 * tk::kMaxK);
    if (!(dt > 0) || !isfinite(dt)) return fail(nullptr, TK_ERR_ARG, "tk_make_grid: dt must be > 0");
    if (substeps < 0) return fail(nullptr, TK_ERR_ARG, "tk_make_grid: substeps < 0");
    if (angular_variable != TK_VAR_LITERAL && angular_variable != TK_VAR_REGULARISED)
        return fail(nullptr, TK_ERR_ARG, "tk_make_grid: bad angular_variable %d", angular_variable);
    if (precision != TK_PREC_F64 && precision != TK_PREC_F32)
        return fail(nullptr, TK_ERR_ARG, "tk_make_grid: bad precision %d", precision);

    tk_solver *S = new (std::nothrow) tk_solver();
    if (!S) return fail(nullptr, TK_ERR_OOM, "tk_make_grid: host allocation failed");
    cudaError_t e = cudaGetDevice(&S->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&S->num_sms, cudaDevAttrMultiProcessorCount, S->device);
    if (e != cudaSuccess) {
        fail(nullptr, TK_ERR_CUDA, "tk_make_grid: %s", cudaGetErrorString(e));
        delete S;
        return TK_ERR_CUDA;
    }
    S->stream = (cudaStream_t)cuda_stream;
    S->Nr = Nr;
    S->Nth = Ntheta;
    S->K = Ntheta <= 32 ? 1 : (Ntheta <= 64 ? 2 : 4);
    S->NP = 32 * S->K;
    S->auto_k = (substeps == 0);
    S->substeps = substeps == 0 ? 1 : substeps;
    S->variable = angular_variable;
    S->precision = precision;
    S->esz = precision == TK_PREC_F64 ? sizeof(double) : sizeof(float);
    S->rs_min = rstar_min;
    S->rs_max = rstar_max;
    S->drs = (rstar_max - rstar_min) / (Nr - 1);
    S->dt = dt;
    S->blocks = tk::step_grid_shape(precision, S->K, Nr, S->num_sms, &S->warps);
    S->adj_blocks = tk::adjoint_grid_shape(precision, S->K, Nr, S->num_sms, &S->adj_warps);
    S->fused_blocks = tk::fused_grid_shape(precision, S->K, Nr, S->num_sms, &S->fused_warps);
    // the persistent launch: FP64 runs the one-step kernel's grid, FP32 the
    // two-step (ring) kernel's, both one wave of resident blocks
    S->persist_blocks = (precision == TK_PREC_F32)
                            ? S->fused_blocks
                            : tk::persistent_grid_blocks(precision, S->K, Nr, S->num_sms, S->warps);
    S->multi_blocks = tk::multi_grid_shape(precision, S->K, Nr, S->num_sms, &S->multi_warps);
    set_launch_mode(S, 0);

    const size_t se = state_elems(S);
    tk_status st = TK_OK;
    if (st == TK_OK) st = alloc(S, &S->u[0], se * S->esz);
    if (st == TK_OK) st = alloc(S, &S->u[1], se * S->esz);
    if (st == TK_OK) st = alloc(S, &S->half, (size_t)Nr * tk::kNCH * S->NP * S->esz);
    if (st == TK_OK) st = alloc(S, &S->node, (size_t)Nr * tk::kNCN * S->NP * S->esz);
    if (st == TK_OK && precision == TK_PREC_F32)
        st = alloc(S, (void **)&S->cmp, (size_t)Nr * tk::kNCC * S->NP * sizeof(float));
    if (st == TK_OK && precision == TK_PREC_F32)
        st = alloc(S, (void **)&S->gpm, (size_t)2 * S->NP * sizeof(float));
    if (st == TK_OK) st = alloc(S, (void **)&S->b_node, (size_t)Nr * S->NP * sizeof(double));
    if (st == TK_OK) st = alloc(S, (void **)&S->w_row, (size_t)S->NP * sizeof(double));
    if (st == TK_OK) st = alloc(S, (void **)&S->x_node, (size_t)Nr * sizeof(double));
    if (st == TK_OK) st = alloc(S, (void **)&S->x_half, (size_t)Nr * sizeof(double));
    if (st == TK_OK) st = alloc(S, (void **)&S->ang, (size_t)2 * S->NP * sizeof(double));
    if (st == TK_OK) st = alloc(S, (void **)&S->flag, sizeof(int));
    if (st == TK_OK) st = alloc(S, (void **)&S->stiff, 2 * sizeof(unsigned long long));
    if (st == TK_OK) st = alloc(S, (void **)&S->ctr, 2 * sizeof(long long));
    if (st != TK_OK) {
        snprintf(g_err, sizeof g_err, "%s", S->err);
        release(S);
        delete S;
        return st;
    }
    e = cudaMemsetAsync(S->u[0], 0, se * S->esz, S->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->u[1], 0, se * S->esz, S->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->ctr, 0, 2 * sizeof(long long), S->stream);
    if (e != cudaSuccess) {
        fail(nullptr, TK_ERR_CUDA, "tk_make_grid: %s", cudaGetErrorString(e));
        release(S);
        delete S;
        return TK_ERR_CUDA;
    }
    *out = S;
    return TK_OK;
}

tk_status tk_precompute_coeffs(tk_solver *S, double a, double M, int s, int m)
{
    tk_status st = enter(S);
    if (st != TK_OK) return st;
    if (!(M > 0) || !isfinite(M) || !(fabs(a) < M))
        return fail(S, TK_ERR_ARG, "tk_precompute_coeffs: need M > 0 and |a| < M (a=%g, M=%g)", a, M);
    if (abs(s) > 4 || abs(m) > 64)
        return fail(S, TK_ERR_ARG, "tk_precompute_coeffs: |s| <= 4 and |m| <= 64 required");
    S->kerr.M = M;
    S->kerr.a = a;
    S->kerr.s = s;
    S->kerr.m = m;
    if (S->auto_k) S->substeps = 1;
    TK_CUDA(S, tk::launch_invert_tortoise(S->kerr, S->rs_min, S->drs, S->Nr, S->x_node, S->x_half,
                                          S->stream));
    TK_CUDA(S, tk::launch_coeff_tables(S->kerr, S->variable, S->Nr, S->Nth, S->NP, S->drs,
                                       S->dt / S->substeps, S->x_node, S->x_half, S->ang,
                                       S->precision, S->half, S->node, S->b_node, S->w_row,
                                       S->cmp, S->gpm, S->stream));
    S->have_coeffs = true;
    S->have_state = false;
    S->epoch++;   // the tables' time step may have changed: recapture graphs
    if (S->auto_k) {
        // substeps from the stability bound at the default growth per step,
        // then the tables again with the inner step it gives
        double dt_max = 0.0;
        int k = 1;
        st = tk_stability_bound(S, kAutoGrowthPerStep, &dt_max, &k);
        if (st != TK_OK) {
            S->have_coeffs = false;
            return st;
        }
        if (k != 1) {
            S->substeps = k;
            TK_CUDA(S, tk::launch_coeff_tables(S->kerr, S->variable, S->Nr, S->Nth, S->NP, S->drs,
                                               S->dt / S->substeps, S->x_node, S->x_half, S->ang,
                                               S->precision, S->half, S->node, S->b_node,
                                               S->w_row, S->cmp, S->gpm, S->stream));
        }
    }
    return TK_OK;
}

tk_status tk_set_coefficients(tk_solver *S, double a, double M, int s, int m, const double *node9,
                              const double *half9, const double *ang2, int on_device)
{
    tk_status st = enter(S);
    if (st != TK_OK) return st;
    if (!(M > 0) || !isfinite(M) || !(fabs(a) < M))
        return fail(S, TK_ERR_ARG, "tk_set_coefficients: need M > 0 and |a| < M (a=%g, M=%g)", a, M);
    if (abs(s) > 4 || abs(m) > 64)
        return fail(S, TK_ERR_ARG, "tk_set_coefficients: |s| <= 4 and |m| <= 64 required");
    if (!node9 || !half9) return fail(S, TK_ERR_ARG, "tk_set_coefficients: node9/half9 are NULL");
    if (S->auto_k)
        return fail(S, TK_ERR_STATE, "tk_set_coefficients: the solver chooses its own substeps; "
                                     "make the grid with substeps > 0");
    S->kerr.M = M;
    S->kerr.a = a;
    S->kerr.s = s;
    S->kerr.m = m;
    const size_t n9 = (size_t)9 * S->Nth * S->Nr;
    double *dev = nullptr;   // node9, half9, ang2 on the device (copies of host inputs)
    const double *dn = node9, *dh = half9;
    if (!on_device) {
        st = alloc(S, (void **)&dev, 2 * n9 * sizeof(double));
        if (st != TK_OK) return st;
        cudaError_t e = cudaMemcpyAsync(dev, node9, n9 * sizeof(double), cudaMemcpyHostToDevice, S->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dev + n9, half9, n9 * sizeof(double), cudaMemcpyHostToDevice, S->stream);
        if (e != cudaSuccess) {
            cudaFree(dev);
            return fail(S, TK_ERR_CUDA, "tk_set_coefficients: %s", cudaGetErrorString(e));
        }
        dn = dev;
        dh = dev + n9;
    }
    cudaError_t e = cudaSuccess;
    const bool ang_given = (ang2 != nullptr) && S->variable != 0;
    if (ang_given) {
        // [2][Ntheta] -> the device layout [2][NP], padding rows zero
        e = cudaMemsetAsync(S->ang, 0, (size_t)2 * S->NP * sizeof(double), S->stream);
        for (int k = 0; k < 2 && e == cudaSuccess; ++k)
            e = cudaMemcpyAsync(S->ang + (size_t)k * S->NP, ang2 + (size_t)k * S->Nth, S->Nth * sizeof(double),
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, S->stream);
    }
    if (e == cudaSuccess)
        e = tk::launch_invert_tortoise(S->kerr, S->rs_min, S->drs, S->Nr, S->x_node, S->x_half, S->stream);
    if (e == cudaSuccess)
        e = tk::launch_coeff_tables(S->kerr, S->variable, S->Nr, S->Nth, S->NP, S->drs, S->dt / S->substeps,
                                    S->x_node, S->x_half, S->ang, S->precision, S->half, S->node, S->b_node,
                                    S->w_row, S->cmp, S->gpm, S->stream, dn, dh, ang_given);
    if (e == cudaSuccess && dev) e = cudaStreamSynchronize(S->stream);
    if (dev) cudaFree(dev);
    if (e != cudaSuccess) return fail(S, TK_ERR_CUDA, "tk_set_coefficients: %s", cudaGetErrorString(e));
    S->have_coeffs = true;
    S->have_state = false;
    S->epoch++;
    return TK_OK;
}

tk_status tk_get_coefficients(tk_solver *S, double *node9, double *half9, int on_device)
{
    tk_status st = enter(S);
    if (st != TK_OK) return st;
    if (!S->have_coeffs) return fail(S, TK_ERR_STATE, "tk_get_coefficients before tk_precompute_coeffs");
    if (!node9 || !half9) return fail(S, TK_ERR_ARG, "tk_get_coefficients: node9/half9 are NULL");
    const size_t n9 = (size_t)9 * S->Nth * S->Nr;
    if (on_device) {
        TK_CUDA(S, tk::launch_raw_export(S->kerr, S->variable, S->Nr, S->Nth, S->x_node, S->x_half, node9,
                                         half9, S->stream));
        return TK_OK;
    }
    double *dev = nullptr;
    st = alloc(S, (void **)&dev, 2 * n9 * sizeof(double));
    if (st != TK_OK) return st;
    cudaError_t e = tk::launch_raw_export(S->kerr, S->variable, S->Nr, S->Nth, S->x_node, S->x_half, dev,
                                          dev + n9, S->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(node9, dev, n9 * sizeof(double), cudaMemcpyDeviceToHost, S->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(half9, dev + n9, n9 * sizeof(double), cudaMemcpyDeviceToHost, S->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
    cudaFree(dev);
    if (e != cudaSuccess) return fail(S, TK_ERR_CUDA, "tk_get_coefficients: %s", cudaGetErrorString(e));
    return TK_OK;
}

tk_status tk_get_substeps(const tk_solver *S, int *substeps)
{
    if (!S || !substeps) return fail(nullptr, TK_ERR_ARG, "tk_get_substeps: NULL argument");
    *substeps = S->substeps;
    return TK_OK;
}

tk_status tk_get_steps_per_launch(const tk_solver *S, int *steps)
{
    if (!S || !steps) return fail(nullptr, TK_ERR_ARG, "tk_get_steps_per_launch: NULL argument");
    *steps = S->persist ? -1 : (S->fuse ? 2 : 1);
    return TK_OK;
}

static tk_status import_planes(tk_solver *S, const double *pr, const double *pi, const double *qr,
                               const double *qi, int on_device)
{
    const size_t plane = (size_t)S->Nth * S->Nr;
    if (!on_device) {
        tk_status st = ensure_staging(S);
        if (st != TK_OK) return st;
        const double *src[4] = {pr, pi, qr, qi};
        for (int c = 0; c < 4; ++c)
            if (src[c])
                TK_CUDA(S, cudaMemcpyAsync(S->staging + c * plane, src[c], plane * sizeof(double),
                                           cudaMemcpyHostToDevice, S->stream));
        // the caller's host buffers may be reused as soon as this call returns
        TK_CUDA(S, cudaStreamSynchronize(S->stream));
        pr = S->staging;
        pi = S->staging + plane;
        qr = qr ? S->staging + 2 * plane : nullptr;
        qi = qi ? S->staging + 3 * plane : nullptr;
    }
    void *dst = S->u[S->cur];
    TK_CUDA(S, tk::launch_import_state(S->precision, S->Nr, S->Nth, S->NP, S->drs, pr, pi, qr, qi,
                                       S->b_node, dst, S->stream));
    return TK_OK;
}

tk_status tk_set_initial_data(tk_solver *S, const double *phi_re, const double *phi_im,
                              const double *pi_re, const double *pi_im, int on_device)
{
    tk_status st = enter(S);
    if (st != TK_OK) return st;
    if (!S->have_coeffs) return fail(S, TK_ERR_STATE, "tk_set_initial_data before tk_precompute_coeffs");
    if (!phi_re || !phi_im) return fail(S, TK_ERR_ARG, "tk_set_initial_data: phi planes are NULL");
    if ((pi_re == nullptr) != (pi_im == nullptr))
        return fail(S, TK_ERR_ARG, "tk_set_initial_data: give both pi planes or neither");
    st = import_planes(S, phi_re, phi_im, pi_re, pi_im, on_device);
    if (st != TK_OK) return st;
    TK_CUDA(S, cudaMemsetAsync(S->ctr, 0, 2 * sizeof(long long), S->stream));
    // keep u^0 (FP64) for the parameter gradients, which recompute the trajectory
    S->init_valid = false;
    if (S->precision == TK_PREC_F64) {
        const size_t bytes = state_elems(S) * S->esz;
        if (!S->u_init) {
            st = alloc(S, &S->u_init, bytes);
            if (st != TK_OK) return st;
        }
        TK_CUDA(S, cudaMemcpyAsync(S->u_init, S->u[S->cur], bytes, cudaMemcpyDeviceToDevice, S->stream));
        S->init_valid = true;
        S->init_pi_derived = (pi_re == nullptr);
    }
    S->have_state = true;
    S->state_valid = true;
    S->count = 0;
    S->steps_done = 0;
    return TK_OK;
}

tk_status tk_set_initial_gaussian(tk_solver *S, double amp, double center, double width,
                                  double noise_amp, uint64_t seed)
{
    tk_status st = enter(S);
    if (st != TK_OK) return st;
    if (!S->have_coeffs)
        return fail(S, TK_ERR_STATE, "tk_set_initial_gaussian before tk_precompute_coeffs");
    if (!isfinite(amp) || !isfinite(center) || !(width > 0.0) || !isfinite(width) ||
        !(noise_amp >= 0.0) || !isfinite(noise_amp))
        return fail(S, TK_ERR_ARG, "tk_set_initial_gaussian: need finite amp and centre, width > 0, "
                                   "noise_amp >= 0");
    st = ensure_staging(S);
    if (st != TK_OK) return st;
    const size_t plane = (size_t)S->Nth * S->Nr;
    TK_CUDA(S, tk::launch_gaussian(S->Nr, S->Nth, S->rs_min, S->drs, amp, center, width, noise_amp,
                                   (unsigned long long)seed, S->staging, S->staging + plane,
                                   S->stream));
    return tk_set_initial_data(S, S->staging, S->staging + plane, nullptr, nullptr, 1);
}

tk_status tk_add_observer(tk_solver *S, double rstar_obs, double theta_obs, int *obs_id)
{
    tk_status st = enter(S);
    if (st != TK_OK) return st;
    if (!obs_id) return fail(S, TK_ERR_ARG, "tk_add_observer: obs_id is NULL");
    if (S->count > 0)
        return fail(S, TK_ERR_STATE, "tk_add_observer: samples already taken; add observers "
                                     "before the first tk_step after tk_set_initial_data");
    if (S->nobs >= tk::kMaxObservers)
        return fail(S, TK_ERR_ARG, "tk_add_observer: at most %d observers", tk::kMaxObservers);
    const double dth = M_PI / S->Nth;
    const double fi = (rstar_obs - S->rs_min) / S->drs;
    const double fj = theta_obs / dth - 0.5;
    if (!(fi >= 0.0) || fi > S->Nr - 1 || !(fj >= 0.0) || fj > S->Nth - 1)
        return fail(S, TK_ERR_ARG, "tk_add_observer: (%g, %g) outside the grid", rstar_obs, theta_obs);
    int i0 = (int)floor(fi), j0 = (int)floor(fj);
    if (i0 > S->Nr - 2) i0 = S->Nr - 2;
    if (j0 > S->Nth - 2) j0 = S->Nth - 2;
    tk_solver::Obs &o = S->obs[S->nobs];
    o.rs = rstar_obs;
    o.th = theta_obs;
    o.i0 = i0;
    o.j0 = j0;
    o.fr = fi - i0;
    o.ft = fj - j0;
    *obs_id = S->nobs++;
    S->epoch++;
    return TK_OK;
}

// Enqueue `outer` outer steps starting from level `cur` on stream `st`;
// returns the level holding the result.  Inner steps run one per launch, or
// in pairs through the two-step kernel when S->fuse; an outer step that ends
// inside a pair is observed there (obs_mask).  Calls start on an outer-step
// boundary, so the inner index t counts from one.
static cudaError_t enqueue_steps(const tk_solver *S, int cur, int outer, cudaStream_t st, int *cur_out)
{
    tk::StepLaunch L;
    tkh::fill_launch(S, L);
    const long long k = S->substeps, total = (long long)outer * k;
    for (long long t = 0; t < total;) {
        L.u_in = S->u[cur];
        L.u_out = S->u[cur ^ 1];
        if (S->fuse && t + 1 < total) {
            L.fused = 1;
            L.blocks = S->fused_blocks;
            L.warps = S->fused_warps;
            L.obs_mask = ((t + 1) % k == 0 ? 1 : 0) | ((t + 2) % k == 0 ? 2 : 0);
            L.write_wave = L.obs_mask != 0 && S->nobs > 0;
            t += 2;
        } else {
            L.fused = 0;
            L.blocks = S->blocks;
            L.warps = S->warps;
            L.obs_mask = 0;
            L.write_wave = (t + 1) % k == 0 && S->nobs > 0;
            t += 1;
        }
        cudaError_t e = tk::launch_lw_step(L, st);
        if (e != cudaSuccess) return e;
        cur ^= 1;
    }
    *cur_out = cur;
    return cudaSuccess;
}

// Outer steps per captured graph: an even number of launches per replay keeps
// the ping-pong level fixed, and with two-step launches the chunk holds whole
// pairs (inner steps a multiple of four).
static int graph_chunk(const tk_solver *S)
{
    int c;
    if (S->graph_chunk >= 0) {
        c = S->graph_chunk;
        if (c == 0) return 0;
    } else {
        // automatic: about 64 launches per replay
        const int per = S->fuse ? (S->substeps + 1) / 2 : S->substeps;
        c = (64 + per - 1) / per;
    }
    const int mult = S->fuse ? 4 : 2;
    while (((long long)c * S->substeps) % mult) ++c;
    return c;
}

static tk_status get_graph(tk_solver *S, int chunk, cudaGraphExec_t *out)
{
    const int p = S->cur;
    if (S->graph[p] && S->graph_epoch[p] == S->epoch && S->graph_outer[p] == chunk) {
        *out = S->graph[p];
        return TK_OK;
    }
    if (S->graph[p]) {
        cudaGraphExecDestroy(S->graph[p]);
        S->graph[p] = nullptr;
    }
    if (!S->capture_stream)
        TK_CUDA(S, cudaStreamCreateWithFlags(&S->capture_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    TK_CUDA(S, cudaStreamBeginCapture(S->capture_stream, cudaStreamCaptureModeThreadLocal));
    int cur_after = p;
    cudaError_t e = enqueue_steps(S, p, chunk, S->capture_stream, &cur_after);
    cudaError_t e2 = cudaStreamEndCapture(S->capture_stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && cur_after != p) e = cudaErrorInvalidValue;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&S->graph[p], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        S->graph[p] = nullptr;
        return fail(S, TK_ERR_CUDA, "tk_step: graph capture failed: %s", cudaGetErrorString(e));
    }
    S->graph_epoch[p] = S->epoch;
    S->graph_outer[p] = chunk;
    *out = S->graph[p];
    return TK_OK;
}

tk_status tk_step(tk_solver *S, int n)
{
    tk_status st = enter(S);
    if (st != TK_OK) return st;
    st = need_state(S, "tk_step");
    if (st != TK_OK) return st;
    if (n < 0) return fail(S, TK_ERR_ARG, "tk_step: n = %d < 0", n);
    if (n == 0) return TK_OK;
    st = ensure_wave(S, S->count + n);
    if (st != TK_OK) return st;
    if (S->persist && (long long)n * S->substeps >= 2) {
        // every inner step of the call in one cooperative launch; its waits
        // are bounded, and a wait that timed out is reported here
        // the one-step sweep keeps two flags per block (its first and last warp)
        const int nflags = 2 * S->persist_blocks > S->multi_blocks ? 2 * S->persist_blocks : S->multi_blocks;
        const size_t fbytes = (size_t)nflags * sizeof(unsigned int) + sizeof(int);
        if (!S->pflags) {
            st = alloc(S, (void **)&S->pflags, fbytes);
            if (st != TK_OK) return st;
        }
        int *perr = (int *)(S->pflags + nflags);
        TK_CUDA(S, cudaMemsetAsync(S->pflags, 0, fbytes, S->stream));
        tk::StepLaunch L;
        tkh::fill_launch(S, L);
        L.blocks = S->persist_blocks;
        L.warps = S->precision == TK_PREC_F32 ? S->fused_warps : S->warps;
        L.u_in = S->u[S->cur];
        L.write_wave = S->nobs > 0;
        const long long inner = (long long)n * S->substeps;
        if (inner > 0x7fffffff) return fail(S, TK_ERR_ARG, "tk_step: %d outer steps are too many for one call", n);
        if (S->precision == TK_PREC_F32) {
            // groups of tk::multi_levels() steps per sweep in one launch (large
            // grids), ending on an outer step's boundary; the rest as pairs of
            // steps in one launch and an odd last step by the one-step kernel
            long long rem = inner;
            int obs_i0[tk::kMaxObservers];
            for (int o = 0; o < S->nobs; ++o) obs_i0[o] = S->obs[o].i0;
            if (S->multi_blocks > 0 &&
                tk::multi_obs_fit(S->Nr, S->multi_blocks, S->multi_warps, obs_i0, S->nobs)) {
                const int lv = tk::multi_levels();
                long long unit = S->substeps;   // groups per run of whole outer steps
                for (int d = lv; d > 1; --d)
                    if (lv % d == 0 && unit % d == 0) {
                        unit /= d;
                        break;
                    }
                const long long groups = rem / lv / unit * unit;
                if (groups > 0 && !S->obs_scr) {
                    st = alloc(S, &S->obs_scr, tk::multi_obs_scratch_bytes(S->K, S->multi_blocks, S->multi_warps));
                    if (st != TK_OK) return st;
                }
                if (groups > 0) {
                    tk::StepLaunch LM = L;
                    LM.blocks = S->multi_blocks;
                    LM.warps = S->multi_warps;
                    TK_CUDA(S, tk::launch_multi_persistent(LM, S->u[S->cur ^ 1], (int)groups, S->substeps,
                                                           S->pflags, perr, S->obs_scr, S->stream));
                    if (groups & 1) S->cur ^= 1;
                    rem -= groups * lv;
                    L.u_in = S->u[S->cur];
                    // the flags count again from zero; the error flag is kept
                    TK_CUDA(S, cudaMemsetAsync(S->pflags, 0, (size_t)nflags * sizeof(unsigned int), S->stream));
                }
            }
            const long long pairs = rem / 2;
            if (pairs > 0) {
                TK_CUDA(S, tk::launch_ring_persistent(L, S->u[S->cur ^ 1], (int)pairs, S->substeps, S->pflags,
                                                      perr, S->stream));
                if (pairs & 1) S->cur ^= 1;
            }
            if (rem & 1) {
                tk::StepLaunch L1;
                tkh::fill_launch(S, L1);
                L1.u_in = S->u[S->cur];
                L1.u_out = S->u[S->cur ^ 1];
                L1.write_wave = S->nobs > 0;
                TK_CUDA(S, tk::launch_lw_step(L1, S->stream));
                S->cur ^= 1;
            }
        } else {
            TK_CUDA(S, tk::launch_lw_persistent(L, S->u[S->cur ^ 1], (int)inner, S->substeps, S->pflags,
                                                perr, S->stream));
            if (inner & 1) S->cur ^= 1;
        }
        int herr = 0;
        TK_CUDA(S, cudaMemcpyAsync(&herr, perr, sizeof(int), cudaMemcpyDeviceToHost, S->stream));
        TK_CUDA(S, cudaStreamSynchronize(S->stream));
        if (S->inject_wait_timeout) {
            S->inject_wait_timeout = false;
            herr = 1;
        }
        if (herr) {
            // the samples before this call stay valid: put the device sample
            // counter back where this call found it and keep the host counts;
            // the state is invalid until it is set again
            long long h[2] = {(long long)S->count, 0};
            TK_CUDA(S, cudaMemcpyAsync(S->ctr, h, sizeof h, cudaMemcpyHostToDevice, S->stream));
            TK_CUDA(S, cudaStreamSynchronize(S->stream));
            S->state_valid = false;
            S->init_valid = false;
            return fail(S, TK_ERR_INTERNAL, "tk_step: a block of the persistent launch waited too long "
                                            "for its neighbours; the state is invalid");
        }
        S->count += n;
        S->steps_done += n;
        return TK_OK;
    }
    const int chunk = graph_chunk(S);
    while (chunk > 0 && n >= chunk) {
        cudaGraphExec_t ge = nullptr;
        st = get_graph(S, chunk, &ge);
        if (st != TK_OK) return st;
        TK_CUDA(S, cudaGraphLaunch(ge, S->stream));
        S->count += chunk;
        S->steps_done += chunk;
        n -= chunk;
    }
    if (n > 0) {
        int cur = S->cur;
        TK_CUDA(S, enqueue_steps(S, S->cur, n, S->stream, &cur));
        S->cur = cur;
        S->count += n;
        S->steps_done += n;
    }
    return TK_OK;
}

tk_status tk_set_steps_per_launch(tk_solver *S, int steps)
{
    tk_status st = enter(S);
    if (st != TK_OK) return st;
    if (steps < -1 || steps > 2)
        return fail(S, TK_ERR_ARG, "tk_set_steps_per_launch: %d is not -1, 0, 1 or 2", steps);
    if (steps == -1 && S->persist_blocks == 0)
        return fail(S, TK_ERR_ARG, "tk_set_steps_per_launch: this grid cannot run as one "
                                   "persistent launch");
    set_launch_mode(S, steps);
    S->epoch++;
    return TK_OK;
}

tk_status tk_set_graph_chunk(tk_solver *S, int outer_steps)
{
    tk_status st = enter(S);
    if (st != TK_OK) return st;
    if (outer_steps < -1) return fail(S, TK_ERR_ARG, "tk_set_graph_chunk: %d < -1", outer_steps);
    S->graph_chunk = outer_steps;
    S->epoch++;
    return TK_OK;
}

tk_status tk_extract(tk_solver *S, int obs_id, double *re, double *im, int capacity, int *count,
                     int on_device)
{
    tk_status st = enter(S);
    if (st != TK_OK) return st;
    if (obs_id < 0 || obs_id >= S->nobs) return fail(S, TK_ERR_ARG, "tk_extract: bad observer id %d", obs_id);
    if (capacity < 0) return fail(S, TK_ERR_ARG, "tk_extract: capacity < 0");
    if (capacity > 0 && (!re || !im)) return fail(S, TK_ERR_ARG, "tk_extract: re/im NULL");
    if (count) *count = (int)S->count;
    const int64_t n = capacity < S->count ? capacity : S->count;
    if (n <= 0) return TK_OK;
    const double *src = S->wave + (size_t)obs_id * S->wave_cap * 4;
    const tk::WaveRead rd = tkh::wave_read(S, obs_id);
    if (on_device) {
        TK_CUDA(S, tk::launch_wave_sum(src, 0, n, rd, re, im, S->stream));
        return TK_OK;
    }
    // host read-out through a device buffer the solver keeps (sized to the
    // waveform buffer's capacity, reallocated only when that grows)
    if (S->xbuf_cap < S->wave_cap) {
        if (S->xbuf) {
            TK_CUDA(S, cudaStreamSynchronize(S->stream));
            cudaFree(S->xbuf);
            S->xbuf = nullptr;
            S->xbuf_cap = 0;
        }
        st = alloc(S, (void **)&S->xbuf, (size_t)2 * S->wave_cap * sizeof(double));
        if (st != TK_OK) return st;
        S->xbuf_cap = S->wave_cap;
    }
    double *tmp = S->xbuf;
    TK_CUDA(S, tk::launch_wave_sum(src, 0, n, rd, tmp, tmp + n, S->stream));
    TK_CUDA(S, cudaMemcpyAsync(re, tmp, n * sizeof(double), cudaMemcpyDeviceToHost, S->stream));
    TK_CUDA(S, cudaMemcpyAsync(im, tmp + n, n * sizeof(double), cudaMemcpyDeviceToHost, S->stream));
    TK_CUDA(S, cudaStreamSynchronize(S->stream));
    return TK_OK;
}

tk_status tk_inject_wait_timeout(tk_solver *S)
{
    tk_status st = enter(S);
    if (st != TK_OK) return st;
    S->inject_wait_timeout = true;
    return TK_OK;
}

tk_status tk_get_state(tk_solver *S, double *planes4, int on_device)
{
    tk_status st = enter(S);
    if (st != TK_OK) return st;
    st = need_state(S, "tk_get_state");
    if (st != TK_OK) return st;
    if (!planes4) return fail(S, TK_ERR_ARG, "tk_get_state: planes4 is NULL");
    if (on_device) {
        TK_CUDA(S, tk::launch_export_state(S->precision, S->Nr, S->Nth, S->NP, S->u[S->cur], planes4,
                                           S->stream));
        return TK_OK;
    }
    st = ensure_staging(S);
    if (st != TK_OK) return st;
    TK_CUDA(S, tk::launch_export_state(S->precision, S->Nr, S->Nth, S->NP, S->u[S->cur], S->staging,
                                       S->stream));
    TK_CUDA(S, cudaMemcpyAsync(planes4, S->staging, (size_t)4 * S->Nth * S->Nr * sizeof(double),
                               cudaMemcpyDeviceToHost, S->stream));
    TK_CUDA(S, cudaStreamSynchronize(S->stream));
    return TK_OK;
}

tk_status tk_set_state(tk_solver *S, const double *planes4, int on_device)
{
    tk_status st = enter(S);
    if (st != TK_OK) return st;
    if (!S->have_state) return fail(S, TK_ERR_STATE, "tk_set_state before tk_set_initial_data");
    if (!planes4) return fail(S, TK_ERR_ARG, "tk_set_state: planes4 is NULL");
    const size_t plane = (size_t)S->Nth * S->Nr;
    S->init_valid = false;   // the trajectory no longer starts from the stored u^0
    st = import_planes(S, planes4, planes4 + plane, planes4 + 2 * plane, planes4 + 3 * plane, on_device);
    if (st == TK_OK) S->state_valid = true;
    return st;
}

tk_status tk_stability_bound(tk_solver *S, double growth_per_step, double *dt_max,
                             int *substeps_needed)
{
    tk_status st = enter(S);
    if (st != TK_OK) return st;
    if (!S->have_coeffs) return fail(S, TK_ERR_STATE, "tk_stability_bound before tk_precompute_coeffs");
    if (!dt_max || !substeps_needed) return fail(S, TK_ERR_ARG, "tk_stability_bound: NULL output");
    if (!(growth_per_step > 0.0) || !(growth_per_step < 1.0))
        return fail(S, TK_ERR_ARG, "tk_stability_bound: growth_per_step must be in (0, 1)");
    unsigned long long h[2] = {0, 0};
    TK_CUDA(S, tk::launch_stiffness(S->kerr, S->variable, S->Nr, S->Nth, S->NP, S->x_node, S->ang,
                                    S->stiff, S->stream));
    TK_CUDA(S, cudaMemcpyAsync(h, S->stiff, sizeof h, cudaMemcpyDeviceToHost, S->stream));
    TK_CUDA(S, cudaStreamSynchronize(S->stream));
    double w2, bmax;
    memcpy(&w2, &h[0], sizeof w2);
    memcpy(&bmax, &h[1], sizeof bmax);
    // radial CFL of the Lax-Wendroff scheme: b dt / dr* <= 1
    double dt = bmax > 0.0 ? S->drs / bmax : INFINITY;
    // angular source term: per step the fastest mode grows by ~ (omega dt)^4 / 8
    const double zmax = pow(8.0 * growth_per_step, 0.25);
    if (w2 > 0.0) dt = fmin(dt, zmax / sqrt(w2));
    *dt_max = dt;
    const double k = ceil(S->dt / dt * (1.0 - 1e-12));
    *substeps_needed = k < 1.0 ? 1 : (k > 1e9 ? 1000000000 : (int)k);
    return TK_OK;
}

tk_status tk_steps_done(const tk_solver *S, int64_t *steps)
{
    if (!S || !steps) return fail(nullptr, TK_ERR_ARG, "tk_steps_done: NULL argument");
    *steps = S->steps_done;
    return TK_OK;
}

tk_status tk_check_finite(tk_solver *S)
{
    tk_status st = enter(S);
    if (st != TK_OK) return st;
    st = need_state(S, "tk_check_finite");
    if (st != TK_OK) return st;
    int h = 0;
    TK_CUDA(S, cudaMemsetAsync(S->flag, 0, sizeof(int), S->stream));
    TK_CUDA(S, tk::launch_finite_check(S->precision, state_elems(S), S->u[S->cur], S->flag, S->stream));
    TK_CUDA(S, cudaMemcpyAsync(&h, S->flag, sizeof(int), cudaMemcpyDeviceToHost, S->stream));
    TK_CUDA(S, cudaStreamSynchronize(S->stream));
    if (h) return fail(S, TK_ERR_UNSTABLE, "non-finite value in the state after %lld steps",
                       (long long)S->steps_done);
    return TK_OK;
}

tk_status tk_synchronize(tk_solver *S)
{
    tk_status st = enter(S);
    if (st != TK_OK) return st;
    TK_CUDA(S, cudaStreamSynchronize(S->stream));
    return TK_OK;
}

tk_status tk_check_bounded_wait(int n_blocks, int silent, int64_t max_polls, int *timed_out)
{
    if (n_blocks < 2 || n_blocks > 64 || silent < -1 || silent >= n_blocks || max_polls < 1 || !timed_out) {
        snprintf(g_err, sizeof g_err, "tk_check_bounded_wait: bad arguments");
        return TK_ERR_ARG;
    }
    unsigned int *flags = nullptr;
    const size_t bytes = (size_t)n_blocks * sizeof(unsigned int) + 3 * sizeof(int);
    cudaError_t e = cudaMalloc((void **)&flags, bytes);
    if (e == cudaSuccess) e = cudaMemset(flags, 0, bytes);
    // [0] the blocks' neighbour barrier, [1] a warp on a global flag, [2] a
    // warp on a shared-memory counter
    int *err = (int *)(flags + n_blocks);
    if (e == cudaSuccess) e = tk::launch_wait_check(n_blocks, silent, (long long)max_polls, flags, err, 0);
    int h[3] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(h, err, sizeof h, cudaMemcpyDeviceToHost);
    if (flags) cudaFree(flags);
    if (e != cudaSuccess) {
        snprintf(g_err, sizeof g_err, "tk_check_bounded_wait: %s", cudaGetErrorString(e));
        return TK_ERR_CUDA;
    }
    const int n_out = (h[0] != 0) + (h[1] != 0) + (h[2] != 0);
    if (n_out != 0 && n_out != 3) {
        snprintf(g_err, sizeof g_err, "tk_check_bounded_wait: only some waits ran out (%d %d %d)", h[0] != 0,
                 h[1] != 0, h[2] != 0);
        return TK_ERR_INTERNAL;
    }
    *timed_out = n_out == 3;
    return TK_OK;
}

const char *tk_last_error(const tk_solver *S) { return S ? S->err : g_err; }

void tk_destroy(tk_solver *S)
{
    if (!S) return;
    cudaSetDevice(S->device);
    cudaStreamSynchronize(S->stream);
    release(S);
    delete S;
}

}  // extern "C"
