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
    double *b_node = nullptr, *w_row = nullptr, *x_node = nullptr, *x_half = nullptr;
    double *ang = nullptr;      // regularised angular stencil [2][NP]
    double *staging = nullptr;  // 4 * Nth * Nr doubles, for host transfers
    int *flag = nullptr;
    // physics
    tk::Kerr kerr{};
    bool have_coeffs = false, have_state = false;
    // observers and waveform samples
    struct Obs {
        double rs, th;
        int i0, j0;
        double fr, ft;
    } obs[tk::kMaxObservers];
    int nobs = 0;
    double *wave = nullptr;  // [obs][cap][2 slots][re, im]
    int64_t wave_cap = 0;
    int64_t count = 0;
    int64_t steps_done = 0;
    // launch shape
    int blocks = 1;
    char err[512] = {0};
};

namespace {

thread_local char g_err[512] = "no error";

tk_status fail(tk_solver *S, tk_status st, const char *fmt, ...)
{
    char *buf = S ? S->err : g_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return st;
}

#define TK_CUDA(S, call)                                                                  \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail((S), e_ == cudaErrorMemoryAllocation ? TK_ERR_OOM : TK_ERR_CUDA,  \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

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
                    S->x_node, S->x_half, S->ang, S->staging, S->flag, S->wave};
    for (void *p : ptrs)
        if (p) cudaFree(p);
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
    return TK_OK;
}

tk_status enter(tk_solver *S)
{
    if (!S) return fail(nullptr, TK_ERR_ARG, "null solver");
    TK_CUDA(S, cudaSetDevice(S->device));
    return TK_OK;
}

}  // namespace

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
    S->substeps = substeps == 0 ? 1 : substeps;
    S->variable = angular_variable;
    S->precision = precision;
    S->esz = precision == TK_PREC_F64 ? sizeof(double) : sizeof(float);
    S->rs_min = rstar_min;
    S->rs_max = rstar_max;
    S->drs = (rstar_max - rstar_min) / (Nr - 1);
    S->dt = dt;
    S->blocks = tk::step_grid_blocks(precision, S->K, Nr, S->num_sms);

    const size_t se = state_elems(S);
    tk_status st = TK_OK;
    if (st == TK_OK) st = alloc(S, &S->u[0], se * S->esz);
    if (st == TK_OK) st = alloc(S, &S->u[1], se * S->esz);
    if (st == TK_OK) st = alloc(S, &S->half, (size_t)Nr * tk::kNCH * S->NP * S->esz);
    if (st == TK_OK) st = alloc(S, &S->node, (size_t)Nr * tk::kNCN * S->NP * S->esz);
    if (st == TK_OK) st = alloc(S, (void **)&S->b_node, (size_t)Nr * S->NP * sizeof(double));
    if (st == TK_OK) st = alloc(S, (void **)&S->w_row, (size_t)S->NP * sizeof(double));
    if (st == TK_OK) st = alloc(S, (void **)&S->x_node, (size_t)Nr * sizeof(double));
    if (st == TK_OK) st = alloc(S, (void **)&S->x_half, (size_t)Nr * sizeof(double));
    if (st == TK_OK) st = alloc(S, (void **)&S->ang, (size_t)2 * S->NP * sizeof(double));
    if (st == TK_OK) st = alloc(S, (void **)&S->flag, sizeof(int));
    if (st != TK_OK) {
        snprintf(g_err, sizeof g_err, "%s", S->err);
        release(S);
        delete S;
        return st;
    }
    e = cudaMemsetAsync(S->u[0], 0, se * S->esz, S->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->u[1], 0, se * S->esz, S->stream);
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
    const double dt_in = S->dt / S->substeps;
    TK_CUDA(S, tk::launch_invert_tortoise(S->kerr, S->rs_min, S->drs, S->Nr, S->x_node, S->x_half,
                                          S->stream));
    TK_CUDA(S, tk::launch_coeff_tables(S->kerr, S->variable, S->Nr, S->Nth, S->NP, S->drs, dt_in,
                                       S->x_node, S->x_half, S->ang, S->precision, S->half, S->node,
                                       S->b_node, S->w_row, S->stream));
    S->have_coeffs = true;
    S->have_state = false;
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
    S->have_state = true;
    S->count = 0;
    S->steps_done = 0;
    return TK_OK;
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
    return TK_OK;
}

tk_status tk_step(tk_solver *S, int n)
{
    tk_status st = enter(S);
    if (st != TK_OK) return st;
    if (!S->have_state) return fail(S, TK_ERR_STATE, "tk_step before tk_set_initial_data");
    if (n < 0) return fail(S, TK_ERR_ARG, "tk_step: n = %d < 0", n);
    if (n == 0) return TK_OK;
    st = ensure_wave(S, S->count + n);
    if (st != TK_OK) return st;
    tk::StepLaunch L;
    L.precision = S->precision;
    L.K = S->K;
    L.Nr = S->Nr;
    L.NP = S->NP;
    L.blocks = S->blocks;
    L.dt_inner = S->dt / S->substeps;
    L.half = S->half;
    L.node = S->node;
    L.wave_cap = S->wave_cap;
    L.wave = S->wave;
    L.w_row = S->w_row;
    L.obs.n = S->nobs;
    for (int k = 0; k < S->nobs; ++k) {
        L.obs.i0[k] = S->obs[k].i0;
        L.obs.j0[k] = S->obs[k].j0;
        L.obs.wr0[k] = 1.0 - S->obs[k].fr;
        L.obs.wr1[k] = S->obs[k].fr;
        L.obs.ft[k] = S->obs[k].ft;
    }
    for (int it = 0; it < n; ++it) {
        for (int k = 0; k < S->substeps; ++k) {
            L.u_in = S->u[S->cur];
            L.u_out = S->u[S->cur ^ 1];
            L.write_wave = (k == S->substeps - 1) && S->nobs > 0;
            L.sample = S->count;
            TK_CUDA(S, tk::launch_lw_step(L, S->stream));
            S->cur ^= 1;
        }
        S->count++;
        S->steps_done++;
    }
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
    if (on_device) {
        TK_CUDA(S, tk::launch_wave_sum(src, n, re, im, S->stream));
        return TK_OK;
    }
    double *tmp = nullptr;
    st = alloc(S, (void **)&tmp, (size_t)2 * n * sizeof(double));
    if (st != TK_OK) return st;
    cudaError_t e = tk::launch_wave_sum(src, n, tmp, tmp + n, S->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(re, tmp, n * sizeof(double), cudaMemcpyDeviceToHost, S->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(im, tmp + n, n * sizeof(double), cudaMemcpyDeviceToHost, S->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return fail(S, TK_ERR_CUDA, "tk_extract: %s", cudaGetErrorString(e));
    return TK_OK;
}

tk_status tk_get_state(tk_solver *S, double *planes4, int on_device)
{
    tk_status st = enter(S);
    if (st != TK_OK) return st;
    if (!S->have_state) return fail(S, TK_ERR_STATE, "tk_get_state before tk_set_initial_data");
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
    return import_planes(S, planes4, planes4 + plane, planes4 + 2 * plane, planes4 + 3 * plane, on_device);
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
    if (!S->have_state) return fail(S, TK_ERR_STATE, "tk_check_finite before tk_set_initial_data");
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
