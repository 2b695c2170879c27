/*
 * tk_oracle.c -- plain, slow FP64 CPU reference of the (2+1)D Teukolsky
 * Lax-Wendroff time step (arXiv 1010.3816, Sec. 3).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle against which the CUDA
 * path is checked.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load it.  It shares no code, header, table or constant
 * generator with the CUDA path, and the CUDA path never calls it.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared [-fopenmp]  (no fast-math).
 *
 * What it computes, in the paper's order and notation:
 *   - Eq. 1, the Teukolsky master equation, reduced with the m-mode ansatz of
 *     Eq. 2 (Psi = e^{i m phi} r^3 Phi) to the first-order system
 *         d_t u + D d_{r*} u = S(u),   u = {Phi_R, Phi_I, Pi_R, Pi_I}
 *     with Pi = d_t Phi + b d_{r*} Phi.  The paper defers D and S to its
 *     reference [klpa]; the coefficients below are derived from Eq. 1 itself
 *     (see tko_coeffs_point) and are pinned in the tests by evaluating Eq. 1
 *     on analytic test functions.
 *   - The two-step Lax-Wendroff update, Eq. (lw1) then Eq. (lw2), with the
 *     averaging stage exactly as the paper's kernel_average1 (Sec. 4).
 *   - 2nd-order centred angular differences (Sec. 3.2) on a cell-centred
 *     theta grid: for the literal field the paper's boundary conditions of
 *     Sec. 3.2 are imposed by ghost parity; for the pole-regularised field
 *     the operator is differenced in self-adjoint form, regular at the poles.
 *     Phi = Pi = 0 on both radial edges.
 *   - The tortoise coordinate r*(r) of Kerr (not printed in the paper) and
 *     its inverse; a pole-regularised angular variable Phi = w(theta) Phi^;
 *     initial momentum for zero time derivative; bilinear waveform
 *     extraction.  These readings are listed in the design notes.
 *
 * Parity status: every exported function is pinned by a test against the
 * paper or the mathematics (Eq. 1 residual, discrete angular spectrum,
 * explicit-matrix brute force, 2nd-order convergence, Schwarzschild l=2
 * quasinormal frequency, exact symmetries, closed forms).
 *
 * Array layout follows the paper (Sec. 4): a plane q is indexed
 * idx(b, a) = Nr*b + a with b the theta index and a the r* index.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(b, a) ((size_t)(Nr) * (size_t)(b) + (size_t)(a))

/* ------------------------------------------------------------------------ */
/* Parameters                                                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
    double M, a;        /* black-hole mass and spin parameter (Eq. 1)         */
    int s, m;           /* spin weight and azimuthal mode (Eq. 1, Eq. 2)      */
    double rs_min;      /* first radial node r*_0                             */
    double drs;         /* radial spacing delta r*                            */
    int Nr, Ntheta;     /* grid sizes                                         */
    double dt;          /* outer time step (one waveform sample per outer step)*/
    int substeps;       /* inner Lax-Wendroff steps per outer step (>= 1)     */
    int variable;       /* 0: literal Phi, 1: pole-regularised Phi^ = Phi / w */
} tko_params;

/* Number of coefficient values stored per location: b, c1(R,I), c2(R,I),
 * c3(R,I), c4, c5. */
#define NCOEF 9
enum { K_B = 0, K_C1R, K_C1I, K_C2R, K_C2I, K_C3R, K_C3I, K_C4, K_C5 };

/* ------------------------------------------------------------------------ */
/* Kerr horizons and the tortoise coordinate (never defined in the paper).   */
/* ------------------------------------------------------------------------ */
static void horizons(double M, double a, double *rp, double *rm)
{
    double d = sqrt(M * M - a * a);
    *rp = M + d;
    *rm = M - d;
}

/* r*(r) = r + 2M r+/(r+ - r-) ln((r - r+)/2M) - 2M r-/(r+ - r-) ln((r - r-)/2M),
 * written in terms of x = r - r+ > 0 so that the horizon is never reached by
 * cancellation.  It satisfies d(r*) / dr = (r^2 + a^2)/Delta. */
double tko_tortoise_x(double M, double a, double x)
{
    double rp, rm;
    horizons(M, a, &rp, &rm);
    double r = rp + x;
    double Ap = 2.0 * M * rp / (rp - rm);
    double Am = 2.0 * M * rm / (rp - rm);
    return r + Ap * log(x / (2.0 * M)) - Am * log((r - rm) / (2.0 * M));
}

/* Inverse of the tortoise map: returns x = r - r+ for a given r*.  The map
 * y = ln x -> r*(e^y) is strictly increasing (its derivative is
 * (r^2+a^2)/(r - r-) > 0), so plain bisection in y brackets the root and is
 * run until the bracket cannot shrink further in FP64. */
double tko_x_of_rstar(double M, double a, double rstar)
{
    double ylo = -700.0, yhi = 1.0;
    while (tko_tortoise_x(M, a, exp(yhi)) < rstar) yhi += 1.0;
    for (int it = 0; it < 400; ++it) {
        double ymid = 0.5 * (ylo + yhi);
        if (ymid <= ylo || ymid >= yhi) break;
        if (tko_tortoise_x(M, a, exp(ymid)) < rstar) ylo = ymid; else yhi = ymid;
    }
    /* pick the end of the final bracket whose image is closer to rstar */
    double xlo = exp(ylo), xhi = exp(yhi);
    double elo = fabs(tko_tortoise_x(M, a, xlo) - rstar);
    double ehi = fabs(tko_tortoise_x(M, a, xhi) - rstar);
    return (elo <= ehi) ? xlo : xhi;
}

/* ------------------------------------------------------------------------ */
/* Coefficients of the first-order system (from Eq. 1 and Eq. 2).            */
/* ------------------------------------------------------------------------ */
/* Angular part that depends on the choice of variable.
 *   literal     Phi : g = cot(theta),                        V = V_theta
 *   regularised Phi^: g = cot(theta) + 2(al cot(theta/2) - be tan(theta/2)),
 *                     V = -lambda0
 * with V_theta = -(m + s cos theta)^2 / sin^2 theta + s (the theta-only terms
 * of Eq. 1 after d_phi -> i m), al = |m+s|/2, be = |m-s|/2, and
 * lambda0 = (l0 - s)(l0 + s + 1), l0 = max(|m|, |s|): w = (1-cos)^al (1+cos)^be
 * is the lowest spin-weighted harmonic, (L_theta + V_theta) w = -lambda0 w. */
static void angular_parts(int s, int m, int variable, double th, double *g, double *V)
{
    double c = cos(th), sn = sin(th);
    if (variable == 0) {
        *g = c / sn;
        *V = -(m + s * c) * (m + s * c) / (sn * sn) + s;
    } else {
        double al = 0.5 * fabs((double)(m + s));
        double be = 0.5 * fabs((double)(m - s));
        int l0 = abs(m) > abs(s) ? abs(m) : abs(s);
        double lam0 = (double)(l0 - s) * (double)(l0 + s + 1);
        *g = c / sn + 2.0 * (al / tan(0.5 * th) - be * tan(0.5 * th));
        *V = -lam0;
    }
}

/* Weight w(theta) relating the physical field to the evolved one: Phi = w Phi^
 * (w = 1 for the literal variable).  1 - cos = 2 sin^2(th/2), 1 + cos =
 * 2 cos^2(th/2), written that way to avoid cancellation near the poles. */
double tko_weight(int s, int m, int variable, double th)
{
    if (variable == 0) return 1.0;
    double al = 0.5 * fabs((double)(m + s));
    double be = 0.5 * fabs((double)(m - s));
    double sh = sin(0.5 * th), ch = cos(0.5 * th);
    return pow(2.0 * sh * sh, al) * pow(2.0 * ch * ch, be);
}

/* Coefficients at one point (x = r - r+, theta).  Output order:
 * b, c1R, c1I, c2R, c2I, c3R, c3I, c4, c5 such that
 *   d_t Phi + b d_* Phi                 = Pi
 *   d_t Pi  - b d_* Pi - c1 d_* Phi     = c2 Pi + c3 Phi + c4 d_thth Phi + c5 d_th Phi
 * i.e. D = [[b, 0], [-c1, -b]] (complex blocks) and
 *      S = (Pi, c2 Pi + c3 Phi + c4 d_thth Phi + c5 d_th Phi).
 * Derivation (Eq. 1 times -Delta/(Sigma^2 r^3), Psi = e^{im phi} r^3 Phi,
 * d_* = (Delta/varpi) d_r):
 *   varpi = r^2 + a^2, Delta = x (r - r-), Sigma^2 = varpi^2 - a^2 Delta sin^2,
 *   b = varpi / Sigma,  b_* = d_* b,
 *   f_* / f = 3 Delta/(r varpi),  f_** / f = (Delta/varpi) r^-3 d_r(3 r^2 Delta/varpi),
 *   C_t = [4 i M a m r + 2 s (r Delta - M (r^2 - a^2)) + 2 i s a Delta cos] / Sigma^2,
 *   E0  = (2 r Delta + s Delta' varpi)/Sigma^2,  E = 2 b^2 f_* / f + E0,
 *   Q   = (m^2 a^2 + 2 i m s a (r - M))/Sigma^2,
 *   c1 = b C_t + E - b b_*,  c2 = -C_t,
 *   c3 = b^2 f_** / f + E0 f_* / f + Q + c4 V,  c4 = Delta/Sigma^2,  c5 = c4 g. */
void tko_coeffs_point(double M, double a, int s, int m, int variable,
                      double x, double th, double *out)
{
    double rp, rm;
    horizons(M, a, &rp, &rm);
    double r = rp + x;
    double varpi = r * r + a * a;
    double Delta = x * (r - rm);
    double dDelta = 2.0 * (r - M);
    double sn = sin(th), cs = cos(th);
    double sn2 = sn * sn;
    double Sig2 = varpi * varpi - a * a * Delta * sn2;
    double Sig = sqrt(Sig2);
    double b = varpi / Sig;
    double db_dr = 2.0 * r / Sig - varpi * (4.0 * r * varpi - a * a * dDelta * sn2) / (2.0 * Sig2 * Sig);
    double b_s = (Delta / varpi) * db_dr;
    double fs = 3.0 * Delta / (r * varpi);
    double d_3r2D = (6.0 * r * Delta + 3.0 * r * r * dDelta) / varpi - 6.0 * r * r * r * Delta / (varpi * varpi);
    double fss = (Delta / varpi) * d_3r2D / (r * r * r);
    double CtR = 2.0 * s * (r * Delta - M * (r * r - a * a)) / Sig2;
    double CtI = (4.0 * M * a * m * r + 2.0 * s * a * Delta * cs) / Sig2;
    double E0 = (2.0 * r * Delta + s * dDelta * varpi) / Sig2;
    double E = 2.0 * b * b * fs + E0;
    double QR = (double)m * m * a * a / Sig2;
    double QI = 2.0 * m * s * a * (r - M) / Sig2;
    double c4 = Delta / Sig2;
    double g, V;
    angular_parts(s, m, variable, th, &g, &V);

    out[K_B] = b;
    out[K_C1R] = b * CtR + E - b * b_s;
    out[K_C1I] = b * CtI;
    out[K_C2R] = -CtR;
    out[K_C2I] = -CtI;
    out[K_C3R] = b * b * fss + E0 * fs + QR + c4 * V;
    out[K_C3I] = QI;
    out[K_C4] = c4;
    out[K_C5] = c4 * g;
}

/* ------------------------------------------------------------------------ */
/* The discrete angular operator (Sec. 3.2: 2nd-order centred differences).  */
/* ------------------------------------------------------------------------ */
/* Ghost parity at theta = 0 and pi.  The paper's condition for the literal
 * field: d_theta Phi = 0 (even |m|, parity +1) or Phi = 0 (odd |m|, parity
 * -1).  The regularised field Phi^ is an even function at both poles. */
int tko_parity(int m, int variable)
{
    if (variable != 0) return 1;
    return (abs(m) % 2 == 0) ? 1 : -1;
}

/* The regularised angular operator written in self-adjoint form.  With
 * Phi = w F and (L_theta + V_theta) w = -lambda0 w,
 *   (L_theta + V_theta)(w F) = w [ (P F')' / P - lambda0 F ],  P = sin(theta) w^2,
 * since P'/P = cot(theta) + 2 w'/w.  Its 2nd-order centred difference on
 * cell j = [j dth, (j+1) dth] is
 *   [ P_{j+1} (F_{j+1} - F_j) - P_j (F_j - F_{j-1}) ] / (Q_j dth^2),
 * with P_f = P(f dth) at the cell faces (P_0 = P_N = 0: no ghost is needed,
 * the field is regular at the poles) and Q_j the mean of P over cell j.
 * The matrix is symmetric in the Q-weighted inner product, so its
 * eigenvalues are real.  Returns Ap_j = P_{j+1}/(Q_j dth^2) and
 * Am_j = P_j/(Q_j dth^2).  Q_j uses composite Simpson with 20000 panels. */
static double sl_weight(int s, int m, double th)
{
    double w = tko_weight(s, m, 1, th);
    return sin(th) * w * w;
}

void tko_regular_stencil(int s, int m, int Ntheta, double *Ap, double *Am)
{
    double dth = M_PI / Ntheta;
    const int n = 20000;
    for (int j = 0; j < Ntheta; ++j) {
        double lo = j * dth, h = dth / n, acc = 0.0;
        for (int k = 0; k <= n; ++k) {
            double wk = (k == 0 || k == n) ? 1.0 : ((k % 2) ? 4.0 : 2.0);
            acc += wk * sl_weight(s, m, lo + k * h);
        }
        double Q = acc * h / 3.0 / dth;
        double Plo = (j == 0) ? 0.0 : sl_weight(s, m, j * dth);
        double Phi = (j == Ntheta - 1) ? 0.0 : sl_weight(s, m, (j + 1) * dth);
        Ap[j] = Phi / (Q * dth * dth);
        Am[j] = Plo / (Q * dth * dth);
    }
}

/* The discrete angular operator divided by c4 (the angular part of S):
 *   literal:     out_j = (F_{j+1} - 2F_j + F_{j-1})/dth^2 + cot(theta_j) (F_{j+1} - F_{j-1})/(2 dth)
 *                        + V_theta(theta_j) F_j,  ghosts F_{-1} = p F_0, F_{N} = p F_{N-1};
 *   regularised: out_j = Ap_j (F_{j+1} - F_j) - Am_j (F_j - F_{j-1}) - lambda0 F_j. */
void tko_angular_apply_many(int s, int m, int variable, int Ntheta, int nvec, const double *F,
                            double *out)
{
    double dth = M_PI / Ntheta;
    int p = tko_parity(m, variable);
    double *Ap = (double *)calloc(Ntheta, sizeof(double));
    double *Am = (double *)calloc(Ntheta, sizeof(double));
    if (variable != 0) tko_regular_stencil(s, m, Ntheta, Ap, Am);
    for (int v = 0; v < nvec; ++v) {
        const double *f = F + (size_t)v * Ntheta;
        double *o = out + (size_t)v * Ntheta;
        for (int j = 0; j < Ntheta; ++j) {
            double th = (j + 0.5) * dth;
            double g, V;
            angular_parts(s, m, variable, th, &g, &V);
            double Fm = (j == 0) ? p * f[0] : f[j - 1];
            double Fp = (j == Ntheta - 1) ? p * f[Ntheta - 1] : f[j + 1];
            if (variable == 0)
                o[j] = (Fp - 2.0 * f[j] + Fm) / (dth * dth) + g * (Fp - Fm) / (2.0 * dth) + V * f[j];
            else
                o[j] = Ap[j] * (Fp - f[j]) - Am[j] * (f[j] - Fm) + V * f[j];
        }
    }
    free(Ap);
    free(Am);
}

void tko_angular_apply(int s, int m, int variable, int Ntheta, const double *F, double *out)
{
    tko_angular_apply_many(s, m, variable, Ntheta, 1, F, out);
}

/* ------------------------------------------------------------------------ */
/* Paper's kernel_average1 (Sec. 4): q_h[b,a] = (q[b,a] + q[b,a-1]) / 2      */
/* for 1 <= a < Nr.  The half-node value between a-1 and a lives at index a. */
/* ------------------------------------------------------------------------ */
void tko_average(const double *q, double *q_h, int Nr, int Ntheta)
{
    for (int b = 0; b < Ntheta; ++b)
        for (int a = 1; a < Nr; ++a)
            q_h[IDX(b, a)] = 0.5 * (q[IDX(b, a)] + q[IDX(b, a - 1)]);
}

/* ------------------------------------------------------------------------ */
/* Solver state                                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
    double rs, th;      /* observer position                                  */
    int i0, j0;         /* lower-left node of the interpolation cell          */
    double fr, fth;     /* bilinear weights                                   */
    double w0, w1;      /* w(theta_j0), w(theta_j0+1)                         */
    double *wave;       /* [cap][2]                                           */
    int count, cap;
} tko_observer;

typedef struct {
    tko_params p;
    double *coef_node;  /* [NCOEF][Ntheta][Nr]: coefficients at r*_a          */
    double *coef_half;  /* [NCOEF][Ntheta][Nr]: at r*_{a-1/2}, index a >= 1   */
    double *q[4];       /* qre, qim, pre, pim (the paper's planes)            */
    double *q_h[4];     /* half-step planes, index a >= 1 is node a-1/2       */
    double *rhs[4];     /* bracketed right-hand sides                         */
    double *avg[4];     /* averaged state used inside S                       */
    double *ang_p, *ang_m; /* regularised angular stencil Ap_j, Am_j          */
    tko_observer obs[16];
    int nobs;
    long long steps_done;
} tko_state;

static double rstar_node(const tko_params *p, int a) { return p->rs_min + a * p->drs; }
static double rstar_half(const tko_params *p, int a) { return p->rs_min + (a - 0.5) * p->drs; }
static double theta_node(const tko_params *p, int b) { return (b + 0.5) * (M_PI / p->Ntheta); }

tko_state *tko_new(const tko_params *p)
{
    if (p->Nr < 3 || p->Ntheta < 2 || p->substeps < 1 || !(p->drs > 0) || !(p->dt > 0)) return NULL;
    if (!(fabs(p->a) < p->M)) return NULL;
    tko_state *S = (tko_state *)calloc(1, sizeof(tko_state));
    S->p = *p;
    int Nr = p->Nr, Nth = p->Ntheta;
    size_t plane = (size_t)Nr * Nth;
    S->coef_node = (double *)calloc(NCOEF * plane, sizeof(double));
    S->coef_half = (double *)calloc(NCOEF * plane, sizeof(double));
    for (int k = 0; k < 4; ++k) {
        S->q[k] = (double *)calloc(plane, sizeof(double));
        S->q_h[k] = (double *)calloc(plane, sizeof(double));
        S->rhs[k] = (double *)calloc(plane, sizeof(double));
        S->avg[k] = (double *)calloc(plane, sizeof(double));
    }
    /* coefficient tables: radial nodes and half nodes, every theta row */
    double *xn = (double *)malloc(sizeof(double) * Nr);
    double *xh = (double *)malloc(sizeof(double) * Nr);
    for (int a = 0; a < Nr; ++a) {
        xn[a] = tko_x_of_rstar(p->M, p->a, rstar_node(p, a));
        xh[a] = (a >= 1) ? tko_x_of_rstar(p->M, p->a, rstar_half(p, a)) : 0.0;
    }
    double c[NCOEF];
    for (int b = 0; b < Nth; ++b) {
        double th = theta_node(p, b);
        for (int a = 0; a < Nr; ++a) {
            tko_coeffs_point(p->M, p->a, p->s, p->m, p->variable, xn[a], th, c);
            for (int k = 0; k < NCOEF; ++k) S->coef_node[k * plane + IDX(b, a)] = c[k];
            if (a >= 1) {
                tko_coeffs_point(p->M, p->a, p->s, p->m, p->variable, xh[a], th, c);
                for (int k = 0; k < NCOEF; ++k) S->coef_half[k * plane + IDX(b, a)] = c[k];
            }
        }
    }
    free(xn);
    free(xh);
    S->ang_p = (double *)calloc(Nth, sizeof(double));
    S->ang_m = (double *)calloc(Nth, sizeof(double));
    if (p->variable != 0) tko_regular_stencil(p->s, p->m, Nth, S->ang_p, S->ang_m);
    return S;
}

void tko_free(tko_state *S)
{
    if (!S) return;
    free(S->coef_node);
    free(S->coef_half);
    free(S->ang_p);
    free(S->ang_m);
    for (int k = 0; k < 4; ++k) { free(S->q[k]); free(S->q_h[k]); free(S->rhs[k]); free(S->avg[k]); }
    for (int o = 0; o < S->nobs; ++o) free(S->obs[o].wave);
    free(S);
}

/* Copy of the coefficient tables, [NCOEF][Ntheta][Nr] each (tests only). */
void tko_get_coeffs(const tko_state *S, double *node, double *half)
{
    size_t n = (size_t)NCOEF * S->p.Nr * S->p.Ntheta;
    memcpy(node, S->coef_node, n * sizeof(double));
    memcpy(half, S->coef_half, n * sizeof(double));
}

/* Initial data.  Planes [Ntheta][Nr] of the evolved variable.  If pi_re is
 * NULL the momentum is set for zero time derivative: Pi = b d_* Phi with the
 * centred difference (Phi_{a+1} - Phi_{a-1})/(2 dr*) at interior nodes.  Both
 * fields are zero on the radial edges. */
void tko_set_initial(tko_state *S, const double *phi_re, const double *phi_im,
                     const double *pi_re, const double *pi_im)
{
    int Nr = S->p.Nr, Nth = S->p.Ntheta;
    size_t plane = (size_t)Nr * Nth;
    memcpy(S->q[0], phi_re, plane * sizeof(double));
    memcpy(S->q[1], phi_im, plane * sizeof(double));
    if (pi_re) {
        memcpy(S->q[2], pi_re, plane * sizeof(double));
        memcpy(S->q[3], pi_im, plane * sizeof(double));
    } else {
        const double *bcoef = S->coef_node + (size_t)K_B * plane;
        for (int b = 0; b < Nth; ++b)
            for (int a = 0; a < Nr; ++a) {
                if (a == 0 || a == Nr - 1) { S->q[2][IDX(b, a)] = 0.0; S->q[3][IDX(b, a)] = 0.0; continue; }
                double bb = bcoef[IDX(b, a)];
                S->q[2][IDX(b, a)] = bb * (S->q[0][IDX(b, a + 1)] - S->q[0][IDX(b, a - 1)]) / (2.0 * S->p.drs);
                S->q[3][IDX(b, a)] = bb * (S->q[1][IDX(b, a + 1)] - S->q[1][IDX(b, a - 1)]) / (2.0 * S->p.drs);
            }
    }
    for (int k = 0; k < 4; ++k)
        for (int b = 0; b < Nth; ++b) { S->q[k][IDX(b, 0)] = 0.0; S->q[k][IDX(b, Nr - 1)] = 0.0; }
    S->steps_done = 0;
    for (int o = 0; o < S->nobs; ++o) S->obs[o].count = 0;
}

void tko_get_state(const tko_state *S, double *out4)
{
    size_t plane = (size_t)S->p.Nr * S->p.Ntheta;
    for (int k = 0; k < 4; ++k) memcpy(out4 + k * plane, S->q[k], plane * sizeof(double));
}

/* Overwrite the current state with in4 (four planes [Ntheta][Nr]), keeping the
 * step count and the waveform samples taken so far.  Used to study the run's
 * sensitivity to perturbations made along the way. */
void tko_replace_state(tko_state *S, const double *in4)
{
    size_t plane = (size_t)S->p.Nr * S->p.Ntheta;
    for (int k = 0; k < 4; ++k) memcpy(S->q[k], in4 + k * plane, plane * sizeof(double));
}

/* Overwrite the coefficient tables (layout of tko_get_coeffs; tests only:
 * the conditioning of a run under a change of its coefficients). */
void tko_replace_coeffs(tko_state *S, const double *node, const double *half)
{
    size_t n = (size_t)NCOEF * S->p.Nr * S->p.Ntheta;
    memcpy(S->coef_node, node, n * sizeof(double));
    memcpy(S->coef_half, half, n * sizeof(double));
}

/* ------------------------------------------------------------------------ */
/* The right-hand side in the square brackets of Eqs. (lw1)/(lw2):           */
/*     (1/dr*) D (u_right - u_left) - S(u_avg)                               */
/* at one point, given the averaged state at theta rows b-1, b, b+1.         */
/* ------------------------------------------------------------------------ */
static void bracket(const double *cf, double drs, const double du[4], const double u0[4],
                    const double ang[2], double out[4])
{
    double bb = cf[K_B];
    /* D as a real 4x4 matrix on (PhiR, PhiI, PiR, PiI): complex blocks
     * [[b, 0], [-c1, -b]], c1 acting as [[c1R, -c1I], [c1I, c1R]]. */
    double D[4][4] = {
        { bb, 0.0, 0.0, 0.0 },
        { 0.0, bb, 0.0, 0.0 },
        { -cf[K_C1R], cf[K_C1I], -bb, 0.0 },
        { -cf[K_C1I], -cf[K_C1R], 0.0, -bb },
    };
    /* S(u): Phi rows = Pi; Pi rows = c2 Pi + c3 Phi + (angular term) */
    double Svec[4];
    Svec[0] = u0[2];
    Svec[1] = u0[3];
    Svec[2] = cf[K_C2R] * u0[2] - cf[K_C2I] * u0[3] + cf[K_C3R] * u0[0] - cf[K_C3I] * u0[1] + ang[0];
    Svec[3] = cf[K_C2R] * u0[3] + cf[K_C2I] * u0[2] + cf[K_C3R] * u0[1] + cf[K_C3I] * u0[0] + ang[1];
    for (int k = 0; k < 4; ++k) {
        double Dd = 0.0;
        for (int l = 0; l < 4; ++l) Dd += D[k][l] * du[l];
        out[k] = Dd / drs - Svec[k];
    }
}

/* Angular part of S acting on the averaged Phi at theta row b (Sec. 3.2,
 * 2nd-order centred differences):
 *   literal:     c4 (F_{b+1} - 2F_b + F_{b-1})/dth^2 + c5 (F_{b+1} - F_{b-1})/(2 dth)
 *   regularised: c4 [Ap_b (F_{b+1} - F_b) - Am_b (F_b - F_{b-1})]           */
static void angular_term(const tko_state *S, const double *cf, int b, double dth,
                         const double um[4], const double u0[4], const double up[4], double ang[2])
{
    for (int k = 0; k < 2; ++k) {
        if (S->p.variable == 0)
            ang[k] = cf[K_C4] * (up[k] - 2.0 * u0[k] + um[k]) / (dth * dth)
                   + cf[K_C5] * (up[k] - um[k]) / (2.0 * dth);
        else
            ang[k] = cf[K_C4] * (S->ang_p[b] * (up[k] - u0[k]) - S->ang_m[b] * (u0[k] - um[k]));
    }
}

/* Averaged state at theta row bn of radial index a (with ghost parity). */
static void avg_row(double *const avg[4], int Nr, int Ntheta, int parity, int b, int a, double out[4])
{
    int bn = b;
    double sgn = 1.0;
    if (b < 0) { bn = 0; sgn = parity; }
    if (b >= Ntheta) { bn = Ntheta - 1; sgn = parity; }
    for (int k = 0; k < 4; ++k) out[k] = sgn * avg[k][IDX(bn, a)];
}

/* One inner Lax-Wendroff step of size dt. */
static void lw_step(tko_state *S, double dt)
{
    const tko_params *p = &S->p;
    int Nr = p->Nr, Nth = p->Ntheta;
    size_t plane = (size_t)Nr * Nth;
    double drs = p->drs, dth = M_PI / Nth;
    int parity = tko_parity(p->m, p->variable);

    /* Eq. (lw1), first term: the paper's kernel_average1 on the 4 planes. */
    for (int k = 0; k < 4; ++k) tko_average(S->q[k], S->avg[k], Nr, Nth);

    /* Eq. (lw1), bracket at the half nodes a-1/2 (index a, 1 <= a < Nr). */
#pragma omp parallel for schedule(static)
    for (int b = 0; b < Nth; ++b) {
        double cf[NCOEF], du[4], um[4], u0[4], up[4], br[4], ang[2];
        for (int a = 1; a < Nr; ++a) {
            for (int k = 0; k < NCOEF; ++k) cf[k] = S->coef_half[k * plane + IDX(b, a)];
            for (int k = 0; k < 4; ++k) du[k] = S->q[k][IDX(b, a)] - S->q[k][IDX(b, a - 1)];
            avg_row(S->avg, Nr, Nth, parity, b - 1, a, um);
            avg_row(S->avg, Nr, Nth, parity, b, a, u0);
            avg_row(S->avg, Nr, Nth, parity, b + 1, a, up);
            angular_term(S, cf, b, dth, um, u0, up, ang);
            bracket(cf, drs, du, u0, ang, br);
            for (int k = 0; k < 4; ++k) S->rhs[k][IDX(b, a)] = br[k];
        }
    }
    /* Eq. (lw1): u^{n+1/2}_{a-1/2} = average - (dt/2) bracket. */
    for (int k = 0; k < 4; ++k)
        for (int b = 0; b < Nth; ++b)
            for (int a = 1; a < Nr; ++a)
                S->q_h[k][IDX(b, a)] = S->avg[k][IDX(b, a)] - 0.5 * dt * S->rhs[k][IDX(b, a)];

    /* Eq. (lw2): average of the half-step values around node a (the half
     * nodes a-1/2 and a+1/2 live at indices a and a+1), for 1 <= a <= Nr-2. */
    for (int k = 0; k < 4; ++k)
        for (int b = 0; b < Nth; ++b)
            for (int a = 1; a < Nr - 1; ++a)
                S->avg[k][IDX(b, a)] = 0.5 * (S->q_h[k][IDX(b, a + 1)] + S->q_h[k][IDX(b, a)]);

    /* Eq. (lw2), bracket at the interior nodes. */
#pragma omp parallel for schedule(static)
    for (int b = 0; b < Nth; ++b) {
        double cf[NCOEF], du[4], um[4], u0[4], up[4], br[4], ang[2];
        for (int a = 1; a < Nr - 1; ++a) {
            for (int k = 0; k < NCOEF; ++k) cf[k] = S->coef_node[k * plane + IDX(b, a)];
            for (int k = 0; k < 4; ++k) du[k] = S->q_h[k][IDX(b, a + 1)] - S->q_h[k][IDX(b, a)];
            avg_row(S->avg, Nr, Nth, parity, b - 1, a, um);
            avg_row(S->avg, Nr, Nth, parity, b, a, u0);
            avg_row(S->avg, Nr, Nth, parity, b + 1, a, up);
            angular_term(S, cf, b, dth, um, u0, up, ang);
            bracket(cf, drs, du, u0, ang, br);
            for (int k = 0; k < 4; ++k) S->rhs[k][IDX(b, a)] = br[k];
        }
    }
    /* Eq. (lw2): u^{n+1}_a = u^n_a - dt bracket, then the radial boundary
     * condition Phi = Pi = 0 on both edges (Sec. 3.2). */
    for (int k = 0; k < 4; ++k)
        for (int b = 0; b < Nth; ++b) {
            for (int a = 1; a < Nr - 1; ++a) S->q[k][IDX(b, a)] -= dt * S->rhs[k][IDX(b, a)];
            S->q[k][IDX(b, 0)] = 0.0;
            S->q[k][IDX(b, Nr - 1)] = 0.0;
        }
}

/* ------------------------------------------------------------------------ */
/* Waveform extraction: bilinear interpolation in (r*, theta) of the         */
/* physical field Phi = w Phi^ after each outer step.                        */
/* ------------------------------------------------------------------------ */
/* Returns the observer id, or -1 if the point is outside
 * [r*_0, r*_{Nr-1}] x [theta_0, theta_{Ntheta-1}]. */
int tko_add_observer(tko_state *S, double rs, double th)
{
    const tko_params *p = &S->p;
    if (S->nobs >= 16) return -1;
    double dth = M_PI / p->Ntheta;
    double fi = (rs - p->rs_min) / p->drs;
    double fj = th / dth - 0.5;
    if (!(fi >= 0.0) || fi > p->Nr - 1 || !(fj >= 0.0) || fj > p->Ntheta - 1) return -1;
    int i0 = (int)floor(fi), j0 = (int)floor(fj);
    if (i0 > p->Nr - 2) i0 = p->Nr - 2;
    if (j0 > p->Ntheta - 2) j0 = p->Ntheta - 2;
    tko_observer *o = &S->obs[S->nobs];
    o->rs = rs;
    o->th = th;
    o->i0 = i0;
    o->j0 = j0;
    o->fr = fi - i0;
    o->fth = fj - j0;
    o->w0 = tko_weight(p->s, p->m, p->variable, theta_node(p, j0));
    o->w1 = tko_weight(p->s, p->m, p->variable, theta_node(p, j0 + 1));
    o->cap = 1024;
    o->count = 0;
    o->wave = (double *)malloc(sizeof(double) * 2 * o->cap);
    return S->nobs++;
}

static void extract(tko_state *S)
{
    int Nr = S->p.Nr;
    for (int n = 0; n < S->nobs; ++n) {
        tko_observer *o = &S->obs[n];
        double v[2];
        for (int k = 0; k < 2; ++k) {
            const double *q = S->q[k];
            double lo = (1.0 - o->fth) * o->w0 * q[IDX(o->j0, o->i0)] + o->fth * o->w1 * q[IDX(o->j0 + 1, o->i0)];
            double hi = (1.0 - o->fth) * o->w0 * q[IDX(o->j0, o->i0 + 1)] + o->fth * o->w1 * q[IDX(o->j0 + 1, o->i0 + 1)];
            v[k] = (1.0 - o->fr) * lo + o->fr * hi;
        }
        if (o->count == o->cap) {
            o->cap *= 2;
            o->wave = (double *)realloc(o->wave, sizeof(double) * 2 * o->cap);
        }
        o->wave[2 * o->count] = v[0];
        o->wave[2 * o->count + 1] = v[1];
        o->count++;
    }
}

/* Advance n outer steps; each outer step is `substeps` Lax-Wendroff steps of
 * size dt/substeps followed by one waveform sample per observer. */
void tko_run(tko_state *S, int n)
{
    double dt_in = S->p.dt / S->p.substeps;
    for (int it = 0; it < n; ++it) {
        for (int k = 0; k < S->p.substeps; ++k) lw_step(S, dt_in);
        extract(S);
        S->steps_done++;
    }
}

/* Copies the waveform of observer `id` into re[], im[] (each of length at
 * least the returned count); returns the number of samples, -1 if bad id. */
int tko_waveform(const tko_state *S, int id, double *re, double *im)
{
    if (id < 0 || id >= S->nobs) return -1;
    const tko_observer *o = &S->obs[id];
    if (re && im)
        for (int k = 0; k < o->count; ++k) { re[k] = o->wave[2 * k]; im[k] = o->wave[2 * k + 1]; }
    return o->count;
}

void tko_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int tko_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
