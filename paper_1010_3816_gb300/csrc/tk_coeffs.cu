// tk_coeffs.cu -- FP64 Kerr coefficient precompute on the device.
//
// 1. The tortoise coordinate (not printed in the paper) is inverted at every
//    radial node r*_i and half node r*_{i+1/2}: x = r - r+ is found by a
//    bracketed Newton iteration in y = ln x, so that Delta = x (r - r-) never
//    suffers the cancellation of r^2 - 2Mr + a^2 near the horizon.
// 2. The coefficients of the first-order system derived from Eq. 1 with the
//    m-mode ansatz of Eq. 2 (Sec. 3.2: "matrices D and S") are evaluated at
//    every (node, theta row) and (half node, theta row), multiplied out with
//    dt, dr*, dtheta into the step kernel's tables, and the angular boundary
//    conditions of Sec. 3.2 are folded into the first and last theta rows.
#include <math.h>
#include <algorithm>

#include "tk_internal.h"

namespace tk {
namespace {

// Horizons r+- = M +- sqrt(M^2 - a^2) and the tortoise log coefficients.
struct Geo {
    double M, a, rp, rm, Ap, Am;
    int s, m;
};

__device__ Geo geometry(const Kerr &K)
{
    Geo g;
    g.M = K.M;
    g.a = K.a;
    g.s = K.s;
    g.m = K.m;
    const double d = sqrt(K.M * K.M - K.a * K.a);
    g.rp = K.M + d;
    g.rm = K.M - d;
    g.Ap = 2.0 * K.M * g.rp / (g.rp - g.rm);
    g.Am = 2.0 * K.M * g.rm / (g.rp - g.rm);
    return g;
}

__device__ double rstar_of_x(const Geo &P, double x)
{
    // r* = r + Ap ln((r - r+)/2M) - Am ln((r - r-)/2M),  Ap = 2M r+/(r+ - r-),
    // Am = 2M r-/(r+ - r-); d r*/dr = (r^2 + a^2)/Delta.
    const double r = P.rp + x;
    return r + P.Ap * log(x / (2.0 * P.M)) - P.Am * log((r - P.rm) / (2.0 * P.M));
}

__device__ double x_of_rstar(const Geo &P, double target)
{
    // r*(e^y) is increasing in y with slope (r^2 + a^2)/(r - r-): keep a
    // bracket [ylo, yhi] around the root and take Newton steps inside it,
    // falling back to bisection when a step leaves the bracket.
    double ylo = -700.0, yhi = 1.0;
    for (int g = 0; g < 64 && rstar_of_x(P, exp(yhi)) < target; ++g) yhi += 1.0;
    double y = (target > P.rp + 4.0 * P.M) ? log(target)
                                           : (target - P.rp) / P.Ap + log(2.0 * P.M);
    if (!(y > ylo && y < yhi)) y = 0.5 * (ylo + yhi);
    for (int it = 0; it < 200; ++it) {
        const double x = exp(y);
        const double r = P.rp + x;
        const double f = rstar_of_x(P, x) - target;
        if (f == 0.0) break;
        if (f < 0.0) ylo = y; else yhi = y;
        double yn = y - f * (r - P.rm) / (r * r + P.a * P.a);
        if (!(yn > ylo && yn < yhi)) yn = 0.5 * (ylo + yhi);
        if (yn == y) break;
        y = yn;
    }
    return exp(y);
}

__global__ void invert_tortoise_kernel(Kerr KP, double rs_min, double drs, int Nr,
                                       double *x_node, double *x_half)
{
    const Geo P = geometry(KP);
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < Nr) {
        x_node[k] = x_of_rstar(P, rs_min + k * drs);
    } else if (k < 2 * Nr - 1) {
        const int i = k - Nr;                       // half node i + 1/2
        x_half[i] = x_of_rstar(P, rs_min + (i + 0.5) * drs);
    }
}

// Coefficients of   d_t Phi + b d_* Phi = Pi,
//                   d_t Pi - b d_* Pi - c1 d_* Phi = c2 Pi + c3 Phi + c4 Phi_thth + c5 Phi_th
// obtained from Eq. 1 x (-Delta/(Sigma^2 r^3)) with Psi = e^{i m phi} r^3 Phi and
// Pi = d_t Phi + b d_* Phi.  With the regularised variable Phi = w Phi^ the
// theta-singular potential is replaced by the constant -lambda0 and c5 gains
// the 2 w'/w term.
struct Raw {
    double b, c1r, c1i, c2r, c2i, c3r, c3i, c4, c5;
};

__device__ Raw raw_coefficients(const Geo &P, int variable, double x, double th)
{
    const double M = P.M, a = P.a, s = P.s, m = P.m;
    const double r = P.rp + x, r2 = r * r, a2 = a * a;
    const double vp = r2 + a2;                 // varpi
    const double Dl = x * (r - P.rm);          // Delta
    const double dDl = 2.0 * (r - M);          // d Delta / dr
    double sn, cs;
    sincos(th, &sn, &cs);
    const double sn2 = sn * sn;
    const double S2 = vp * vp - a2 * Dl * sn2; // Sigma^2
    const double Sg = sqrt(S2);
    const double b = vp / Sg;
    const double tor = Dl / vp;                // dr/dr*
    const double db = tor * (2.0 * r / Sg - vp * (4.0 * r * vp - a2 * dDl * sn2) / (2.0 * S2 * Sg));
    const double fs = 3.0 * Dl / (r * vp);     // (d_* r^3)/r^3
    const double fss = tor * ((6.0 * r * Dl + 3.0 * r2 * dDl) / vp - 6.0 * r2 * r * Dl / (vp * vp)) / (r2 * r);
    const double Ctr = 2.0 * s * (r * Dl - M * (r2 - a2)) / S2;
    const double Cti = (4.0 * M * a * m * r + 2.0 * s * a * Dl * cs) / S2;
    const double E0 = (2.0 * r * Dl + s * dDl * vp) / S2;
    const double c4 = Dl / S2;
    double g, V;
    if (variable == 0) {
        g = cs / sn;
        V = -(m + s * cs) * (m + s * cs) / sn2 + s;
    } else {
        const double al = 0.5 * fabs(m + s), be = 0.5 * fabs(m - s);
        const int l0 = max(abs(P.m), abs(P.s));
        const double t2 = tan(0.5 * th);
        g = cs / sn + 2.0 * (al / t2 - be * t2);
        V = -(double)(l0 - P.s) * (double)(l0 + P.s + 1);
    }
    Raw o;
    o.b = b;
    o.c1r = b * Ctr + (2.0 * b * b * fs + E0) - b * db;
    o.c1i = b * Cti;
    o.c2r = -Ctr;
    o.c2i = -Cti;
    o.c3r = b * b * fss + E0 * fs + m * m * a2 / S2 + c4 * V;
    o.c3i = 2.0 * m * s * a * (r - M) / S2;
    o.c4 = c4;
    o.c5 = c4 * g;
    return o;
}

// w(theta) = (1 - cos)^{|m+s|/2} (1 + cos)^{|m-s|/2}, written with half angles
// (1 - cos = 2 sin^2, 1 + cos = 2 cos^2) so that nothing cancels near the poles.
__device__ double weight_w(int s, int m, double th)
{
    const double sh = sin(0.5 * th), ch = cos(0.5 * th);
    return pow(2.0 * sh * sh, 0.5 * fabs((double)(m + s))) * pow(2.0 * ch * ch, 0.5 * fabs((double)(m - s)));
}

__device__ double sl_weight(int s, int m, double th)
{
    const double w = weight_w(s, m, th);
    return sin(th) * w * w;
}

// Self-adjoint stencil of the regularised angular operator on cell j:
//   (1/P)(P F')'  ->  [P_{j+1}(F_{j+1} - F_j) - P_j (F_j - F_{j-1})] / (Q_j dth^2),
// P = sin(theta) w^2 at the faces theta = f dth (zero on both poles), Q_j the
// mean of P over the cell by 4-point Gauss-Legendre on 64 sub-panels.
// ang[j] = P_{j+1}/(Q_j dth^2), ang[NP + j] = P_j/(Q_j dth^2); zero on padding rows.
// One warp per row j: lane l integrates sub-panels l and l + 32, then the
// warp sums the 32 partial sums in a fixed tree order.
constexpr int kStencilPanels = 64;

__global__ void regular_stencil_kernel(int s, int m, int Nth, int NP, double *__restrict__ ang)
{
    const int j = blockIdx.x;
    const int lane = threadIdx.x;
    if (j >= NP) return;
    if (j >= Nth) {
        if (lane == 0) {
            ang[j] = 0.0;
            ang[NP + j] = 0.0;
        }
        return;
    }
    const double dth = M_PI / Nth;
    const double xg[2] = {0.3399810435848563, 0.8611363115940526};
    const double wg[2] = {0.6521451548625461, 0.3478548451374538};
    const double h = dth / kStencilPanels;
    double acc = 0.0;
    for (int k = lane; k < kStencilPanels; k += 32) {
        const double c = j * dth + (k + 0.5) * h;
        for (int g = 0; g < 2; ++g)
            acc += wg[g] * (sl_weight(s, m, c - 0.5 * h * xg[g]) + sl_weight(s, m, c + 0.5 * h * xg[g]));
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane != 0) return;
    const double Q = 0.5 * h * acc / dth;
    const double Plo = (j == 0) ? 0.0 : sl_weight(s, m, j * dth);
    const double Phi = (j == Nth - 1) ? 0.0 : sl_weight(s, m, (j + 1) * dth);
    ang[j] = Phi / (Q * dth * dth);
    ang[NP + j] = Plo / (Q * dth * dth);
}

// Raw coefficients supplied by the caller: [9][Nth][Nr] in the order of Raw
// (b, c1 re/im, c2 re/im, c3 re/im, c4, c5).
__device__ Raw raw_from(const double *__restrict__ r, int Nth, int Nr, int jp, int i)
{
    const size_t plane = (size_t)Nth * Nr, k = (size_t)jp * Nr + i;
    Raw c;
    c.b = r[k];
    c.c1r = r[plane + k];
    c.c1i = r[2 * plane + k];
    c.c2r = r[3 * plane + k];
    c.c2i = r[4 * plane + k];
    c.c3r = r[5 * plane + k];
    c.c3i = r[6 * plane + k];
    c.c4 = r[7 * plane + k];
    c.c5 = r[8 * plane + k];
    return c;
}

template <typename T>
__global__ void coeff_tables_kernel(Kerr KP, int variable, int Nr, int Nth, int NP, double drs,
                                    double dt, const double *__restrict__ x_node,
                                    const double *__restrict__ x_half,
                                    const double *__restrict__ ang, T *__restrict__ half,
                                    T *__restrict__ node, double *__restrict__ b_node,
                                    double *__restrict__ w_row, float *__restrict__ cmp,
                                    float *__restrict__ gpm, F32Derive fd,
                                    const double *__restrict__ raw_node,
                                    const double *__restrict__ raw_half)
{
    const int jp = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (jp >= NP || i >= Nr) return;
    const Geo P = geometry(KP);
    T *hcol = half + (size_t)i * kNCH * NP + jp;
    T *ncol = node + (size_t)i * kNCN * NP + jp;
    double hv[kNCH], nv[kNCN];
    for (int q = 0; q < kNCH; ++q) hv[q] = 0.0;
    for (int q = 0; q < kNCN; ++q) nv[q] = 0.0;
    double bn = 0.0;
    double c4n = 0.0, c4h = 0.0;   // c4 at the node and at the half node
    double gpv = 0.0, gmv = 0.0;   // theta-only stencil factors of the row
    const double dth = M_PI / Nth;
    const double ith2 = 1.0 / (dth * dth), i2th = 1.0 / (2.0 * dth);
    const double p = (variable == 0 && (abs(P.m) & 1)) ? -1.0 : 1.0;   // ghost parity
    if (jp < Nth) {
        const double th = (jp + 0.5) * dth;
        if (i == 0 && w_row) w_row[jp] = (variable != 0) ? weight_w(P.s, P.m, th) : 1.0;
        // angular stencil A+ (row j+1), A- (row j-1); the centre gets -(A+ + A-)
        //   literal:     A+- = 1/dth^2 +- cot(theta)/(2 dth) times c4, i.e. c4/dth^2 +- c5/(2 dth)
        //   regularised: A+- = c4 ang[.]  (self-adjoint form, no ghosts)
        const double Ap = (variable != 0) ? ang[jp] : 0.0;
        const double Am = (variable != 0) ? ang[NP + jp] : 0.0;
        if (variable != 0) {
            gpv = Ap;
            gmv = Am;
        } else {
            double sn, cs;
            sincos(th, &sn, &cs);
            gpv = (jp == Nth - 1) ? 0.0 : ith2 + (cs / sn) * i2th;   // ghosts folded on the edge rows
            gmv = (jp == 0) ? 0.0 : ith2 - (cs / sn) * i2th;
        }
        {   // node r*_i, Eq. (lw2), step dt
            const Raw c = raw_node ? raw_from(raw_node, Nth, Nr, jp, i)
                                   : raw_coefficients(P, variable, x_node[i], th);
            bn = c.b;
            if (i > 0 && i < Nr - 1) {
                c4n = c.c4;
                const double h2 = 0.5 * dt;
                const double B = dt * c.b / drs;
                const double g1r = dt * c.c1r / drs, g1i = dt * c.c1i / drs;
                double kp, km;
                if (variable == 0) {
                    kp = h2 * (c.c4 * ith2 + c.c5 * i2th);
                    km = h2 * (c.c4 * ith2 - c.c5 * i2th);
                } else {
                    kp = h2 * c.c4 * Ap;
                    km = h2 * c.c4 * Am;
                }
                const double dg = kp + km;
                double fpr = g1r + h2 * c.c3r - dg, fmr = -g1r + h2 * c.c3r - dg;
                if (variable == 0 && jp == 0) { fpr += p * km; fmr += p * km; km = 0.0; }
                if (variable == 0 && jp == Nth - 1) { fpr += p * kp; fmr += p * kp; kp = 0.0; }
                // entries that multiply half-node Phi values carry the factor eh
                // (the half node returns Phi / eh, see the half-node tables)
                const double eh = 0.25 * dt;
                nv[N_B] = eh * B;
                nv[N_PPR] = B + h2 * c.c2r;
                nv[N_PMR] = -B + h2 * c.c2r;
                nv[N_C2I] = h2 * c.c2i;
                nv[N_FPR] = eh * fpr;
                nv[N_FPI] = eh * (g1i + h2 * c.c3i);
                nv[N_FMR] = eh * fmr;
                nv[N_FMI] = eh * (-g1i + h2 * c.c3i);
                nv[N_KP] = eh * kp;
                nv[N_KM] = eh * km;
            }
        }
        if (i < Nr - 1) {   // half node r*_{i+1/2}, Eq. (lw1), step dt/2
            const Raw c = raw_half ? raw_from(raw_half, Nth, Nr, jp, i)
                                   : raw_coefficients(P, variable, x_half[i], th);
            c4h = c.c4;
            const double dtau = 0.5 * dt, e2 = 0.5 * dtau;
            const double B = dtau * c.b / drs;
            const double g1r = dtau * c.c1r / drs, g1i = dtau * c.c1i / drs;
            double kp, km;
            if (variable == 0) {
                kp = e2 * (c.c4 * ith2 + c.c5 * i2th);
                km = e2 * (c.c4 * ith2 - c.c5 * i2th);
            } else {
                kp = e2 * c.c4 * Ap;
                km = e2 * c.c4 * Am;
            }
            const double dg = kp + km;
            double far = -g1r + e2 * c.c3r - dg, fcr = g1r + e2 * c.c3r - dg;
            if (variable == 0 && jp == 0) { far += p * km; fcr += p * km; km = 0.0; }
            if (variable == 0 && jp == Nth - 1) { far += p * kp; fcr += p * kp; kp = 0.0; }
            // the Phi half-node value is returned divided by e2 (= eh): its
            // Pi term e2 (Pi_a + Pi_c) then needs no multiplication
            hv[H_HP] = (0.5 + B) / e2;
            hv[H_HQ] = (0.5 - B) / e2;
            hv[H_PAR] = 0.5 - B + e2 * c.c2r;
            hv[H_PCR] = 0.5 + B + e2 * c.c2r;
            hv[H_PI] = e2 * c.c2i;
            hv[H_FAR] = far;
            hv[H_FAI] = -g1i + e2 * c.c3i;
            hv[H_FCR] = fcr;
            hv[H_FCI] = g1i + e2 * c.c3i;
            hv[H_KP] = kp;
            hv[H_KM] = km;
        }
    } else if (i == 0 && w_row) {
        w_row[jp] = 0.0;
    }
    if constexpr (sizeof(T) == 4) {
        // FP32: sixteen entries rounded from FP64, the other five derived from
        // them in FP32 exactly as the compact-table kernel derives them
        float cv[kNCC];
        cv[C_HP] = (float)hv[H_HP];
        cv[C_PAR] = (float)hv[H_PAR];
        cv[C_PI] = (float)hv[H_PI];
        cv[C_FAR] = (float)hv[H_FAR];
        cv[C_FAI] = (float)hv[H_FAI];
        cv[C_FCR] = (float)hv[H_FCR];
        cv[C_FCI] = (float)hv[H_FCI];
        cv[C_C4H] = (jp < Nth && i < Nr - 1) ? (float)(0.25 * dt * c4h) : 0.0f;
        cv[C_B] = (float)nv[N_B];
        cv[C_PMR] = (float)nv[N_PMR];
        cv[C_C2I] = (float)nv[N_C2I];
        cv[C_FPR] = (float)nv[N_FPR];
        cv[C_FPI] = (float)nv[N_FPI];
        cv[C_FMR] = (float)nv[N_FMR];
        cv[C_FMI] = (float)nv[N_FMI];
        cv[C_C4N] = (jp < Nth && i > 0 && i < Nr - 1) ? (float)(0.25 * dt * 0.5 * dt * c4n) : 0.0f;
        const float gp = (float)gpv, gm = (float)gmv;
        if (i == 0 && gpm) {
            gpm[jp] = gp;
            gpm[NP + jp] = gm;
        }
        float h32[kNCH], n32[kNCN];
        h32[H_HP] = cv[C_HP];
        h32[H_HQ] = __fadd_rn(fd.ih, -cv[C_HP]);
        h32[H_PAR] = cv[C_PAR];
        h32[H_PCR] = __fadd_rn(cv[C_PAR], __fmaf_rn(fd.t2, cv[C_HP], -1.0f));
        h32[H_PI] = cv[C_PI];
        h32[H_FAR] = cv[C_FAR];
        h32[H_FAI] = cv[C_FAI];
        h32[H_FCR] = cv[C_FCR];
        h32[H_FCI] = cv[C_FCI];
        h32[H_KP] = __fmul_rn(cv[C_C4H], gp);
        h32[H_KM] = __fmul_rn(cv[C_C4H], gm);
        n32[N_B] = cv[C_B];
        n32[N_PPR] = __fmaf_rn(fd.bn2, cv[C_B], cv[C_PMR]);
        n32[N_PMR] = cv[C_PMR];
        n32[N_C2I] = cv[C_C2I];
        n32[N_FPR] = cv[C_FPR];
        n32[N_FPI] = cv[C_FPI];
        n32[N_FMR] = cv[C_FMR];
        n32[N_FMI] = cv[C_FMI];
        n32[N_KP] = __fmul_rn(cv[C_C4N], gp);
        n32[N_KM] = __fmul_rn(cv[C_C4N], gm);
        for (int q = 0; q < kNCH; ++q) hcol[(size_t)q * NP] = h32[q];
        for (int q = 0; q < kNCN; ++q) ncol[(size_t)q * NP] = n32[q];
        if (cmp) {
            float *ccol = cmp + (size_t)i * kNCC * NP + jp;
            for (int q = 0; q < kNCC; ++q) ccol[(size_t)q * NP] = cv[q];
        }
    } else {
        for (int q = 0; q < kNCH; ++q) hcol[(size_t)q * NP] = (T)hv[q];
        for (int q = 0; q < kNCN; ++q) ncol[(size_t)q * NP] = (T)nv[q];
    }
    b_node[(size_t)i * NP + jp] = bn;
}

// The raw coefficients the precompute forms, [9][Nth][Nr] in the order of Raw,
// at the nodes and (column i < Nr - 1) the half nodes r*_{i+1/2}; column
// Nr - 1 of the half table is zero.  Grid-stride over the Nth * Nr points.
__global__ void raw_export_kernel(Kerr KP, int variable, int Nr, int Nth,
                                  const double *__restrict__ x_node, const double *__restrict__ x_half,
                                  double *__restrict__ out_node, double *__restrict__ out_half)
{
    const Geo P = geometry(KP);
    const size_t plane = (size_t)Nth * Nr;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < plane;
         k += (size_t)gridDim.x * blockDim.x) {
        const int jp = (int)(k / Nr), i = (int)(k % Nr);
        const double th = (jp + 0.5) * (M_PI / Nth);
        const Raw c = raw_coefficients(P, variable, x_node[i], th);
        const double v[9] = {c.b, c.c1r, c.c1i, c.c2r, c.c2i, c.c3r, c.c3i, c.c4, c.c5};
        for (int q = 0; q < 9; ++q) out_node[q * plane + k] = v[q];
        Raw h = {};
        if (i < Nr - 1) h = raw_coefficients(P, variable, x_half[i], th);
        const double w[9] = {h.b, h.c1r, h.c1i, h.c2r, h.c2i, h.c3r, h.c3i, h.c4, h.c5};
        for (int q = 0; q < 9; ++q) out_half[q * plane + k] = w[q];
    }
}

// Stiffness of the source term at every interior node: a Gershgorin bound on
// the spectrum of the Phi -> Pi coupling c3 + c4 (angular stencil), i.e. on
// omega^2 of the fastest angular oscillation, and the radial speed b.  The two
// maxima are written as the bit patterns of non-negative doubles, which order
// like unsigned integers: out[0] = max omega^2, out[1] = max b.
__global__ void stiffness_kernel(Kerr KP, int variable, int Nr, int Nth, int NP,
                                 const double *__restrict__ x_node, const double *__restrict__ ang,
                                 unsigned long long *__restrict__ out)
{
    const int jp = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    double w2 = 0.0, bb = 0.0;
    if (jp < Nth && i > 0 && i < Nr - 1) {
        const Geo P = geometry(KP);
        const double dth = M_PI / Nth;
        const double th = (jp + 0.5) * dth;
        const Raw c = raw_coefficients(P, variable, x_node[i], th);
        const double asum = (variable != 0) ? ang[jp] + ang[NP + jp] : 2.0 / (dth * dth);
        w2 = sqrt(c.c3r * c.c3r + c.c3i * c.c3i) + 2.0 * c.c4 * asum;
        bb = c.b;
    }
    // warp maximum, then one atomic per warp
    for (int off = 16; off > 0; off >>= 1) {
        w2 = fmax(w2, __shfl_xor_sync(0xffffffffu, w2, off));
        bb = fmax(bb, __shfl_xor_sync(0xffffffffu, bb, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, (unsigned long long)__double_as_longlong(w2));
        atomicMax(out + 1, (unsigned long long)__double_as_longlong(bb));
    }
}

}  // namespace

cudaError_t launch_stiffness(const Kerr &P, int variable, int Nr, int Ntheta, int NP,
                             const double *x_node, const double *ang, unsigned long long *out,
                             cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    dim3 block(32, 8), grid((NP + 31) / 32, (Nr + 7) / 8);
    stiffness_kernel<<<grid, block, 0, st>>>(P, variable, Nr, Ntheta, NP, x_node, ang, out);
    return cudaGetLastError();
}

cudaError_t launch_raw_export(const Kerr &P, int variable, int Nr, int Ntheta, const double *x_node,
                              const double *x_half, double *out_node, double *out_half, cudaStream_t st)
{
    const size_t n = (size_t)Ntheta * Nr;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 8);
    raw_export_kernel<<<blocks, 256, 0, st>>>(P, variable, Nr, Ntheta, x_node, x_half, out_node, out_half);
    return cudaGetLastError();
}

cudaError_t launch_invert_tortoise(const Kerr &P, double rs_min, double drs, int Nr,
                                   double *x_node, double *x_half, cudaStream_t st)
{
    const int n = 2 * Nr - 1;
    invert_tortoise_kernel<<<(n + 127) / 128, 128, 0, st>>>(P, rs_min, drs, Nr, x_node, x_half);
    return cudaGetLastError();
}

cudaError_t launch_coeff_tables(const Kerr &P, int variable, int Nr, int Ntheta, int NP,
                                double drs, double dt_inner, const double *x_node,
                                const double *x_half, double *ang, int precision, void *half,
                                void *node, double *b_node, double *w_row, float *cmp, float *gpm,
                                cudaStream_t st, const double *raw_node, const double *raw_half,
                                bool ang_given)
{
    const F32Derive fd = f32_derive(dt_inner);
    if (variable != 0 && !ang_given) {
        regular_stencil_kernel<<<NP, 32, 0, st>>>(P.s, P.m, Ntheta, NP, ang);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    dim3 block(32, 8);
    dim3 grid((NP + 31) / 32, (Nr + 7) / 8);
    if (precision == 0)
        coeff_tables_kernel<double><<<grid, block, 0, st>>>(P, variable, Nr, Ntheta, NP, drs, dt_inner,
                                                             x_node, x_half, ang, (double *)half,
                                                             (double *)node, b_node, w_row, nullptr,
                                                             nullptr, fd, raw_node, raw_half);
    else
        coeff_tables_kernel<float><<<grid, block, 0, st>>>(P, variable, Nr, Ntheta, NP, drs, dt_inner,
                                                            x_node, x_half, ang, (float *)half,
                                                            (float *)node, b_node, w_row, cmp, gpm, fd,
                                                            raw_node, raw_half);
    return cudaGetLastError();
}

}  // namespace tk
