// tk_internal.h -- declarations shared by the CUDA translation units of libtk.
//
// Device-resident layout (differs from the ABI's [Ntheta][Nr] planes):
//   state   u[i][c][jp]     i: r* column, c: 0..3 = Phi_R, Phi_I, Pi_R, Pi_I,
//                           jp: theta row padded to NP = 32*K (rows >= Ntheta are 0)
//   tables  half[i][q][jp]  q < kNCH: folded coefficients of Eq. (lw1) at r*_{i+1/2}
//           node[i][q][jp]  q < kNCN: folded coefficients of Eq. (lw2) at r*_i
// One warp owns every theta row of a column (lane l holds rows K*l .. K*l+K-1),
// so a column of any plane or table is one contiguous, coalesced vector load.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tk {

constexpr int kMaxObservers = 16;
constexpr int kMaxK = 4;          // theta rows per lane: Ntheta <= 32 * kMaxK
constexpr int kNarrowWarps = 4;   // warps per block of a narrow launch (small grids)
constexpr int kNCH = 11;          // half-node table entries
constexpr int kNCN = 10;          // node table entries

// Half-node table entries (Eq. lw1 with dtau = dt/2, rho = 1/dr*):
//   HP  = 1/2 + dtau rho b        coefficient of Phi_i   in Phi^{n+1/2}
//   HQ  = 1/2 - dtau rho b        coefficient of Phi_i+1 in Phi^{n+1/2}
//   PAR = 1/2 - dtau rho b + dtau/2 c2R     Pi_i   -> Pi^{n+1/2} (real part)
//   PCR = 1/2 + dtau rho b + dtau/2 c2R     Pi_i+1 -> Pi^{n+1/2} (real part)
//   PI  = dtau/2 c2I                        imaginary part of both
//   FA  = -dtau rho c1 + dtau/2 c3 - dtau c4/dth^2   Phi_i   -> Pi^{n+1/2} (complex)
//   FC  = +dtau rho c1 + dtau/2 c3 - dtau c4/dth^2   Phi_i+1 -> Pi^{n+1/2} (complex)
//   KP  = dtau/2 (c4/dth^2 + c5/(2 dth))    (Phi_i + Phi_i+1) at row j+1
//   KM  = dtau/2 (c4/dth^2 - c5/(2 dth))    (Phi_i + Phi_i+1) at row j-1
// plus the uniform dtau/2 on (Pi_i + Pi_i+1) in Phi^{n+1/2}.
enum { H_HP = 0, H_HQ, H_PAR, H_PCR, H_PI, H_FAR, H_FAI, H_FCR, H_FCI, H_KP, H_KM };
// Node table entries (Eq. lw2 with dt, applied to h+ = u^{n+1/2}_{i+1/2},
// h- = u^{n+1/2}_{i-1/2}):
//   B   = dt rho b              Phi^{n+1} = Phi_i - B Phi+ + B Phi- + dt/2 (Pi+ + Pi-)
//   PPR = B + dt/2 c2R, PMR = -B + dt/2 c2R, C2I = dt/2 c2I
//   FP  = dt rho c1 + dt/2 c3 - dt c4/dth^2,  FM = -dt rho c1 + dt/2 c3 - dt c4/dth^2
//   KP, KM as above with dt/2.
// Literal variable: the theta ghosts of Sec. 3.2 (u_{-1} = p u_0, u_{N} = p u_{N-1})
// are folded into rows 0 and Ntheta-1: KM (resp. KP) is added, times p, to the
// real parts of the two Phi coefficients and then set to 0.  Regularised
// variable: KP, KM come from the self-adjoint stencil, which has no flux through
// the poles (KM = 0 on row 0, KP = 0 on row Ntheta-1).  Padding rows are all 0.
enum { N_B = 0, N_PPR, N_PMR, N_C2I, N_FPR, N_FPI, N_FMR, N_FMI, N_KP, N_KM };

// FP32 tables.  Five of the 21 entries follow from the others and from
// theta-only factors: HQ = 1/e2 - HP, PCR = PAR + (2 e2 HP - 1) (both from
// HP e2 = 1/2 + B at the half node), PPR = PMR + (2/eh) B_tab (B_tab = eh B at
// the node), and KP, KM = C4 gp_j, C4 gm_j with C4 the 2-D factor (e2 c4 at
// the half node, eh dt/2 c4 at the node) and gp, gm the theta-only stencil
// factors of row j (regularised: the self-adjoint stencil's face weights;
// literal: 1/dth^2 +- cot(theta_j)/(2 dth); zero where a ghost was folded).
// The FP32 tables hold those five entries as exactly these FP32 operations on
// the FP32 values of the others (F32Derive), so that a kernel may read all 21
// or read the 16 of the compact copy cmp[i][kNCC][jp] (the four-step sweep:
// 24 % fewer table bytes) and derive the rest with the same operations,
// bit-identically.
constexpr int kNCC = 16;
enum { C_HP = 0, C_PAR, C_PI, C_FAR, C_FAI, C_FCR, C_FCI, C_C4H,
       C_B, C_PMR, C_C2I, C_FPR, C_FPI, C_FMR, C_FMI, C_C4N };
struct F32Derive {
    float ih;    // 1 / e2 (e2 = eh = dt/4)
    float t2;    // 2 e2
    float bn2;   // 2 / eh
};
// The FP32 constants of the derivation for an inner step dt.
inline F32Derive f32_derive(double dt_inner)
{
    const double e2 = 0.25 * dt_inner;
    return F32Derive{(float)(1.0 / e2), (float)(2.0 * e2), (float)(2.0 / e2)};
}

struct Kerr {
    double M, a;  // black-hole mass and spin
    int s, m;     // spin weight, azimuthal mode
};

struct ObsDev {
    int n;                          // number of observers
    int i0[kMaxObservers];          // lower r* column of the interpolation cell
    int j0[kMaxObservers];          // lower theta row
    double wr0[kMaxObservers];      // 1 - fr
    double wr1[kMaxObservers];      // fr
    double ft[kMaxObservers];       // theta weight fth
};

// How the read-out forms an observer's samples from its buffer entries.  An
// entry is 4 doubles per outer step.  FP64 solvers store two weighted partial
// sums (slot 0 from column i0, slot 1 from column i0 + 1) as (re, im) pairs
// and the sample is slot 0 + slot 1.  FP32 solvers store the FP32 values
// themselves, 8 floats: for slot s, Phi_R and Phi_I at rows j0 and j0 + 1
// (floats 4s .. 4s + 3 = R_j0, I_j0, R_j0+1, I_j0+1); the read-out converts
// them to FP64 (exactly) and forms the same bilinear sample as the FP64 path,
// in FP64.
struct WaveRead {
    int precision;
    int j0;                 // lower theta row
    double ft;              // theta weight fth
    double wr0, wr1;        // 1 - fr, fr
    const double *w_row;    // w(theta_j) on the device
};

// ---- coefficient precompute (tk_coeffs.cu) ----
cudaError_t launch_invert_tortoise(const Kerr &P, double rs_min, double drs, int Nr,
                                   double *x_node, double *x_half, cudaStream_t st);
// FP32 (precision 1) also writes the compact tables cmp and the theta
// factors gpm[2][NP] (gp, then gm); both may be NULL for FP64.  raw_node,
// raw_half (device, [9][Ntheta][Nr], half node i at r*_{i+1/2}): coefficients
// supplied by the caller instead of computed (x_node, x_half then unused);
// ang_given: ang already holds the regularised stencil.
cudaError_t launch_coeff_tables(const Kerr &P, int variable, int Nr, int Ntheta, int NP,
                                double drs, double dt_inner, const double *x_node,
                                const double *x_half, double *ang, int precision, void *half,
                                void *node, double *b_node, double *w_row, float *cmp, float *gpm,
                                cudaStream_t st, const double *raw_node = nullptr,
                                const double *raw_half = nullptr, bool ang_given = false);

// The raw coefficients of the precompute, [9][Ntheta][Nr] at nodes and half
// nodes (device output buffers).
cudaError_t launch_raw_export(const Kerr &P, int variable, int Nr, int Ntheta, const double *x_node,
                              const double *x_half, double *out_node, double *out_half, cudaStream_t st);

cudaError_t launch_stiffness(const Kerr &P, int variable, int Nr, int Ntheta, int NP,
                             const double *x_node, const double *ang, unsigned long long *out,
                             cudaStream_t st);

// ---- state import / export (tk_layout.cu) ----
cudaError_t launch_import_state(int precision, int Nr, int Ntheta, int NP, double drs,
                                const double *phi_re, const double *phi_im, const double *pi_re,
                                const double *pi_im, const double *b_node, void *u,
                                cudaStream_t st);
cudaError_t launch_export_state(int precision, int Nr, int Ntheta, int NP, const void *u,
                                double *planes4, cudaStream_t st);
cudaError_t launch_gaussian(int Nr, int Ntheta, double rs_min, double drs, double amp,
                            double center, double width, double noise, unsigned long long seed,
                            double *re, double *im, cudaStream_t st);
cudaError_t launch_finite_check(int precision, size_t n, const void *u, int *flag,
                                cudaStream_t st);
// Samples [first, first + count) of one observer's buffer to re[0..count),
// im[0..count) (device pointers).
cudaError_t launch_wave_sum(const double *wave_obs, int64_t first, int64_t count, const WaveRead &r,
                            double *re, double *im, cudaStream_t st);

// ---- time step (tk_step.cu) ----
struct StepLaunch {
    int precision, K;
    int Nr, NP;
    int blocks;           // grid size (columns are split evenly over its warps)
    int warps;            // warps per block (from step_grid_shape or fused_grid_shape)
    int fused;            // 1: two Lax-Wendroff steps in this launch (lw_step2_kernel)
    int obs_mask;         // fused: bit 0, an outer step ends after the first step; bit 1, after the second
    double dt_inner;      // Lax-Wendroff step
    const void *u_in;
    void *u_out;
    const void *half;
    const void *node;
    const float *cmp;     // FP32: compact tables [i][kNCC][jp] (the four-step sweep)
    const float *gpm;     // FP32: theta factors gp[NP], gm[NP]
    // waveform (only on the last inner step of an outer step)
    int write_wave;
    const long long *sample_ctr;  // device: index of the sample the outer step writes
    unsigned int *done_ctr;       // device: blocks finished (reset by the last one)
    int64_t wave_cap;     // samples per observer in the buffer
    double *wave;         // [obs][cap][slot 2][re, im]
    const double *w_row;  // w(theta_j)
    ObsDev obs;
};
cudaError_t launch_lw_step(const StepLaunch &L, cudaStream_t st);
// Launch shape of the step kernel for a grid: returns the number of blocks
// and sets *warps to the warps per block.
int step_grid_shape(int precision, int K, int Nr, int num_sms, int *warps);
// Many steps in one cooperative launch (small grids): the grid size for it,
// 0 if it cannot run; the launch itself (L.u_in holds u^n, u_other is the
// second level; flags: one zeroed unsigned int per block; *err set on a wait
// that timed out).
int persistent_grid_blocks(int precision, int K, int Nr, int num_sms, int warps);
// Diagnostic of the persistent launches' bounded neighbour wait (one-warp
// blocks; flags: n_blocks zeroed unsigned ints).
cudaError_t launch_wait_check(int n_blocks, int silent, long long max_spins, unsigned int *flags,
                              int *err, cudaStream_t st);
cudaError_t launch_lw_persistent(const StepLaunch &L, void *u_other, int n_inner, int substeps,
                                 unsigned int *flags, int *err, cudaStream_t st);
// Pairs of steps in one cooperative launch (FP32, the two-step kernel's grid
// and shared-memory ring): L.u_in holds u^n, u_other the second level.
cudaError_t launch_ring_persistent(const StepLaunch &L, void *u_other, int n_pairs, int k,
                                   unsigned int *flags, int *err, cudaStream_t st);
// Launch shape of the two-step kernel.
int fused_grid_shape(int precision, int K, int Nr, int num_sms, int *warps);
// FP32, large grids: groups of multi_levels() steps per sweep in one
// cooperative launch (one block per SM); 0 blocks where it does not apply.
// The call must start on an outer step's boundary.
int multi_grid_shape(int precision, int K, int Nr, int num_sms, int *warps);
int multi_levels();
// scratch: multi_obs_scratch_bytes(K, blocks, warps) of device memory for the
// waveform samples; the sweep applies only if multi_obs_fit (no warp holds
// more than four distinct observer columns).
size_t multi_obs_scratch_bytes(int K, int blocks, int warps);
bool multi_obs_fit(int Nr, int blocks, int warps, const int *obs_i0, int nobs);
cudaError_t launch_multi_persistent(const StepLaunch &L, void *u_other, int n_groups, int k,
                                    unsigned int *flags, int *err, void *scratch, cudaStream_t st);
// Launch shape of the adjoint step kernel: returns the number of blocks and
// sets *warps to the warps per block.
int adjoint_grid_shape(int precision, int K, int Nr, int num_sms, int *warps);

}  // namespace tk
