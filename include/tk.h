/*
 * tk.h -- C ABI of a GB300 (sm_103a) solver for the homogeneous (2+1)D
 * Teukolsky equation, time-stepped with the two-step 2nd-order Lax-Wendroff
 * scheme of arXiv 1010.3816 (Choudhary, Navada, Ginjupalli, Khanna), Sec. 3.
 *
 * One solver evolves one azimuthal mode m of a spin-weight-s field on a Kerr
 * black hole of mass M and spin a, on a uniform grid in the tortoise
 * coordinate r* and the polar angle theta.  The state is the solution vector
 * of Eq. (lw1)/(lw2), u = {Phi_R, Phi_I, Pi_R, Pi_I}, with Pi the momentum of
 * Sec. 3.2.  All arithmetic of the path runs in CUDA kernels; the host code
 * behind this header only validates arguments, allocates device memory and
 * enqueues work.
 *
 * Conventions shared by every entry point
 *   - Field planes: four planes Phi_R, Phi_I, Pi_R, Pi_I, each laid out as
 *     plane[j * Nr + i] (theta row j, r* index i fastest), the layout of the
 *     paper's kernels (Sec. 4: idx(b,a) = N*b + a).  "planes4" means the four
 *     planes back to back in that order (4 * Ntheta * Nr doubles).
 *   - Grid: r*_i = rstar_min + i * dr*, dr* = (rstar_max - rstar_min)/(Nr-1);
 *     theta_j = (j + 1/2) * dtheta, dtheta = pi/Ntheta (cell-centred, no
 *     node on a pole).
 *   - Pointers are plain host or device pointers as the on_device flag says;
 *     device pointers must be in this GPU's memory.  The caller owns every
 *     buffer it passes; the solver copies inputs and never keeps a caller
 *     pointer.  Host buffers may be pageable or pinned.
 *   - Every call is asynchronous on the CUDA stream given to tk_make_grid,
 *     except calls that return data to host memory, which synchronize that
 *     stream before returning.
 *   - Errors: every call returns a tk_status.  No call aborts or throws.  On
 *     error the solver keeps its previous state and tk_last_error() returns a
 *     one-line message.  A CUDA error is returned as TK_ERR_CUDA.
 *   - Calls must come in the order make_grid -> precompute_coeffs ->
 *     set_initial_data -> (add_observer | step | extract | get_state)*;
 *     out-of-order calls return TK_ERR_STATE.
 *   - A solver may be used by one host thread at a time.
 */
#ifndef TK_H
#define TK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tk_solver tk_solver;

typedef enum {
    TK_OK = 0,
    TK_ERR_ARG = 1,       /* invalid argument (null pointer, size, range)        */
    TK_ERR_STATE = 2,     /* call out of order                                   */
    TK_ERR_CUDA = 3,      /* a CUDA runtime call failed                          */
    TK_ERR_OOM = 4,       /* device allocation failed                            */
    TK_ERR_UNSTABLE = 5,  /* non-finite values detected in the state             */
    TK_ERR_INTERNAL = 6   /* device-side consistency check failed                */
} tk_status;

/* Angular variable evolved by the solver. */
enum {
    TK_VAR_LITERAL = 0,     /* Phi itself; ghost parity (-1)^|m| (Sec. 3.2)      */
    TK_VAR_REGULARISED = 1  /* Phi^ = Phi / w(theta), w = (1-cos)^{|m+s|/2}
                               (1+cos)^{|m-s|/2}; ghost parity +1               */
};

/* Arithmetic of the time step. */
enum {
    TK_PREC_F64 = 0,        /* FP64 planes, tables and arithmetic                */
    TK_PREC_F32 = 1         /* FP32 planes, tables and stencil arithmetic; FP64
                               coefficient precompute, and waveform samples
                               formed in FP64 from the FP32 state values        */
};

/* Create a solver for an Nr x Ntheta grid (Sec. 3.2).
 *   rstar_min < rstar_max   radial extent (tortoise coordinate, units of M)
 *   Nr >= 3, 2 <= Ntheta <= 128
 *   dt > 0                  outer time step: one waveform sample per outer step
 *   substeps >= 0           Lax-Wendroff steps per outer step (each dt/substeps);
 *                           0: chosen by every tk_precompute_coeffs as the
 *                           tk_stability_bound count for a growth of 2.5e-5
 *                           per step (read it back with tk_get_substeps)
 *   angular_variable        TK_VAR_LITERAL or TK_VAR_REGULARISED
 *   precision               TK_PREC_F64 or TK_PREC_F32
 *   cuda_stream             cudaStream_t to run on (NULL: the legacy default stream)
 * Allocates the device state (two time levels) and nothing else yet.
 * Returns TK_ERR_ARG on a bad size, TK_ERR_OOM if allocation fails. */
tk_status tk_make_grid(tk_solver **out, double rstar_min, double rstar_max, int Nr, int Ntheta,
                       double dt, int substeps, int angular_variable, int precision,
                       void *cuda_stream);

/* Kerr coefficient precompute for black-hole spin a and mass M (|a| < M),
 * spin weight s and azimuthal mode m (Eq. 1, Eq. 2).  Runs in FP64 on the
 * device: inverts the tortoise map r*(r) at every node and half node, forms
 * the coefficients of the first-order system derived from Eq. 1 (matrices D
 * and S of Eqs. lw1/lw2), folds in dt, dr*, dtheta and the angular boundary
 * conditions of Sec. 3.2, and stores them as the step kernel's tables.  May
 * be called again to change (a, M, s, m); the state must then be set again.
 * Returns TK_ERR_ARG unless M > 0 and |a| < M. */
tk_status tk_precompute_coeffs(tk_solver *S, double a, double M, int s, int m);

/* Coefficients supplied by the caller instead of computed (the paper leaves
 * the precompute to its host code): the raw coefficients of the first-order
 * system (matrices D and S of Eqs. lw1/lw2) in the order b, c1_re, c1_im,
 * c2_re, c2_im, c3_re, c3_im, c4, c5, at the nodes r*_i (node9) and at the
 * half nodes r*_{i+1/2} (half9, column i for i < Nr - 1; column Nr - 1 is not
 * read), each [9][Ntheta][Nr] with r* fastest; for the regularised variable
 * optionally the angular stencil weights ang2 [2][Ntheta] (A+ toward row
 * j + 1, then A- toward row j - 1), or NULL to compute them.  They are folded
 * into the step's tables exactly as tk_precompute_coeffs folds its own.
 * a, M, s, m are those of tk_precompute_coeffs (w(theta), the stability
 * bound and the parameter gradients use them; both of the latter evaluate
 * the library's own coefficients).  Host or device pointers as on_device
 * says; host inputs go through a temporary device buffer (allocated and
 * freed; the call synchronizes).  TK_ERR_STATE for a solver made with
 * substeps = 0; the state must be set again afterwards. */
tk_status tk_set_coefficients(tk_solver *S, double a, double M, int s, int m, const double *node9,
                              const double *half9, const double *ang2, int on_device);

/* The raw coefficients of the library's own precompute for the current
 * (a, M, s, m), in the layout of tk_set_coefficients (half9 column Nr - 1 is
 * zero), evaluated again from the stored r(r*) inversion; for inspecting or
 * exporting the precompute (the paper leaves it to its host code).  Host or
 * device buffers of 9 * Ntheta * Nr doubles each; a host read-out allocates
 * and frees a temporary device buffer and synchronizes.  TK_ERR_STATE before
 * tk_precompute_coeffs. */
tk_status tk_get_coefficients(tk_solver *S, double *node9, double *half9, int on_device);

/* Initial data (Sec. 3.2).  phi_re, phi_im: planes [Ntheta][Nr] of the evolved
 * field (Phi, or Phi^ = Phi/w in the regularised variable).  pi_re, pi_im: the
 * momentum planes, or both NULL for zero time derivative, Pi = b d_{r*} Phi
 * with the centred difference at interior nodes.  Both fields are set to zero
 * on the two radial edges (Sec. 3.2).  on_device: 1 if the pointers are device
 * pointers, 0 if host.  Resets the step counter and every observer. */
tk_status tk_set_initial_data(tk_solver *S, const double *phi_re, const double *phi_im,
                              const double *pi_re, const double *pi_im, int on_device);

/* Initial data generated on the device (the synthetic pulses of the
 * benchmarks): the evolved field's real plane is
 *   amp * exp(-(r*_i - center)^2 / (2 width^2)) * sin^2(theta_j) + noise_amp * (2 u - 1)
 * and its imaginary plane noise_amp * (2 u' - 1), where u and u' are uniform
 * doubles in [0, 1) from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) with
 * this seed: output j*Nr + i for u and Nr*Ntheta + j*Nr + i for u', each the
 * top 53 bits of the 64-bit output times 2^-53.  In the regularised variable
 * this sets Phi^ (so Phi = w(theta) * Phi^).  The momentum is that of zero time
 * derivative, as for tk_set_initial_data with NULL pi planes.  width > 0,
 * noise_amp >= 0 (0: no noise), amp and center finite (TK_ERR_ARG otherwise).
 * Requires tk_precompute_coeffs (TK_ERR_STATE). */
tk_status tk_set_initial_gaussian(tk_solver *S, double amp, double center, double width,
                                  double noise_amp, uint64_t seed);

/* Register a waveform observer at (rstar_obs, theta_obs); writes its id.  Not
 * in the paper, which prints no extraction rule: the sample after every outer
 * step is taken here as the bilinear interpolant in (r*, theta) of the
 * physical field Phi = w Phi^ (w = 1 for the literal variable), formed in FP64
 * for both precisions.  The point
 * must lie in [r*_0, r*_{Nr-1}] x [theta_0, theta_{Ntheta-1}] (TK_ERR_ARG
 * otherwise).  At most 16 observers.  Observers are added after
 * tk_set_initial_data and before the first tk_step (TK_ERR_STATE otherwise);
 * they persist across later tk_set_initial_data calls. */
tk_status tk_add_observer(tk_solver *S, double rstar_obs, double theta_obs, int *obs_id);

/* Advance n >= 0 outer steps (Eqs. lw1 then lw2, with the theta-pole ghosts
 * and radial-edge zeros folded in), appending one sample per observer per
 * outer step.  In the persistent mode of tk_set_steps_per_launch (-1, the
 * default) every step of the call runs in one cooperative launch and the call
 * synchronizes the stream to check that launch's bounded waits; in the other
 * modes it is asynchronous.  The persistent launch needs all its blocks
 * resident at once, as the grid was sized for at tk_make_grid; where fewer
 * fit (a limit on active threads set for the process) the launch fails with
 * TK_ERR_CUDA and nothing is stepped, and tk_set_steps_per_launch(S, 1) runs
 * the same steps one launch at a time.  If one ran out, tk_step returns TK_ERR_INTERNAL,
 * the step and sample counts stay where the call found them (the samples
 * taken before it stay readable), and the state is invalid: tk_step,
 * tk_get_state, tk_check_finite, tk_adjoint and tk_param_gradient return
 * TK_ERR_STATE until tk_set_state or tk_set_initial_data sets it again.
 * Otherwise
 * whole chunks of outer steps are replayed from a CUDA graph captured on
 * first use (see tk_set_graph_chunk) and the rest are launched one by one.
 * Every path gives identical results.  The first call after tk_add_observer,
 * or after the waveform buffer grew, captures a new graph (host work of ~1 ms). */
tk_status tk_step(tk_solver *S, int n);

/* Outer steps per CUDA-graph replay in tk_step: -1 (default) picks about 64
 * kernel launches per replay, 0 launches every step directly, c > 0 replays
 * c outer steps (rounded up to an even number of launches). */
tk_status tk_set_graph_chunk(tk_solver *S, int outer_steps);

/* Waveform of observer obs_id (the samples of tk_add_observer; not in the
 * paper): copies the first min(count, capacity) samples into re[], im[]
 * (device pointers if on_device) and writes the total sample count to *count.
 * re/im may be NULL with capacity 0 to query the count.  A host read-out goes
 * through a device buffer of 16 bytes per sample of the waveform buffer's
 * capacity, which the solver allocates on the first such call and again only
 * when that capacity has grown (see tk_extract_noalloc for a read-out that
 * never allocates); it synchronizes the stream. */
tk_status tk_extract(tk_solver *S, int obs_id, double *re, double *im, int capacity, int *count,
                     int on_device);

/* Allocation-free read-out of a waveform into host memory.  The paper has no
 * counterpart.  It is for callers that must not allocate device memory once
 * they are set up: hosts that hand all device memory to their own pool and
 * treat any other allocation as a failure, and loops whose device-memory
 * budget is fixed in advance (tk_extract allocates its read-out buffer on
 * first use and when the waveform grows, and a cudaMalloc can also
 * synchronize the device).  Copies samples [first, first + count) of observer
 * obs_id to re[0..count) and im[0..count) (host pointers, pageable or pinned),
 * bit-identical to what tk_extract returns, and synchronizes the solver's
 * stream.  Device work goes through a 1 MiB array compiled into the library,
 * so count is limited to 65536 per call (TK_ERR_ARG beyond; read a longer
 * waveform in pieces).  The array is shared by every call in the process and
 * keeps the last call's contents: calls whose work overlaps on the GPU (other
 * threads, other streams) race on it and must be serialized by the caller.
 * Every call looks up the array's device address (cudaGetSymbolAddress); the
 * first lookup on a device may load the library's device code, so make the
 * first call on each device before any stream capture.  Allocates nothing: no
 * cudaMalloc, cudaFree or allocating library call. */
tk_status tk_extract_noalloc(tk_solver *S, int obs_id, int first, int count, double *re,
                             double *im);

/* Gradient of a loss with respect to the initial data, by the transposed
 * Lax-Wendroff step run backward over the steps taken since
 * tk_set_initial_data.  The step of Eqs. (lw1)/(lw2) is linear and
 * time-invariant, so the backward sweep needs no stored trajectory: only the
 * loss gradients.
 *   dL_dwave   [nobs][count][2]: dL/d(Re W), dL/d(Im W) for every sample of
 *              every observer (count = outer steps taken), or NULL
 *   dL_dfinal  planes4: dL/d(final state), or NULL (not both NULL)
 *   on_device  location of dL_dwave / dL_dfinal
 *   grad       output: with independent_pi = 0, two planes [Ntheta][Nr],
 *              dL/d(phi_re), dL/d(phi_im) of tk_set_initial_data with the
 *              momentum derived from Phi (pi planes NULL); with
 *              independent_pi = 1, planes4 including dL/d(pi planes)
 *   grad_on_device location of grad
 * The solver's state is not touched.  Allocates two adjoint state levels on
 * first use (kept until tk_destroy) and temporary buffers for host inputs.
 * Synchronizes the stream when an input or the output is in host memory. */
tk_status tk_adjoint(tk_solver *S, const double *dL_dwave, const double *dL_dfinal, int on_device,
                     double *grad, int grad_on_device, int independent_pi);

/* Gradient of a waveform loss with respect to a black-hole parameter of the
 * coefficients (Eq. 1): param 0 the spin a, param 1 the mass M, for the
 * trajectory taken since tk_set_initial_data (FP64 solvers; TK_ERR_STATE if
 * the state was replaced by tk_set_state since).  dL_dwave as for tk_adjoint:
 * [obs][samples][2] = dL/dRe W, dL/dIm W for every sample taken.  The
 * gradient is the exact one of the discrete scheme up to the derivative of
 * the coefficient tables, which is a 4-point central difference in the
 * parameter (step 1e-3 M, or a quarter of M - |a| if smaller): of relative
 * accuracy ~1e-10.  It includes the momentum's dependence on the parameter
 * when Pi^0 was derived from Phi^0 (NULL pi planes).
 * The adjoint state at inner step j needs u^j, so the trajectory is
 * recomputed: checkpoints of the state every checkpoint_every outer steps
 * (<= 0: about sqrt(samples / substeps), the choice that minimises memory),
 * then, segment by segment from the last, the segment's inner states from its
 * checkpoint, against which the adjoint sweep runs.  Device memory:
 * (samples / C + C * substeps) states plus three table-sized arrays; the cost
 * is about two forward runs plus one adjoint run plus the tangent
 * contractions.  Writes the gradient to *grad (host).  Synchronizes. */
tk_status tk_param_gradient(tk_solver *S, int param, const double *dL_dwave, int on_device,
                            int checkpoint_every, double *grad);

/* Current state as planes4 (4 * Ntheta * Nr doubles), host or device.  (The
 * paper's solver keeps its state on the device; this read-back and
 * tk_set_state are checkpoint and test plumbing, not steps of the method.) */
tk_status tk_get_state(tk_solver *S, double *planes4, int on_device);

/* Overwrite the state from planes4 (checkpoint restore); keeps observers and
 * the step counter, and makes an invalid state (see tk_step) valid again. */
tk_status tk_set_state(tk_solver *S, const double *planes4, int on_device);

/* Largest stable inner step for the current coefficients, and the number of
 * Lax-Wendroff steps per outer step it implies for this solver's dt.  Not in
 * the paper, which gives no time step; the outer dt is read as the sampling
 * cadence, split into this many inner steps where the angular source needs
 * it.  Two
 * limits, both evaluated on the device over every interior node: the radial
 * CFL condition of the Lax-Wendroff scheme, b dt / dr* <= 1, and the angular
 * source term, which the two-step scheme advances like a 2nd-order
 * Runge-Kutta method and therefore amplifies an oscillation of frequency
 * omega by about 1 + (omega dt)^4 / 8 per step; omega^2 is bounded by the
 * Gershgorin radius |c3| + 2 c4 (A+ + A-) of the discrete angular operator.
 * growth_per_step in (0, 1) is the tolerated amplification per step (e.g.
 * 2.5e-5: a factor e over 40000 steps).  Requires tk_precompute_coeffs;
 * synchronizes the stream.  The stiffness bound ignores a^2 couplings in the
 * principal part and is conservative by up to ~2x in dt. */
tk_status tk_stability_bound(tk_solver *S, double growth_per_step, double *dt_max,
                             int *substeps_needed);

/* Lax-Wendroff steps per kernel launch: 1, 2, -1 (every inner step of a
 * tk_step call in one persistent launch: single steps for TK_PREC_F64; for
 * TK_PREC_F32 sweeps of four steps over the grid where it has at least four
 * columns per warp of one block per SM -- the sweeps cover whole outer steps
 * -- and pairs of steps, in a second launch, for the rest, with an odd last
 * step launched alone), or 0 for the default: -1 (1 for TK_PREC_F64 and 2
 * for TK_PREC_F32 on a grid whose blocks could not all be resident at once).
 * With 2,
 * pairs of inner steps run in one launch that reads the state and the
 * coefficient tables once; each warp recomputes the intermediate level one
 * column beyond its range, which adds arithmetic but no DRAM traffic.  With
 * -1, all blocks stay resident (cooperative launch) and a block waits for
 * its two neighbouring blocks' previous step (or sweep) only where its
 * columns involve theirs; the waits are bounded, and tk_step then
 * synchronizes the stream and returns TK_ERR_INTERNAL if one ran out.  Results are bit-identical in every mode.  Returns TK_ERR_ARG for
 * other values. */
tk_status tk_set_steps_per_launch(tk_solver *S, int steps);

/* The launch structure tk_step uses now: -1, 1 or 2 as in
 * tk_set_steps_per_launch, with the default (0) resolved to the choice it
 * made for this grid and precision.  The paper has no counterpart. */
tk_status tk_get_steps_per_launch(const tk_solver *S, int *steps);

/* Lax-Wendroff steps per outer step in use (the count chosen at the last
 * tk_precompute_coeffs when the grid was made with substeps = 0). */
tk_status tk_get_substeps(const tk_solver *S, int *substeps);

/* Outer steps taken since the initial data. */
tk_status tk_steps_done(const tk_solver *S, int64_t *steps);

/* Check that every value of the state is finite; returns TK_ERR_UNSTABLE if
 * not.  Synchronizes the stream. */
tk_status tk_check_finite(tk_solver *S);

/* Wait for all work queued by this solver. */
tk_status tk_synchronize(tk_solver *S);

/* ---- Batches: many solvers advanced together ----------------------------
 * A batch groups n solvers (each past tk_set_initial_data, all with the same
 * precision and outer dt, on one device) so that one kernel launch per inner
 * Lax-Wendroff tick advances all of them.  Members may differ in every other
 * parameter; with k_i inner steps per outer step each, an outer step is
 * lcm(k_i) <= 64 ticks and member i steps on every (lcm/k_i)-th tick.  The
 * batch kernel is persistent: its warps take (member, column range) items,
 * longest first, from a queue in device memory.  Whole chunks of outer steps
 * are replayed from a captured CUDA graph.  Results are bit-identical to
 * stepping each member alone with tk_step.  Everything runs on the first
 * member's stream; members must not be stepped otherwise while the batch
 * holds them.  The batch does not own its members. */
typedef struct tk_batch tk_batch;

/* Create a batch of members[0..n-1].  TK_ERR_ARG if the members do not share
 * device, precision and dt, or lcm(k_i) > 64. */
tk_status tk_batch_create(tk_batch **out, tk_solver *const *members, int n);

/* Advance every member by n outer steps (samples appended as by tk_step). */
tk_status tk_batch_step(tk_batch *B, int n);

/* Autotuner (the counterpart of the paper's tuning of the work-group size,
 * Sec. 4): time trial_steps outer steps for every pair of a segment length
 * (columns per work item: 4 .. 128) and a grid size (1 .. the resident
 * maximum of blocks per SM) on the batch's own data; then, when every member
 * fills the GPU alone (its own persistent launch has one block per SM),
 * compare the best pair with the members stepped one after another as
 * tk_step would step each alone, both timed on the device at trial_steps and 2 trial_steps outer
 * steps and compared by the difference (so that fixed start-up costs count
 * for neither); restore every member's state and sample counter after each
 * trial, and keep the faster.  Writes the chosen segment length
 * (0 for the members one after another) and its time per outer step (ms);
 * the chosen grid is reported by tk_batch_info.  Results are bit-identical
 * either way.  Needs device memory for one copy of every member's state. */
tk_status tk_batch_tune(tk_batch *B, int trial_steps, int *best_seg, double *best_ms_per_step);

/* Set the segment length directly (>= 2), or 0 to step the members one after
 * another as tk_step would (synchronizing as tk_step does). */
tk_status tk_batch_set_segment(tk_batch *B, int seg);

/* Outer steps per graph replay: -1 automatic, 0 no graph, c > 0 about c. */
tk_status tk_batch_set_graph_chunk(tk_batch *B, int outer_steps);

/* Ticks per outer step, segment length, grid size (segment and grid 0 when
 * the members are stepped one after another). */
tk_status tk_batch_info(const tk_batch *B, int *kmax, int *seg, int *blocks);

const char *tk_batch_last_error(const tk_batch *B);
void tk_batch_destroy(tk_batch *B);

/* Diagnostic of the bounded waits of the persistent launches (tk_step with
 * tk_set_steps_per_launch -1): a cooperative launch of n_blocks (2..64)
 * one-warp blocks, each publishing a flag and then waiting, at most max_polls
 * polls each time, for its two neighbours' flags, first as the persistent
 * kernels' blocks do between steps and then as the one-step sweep's edge
 * warps do -- except block `silent` (-1: none), which never publishes and
 * instead waits on a shared-memory counter that nothing sets, as the one-step
 * sweep's warps wait for their siblings.  All three kinds of wait run out,
 * each sets its own error flag, and every block returns; the context stays
 * usable.  *timed_out = 1 if all three error flags were set (where tk_step
 * reports TK_ERR_INTERNAL), 0 if none was; TK_ERR_INTERNAL if only some were.  The persistent kernels use 2^24 polls.
 * Runs on the legacy default stream and synchronizes.  TK_ERR_ARG for
 * arguments out of range (message in tk_last_error(NULL)). */
tk_status tk_check_bounded_wait(int n_blocks, int silent, int64_t max_polls, int *timed_out);

/* Measured rate of this GPU's FP64 fused multiply-add pipe (not in the
 * paper; the roofline of the FP64 step, which is bound by that pipe).  Runs
 * blocks_per_sm * (SM count) blocks of `threads` threads (a multiple of 32,
 * <= 1024), each thread advancing 8 independent FP64 FMA chains `iters`
 * times, on the legacy default stream after a short warm-up launch, and
 * writes the launch's duration (CUDA events) to *seconds and the FP64 flops
 * it did (2 per FMA) to *flop.  Allocates and frees a few bytes of device
 * memory; synchronizes.  TK_ERR_ARG for arguments out of range (message in
 * tk_last_error(NULL)). */
tk_status tk_probe_fp64_fma(int blocks_per_sm, int threads, int iters, double *seconds,
                            double *flop);

/* Test hook, host-side fault injection (not in the paper): the next tk_step
 * on this solver that runs a persistent launch completes its device work
 * normally and then reports its bounded waits as having run out, with the
 * consequences described at tk_step.  For testing a caller's recovery path
 * without a device fault.  Cleared when it fires. */
tk_status tk_inject_wait_timeout(tk_solver *S);

/* One-line description of the last error on this solver (never NULL). */
const char *tk_last_error(const tk_solver *S);

/* Release every device buffer of the solver.  NULL is ignored. */
void tk_destroy(tk_solver *S);

#ifdef __cplusplus
}
#endif

#endif /* TK_H */
