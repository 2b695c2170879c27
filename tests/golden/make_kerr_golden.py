"""Writes tests/golden/kerr_25601x64_oracle.npz: the CPU oracle's full run of
the Kerr a = 0.9, 25601 x 64, 38400-outer-step workload (two Lax-Wendroff
steps per outer step).  Calls only oracle/ and the shared input generator.

Stored: both waveforms (every sample), the physical state Phi = w Phi^,
Pi = w Pi^ on every theta row and every 4th r* column, and the L2 norm of
each full physical plane.  Takes about two hours on 6 cores.

With --fma it writes kerr_25601x64_oracle_fma.npz: the same run through the
same oracle source compiled with FMA contraction (oracle.Solver(build="fma")),
a second correct rounding order of the scheme.  With --coeffs it writes
kerr_25601x64_oracle_coeffs.npz: the run with every coefficient of the tables
multiplied by 1 + 4.4e-16 * N(0, 1) (seed 12347), i.e. changed by about two
ulps, the size of the differences between two correct FP64 evaluations of the
coefficient formulas (their transcendental functions are not correctly
rounded); stored on every 8th theta row and 16th r* column.  With --extcoeffs
it writes kerr_25601x64_oracle_extcoeffs.npz: the run from coefficient tables
evaluated in extended precision and rounded to FP64 once
(oracle.coeffs_ext.tables), which differ from the FP64 tables where the
coefficient formulas cancel (c1R near the horizon keeps two or three digits in
FP64); stored like the --coeffs run.

With --perturbed it writes kerr_25601x64_oracle_perturbed.npz instead: the same
run from the real initial plane times 1 + 2.2e-16 * N(0, 1) (numpy's default
generator, seed 12345), i.e. a change of about one ulp.  The perturbed and
noisy runs store the state on every 8th theta row and every 16th r* column
only.  With --noisy it writes
kerr_25601x64_oracle_noisy.npz: the run with every value of the state
multiplied by 1 + 8.8e-16 * N(0, 1) after every 16th outer step (seed 12346),
a random walk of about one ulp per outer step, the size of the rounding
differences two correct implementations accumulate.  The differences of these
runs from the plain one are the run's own conditioning, which sets the parity
bar of the full-length test.

    python tests/golden/make_kerr_golden.py [threads] [--perturbed | --noisy | --fma | --coeffs | --extcoeffs]
"""
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from inputs import KERR_25601x64, initial_planes  # noqa: E402

ROWS = slice(0, None, 1)
COLS = slice(0, None, 4)
SPARSE_ROWS = slice(0, None, 8)      # the perturbed and noisy runs
SPARSE_COLS = slice(0, None, 16)


EPS = 2.2e-16
SEED = 12345
NOISE_EVERY = 16                 # outer steps between the noisy run's perturbations
NOISE_EPS = 4 * EPS              # sqrt(16) ulps: one ulp per outer step as a random walk
COEF_EPS = 2 * EPS               # about two ulps of every coefficient


def main():
    args = [a for a in sys.argv[1:] if not a.startswith("--")]
    perturbed = "--perturbed" in sys.argv
    noisy = "--noisy" in sys.argv
    fma = "--fma" in sys.argv
    coeffs = "--coeffs" in sys.argv
    extcoeffs = "--extcoeffs" in sys.argv
    assert perturbed + noisy + fma + coeffs + extcoeffs <= 1, "one variant at a time"
    sparse = perturbed or noisy or coeffs or extcoeffs
    rows, cols = (SPARSE_ROWS, SPARSE_COLS) if sparse else (ROWS, COLS)
    if args:
        oracle.set_threads(int(args[0]))
    w = KERR_25601x64
    sol = oracle.Solver(M=w.M, a=w.a, s=w.s, m=w.m, rs_min=w.rs_min, rs_max=w.rs_max, Nr=w.Nr,
                        Ntheta=w.Ntheta, dt=w.dt, substeps=w.substeps, variable=w.variable,
                        build="fma" if fma else "plain")
    ids = [sol.add_observer(r, t) for r, t in w.observers]
    if coeffs:
        node, half = sol.coeffs()
        crng = np.random.default_rng(SEED + 2)
        sol.replace_coeffs(node * (1.0 + COEF_EPS * crng.standard_normal(node.shape)),
                           half * (1.0 + COEF_EPS * crng.standard_normal(half.shape)))
    if extcoeffs:
        from oracle import coeffs_ext
        sol.replace_coeffs(*coeffs_ext.tables(w.M, w.a, w.s, w.m, w.variable, w.rs_min, sol.drs,
                                              w.Nr, w.Ntheta))
    re, im = initial_planes(w)
    if perturbed:
        re = re * (1.0 + EPS * np.random.default_rng(SEED).standard_normal(re.shape))
    sol.set_initial(re, im)
    t0 = time.time()
    chunk = 1200
    rng = np.random.default_rng(SEED + 1)
    for k in range(0, w.steps, chunk):
        n = min(chunk, w.steps - k)
        if noisy:
            for _ in range(0, n, NOISE_EVERY):
                sol.run(NOISE_EVERY)
                st = sol.state()
                sol.replace_state(st * (1.0 + NOISE_EPS * rng.standard_normal(st.shape)))
        else:
            sol.run(n)
        print(f"{k + chunk}/{w.steps} outer steps, {time.time() - t0:.0f} s", flush=True)
    st = sol.state()
    th = (np.arange(w.Ntheta) + 0.5) * (math.pi / w.Ntheta)
    wt = np.array([oracle.weight(w.s, w.m, w.variable, t) for t in th])[None, :, None]
    phys = st * wt
    np.savez_compressed(
        os.path.join(HERE, "kerr_25601x64_oracle" + ("_perturbed" if perturbed else "")
                     + ("_noisy" if noisy else "") + ("_fma" if fma else "")
                     + ("_coeffs" if coeffs else "") + ("_extcoeffs" if extcoeffs else "") + ".npz"),
        wave0=sol.waveform(ids[0]), wave1=sol.waveform(ids[1]),
        state_sub=phys[:, rows, cols], plane_norms=np.linalg.norm(phys.reshape(4, -1), axis=1),
        rows=np.arange(w.Ntheta)[rows], cols=np.arange(w.Nr)[cols],
        note=np.array("oracle full run of " + w.name + f", {w.substeps} LW steps per outer step"
                      + (f", real initial plane times 1 + {EPS} N(0,1), seed {SEED}" if perturbed else "")
                      + (f", state times 1 + {NOISE_EPS} N(0,1) every {NOISE_EVERY} outer steps, seed "
                         f"{SEED + 1}" if noisy else "")
                      + (", oracle compiled with FMA contraction" if fma else "")
                      + (f", coefficients times 1 + {COEF_EPS} N(0,1), seed {SEED + 2}" if coeffs else "")
                      + (", coefficients evaluated in extended precision" if extcoeffs else "")))


if __name__ == "__main__":
    main()
