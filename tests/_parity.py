"""Helpers for the CUDA-vs-oracle parity tests: run the same seeded workload
through the C ABI (GPU) and through the CPU oracle, and compare.

Parity is measured on the paper's fields u = {Phi_R, Phi_I, Pi_R, Pi_I}
(Sec. 3.2).  With the pole-regularised variable the solver evolves
Phi^ = Phi / w(theta); the physical planes are w(theta_j) times the evolved
ones.  (Phi^ itself is badly scaled next to the poles, where w is ~1e-7: an
O(eps) difference anywhere maps to O(eps / w) there, so Phi^ is reported
but the bar applies to Phi.)

Norms (the parity bar is 1e-12 relative L2 in FP64):
  * per physical plane over the whole grid,
  * per physical plane over r* >= 0 (the field near the horizon can dominate
    the whole-grid norm on long runs),
  * per waveform.
A plane that is exactly zero in the oracle must be exactly zero on the GPU.
"""
from __future__ import annotations

import numpy as np

from inputs import Workload, initial_planes


def run_oracle(w: Workload, steps=None, threads=None, build="plain"):
    """The oracle's run of the workload; build="fma" runs the same source
    compiled with FMA contraction (a second correct rounding order)."""
    import oracle
    if threads:
        oracle.set_threads(threads)
    sol = oracle.Solver(M=w.M, a=w.a, s=w.s, m=w.m, rs_min=w.rs_min, rs_max=w.rs_max, Nr=w.Nr,
                        Ntheta=w.Ntheta, dt=w.dt, substeps=w.substeps, variable=w.variable,
                        build=build)
    ids = [sol.add_observer(r, t) for r, t in w.observers]
    re, im = initial_planes(w)
    sol.set_initial(re, im)
    sol.run(w.steps if steps is None else steps)
    return sol.state(), [sol.waveform(k) for k in ids]


def run_gpu(w: Workload, steps=None, precision=0, device_inputs=True, chunks=1):
    import torch
    import paper_1010_3816_gb300 as tk
    g = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt,
                  substeps=w.substeps, variable=w.variable, precision=precision)
    try:
        g.precompute(w.a, w.M, w.s, w.m)
        re, im = initial_planes(w)
        if device_inputs:
            g.set_initial(torch.from_numpy(re).cuda(), torch.from_numpy(im).cuda())
        else:
            g.set_initial(re, im)
        ids = [g.add_observer(r, t) for r, t in w.observers]
        n = w.steps if steps is None else steps
        done = 0
        for c in range(chunks):
            k = n // chunks + (1 if c < n % chunks else 0)
            g.step(k)
            done += k
        assert done == n
        return g.state(), [g.waveform(k) for k in ids]
    finally:
        g.close()


def rel_l2(a, b):
    den = np.linalg.norm(b)
    num = np.linalg.norm(a - b)
    if den == 0.0:
        return 0.0 if num == 0.0 else np.inf
    return num / den


def row_weights(w: Workload) -> np.ndarray:
    """w(theta_j) per theta row (1 for the literal variable), from the oracle."""
    import math
    import oracle
    th = (np.arange(w.Ntheta) + 0.5) * (math.pi / w.Ntheta)
    return np.array([oracle.weight(w.s, w.m, w.variable, t) for t in th])


def sensitivity(w: Workload, steps=None, eps=2.2e-16, seed=12345):
    """The run's own conditioning: parity numbers between the oracle on the
    workload's inputs and the oracle on inputs changed by ~1 ulp (each value
    of the real initial plane times 1 + eps * N(0, 1))."""
    import oracle
    sol = oracle.Solver(M=w.M, a=w.a, s=w.s, m=w.m, rs_min=w.rs_min, rs_max=w.rs_max, Nr=w.Nr,
                        Ntheta=w.Ntheta, dt=w.dt, substeps=w.substeps, variable=w.variable)
    ids = [sol.add_observer(r, t) for r, t in w.observers]
    re, im = initial_planes(w)
    re = re * (1.0 + eps * np.random.default_rng(seed).standard_normal(re.shape))
    sol.set_initial(re, im)
    sol.run(w.steps if steps is None else steps)
    pert = (sol.state(), [sol.waveform(k) for k in ids])
    return pert


def compare(w: Workload, gpu, ref, tol=1e-12, perturbed=None):
    """Returns a dict of the parity numbers; asserts those of the physical
    planes and the waveforms are <= tol (evolved-variable numbers, key
    suffix '_evolved', are reported only).

    ``perturbed``: other oracle runs of the same workload that differ from
    ``ref`` only by rounding -- the same source built with FMA contraction
    (``run_oracle(w, build="fma")``) and the run from inputs changed by ~1 ulp
    (``sensitivity``) -- one run or a list.  Each quantity's bar is then
    max(tol, 2 kappa), kappa the largest difference of that quantity between
    ``ref`` and those runs: a run that amplifies rounding differences beyond
    tol cannot be matched closer than two correct rounding orders match each
    other."""
    gs, gw = gpu
    os_, ow = ref
    assert gs.shape == os_.shape
    wt = row_weights(w)[None, :, None]
    gp, op = gs * wt, os_ * wt
    rs = w.rs_min + np.arange(w.Nr) * w.drs
    outer = rs >= 0.0
    out, info = {}, {}
    for c, name in enumerate(("PhiR", "PhiI", "PiR", "PiI")):
        out[name] = rel_l2(gp[c], op[c])
        if outer.any():
            out[name + "_outer"] = rel_l2(gp[c][:, outer], op[c][:, outer])
        info[name + "_evolved"] = rel_l2(gs[c], os_[c])
    for k, (a, b) in enumerate(zip(gw, ow)):
        assert len(a) == len(b), (len(a), len(b))
        out[f"wave{k}"] = rel_l2(a, b)
    bars = {k: tol for k in out}
    if perturbed is not None:
        runs = perturbed if isinstance(perturbed, list) else [perturbed]
        kaps = [compare(w, r, ref, tol=np.inf) for r in runs]
        for k in out:
            kap = max(kk[k] for kk in kaps)
            bars[k] = max(tol, 2.0 * kap)
            info["kappa_" + k] = kap
    bad = {k: (v, bars[k]) for k, v in out.items() if not v <= bars[k]}
    assert not bad, f"parity above bar: {bad} (evolved variable: {info})"
    out.update(info)
    return out
