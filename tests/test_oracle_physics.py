"""Pins of the whole oracle scheme against the mathematics and the physics.

* 2nd-order convergence of the two-step Lax-Wendroff scheme (Sec. 3.2): the
  waveform differences between successive grid halvings (dr*, dtheta and dt
  halved together) shrink by ~4.
* The Schwarzschild l = 2 fundamental quasinormal frequency fitted from the
  extracted waveform (golden value with its citation in tests/golden/).
"""
import math
import os

import numpy as np
import pytest

from inputs import Workload, initial_planes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _run(oracle_mod, w: Workload):
    sol = oracle_mod.Solver(M=w.M, a=w.a, s=w.s, m=w.m, rs_min=w.rs_min, rs_max=w.rs_max,
                            Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt, substeps=w.substeps,
                            variable=w.variable)
    ids = [sol.add_observer(r, t) for r, t in w.observers]
    re, im = initial_planes(w)
    sol.set_initial(re, im)
    sol.run(w.steps)
    return [sol.waveform(k) for k in ids], sol


@pytest.mark.parametrize("a,m", [(0.0, 2), (0.9, 2), (0.5, -1)])
def test_second_order_convergence(oracle_mod, a, m):
    # r* in [-30, 70]: the pulse leaves r* = 20; no reflection from either
    # edge reaches the observer at r* = 50 before t = 58 > T.
    T = 40.0
    base = Workload(name="conv", a=a, m=m, rs_min=-30.0, rs_max=70.0, center=20.0, width=4.0,
                    observers=((50.0, math.pi / 2),))
    waves = []
    levels = [(201, 8), (401, 16), (801, 32), (1601, 64)]
    for Nr, Nth in levels:
        drs = 100.0 / (Nr - 1)
        dt = 0.5 * drs
        w = base.with_(Nr=Nr, Ntheta=Nth, dt=dt, steps=int(round(T / dt)))
        (wave,), _ = _run(oracle_mod, w)
        waves.append(wave)
    n0 = len(waves[0])
    common = []
    for L, wv in enumerate(waves):
        idx = (np.arange(1, n0 + 1) << L) - 1
        common.append(wv[idx])
    e = [np.max(np.abs(common[L] - common[L + 1])) for L in range(len(levels) - 1)]
    r1, r2 = e[0] / e[1], e[1] / e[2]
    # second order: the ratio tends to 4 (first order would give 2).  The
    # coarsest level, Ntheta = 8, is still pre-asymptotic for the self-adjoint
    # angular stencil: measured (a, m) = (0, 2): 3.37, 3.68; (0.9, 2): 3.42,
    # 3.68; (0.5, -1): 4.07, 4.03.
    assert 3.3 < r2 < 4.6, (e, r1, r2)
    assert 2.5 < r1 < 5.0, (e, r1, r2)


def _prony_single_mode(x, dt):
    """Fit x_n = Re(C z^n) with one damped mode by linear prediction
    x_{n+1} = p x_n + q x_{n-1}; returns omega with z = exp(-i omega dt)."""
    A = np.stack([x[1:-1], x[:-2]], axis=1)
    p, q = np.linalg.lstsq(A, x[2:], rcond=None)[0]
    z = np.roots([1.0, -p, -q])
    z = z[np.argmax(z.imag)] if np.iscomplexobj(z) else z[0]
    lam = np.log(z) / dt          # = -gamma + i omega_R
    return abs(lam.imag) - 1j * (-lam.real)


def test_schwarzschild_l2_quasinormal_frequency(oracle_mod):
    golden = dict(l.split() for l in open(os.path.join(GOLDEN, "qnm_schwarzschild_l2.txt"))
                  if l.strip() and not l.startswith("#"))
    w_ref = float(golden["omega_re"]) + 1j * float(golden["omega_im"])
    # a = 0, s = -2, m = 2: in the regularised variable w = (1 + cos)^2 is the
    # l = 2 harmonic, so theta-independent data are a pure l = 2 mode.
    # r* in [-100, 250]: neither edge is causally connected to the observer at
    # r* = 50 before t = 180, the end of the fit window.
    w = Workload(name="qnm", a=0.0, s=-2, m=2, rs_min=-100.0, rs_max=250.0, Nr=5601, Ntheta=4,
                 dt=1.0 / 32.0, steps=int(180 * 32), center=20.0, width=4.0, angular="one",
                 observers=((50.0, math.pi / 2),))
    (wave,), _ = _run(oracle_mod, w)
    t = (np.arange(len(wave)) + 1) * w.dt
    assert np.max(np.abs(wave.imag)) == 0.0
    sel = (t >= 120.0) & (t <= 180.0)
    step = 16                                   # resample at dt = 0.5
    x = wave.real[sel][::step]
    om = _prony_single_mode(x, w.dt * step)
    assert abs(om - w_ref) < 1e-3, (om, w_ref)
