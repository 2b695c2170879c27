"""Gradients of a waveform misfit with respect to the black-hole spin a and
mass M (tk_param_gradient): the exact gradient of the discrete scheme through
the adjoint sweep, with the trajectory recomputed from checkpoints.

* Against 4-point central finite differences of the loss itself (every
  evaluation re-runs the precompute and the whole solve at the shifted
  parameter): agreement to 1e-7 relative, for a and M, both angular
  variables, a momentum derived from Phi (it then depends on a and M through
  b) or given.
* Independent of the checkpoint interval (bit-identical sums: the same
  contributions are added in the same order).
* Refused where the trajectory is unknown (tk_set_state), for FP32 solvers
  and before any step.
"""
import math

import numpy as np
import pytest

from inputs import Workload, initial_planes, uniform01

pytestmark = pytest.mark.gpu

BASE = Workload(name="pg", a=0.7, m=2, rs_min=-20.0, rs_max=30.0, Nr=401, Ntheta=32, dt=0.0625,
                substeps=2, steps=200, center=2.0, width=2.5,
                observers=((12.0, math.pi / 2), (6.7, 1.1)))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1010_3816_gb300 as tk
    tk.load_library()


def _solve(w, planes):
    import paper_1010_3816_gb300 as tk
    g = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt,
                  substeps=w.substeps, variable=w.variable)
    g.precompute(w.a, w.M, w.s, w.m)
    g.set_initial(*planes)
    ids = [g.add_observer(r, t) for r, t in w.observers]
    g.step(w.steps)
    return g, np.stack([g.waveform(k) for k in ids])


def _target(w):
    re, im = initial_planes(w.with_(center=w.center + 0.7, width=w.width * 1.1, amp=0.9))
    g, W = _solve(w, (re, im))
    g.close()
    return W


def _loss(W, target):
    return float(np.sum(np.abs(W - target) ** 2))


def _shifted(w, param, d):
    return w.with_(a=w.a + d) if param == "a" else w.with_(M=w.M + d)


def _fd(w, param, planes, target, h):
    vals = []
    for d in (h, -h, 2 * h, -2 * h):
        g, W = _solve(_shifted(w, param, d), planes)
        g.close()
        vals.append(_loss(W, target))
    return (8 * (vals[0] - vals[1]) - (vals[2] - vals[3])) / (12 * h)


def _adjoint_gradient(w, param, planes, target, checkpoint_every=0):
    g, W = _solve(w, planes)
    dW = 2.0 * (W - target)
    dwave = np.stack([dW.real, dW.imag], axis=-1)       # [obs][samples][2]
    out = g.param_gradient(param, dwave, checkpoint_every)
    g.close()
    return out


@pytest.mark.parametrize("param,kw,given_pi", [
    ("a", dict(), False),
    ("M", dict(), False),
    ("a", dict(variable=0, m=1, dt=0.02, substeps=1, steps=500), False),
    ("a", dict(Ntheta=64, a=0.9, substeps=3, steps=150), True),
    ("M", dict(s=0, m=0, a=0.5), True),
])
def test_gradient_matches_finite_differences(param, kw, given_pi):
    w = BASE.with_(**kw)
    re, im = initial_planes(w)
    planes = (re, im)
    if given_pi:
        n = re.size
        pr = 0.3 * (2.0 * uniform01(41, n) - 1.0).reshape(re.shape) * re
        pi = 0.2 * (2.0 * uniform01(42, n) - 1.0).reshape(re.shape) * re
        planes = (re, im, pr, pi)
    target = _target(w)
    grad = _adjoint_gradient(w, param, planes, target)
    fd = _fd(w, param, planes, target, 1e-3 * w.M)
    assert abs(grad - fd) <= 1e-7 * abs(fd), (param, grad, fd)


def test_checkpoint_interval_does_not_change_the_sum():
    w = BASE
    planes = initial_planes(w)
    target = _target(w)
    g0 = _adjoint_gradient(w, "a", planes, target, 0)
    for c in (1, 4, 7, w.steps):
        assert _adjoint_gradient(w, "a", planes, target, c) == g0


def test_refusals():
    import paper_1010_3816_gb300 as tk
    w = BASE.with_(steps=5)
    planes = initial_planes(w)
    dw = np.zeros((len(w.observers), w.steps, 2))
    g, _ = _solve(w, planes)
    g.set_state(g.state())                      # trajectory no longer from u^0
    with pytest.raises(tk.TkError):
        g.param_gradient("a", dw)
    g.close()
    g = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt,
                  precision=tk.TK_PREC_F32)
    g.precompute(w.a, w.M, w.s, w.m)
    g.set_initial(*planes)
    g.add_observer(*w.observers[0])
    g.step(5)
    with pytest.raises(tk.TkError):
        g.param_gradient("a", dw[:1])
    g.close()
    g = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt)
    g.precompute(w.a, w.M, w.s, w.m)
    g.set_initial(*planes)
    g.add_observer(*w.observers[0])
    with pytest.raises(tk.TkError):
        g.param_gradient("a", dw[:1])            # no steps taken
    with pytest.raises(tk.TkError):
        g.param_gradient(2, dw[:1])
    g.close()


def test_autograd_through_spin_mass_and_pulse():
    """waveforms_with_params: torch gradients of a misfit with respect to a, M
    and the pulse amplitude against 4-point finite differences."""
    import torch
    import paper_1010_3816_gb300 as tk
    w = BASE.with_(steps=160)
    g = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt,
                  substeps=w.substeps)
    g.precompute(w.a, w.M, w.s, w.m)
    for r, t in w.observers:
        g.add_observer(r, t)
    re, _ = initial_planes(w)
    shape = torch.tensor(re, device="cuda")
    target = torch.tensor(np.stack([np.stack([x.real, x.imag], -1) for x in _target(w)]),
                          device="cuda")

    def loss(a, M, A):
        W = tk.waveforms_with_params(g, a, M, w.s, w.m, A * shape, torch.zeros_like(shape), w.steps)
        return ((W - target) ** 2).sum()

    p = [torch.tensor(v, dtype=torch.float64, device="cuda", requires_grad=True)
         for v in (w.a, w.M, 1.0)]
    L = loss(*p)
    L.backward()
    for k in range(3):
        h = 1e-3
        vals = []
        for d in (h, -h, 2 * h, -2 * h):
            q = [x.detach().clone() for x in p]
            q[k] += d
            with torch.no_grad():
                vals.append(loss(*q).item())
        fd = (8 * (vals[0] - vals[1]) - (vals[2] - vals[3])) / (12 * h)
        assert abs(p[k].grad.item() - fd) <= 1e-7 * abs(fd), (k, p[k].grad.item(), fd)
    g.close()
