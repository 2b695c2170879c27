"""The adjoint (transposed) Lax-Wendroff step, tk_adjoint.

* Dot-product test: for the linear map J from the initial data to the
  waveforms (and the final state), <g, J u> = <J^T g, u> to 1e-12, for every
  theta packing, both angular variables, sub-stepping, with the momentum given
  or derived from Phi.
* The same identity with J applied by the CPU oracle instead of the GPU.
* Finite differences of a waveform misfit with respect to the amplitude,
  centre and width of the initial Gaussian, through the torch.autograd
  function built on the adjoint.
"""
import math

import numpy as np
import pytest

from inputs import Workload, initial_planes, uniform01

pytestmark = pytest.mark.gpu

BASE = Workload(name="adj", a=0.7, m=2, rs_min=-30.0, rs_max=50.0, Nr=401, Ntheta=32, dt=0.1,
                steps=60, observers=((20.0, math.pi / 2), (9.3, 1.1)))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1010_3816_gb300 as tk
    tk.load_library()


def _rand(shape, seed):
    return (2.0 * uniform01(seed, int(np.prod(shape))) - 1.0).reshape(shape)


def _solver(w):
    import paper_1010_3816_gb300 as tk
    g = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt,
                  substeps=w.substeps, variable=w.variable)
    g.precompute(w.a, w.M, w.s, w.m)
    return g


def _forward(g, w, planes, ids=None):
    """Waveforms [nobs][steps][2] and final state of the GPU run from planes
    (2 planes: momentum derived; 4 planes: given)."""
    if len(planes) == 2:
        g.set_initial(planes[0], planes[1])
    else:
        g.set_initial(planes[0], planes[1], planes[2], planes[3])
    if ids is None:
        ids = [g.add_observer(r, t) for r, t in w.observers]
    g.step(w.steps)
    waves = np.stack([np.stack([x.real, x.imag], axis=1) for x in (g.waveform(k) for k in ids)])
    return waves, g.state(), ids


def _edge0(p):
    p = p.copy()
    p[..., 0] = 0.0
    p[..., -1] = 0.0
    return p


@pytest.mark.parametrize("kw,indep", [
    (dict(), True), (dict(), False),
    (dict(Ntheta=64, substeps=3, a=0.9), True),
    (dict(Ntheta=128, Nr=201, substeps=4, m=3), False),
    (dict(variable=0, m=-1, dt=0.02), True),
    (dict(Ntheta=40, s=0, m=1), False),
])
def test_dot_product(kw, indep):
    w = BASE.with_(**kw)
    g = _solver(w)
    np_ = 4 if indep else 2
    u0 = _edge0(_rand((np_, w.Ntheta, w.Nr), 11))
    dwave = _rand((len(w.observers), w.steps, 2), 12)
    dfin = _rand((4, w.Ntheta, w.Nr), 13)
    waves, final, _ = _forward(g, w, u0)
    grad = np.zeros((np_, w.Ntheta, w.Nr))
    g.adjoint(grad, dL_dwave=dwave, dL_dfinal=dfin, independent_pi=indep)
    lhs = float(np.sum(dwave * waves) + np.sum(dfin * final))
    rhs = float(np.sum(grad * u0))
    scale = float(np.sum(np.abs(dwave * waves)) + np.sum(np.abs(dfin * final)))
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs, scale)
    # the gradient of a waveform-only loss does not touch the solver's state
    before = g.state()
    g.adjoint(np.zeros((np_, w.Ntheta, w.Nr)), dL_dwave=dwave, independent_pi=indep)
    assert np.array_equal(g.state(), before)
    g.close()


def test_dot_product_against_oracle_forward():
    """J applied by the oracle, J^T by the GPU adjoint."""
    import oracle
    w = BASE.with_(a=0.9, Ntheta=64, steps=40)
    u0 = _edge0(_rand((2, w.Ntheta, w.Nr), 21))
    dwave = _rand((len(w.observers), w.steps, 2), 22)
    sol = oracle.Solver(M=w.M, a=w.a, s=w.s, m=w.m, rs_min=w.rs_min, rs_max=w.rs_max, Nr=w.Nr,
                        Ntheta=w.Ntheta, dt=w.dt, substeps=w.substeps, variable=w.variable)
    ids = [sol.add_observer(r, t) for r, t in w.observers]
    sol.set_initial(u0[0], u0[1])
    sol.run(w.steps)
    waves = np.stack([np.stack([x.real, x.imag], axis=1) for x in (sol.waveform(k) for k in ids)])
    g = _solver(w)
    g.set_initial(u0[0], u0[1])
    for r, t in w.observers:
        g.add_observer(r, t)
    g.step(w.steps)
    grad = np.zeros((2, w.Ntheta, w.Nr))
    g.adjoint(grad, dL_dwave=dwave)
    lhs = float(np.sum(dwave * waves))
    rhs = float(np.sum(grad * u0))
    scale = float(np.sum(np.abs(dwave * waves)))
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs)
    g.close()


def test_gaussian_parameter_gradients_match_finite_differences():
    import torch
    import paper_1010_3816_gb300 as tk
    w = BASE.with_(a=0.7, Ntheta=32, steps=80, center=5.0, width=3.0)
    g = _solver(w)
    for r, t in w.observers:
        g.add_observer(r, t)
    rs = torch.tensor(w.rs_min + np.arange(w.Nr) * w.drs, dtype=torch.float64, device="cuda")
    th = torch.tensor((np.arange(w.Ntheta) + 0.5) * (math.pi / w.Ntheta), dtype=torch.float64,
                      device="cuda")
    ang = torch.sin(th)[:, None] ** 2

    def planes(A, c, s):
        G = A * torch.exp(-((rs - c) ** 2) / (2.0 * s ** 2))
        re = ang * G[None, :]
        return re, torch.zeros_like(re)

    with torch.no_grad():
        tr, ti = planes(torch.tensor(1.07, device="cuda", dtype=torch.float64),
                        torch.tensor(5.4, device="cuda", dtype=torch.float64),
                        torch.tensor(2.8, device="cuda", dtype=torch.float64))
        target = tk.waveforms(g, tr, ti, w.steps).clone()

    def loss(A, c, s):
        re, im = planes(A, c, s)
        W = tk.waveforms(g, re, im, w.steps)
        return ((W - target) ** 2).sum()

    p = [torch.tensor(v, dtype=torch.float64, device="cuda", requires_grad=True) for v in (1.0, 5.0, 3.0)]
    L = loss(*p)
    L.backward()
    grads = [x.grad.item() for x in p]
    for k in range(3):
        h = 1e-5
        q = [x.detach().clone() for x in p]
        q[k] += h
        Lp = loss(*q).item()
        q[k] -= 2 * h
        Lm = loss(*q).item()
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - grads[k]) <= 1e-6 * max(abs(fd), 1e-12), (k, fd, grads[k])
    g.close()


def test_dot_product_full_size_adjoint_grid():
    """The 16001 x 128 Kerr a = 0.7 grid of the adjoint workload (k = 8), 15
    outer steps: <g, J u> = <J^T g, u>."""
    from inputs import ADJOINT_16001x128
    w = ADJOINT_16001x128.with_(steps=15, observers=((20.0, math.pi / 2), (40.0, 1.0)))
    g = _solver(w)
    u0 = _edge0(_rand((2, w.Ntheta, w.Nr), 31))
    dwave = _rand((len(w.observers), w.steps, 2), 32)
    dfin = _rand((4, w.Ntheta, w.Nr), 33)
    waves, final, _ = _forward(g, w, u0)
    grad = np.zeros((2, w.Ntheta, w.Nr))
    g.adjoint(grad, dL_dwave=dwave, dL_dfinal=dfin)
    lhs = float(np.sum(dwave * waves) + np.sum(dfin * final))
    rhs = float(np.sum(grad * u0))
    scale = float(np.sum(np.abs(dwave * waves)) + np.sum(np.abs(dfin * final)))
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs, scale)
    g.close()


@pytest.mark.parametrize("kw,indep", [
    (dict(), True),
    (dict(Ntheta=64, substeps=3, a=0.9), False),
    (dict(Ntheta=128, Nr=201, substeps=4, m=3), True),
    (dict(variable=0, m=-1, dt=0.02), False),
    (dict(Nr=2561, Ntheta=64, substeps=2, rs_max=130.0, steps=12), True),   # one 16-warp block per SM
    (dict(Nr=3701, Ntheta=32, rs_max=200.0, steps=10), False),               # one 24-warp block per SM
])
def test_persistent_adjoint_is_bit_identical_to_one_launch_per_step(kw, indep):
    """By default tk_adjoint runs every transposed step in one persistent
    launch (as tk_step runs the forward steps); with one launch per step set
    it launches each transposed step alone.  Same gradient, bit for bit."""
    import paper_1010_3816_gb300 as tk
    w = BASE.with_(**kw)
    np_ = 4 if indep else 2
    u0 = _edge0(_rand((np_, w.Ntheta, w.Nr), 31))
    dwave = _rand((len(w.observers), w.steps, 2), 32)
    dfin = _rand((4, w.Ntheta, w.Nr), 33)
    grads = []
    for spl in (-1, 1):
        g = _solver(w)
        g.set_steps_per_launch(spl)
        assert tk.tk_get_steps_per_launch(g.h) == spl
        _forward(g, w, u0)
        grad = np.zeros((np_, w.Ntheta, w.Nr))
        g.adjoint(grad, dL_dwave=dwave, dL_dfinal=dfin, independent_pi=indep)
        grads.append(grad)
        g.close()
    assert np.isfinite(grads[0]).all() and np.abs(grads[0]).max() > 0
    assert np.array_equal(grads[0], grads[1])
