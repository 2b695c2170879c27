"""CUDA path (through the C ABI) versus the CPU oracle, FP64.

The bar is 1e-12 relative L2 per plane (whole grid and r* >= 0) and per
waveform.  Grids span several warps' segments with a ragged last segment, all
three theta-row packings (1, 2, 4 rows per lane, with padding), both angular
variables, odd and even m, Kerr and Schwarzschild, sub-stepping, and the
degenerate sizes (Nr = 3, Ntheta = 2).
"""
import math

import numpy as np
import pytest

from inputs import KERR_25601x64, SCHWARZSCHILD_1601x32, Workload, initial_planes

from _parity import compare, rel_l2, run_gpu, run_oracle, sensitivity

pytestmark = pytest.mark.gpu

BASE = Workload(name="base", rs_min=-40.0, rs_max=60.0, Nr=803, Ntheta=32, dt=0.0625, steps=160,
                center=10.0, width=3.0, observers=((30.0, math.pi / 2), (17.31, 1.0), (60.0, 0.2)))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1010_3816_gb300 as tk
    tk.load_library()
    torch.zeros(1, device="cuda")


CASES = [
    dict(a=0.0, m=2, variable=1, Ntheta=32),
    dict(a=0.9, m=2, variable=1, Ntheta=64, noise=1e-3, seed=1),
    dict(a=0.99, m=3, variable=1, Ntheta=128, Nr=401, substeps=4),   # K = 4
    dict(a=0.7, m=-1, variable=0, Ntheta=32, dt=0.01),            # literal, odd m: parity -1
    dict(a=0.5, m=0, s=0, variable=1, Ntheta=33),                   # padding rows, K = 2
    dict(a=0.3, m=4, variable=0, Ntheta=16, dt=0.005),              # literal, even m
    dict(a=0.9, m=1, variable=1, Ntheta=100, Nr=301, substeps=3),   # K = 4 with padding
    dict(a=-0.6, m=2, variable=1, Ntheta=8, Nr=1999, dt=0.025),     # negative spin, many segments
    dict(a=0.8, m=-2, s=1, variable=1, Ntheta=48, angular="cos"),
]


@pytest.mark.parametrize("kw", CASES, ids=[f"case{k}" for k in range(len(CASES))])
def test_parity_small(kw):
    w = BASE.with_(**kw)
    res = compare(w, run_gpu(w), run_oracle(w))
    assert np.isfinite(list(res.values())).all()


def test_parity_host_inputs_and_chunked_steps():
    w = BASE.with_(a=0.9, Ntheta=64, noise=1e-3, seed=4)
    ref = run_oracle(w)
    compare(w, run_gpu(w, device_inputs=False, chunks=7), ref)


def test_initial_state_matches():
    w = BASE.with_(a=0.9, Ntheta=64, noise=1e-3, seed=5)
    gs, _ = run_gpu(w, steps=0)
    os_, _ = run_oracle(w, steps=0)
    assert np.array_equal(gs[:2], os_[:2])          # Phi is copied verbatim
    assert rel_l2(gs[2], os_[2]) < 1e-14 and rel_l2(gs[3], os_[3]) < 1e-14


def test_degenerate_sizes():
    for kw in (dict(Nr=3, Ntheta=2, rs_min=-1.0, rs_max=1.0, observers=((0.0, math.pi / 2),)),
               dict(Nr=4, Ntheta=2, rs_min=-1.0, rs_max=2.0, observers=((2.0, 0.75 * math.pi / 2),)),
               dict(Nr=5, Ntheta=3, rs_min=0.0, rs_max=4.0, a=0.9, observers=())):
        w = BASE.with_(center=0.0, width=0.7, steps=7, dt=0.2, **kw)
        compare(w, run_gpu(w), run_oracle(w))


def test_a0_imaginary_planes_exactly_zero():
    w = BASE.with_(a=0.0, steps=300)
    gs, gw = run_gpu(w)
    assert np.all(gs[1] == 0.0) and np.all(gs[3] == 0.0)
    assert all(np.all(x.imag == 0.0) for x in gw)


def test_spin_reversal_is_bitwise_conjugation_on_gpu():
    """a -> -a with real data conjugates the solution exactly; FMA and the
    folded tables preserve this to the bit."""
    w = BASE.with_(a=0.9, Ntheta=64)
    s1, w1 = run_gpu(w)
    s2, w2 = run_gpu(w.with_(a=-0.9))
    assert np.array_equal(s1[0], s2[0]) and np.array_equal(s1[2], s2[2])
    assert np.array_equal(s1[1], -s2[1]) and np.array_equal(s1[3], -s2[3])
    assert all(np.array_equal(x, np.conj(y)) for x, y in zip(w1, w2))


def test_schwarzschild_1601x32_full_run():
    """The 1601 x 32, 2000-step Schwarzschild workload in full.  The s = -2
    evolution amplifies rounding differences to ~2.5e-11 in Pi by t = 125 M:
    the oracle built with FMA contraction and the oracle from initial data
    changed by one ulp both differ from the plain oracle by that much, so each
    quantity is held to max(1e-12, 2 x the larger of the two); waveforms and
    Phi stay at 1e-12."""
    w = SCHWARZSCHILD_1601x32
    ref = run_oracle(w)
    res = compare(w, run_gpu(w), ref, perturbed=[sensitivity(w), run_oracle(w, build="fma")])
    assert res["wave0"] <= 1e-12 and res["PhiR"] <= 1e-12
    print(res)


def test_kerr_25601x64_full_grid_first_steps():
    """The 25601 x 64 Kerr grid in the launch configuration the benchmark
    times, compared element by element with the oracle over its first 120
    steps (the oracle cannot run all 38400 in a test)."""
    w = KERR_25601x64
    res = compare(w, run_gpu(w, steps=120), run_oracle(w, steps=120))
    print(res)


def test_schwarzschild_1601x32_literal_variable():
    """The 1601 x 32 workload in the literal variable Phi with the sin^2 data
    taken literally (not regular at theta = pi for s = -2, m = 2), four
    Lax-Wendroff steps per outer step (the literal pole stiffness needs
    dt <= dr*/8), 400 outer steps; held to the conditioned bar."""
    w = SCHWARZSCHILD_1601x32.with_(variable=0, substeps=4, steps=400)
    ref = run_oracle(w)
    res = compare(w, run_gpu(w), ref, perturbed=[sensitivity(w), run_oracle(w, build="fma")])
    print(res)


def test_kerr_25601x64_scalar_field_first_steps():
    """The scalar field (s = 0) on the full 25601 x 64 Kerr grid, 120 steps."""
    w = KERR_25601x64.with_(s=0)
    res = compare(w, run_gpu(w, steps=120), run_oracle(w, steps=120))
    print(res)


def test_kerr_25601x64_full_length_properties():
    """All 38400 steps of the 25601 x 64 Kerr workload: finite, waveform of the
    right length, and exact a -> -a conjugation on the full run."""
    import paper_1010_3816_gb300 as tk
    w = KERR_25601x64.with_(noise=0.0)     # real data for the conjugation property
    s1, w1 = run_gpu(w)
    s2, w2 = run_gpu(w.with_(a=-w.a))
    assert np.isfinite(s1).all()
    assert all(len(x) == w.steps for x in w1)
    assert np.array_equal(s1[1], -s2[1]) and np.array_equal(s1[0], s2[0])
    assert all(np.array_equal(x, np.conj(y)) for x, y in zip(w1, w2))


def test_state_round_trip_and_restart():
    """get_state / set_state restore bit-for-bit; a run split by a restore
    equals the uninterrupted run."""
    import torch
    import paper_1010_3816_gb300 as tk
    w = BASE.with_(a=0.7, Ntheta=64, noise=1e-3, seed=6)
    re, im = initial_planes(w)
    g = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt)
    g.precompute(w.a, w.M, w.s, w.m).set_initial(re, im)
    g.step(40)
    mid = g.state()
    dev = torch.empty((4, w.Ntheta, w.Nr), dtype=torch.float64, device="cuda")
    g.state(dev)
    assert np.array_equal(dev.cpu().numpy(), mid)
    g.step(40)
    end = g.state()
    g.set_state(mid)
    assert np.array_equal(g.state(), mid)
    g.step(40)
    assert np.array_equal(g.state(), end)
    g.set_state(dev)
    g.step(40)
    assert np.array_equal(g.state(), end)
    assert g.steps_done() == 160
    g.close()


def test_api_errors_and_order():
    import paper_1010_3816_gb300 as tk
    with pytest.raises(tk.TkError) as e:
        tk.tk_make_grid(1.0, 0.0, 10, 8, 0.1)
    assert e.value.status == tk.TK_ERR_ARG
    with pytest.raises(tk.TkError):
        tk.tk_make_grid(0.0, 1.0, 10, 129, 0.1)
    h = tk.tk_make_grid(-10.0, 10.0, 41, 8, 0.1)
    try:
        with pytest.raises(tk.TkError) as e:
            tk.tk_step(h, 1)
        assert e.value.status == tk.TK_ERR_STATE
        with pytest.raises(tk.TkError) as e:
            tk.tk_precompute_coeffs(h, 1.0, 1.0, -2, 2)
        assert e.value.status == tk.TK_ERR_ARG
        tk.tk_precompute_coeffs(h, 0.5, 1.0, -2, 2)
        z = np.zeros((8, 41))
        tk.tk_set_initial_data(h, z, z)
        with pytest.raises(tk.TkError):
            tk.tk_add_observer(h, 11.0, 1.0)
        k = tk.tk_add_observer(h, 10.0, 7.4 * (math.pi / 8))     # r*_max edge, last theta cell
        tk.tk_step(h, 0)
        tk.tk_step(h, 3)
        with pytest.raises(tk.TkError) as e:
            tk.tk_add_observer(h, 0.0, 1.0)
        assert e.value.status == tk.TK_ERR_STATE
        assert np.all(tk.tk_extract(h, k) == 0.0) and len(tk.tk_extract(h, k)) == 3
        tk.tk_check_finite(h)
    finally:
        tk.tk_destroy(h)


def test_nonfinite_detection():
    import paper_1010_3816_gb300 as tk
    h = tk.tk_make_grid(-10.0, 10.0, 41, 8, 0.1)
    try:
        tk.tk_precompute_coeffs(h, 0.5, 1.0, -2, 2)
        z = np.zeros((8, 41))
        bad = z.copy()
        bad[3, 7] = np.nan
        tk.tk_set_initial_data(h, bad, z)
        with pytest.raises(tk.TkError) as e:
            tk.tk_check_finite(h)
        assert e.value.status == tk.TK_ERR_UNSTABLE
    finally:
        tk.tk_destroy(h)


def test_stability_bound():
    """tk_stability_bound: the literal variable is far stiffer than the
    regularised one (R7: the 1601 x 32 literal run needs dt ~ dr*/8), the
    bound tightens with Ntheta, and a radial CFL violation is caught."""
    import paper_1010_3816_gb300 as tk
    w = SCHWARZSCHILD_1601x32

    def bound(**kw):
        v = w.with_(**kw)
        g = tk.Solver(rstar_min=v.rs_min, rstar_max=v.rs_max, Nr=v.Nr, Ntheta=v.Ntheta, dt=v.dt,
                      variable=v.variable)
        g.precompute(v.a, v.M, v.s, v.m)
        r = g.stability_bound(2.5e-5)
        g.close()
        return r

    dl, kl = bound(variable=0)
    dr, kr = bound(variable=1)
    d64, k64 = bound(variable=1, Ntheta=64)
    assert kl >= 3 and kl > kr >= 1, (kl, kr)
    assert d64 < dr
    dc, kc = bound(variable=1, dt=2.0 * w.drs)
    assert kc >= 2 and dc <= w.drs * 1.0001
    print({"literal": (dl, kl), "regularised": (dr, kr), "regularised Ntheta=64": (d64, k64)})


def test_graph_replay_matches_direct_launches():
    """Chunks replayed from a captured CUDA graph give bit-identical states and
    waveforms to step-by-step launches (odd substep counts included)."""
    import paper_1010_3816_gb300 as tk
    w = BASE.with_(a=0.9, Ntheta=64, noise=1e-3, seed=8, substeps=3)
    re, im = initial_planes(w)
    out = []
    for chunk in (0, -1, 5, 1):
        g = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt,
                      substeps=w.substeps)
        g.precompute(w.a, w.M, w.s, w.m).set_initial(re, im)
        ids = [g.add_observer(r, t) for r, t in w.observers]
        g.set_steps_per_launch(1)        # this grid would otherwise run as one persistent launch
        g.set_graph_chunk(chunk)
        g.step(100)
        g.step(3)
        g.step(100)
        out.append((g.state(), [g.waveform(k) for k in ids]))
        assert g.steps_done() == 203
        g.close()
    for s, wv in out[1:]:
        assert np.array_equal(s, out[0][0])
        assert all(np.array_equal(a, b) for a, b in zip(wv, out[0][1]))


def _oracle_coefficients(w):
    """The oracle's raw coefficient tables in the layout of tk_set_coefficients
    (half node i at r*_{i+1/2}) and its regularised angular stencil."""
    import oracle
    sol = oracle.Solver(M=w.M, a=w.a, s=w.s, m=w.m, rs_min=w.rs_min, rs_max=w.rs_max, Nr=w.Nr,
                        Ntheta=w.Ntheta, dt=w.dt, substeps=w.substeps, variable=w.variable)
    node, half = sol.coeffs()
    half9 = np.zeros_like(half)
    half9[:, :, :-1] = half[:, :, 1:]
    ang2 = np.stack(oracle.regular_stencil(w.s, w.m, w.Ntheta)) if w.variable else None
    return np.ascontiguousarray(node), half9, ang2


def run_gpu_with_coefficients(w, node9, half9, ang2, steps=None, precision=0):
    """run_gpu with the coefficients supplied through tk_set_coefficients."""
    import torch
    import paper_1010_3816_gb300 as tk
    g = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt,
                  substeps=w.substeps, variable=w.variable, precision=precision)
    try:
        tk.tk_set_coefficients(g.h, w.a, w.M, w.s, w.m, node9, half9, ang2)
        re, im = initial_planes(w)
        g.set_initial(torch.from_numpy(re).cuda(), torch.from_numpy(im).cuda())
        ids = [g.add_observer(r, t) for r, t in w.observers]
        g.step(w.steps if steps is None else steps)
        return g.state(), [g.waveform(k) for k in ids]
    finally:
        g.close()


@pytest.mark.parametrize("kw", [dict(a=0.9, Ntheta=64, noise=1e-3, seed=6),
                                dict(a=0.7, m=-1, variable=0, Ntheta=32, dt=0.01)])
def test_parity_with_the_oracles_coefficients(kw):
    """tk_set_coefficients: the step from the oracle's own coefficient tables
    (and its angular stencil) matches the oracle at the 1e-12 bar, and differs
    from the step from the library's precompute only by the rounding of the
    coefficients."""
    w = BASE.with_(**kw)
    node9, half9, ang2 = _oracle_coefficients(w)
    ref = run_oracle(w)
    mine = run_gpu_with_coefficients(w, node9, half9, ang2)
    compare(w, mine, ref)
    own = run_gpu(w)
    d = rel_l2(mine[0], own[0])
    assert 0.0 <= d < 1e-12, d


def test_set_coefficients_rejects_bad_calls():
    import paper_1010_3816_gb300 as tk
    w = BASE
    node9, half9, ang2 = _oracle_coefficients(w)
    g = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt,
                  substeps=0)
    with pytest.raises(tk.TkError) as e:            # the solver picks its own substeps
        tk.tk_set_coefficients(g.h, w.a, w.M, w.s, w.m, node9, half9, ang2)
    assert e.value.status == tk.TK_ERR_STATE
    g.close()
    g = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt)
    with pytest.raises(tk.TkError) as e:
        tk.tk_set_coefficients(g.h, 1.0, 1.0, w.s, w.m, node9, half9, ang2)    # |a| = M
    assert e.value.status == tk.TK_ERR_ARG
    g.close()


@pytest.mark.parametrize("kw", [dict(a=0.9, Ntheta=64, noise=1e-3, seed=6),
                                dict(a=0.7, m=-1, variable=0, Ntheta=32, dt=0.01),
                                dict(a=0.9, rs_min=-100.0, rs_max=40.0, Nr=1121, Ntheta=16, steps=40,
                                     observers=((30.0, math.pi / 2), (-90.0, 1.0)))])
def test_get_coefficients_round_trip_and_oracle_agreement(kw):
    """tk_get_coefficients exports the precompute's raw coefficients: they are
    the oracle's to FP64 evaluation error (c1R, which cancels near the horizon
    and far out, only where it does not), and fed back through
    tk_set_coefficients they reproduce the default run bit for bit (the fold is
    the same code from the same values)."""
    import paper_1010_3816_gb300 as tk
    w = BASE.with_(**kw)
    g = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt,
                  substeps=w.substeps, variable=w.variable)
    with pytest.raises(tk.TkError) as e:
        tk.tk_get_coefficients(g.h, (w.Ntheta, w.Nr))
    assert e.value.status == tk.TK_ERR_STATE              # before the precompute
    g.precompute(w.a, w.M, w.s, w.m)
    node9, half9 = tk.tk_get_coefficients(g.h, (w.Ntheta, w.Nr))
    g.close()
    assert np.all(half9[:, :, -1] == 0)
    on, oh9, _ = _oracle_coefficients(w)
    rs = w.rs_min + np.arange(w.Nr) * w.drs
    import oracle
    for mine, ref in ((node9, on), (half9, oh9)):
        for q, name in enumerate(oracle.COEF_NAMES):
            colmax = np.abs(ref[q]).max(axis=0, keepdims=True)
            d = np.abs(mine[q] - ref[q]) / np.where(colmax > 0, colmax, 1.0)
            if name == "c1R":
                d = d[:, (rs > -30.0) & (rs < 60.0)]
                assert d.max() < 1e-9, name
            else:
                assert d.max() < 1e-10, (name, d.max())
    mine = run_gpu_with_coefficients(w, node9, half9, None)
    own = run_gpu(w)
    assert np.array_equal(mine[0], own[0])
    for a, b in zip(mine[1], own[1]):
        assert np.array_equal(a, b)
