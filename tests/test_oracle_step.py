"""Pins of the oracle's Lax-Wendroff step (Eqs. lw1, lw2; Sec. 3.2 and 4).

* kernel_average1 (Sec. 4): bit-exact half-sums.
* Brute force: the one-step map is assembled as an explicit matrix from the
  formulas of Eqs. (lw1) and (lw2) -- averaging and difference matrices, the
  4x4 D blocks, the source S with its centred angular stencils (ghost parity
  for the literal field, the self-adjoint form for the regularised one), the
  radial edge condition -- and must reproduce the oracle's step.
* Exact symmetries of Eq. 1: a = 0 keeps real data real; a -> -a conjugates;
  m -> -m mirrors theta -> pi - theta and conjugates.
* The initial momentum rule and the radial boundary condition.
"""
import math

import numpy as np
import pytest

from inputs import Workload, initial_planes


def _solver(oracle_mod, w: Workload):
    return oracle_mod.Solver(M=w.M, a=w.a, s=w.s, m=w.m, rs_min=w.rs_min, rs_max=w.rs_max,
                             Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt, substeps=w.substeps,
                             variable=w.variable)


def test_kernel_average1_bit_exact(oracle_mod):
    rng = np.random.default_rng(5)
    q = rng.standard_normal((7, 33)) * 10.0 ** rng.integers(-5, 5, size=(7, 33))
    h = oracle_mod.average(q)
    want = 0.5 * (q[:, 1:] + q[:, :-1])
    assert np.array_equal(h[:, 1:], want)
    assert np.all(h[:, 0] == 0.0)


# --- brute-force explicit matrix ---------------------------------------------------
def _angular_mats(N, parity):
    """Centred second and first theta differences on the cell-centred grid
    theta_j = (j + 1/2) pi/N with ghosts F_{-1} = p F_0, F_N = p F_{N-1}."""
    dth = math.pi / N
    T2 = np.zeros((N, N))
    T1 = np.zeros((N, N))
    for j in range(N):
        for jj, c2, c1 in ((j - 1, 1.0, -1.0), (j, -2.0, 0.0), (j + 1, 1.0, 1.0)):
            if jj < 0:
                jj, f = 0, parity
            elif jj >= N:
                jj, f = N - 1, parity
            else:
                f = 1.0
            T2[j, jj] += f * c2 / dth ** 2
            T1[j, jj] += f * c1 / (2 * dth)
    return T2, T1


def _regular_mat(N, s, m):
    """Self-adjoint centred stencil of (1/P) d_th (P d_th F), P = sin w^2, on the
    cell-centred grid: faces at j dth carry P (zero at the poles), cells carry
    the mean of P over the cell (here by adaptive quadrature)."""
    from scipy.integrate import quad
    dth = math.pi / N
    al, be = abs(m + s) / 2, abs(m - s) / 2

    def P(t):
        return math.sin(t) * ((1 - math.cos(t)) ** al * (1 + math.cos(t)) ** be) ** 2

    faces = [0.0] + [P(f * dth) for f in range(1, N)] + [0.0]
    T = np.zeros((N, N))
    for j in range(N):
        Q = quad(P, j * dth, (j + 1) * dth, epsabs=0, epsrel=2e-14, limit=200)[0] / dth
        if j > 0:
            T[j, j - 1] += faces[j] / (Q * dth * dth)
            T[j, j] -= faces[j] / (Q * dth * dth)
        if j < N - 1:
            T[j, j + 1] += faces[j + 1] / (Q * dth * dth)
            T[j, j] -= faces[j + 1] / (Q * dth * dth)
    return T


def _lw_matrix(C_node, C_half, Nr, N, drs, dt, parity, regular=None):
    """Explicit matrix of one step u^n -> u^{n+1}.  State ordering: component
    k (PhiR, PhiI, PiR, PiI), then theta row j, then radial index i.
    Half nodes i + 1/2, i = 0..Nr-2, are indexed by i; the coefficient table
    C_half stores them at column i + 1 (the paper's kernel_average1 places the
    average of columns i and i+1 at index i + 1)."""
    nh = Nr - 1

    def vid(k, j, i, ncol):
        return (k * N + j) * ncol + i

    n_full, n_half = 4 * N * Nr, 4 * N * nh
    T2, T1 = _angular_mats(N, parity)
    TR = None if regular is None else _regular_mat(N, *regular)

    def blocks(C):
        b, c1, c2, c3 = C[0], C[1] + 1j * C[2], C[3] + 1j * C[4], C[5] + 1j * C[6]
        return b, c1, c2, c3, C[7], C[8]

    def cmat(z):
        return np.array([[z.real, -z.imag], [z.imag, z.real]])

    def bracket_ops(coef_at, ncol_out, cols_out):
        """Matrices (Dm, Sm) with bracket = Dm @ du / drs - Sm @ ubar, both on
        vectors indexed over the output columns."""
        n = 4 * N * ncol_out
        Dm = np.zeros((n, n))
        Sm = np.zeros((n, n))
        for j in range(N):
            for c, i in enumerate(cols_out):
                b, c1, c2, c3, c4, c5 = blocks(coef_at(j, i))
                P = [vid(0, j, c, ncol_out), vid(1, j, c, ncol_out)]
                Q = [vid(2, j, c, ncol_out), vid(3, j, c, ncol_out)]
                for r in range(2):
                    Dm[P[r], P[r]] = b
                    Dm[Q[r], Q[r]] = -b
                    Sm[P[r], Q[r]] = 1.0                      # S_Phi = Pi
                C1, C2, C3 = cmat(c1), cmat(c2), cmat(c3)
                for r in range(2):
                    for s_ in range(2):
                        Dm[Q[r], P[s_]] = -C1[r, s_]
                        Sm[Q[r], Q[s_]] += C2[r, s_]
                        Sm[Q[r], P[s_]] += C3[r, s_]
                for jj in range(N):
                    ang = c4 * T2[j, jj] + c5 * T1[j, jj] if TR is None else c4 * TR[j, jj]
                    for r in range(2):
                        Sm[Q[r], vid(r, jj, c, ncol_out)] += ang
        return Dm, Sm

    # averaging / difference from full columns to half columns
    A1 = np.zeros((n_half, n_full))
    G1 = np.zeros((n_half, n_full))
    for k in range(4):
        for j in range(N):
            for i in range(nh):
                A1[vid(k, j, i, nh), vid(k, j, i, Nr)] = 0.5
                A1[vid(k, j, i, nh), vid(k, j, i + 1, Nr)] = 0.5
                G1[vid(k, j, i, nh), vid(k, j, i, Nr)] = -1.0
                G1[vid(k, j, i, nh), vid(k, j, i + 1, Nr)] = 1.0
    Dh, Sh = bracket_ops(lambda j, i: C_half[:, j, i + 1], nh, list(range(nh)))
    # Eq. (lw1)
    Mh = A1 - 0.5 * dt * (Dh @ G1 / drs - Sh @ A1)

    # from half columns to interior full columns 1..Nr-2
    ni = Nr - 2
    n_int = 4 * N * ni
    A2 = np.zeros((n_int, n_half))
    G2 = np.zeros((n_int, n_half))
    E = np.zeros((n_int, n_full))     # restriction of u^n to interior nodes
    for k in range(4):
        for j in range(N):
            for c in range(ni):
                i = c + 1
                A2[vid(k, j, c, ni), vid(k, j, i - 1, nh)] = 0.5
                A2[vid(k, j, c, ni), vid(k, j, i, nh)] = 0.5
                G2[vid(k, j, c, ni), vid(k, j, i - 1, nh)] = -1.0
                G2[vid(k, j, c, ni), vid(k, j, i, nh)] = 1.0
                E[vid(k, j, c, ni), vid(k, j, i, Nr)] = 1.0
    Dn, Sn = bracket_ops(lambda j, i: C_node[:, j, i], ni, list(range(1, Nr - 1)))
    # Eq. (lw2)
    Mint = E - dt * (Dn @ G2 / drs - Sn @ A2) @ Mh
    # radial edges stay zero: scatter the interior rows back into the full state
    M = np.zeros((n_full, n_full))
    for k in range(4):
        for j in range(N):
            for c in range(ni):
                M[vid(k, j, c + 1, Nr), :] = Mint[vid(k, j, c, ni), :]
    return M


@pytest.mark.parametrize("a,s,m,variable,Nr,N", [
    (0.7, -2, 3, 0, 9, 4),       # literal, odd m: ghost parity -1
    (0.9, -2, 2, 1, 9, 5),       # regularised, odd Ntheta
    (0.5, 0, 1, 1, 11, 4),
    (0.0, -2, 2, 0, 8, 3),
])
def test_one_step_matches_explicit_matrix(oracle_mod, a, s, m, variable, Nr, N):
    w = Workload(name="tiny", a=a, s=s, m=m, variable=variable, rs_min=-3.0, rs_max=5.0,
                 Nr=Nr, Ntheta=N, dt=0.5, substeps=1, steps=1)
    sol = _solver(oracle_mod, w)
    rng = np.random.default_rng(11)
    u0 = rng.standard_normal((4, N, Nr))
    u0[:, :, 0] = 0.0
    u0[:, :, -1] = 0.0
    sol.set_initial(u0[0], u0[1], u0[2], u0[3])
    node, half = sol.coeffs()
    M = _lw_matrix(node, half, Nr, N, w.drs, w.dt, oracle_mod.parity(m, variable),
                   regular=(s, m) if variable == 1 else None)
    want = (M @ u0.reshape(-1)).reshape(4, N, Nr)
    sol.run(1)
    got = sol.state()
    err = np.max(np.abs(got - want)) / np.max(np.abs(want))
    assert err < 1e-14, err
    # two steps and the substep split: one outer step of 2 dt in 2 inner steps
    want2 = (M @ (M @ u0.reshape(-1))).reshape(4, N, Nr)
    sol.run(1)
    err2 = np.max(np.abs(sol.state() - want2)) / np.max(np.abs(want2))
    assert err2 < 1e-14, err2
    w2 = w.with_(dt=2 * w.dt, substeps=2)
    sol2 = _solver(oracle_mod, w2)
    sol2.set_initial(u0[0], u0[1], u0[2], u0[3])
    sol2.run(1)
    assert np.array_equal(sol2.state(), sol.state())


# --- symmetries -------------------------------------------------------------------
SMALL = Workload(name="small", rs_min=-30.0, rs_max=70.0, Nr=401, Ntheta=8, dt=0.125,
                 steps=160, center=10.0, width=3.0)


def test_a0_real_data_stay_real(oracle_mod):
    sol = _solver(oracle_mod, SMALL)
    re, im = initial_planes(SMALL)
    sol.set_initial(re, im)
    sol.run(SMALL.steps)
    st = sol.state()
    assert np.max(np.abs(st[0])) > 1e-3
    assert np.all(st[1] == 0.0) and np.all(st[3] == 0.0)


@pytest.mark.parametrize("variable", [0, 1])
def test_spin_reversal_conjugates_bitwise(oracle_mod, variable):
    """Eq. 1 with a -> -a is the complex conjugate equation: real initial data
    give Phi(-a) = conj Phi(a) exactly."""
    wl = SMALL.with_(a=0.9, m=2, variable=variable, steps=120)
    re, im = initial_planes(wl)
    out = []
    for a in (0.9, -0.9):
        sol = _solver(oracle_mod, wl.with_(a=a))
        o = sol.add_observer(20.0, 1.0)
        sol.set_initial(re, im)
        sol.run(wl.steps)
        out.append((sol.state(), sol.waveform(o)))
    (s1, w1), (s2, w2) = out
    assert np.max(np.abs(s1[1])) > 1e-6
    assert np.array_equal(s1[0], s2[0]) and np.array_equal(s1[2], s2[2])
    assert np.array_equal(s1[1], -s2[1]) and np.array_equal(s1[3], -s2[3])
    assert np.array_equal(w1, np.conj(w2))


@pytest.mark.parametrize("variable", [0, 1])
def test_mode_reversal_mirrors_theta(oracle_mod, variable):
    """Phi_{-m}(t, r, theta) = conj Phi_m(t, r, pi - theta) for real initial
    data symmetric about the equator; equal up to rounding."""
    wl = SMALL.with_(a=0.7, m=3, variable=variable, steps=120)
    re, im = initial_planes(wl)
    assert np.allclose(re, re[::-1], rtol=0, atol=1e-15)
    res = []
    for m in (3, -3):
        sol = _solver(oracle_mod, wl.with_(m=m))
        sol.set_initial(re, im)
        sol.run(wl.steps)
        res.append(sol.state())
    s1, s2 = res
    mir = s2[:, ::-1, :].copy()
    mir[1] *= -1
    mir[3] *= -1
    scale = np.max(np.abs(s1))
    assert np.max(np.abs(s1 - mir)) < 1e-12 * scale


def test_initial_momentum_and_edges(oracle_mod):
    """Pi(0) = b (Phi_{i+1} - Phi_{i-1}) / (2 dr*) at interior nodes (zero time
    derivative, Pi = d_t Phi + b d_* Phi), and Phi = Pi = 0 on the radial edges.
    For a field linear in r*, the centred difference is exact."""
    wl = Workload(name="lin", a=0.6, rs_min=-10.0, rs_max=10.0, Nr=41, Ntheta=6, dt=0.25)
    sol = _solver(oracle_mod, wl)
    rs = wl.rs_min + np.arange(wl.Nr) * wl.drs
    re = np.tile(3.0 * rs + 1.0, (wl.Ntheta, 1))
    im = np.tile(-2.0 * rs, (wl.Ntheta, 1))
    sol.set_initial(re, im)
    st = sol.state()
    node, _ = sol.coeffs()
    b = node[0]
    assert np.all(st[:, :, 0] == 0.0) and np.all(st[:, :, -1] == 0.0)
    assert np.allclose(st[2][:, 1:-1], 3.0 * b[:, 1:-1], rtol=1e-13, atol=0)
    assert np.allclose(st[3][:, 1:-1], -2.0 * b[:, 1:-1], rtol=1e-13, atol=0)
    assert np.array_equal(st[0][:, 1:-1], re[:, 1:-1])
    # edges stay zero after steps
    sol.run(3)
    st = sol.state()
    assert np.all(st[:, :, 0] == 0.0) and np.all(st[:, :, -1] == 0.0)


def test_extraction_is_bilinear(oracle_mod):
    """The waveform sample is the bilinear interpolant of Phi = w Phi^.  With
    dt tiny the state barely moves in one step; compare against the formula on
    the stepped state."""
    wl = Workload(name="ext", a=0.3, m=1, rs_min=-10.0, rs_max=10.0, Nr=81, Ntheta=10, dt=1e-3,
                  variable=1)
    sol = _solver(oracle_mod, wl)
    re, im = initial_planes(wl.with_(center=0.0, width=3.0, noise=0.2, seed=9))
    sol.set_initial(re, im)
    rs_obs, th_obs = 1.13, 1.0
    o = sol.add_observer(rs_obs, th_obs)
    sol.run(1)
    st = sol.state()
    dth = math.pi / wl.Ntheta
    fi = (rs_obs - wl.rs_min) / wl.drs
    fj = th_obs / dth - 0.5
    i0, j0 = int(math.floor(fi)), int(math.floor(fj))
    fr, ft = fi - i0, fj - j0
    wts = [oracle_mod.weight(wl.s, wl.m, 1, (j + 0.5) * dth) for j in (j0, j0 + 1)]
    phi = (st[0] + 1j * st[1])
    lo = (1 - ft) * wts[0] * phi[j0, i0] + ft * wts[1] * phi[j0 + 1, i0]
    hi = (1 - ft) * wts[0] * phi[j0, i0 + 1] + ft * wts[1] * phi[j0 + 1, i0 + 1]
    want = (1 - fr) * lo + fr * hi
    got = sol.waveform(o)
    assert got.shape == (1,)
    assert abs(got[0] - want) <= 1e-14 * abs(want)
    with pytest.raises(ValueError):
        sol.add_observer(wl.rs_max + 1.0, 1.0)
    with pytest.raises(ValueError):
        sol.add_observer(0.0, 0.5 * dth * 0.9)


def test_coefficient_tables_sit_at_nodes_and_half_nodes(oracle_mod):
    """Eq. (lw1) takes D and S at r*_{i+1/2}, Eq. (lw2) at r*_i: the tables
    hold the coefficients evaluated exactly there (not averaged), on the
    cell-centred theta rows."""
    wl = Workload(name="tab", a=0.8, m=-1, rs_min=-20.0, rs_max=30.0, Nr=51, Ntheta=6, dt=0.5)
    sol = _solver(oracle_mod, wl)
    node, half = sol.coeffs()
    for b in (0, 2, 5):
        th = (b + 0.5) * (math.pi / wl.Ntheta)     # theta_b = (b + 1/2) dtheta
        for a in (1, 7, 25, 50):
            xn = oracle_mod.x_of_rstar(wl.M, wl.a, wl.rs_min + a * wl.drs)
            xh = oracle_mod.x_of_rstar(wl.M, wl.a, wl.rs_min + (a - 0.5) * wl.drs)
            cn = oracle_mod.coeffs_point(wl.M, wl.a, wl.s, wl.m, wl.variable, xn, th)
            ch = oracle_mod.coeffs_point(wl.M, wl.a, wl.s, wl.m, wl.variable, xh, th)
            assert list(node[:, b, a]) == list(cn.values())
            assert list(half[:, b, a]) == list(ch.values())


def test_fma_build_is_another_rounding_of_the_same_scheme():
    """The oracle source compiled with FMA contraction (the second rounding
    order the full-length parity bar is measured with) computes the same
    scheme: after 60 steps of a Kerr case its fields differ from the plain
    build's by rounding only -- not at all in the bits would mean the
    contraction did not happen."""
    import math
    import oracle
    from inputs import Workload, initial_planes
    w = Workload(name="fma", a=0.9, rs_min=-30.0, rs_max=50.0, Nr=321, Ntheta=16, dt=0.125,
                 steps=60, center=5.0, width=3.0, noise=1e-3, seed=11, observers=((20.0, math.pi / 2),))
    out = []
    for build in ("plain", "fma"):
        sol = oracle.Solver(M=w.M, a=w.a, s=w.s, m=w.m, rs_min=w.rs_min, rs_max=w.rs_max, Nr=w.Nr,
                            Ntheta=w.Ntheta, dt=w.dt, substeps=w.substeps, variable=w.variable,
                            build=build)
        k = sol.add_observer(*w.observers[0])
        sol.set_initial(*initial_planes(w))
        sol.run(w.steps)
        out.append((sol.state(), sol.waveform(k)))
    (s0, w0), (s1, w1) = out
    d = np.linalg.norm(s1 - s0) / np.linalg.norm(s0)
    dw = np.linalg.norm(w1 - w0) / np.linalg.norm(w0)
    assert 0.0 < d < 1e-12 and dw < 1e-12, (d, dw)


def test_replace_coeffs_round_trip():
    """replace_coeffs writes exactly what coeffs() reads, and a run with the
    tables put back unchanged is bit-identical to one never touched."""
    import math
    import oracle
    from inputs import Workload, initial_planes
    w = Workload(name="rc", a=0.7, rs_min=-20.0, rs_max=30.0, Nr=201, Ntheta=8, dt=0.125, steps=20,
                 center=3.0, width=2.0, observers=((10.0, math.pi / 2),))
    out = []
    for touch in (False, True):
        sol = oracle.Solver(M=w.M, a=w.a, s=w.s, m=w.m, rs_min=w.rs_min, rs_max=w.rs_max, Nr=w.Nr,
                            Ntheta=w.Ntheta, dt=w.dt, substeps=w.substeps, variable=w.variable)
        if touch:
            node, half = sol.coeffs()
            sol.replace_coeffs(node.copy(), half.copy())
            n2, h2 = sol.coeffs()
            assert np.array_equal(n2, node) and np.array_equal(h2, half)
        sol.set_initial(*initial_planes(w))
        sol.run(w.steps)
        out.append(sol.state())
    assert np.array_equal(out[0], out[1])
