"""Pins of the oracle's angular discretisation (Sec. 3.2: 2nd-order centred
angular differences; angular boundary conditions from the symmetries of the
harmonics).

At a = 0 the angular part of the source divided by c4 is the spin-weighted
spherical-harmonic operator
    L = d_thth + cot d_th - (m + s cos)^2 / sin^2 + s,
whose eigenvalues are -(l - s)(l + s + 1), l = max(|m|, |s|), max+1, ...
The discrete operator on the cell-centred grid must reproduce them with an
O(dtheta^2) error, in both the literal and the pole-regularised variable (the
latter is a similarity transform of the former).
"""
import math

import numpy as np
import pytest


def _matrix(oracle_mod, s, m, variable, N):
    A = oracle_mod.angular_matrix(s, m, variable, N)
    e = np.zeros(N)
    e[N // 3] = 1.0
    assert np.array_equal(A[:, N // 3], oracle_mod.angular_apply(s, m, variable, e))
    return A


def _top_eigs(A, n):
    """The n eigenvalues with the largest real part (the low-l modes)."""
    ev = np.linalg.eigvals(A)
    ev = ev[np.argsort(-ev.real)][:n]
    assert np.max(np.abs(ev.imag)) < 1e-8 * np.max(np.abs(ev.real))
    return ev.real


@pytest.mark.parametrize("variable", [0, 1])
@pytest.mark.parametrize("s,m", [(-2, 2), (-2, 3), (-2, -4), (0, 1), (-1, 2)])
def test_angular_operator_has_real_negative_spectrum(oracle_mod, s, m, variable):
    """Every eigenvalue of the discrete operator is real and negative, at every
    resolution: angular modes oscillate in time, none grows.  (A centred
    non-self-adjoint differencing of the regularised operator fails this near
    the poles for Ntheta >= 64, with complex pairs that make rounding errors grow.)"""
    if variable == 0 and s % 2 != 0:
        pytest.skip("literal parity rule matches regularity only for even s")
    for N in (32, 64, 128):
        ev = np.linalg.eigvals(_matrix(oracle_mod, s, m, variable, N))
        assert np.max(np.abs(ev.imag)) == 0.0, (N, np.max(np.abs(ev.imag)))
        assert np.max(ev.real) < 0.0


def test_regularised_stencil_is_self_adjoint(oracle_mod):
    """Q_j Ap_j = Q_{j+1} Am_{j+1} (symmetry in the Q-weighted inner product,
    checked through the face weights) and no flux through the poles."""
    for s, m in [(-2, 2), (-2, 3), (0, 0), (-2, -1)]:
        N = 48
        Ap, Am = oracle_mod.regular_stencil(s, m, N)
        assert Am[0] == 0.0 and Ap[-1] == 0.0
        # Ap_j / Am_{j+1} = Q_{j+1} / Q_j > 0: the off-diagonal products are positive
        assert np.all(Ap[:-1] > 0) and np.all(Am[1:] > 0)


def _exact(s, m, n):
    l0 = max(abs(m), abs(s))
    return np.array([-(l - s) * (l + s + 1) for l in range(l0, l0 + n)], dtype=float)


@pytest.mark.parametrize("variable", [0, 1])
@pytest.mark.parametrize("s,m", [(-2, 2), (-2, 3), (-2, -2), (-2, 0), (0, 0), (0, 1), (-2, 4)])
def test_discrete_angular_spectrum_converges(oracle_mod, s, m, variable):
    """Even s: the paper's parity (-1)^|m| equals the harmonics' regularity
    parity (-1)^(m+s), so the literal scheme is consistent."""
    n = 3
    exact = _exact(s, m, n)
    errs = []
    for N in (32, 64, 128):
        ev = _top_eigs(_matrix(oracle_mod, s, m, variable, N), n)
        errs.append(np.max(np.abs(ev - exact)))
    # s = -2, m = 2: the exact values are -(l-s)(l+s+1) = -4, -10, -18 for l = 2, 3, 4
    assert errs[-1] < 2e-2 * np.max(np.abs(exact))
    # second order: halving dtheta divides the error by ~4
    assert errs[0] / errs[1] > 3.3 and errs[1] / errs[2] > 3.3, errs


def test_spectrum_values_s_minus2_m2(oracle_mod):
    """Nθ = 32 and 64 give eigenvalues close to -4, -10, -18 (l = 2, 3, 4)."""
    for N, tol in ((32, 0.05), (64, 0.012)):
        ev = _top_eigs(_matrix(oracle_mod, -2, 2, 1, N), 3)
        assert np.allclose(ev, [-4.0, -10.0, -18.0], atol=tol * 18), ev


def test_regularised_weight_is_lowest_harmonic():
    """(L_theta + V_theta) w = -lambda0 w for w = (1-cos)^al (1+cos)^be,
    al = |m+s|/2, be = |m-s|/2, lambda0 = (l0-s)(l0+s+1), l0 = max(|m|,|s|):
    the identity behind the pole-regularised variable."""
    sp = pytest.importorskip("sympy")
    th = sp.symbols("th", real=True)
    for s in (-2, -1, 0, 1, 2):
        for m in range(-4, 5):
            al = sp.Rational(abs(m + s), 2)
            be = sp.Rational(abs(m - s), 2)
            l0 = max(abs(m), abs(s))
            lam0 = (l0 - s) * (l0 + s + 1)
            w = (1 - sp.cos(th)) ** al * (1 + sp.cos(th)) ** be
            L = (sp.diff(w, th, 2) + sp.cos(th) / sp.sin(th) * sp.diff(w, th)
                 - (m + s * sp.cos(th)) ** 2 / sp.sin(th) ** 2 * w + s * w)
            for tv in (0.3, 1.2, 2.5):
                tvh = sp.Float(tv, 50)
                val = complex((L + lam0 * w).subs(th, tvh).evalf(50))
                ref = abs(complex(w.subs(th, tvh).evalf(50))) * (1 + lam0)
                assert abs(val) < 1e-30 * max(ref, 1.0), (s, m, tv, val)


def test_ghost_parity_rules(oracle_mod):
    """The paper: d_theta Phi = 0 at the poles for even |m| (ghost equal),
    Phi = 0 for odd |m| (ghost opposite); the regularised field is even."""
    assert oracle_mod.parity(2, 0) == 1
    assert oracle_mod.parity(-4, 0) == 1
    assert oracle_mod.parity(3, 0) == -1
    assert oracle_mod.parity(-1, 0) == -1
    for m in range(-4, 5):
        assert oracle_mod.parity(m, 1) == 1


def test_weight_values(oracle_mod):
    """w(theta) = (1-cos)^al (1+cos)^be; literal variable has w = 1."""
    for s, m in [(-2, 2), (-2, 3), (0, 1), (-2, -1)]:
        al, be = abs(m + s) / 2, abs(m - s) / 2
        for th in (0.01, 0.7, math.pi / 2, 2.9):
            want = (1 - math.cos(th)) ** al * (1 + math.cos(th)) ** be
            got = oracle_mod.weight(s, m, 1, th)
            assert abs(got - want) <= 1e-12 * max(want, 1e-300) + 1e-300
            assert oracle_mod.weight(s, m, 0, th) == 1.0
