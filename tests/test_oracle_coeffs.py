"""Pins of the oracle's coefficients and tortoise coordinate against Eq. 1.

The coefficients of the first-order system are not printed in the paper
(Sec. 3.2 defers D and S to its reference [klpa]).  The oracle derives them
from Eq. 1; these tests evaluate Eq. 1 itself, typed from the paper, on
analytic test functions and require the oracle's first-order operator to
reproduce it:

  for any Phi, with Pi := d_t Phi + b d_* Phi,
  d_t Pi - b d_* Pi - c1 d_* Phi - c2 Pi - c3 Phi - c4 Phi_thth - c5 Phi_th
      = -(Delta / (Sigma^2 r^3 w)) e^{-i m phi} [Eq. 1 applied to Psi],
  Psi = e^{i m phi} r^3 w(theta) Phi   (w = 1 for the literal field).

Expanding the left side gives Phi_tt - b^2 Phi_** - (b b_* + c1 + c2 b) Phi_*
- c2 Phi_t - c3 Phi - c4 Phi_thth - c5 Phi_th; b_* is taken from the oracle's
own b by a Richardson-extrapolated central difference.
"""
import math

import numpy as np
import pytest

sp = pytest.importorskip("sympy")

CASES = [
    # (a, s, m)
    (0.0, -2, 2),
    (0.9, -2, 2),
    (0.7, -2, -3),
    (0.5, 0, 1),
    (0.99, 1, 3),
    (0.3, -1, 0),
    (0.6, 2, -1),
]
POINTS = [(2.9, 0.35), (3.7, 1.1), (8.0, 2.05), (25.0, 2.8), (5.0, 1.5707963267948966)]


def _eq1_sympy(M, a, s, m, variable):
    """Eq. 1 of the paper applied to Psi = e^{i m phi} r^3 w Phi, as a sympy
    expression in (t, r, th) with the e^{i m phi} factor removed, plus the
    derivatives of the test function Phi needed on the left side."""
    t, r, th, ph = sp.symbols("t r th ph", real=True)
    I = sp.I
    Ms, as_ = sp.nsimplify(M), sp.nsimplify(a)
    Delta = r ** 2 - 2 * Ms * r + as_ ** 2
    # generic analytic test function
    omega = sp.Rational(7, 10) + sp.Rational(2, 10) * I
    g = sp.exp(-(r - 6) ** 2 / 10) + sp.Rational(3, 10) * sp.sin(r) + sp.Rational(1, 5)
    h = sp.cos(th) + sp.Rational(1, 2) * sp.sin(th) ** 2 + sp.Rational(1, 5) * sp.cos(3 * th) + sp.Rational(3, 10)
    Phi = sp.exp(-I * omega * t) * g * h
    if variable == 1:
        al = sp.Rational(abs(m + s), 2)
        be = sp.Rational(abs(m - s), 2)
        w = (1 - sp.cos(th)) ** al * (1 + sp.cos(th)) ** be
    else:
        w = sp.Integer(1)
    Psi = sp.exp(I * m * ph) * r ** 3 * w * Phi
    # Eq. 1 (Sec. 3.1), term by term
    e1 = (-((r ** 2 + as_ ** 2) ** 2 / Delta - as_ ** 2 * sp.sin(th) ** 2) * sp.diff(Psi, t, 2)
          - (4 * Ms * as_ * r / Delta) * sp.diff(Psi, t, ph)
          - 2 * s * (r - Ms * (r ** 2 - as_ ** 2) / Delta + I * as_ * sp.cos(th)) * sp.diff(Psi, t)
          + Delta ** (-s) * sp.diff(Delta ** (s + 1) * sp.diff(Psi, r), r)
          + 1 / sp.sin(th) * sp.diff(sp.sin(th) * sp.diff(Psi, th), th)
          + (1 / sp.sin(th) ** 2 - as_ ** 2 / Delta) * sp.diff(Psi, ph, 2)
          + 2 * s * (as_ * (r - Ms) / Delta + I * sp.cos(th) / sp.sin(th) ** 2) * sp.diff(Psi, ph)
          - (s ** 2 * sp.cot(th) ** 2 - s) * Psi)
    e1 = sp.exp(-I * m * ph) * e1
    varpi = r ** 2 + as_ ** 2
    Sig2 = varpi ** 2 - as_ ** 2 * Delta * sp.sin(th) ** 2
    rhs = -Delta / (Sig2 * r ** 3 * w) * e1
    tort = Delta / varpi                      # d_* = (Delta / varpi) d_r
    d = {
        "Phi": Phi,
        "Phi_t": sp.diff(Phi, t),
        "Phi_tt": sp.diff(Phi, t, 2),
        "Phi_s": tort * sp.diff(Phi, r),
        "Phi_ss": tort * sp.diff(tort * sp.diff(Phi, r), r),
        "Phi_th": sp.diff(Phi, th),
        "Phi_thth": sp.diff(Phi, th, 2),
        "rhs": rhs,
    }
    return (t, r, th, ph), d


def _num(expr, syms, vals):
    t, r, th, ph = syms
    v = complex(expr.subs({t: vals[0], r: vals[1], th: vals[2], ph: 0}).evalf(30))
    return v


def _b_star(oracle_mod, M, a, s, m, variable, x, th):
    """d_* b = (Delta/varpi) d_r b from the oracle's b, central differences
    with one Richardson extrapolation."""
    rp, rm = oracle_mod.horizons(M, a)
    r = rp + x

    def b(xx):
        return oracle_mod.coeffs_point(M, a, s, m, variable, xx, th)["b"]

    def cd(h):
        return (b(x + h) - b(x - h)) / (2 * h)

    h = 1e-3 * max(1.0, r)
    db = (4 * cd(h / 2) - cd(h)) / 3
    Delta = (r - rp) * (r - rm)
    return Delta / (r * r + a * a) * db


@pytest.mark.parametrize("variable", [0, 1])
@pytest.mark.parametrize("a,s,m", CASES)
def test_first_order_system_reproduces_eq1(oracle_mod, a, s, m, variable):
    M = 1.0
    syms, d = _eq1_sympy(M, a, s, m, variable)
    rp, _ = oracle_mod.horizons(M, a)
    tval = 0.4
    for r, th in POINTS:
        vals = (tval, r, th)
        x = r - rp
        c = oracle_mod.coeffs_point(M, a, s, m, variable, x, th)
        c1 = c["c1R"] + 1j * c["c1I"]
        c2 = c["c2R"] + 1j * c["c2I"]
        c3 = c["c3R"] + 1j * c["c3I"]
        b, c4, c5 = c["b"], c["c4"], c["c5"]
        bs = _b_star(oracle_mod, M, a, s, m, variable, x, th)
        D = {k: _num(v, syms, vals) for k, v in d.items()}
        terms = [D["Phi_tt"], -b * b * D["Phi_ss"], -(b * bs + c1 + c2 * b) * D["Phi_s"],
                 -c2 * D["Phi_t"], -c3 * D["Phi"], -c4 * D["Phi_thth"], -c5 * D["Phi_th"]]
        lhs = sum(terms)
        scale = sum(abs(z) for z in terms) + abs(D["rhs"])
        err = abs(lhs - D["rhs"]) / scale
        assert err < 1e-9, (a, s, m, variable, r, th, lhs, D["rhs"], err)


def test_a0_coefficients_are_real_and_b_is_one(oracle_mod):
    for s, m in [(-2, 2), (0, 1), (-1, -3)]:
        for x in (0.01, 1.0, 30.0):
            for th in (0.2, 1.3, 2.9):
                c = oracle_mod.coeffs_point(1.0, 0.0, s, m, 1, x, th)
                assert c["b"] == 1.0
                assert c["c1I"] == 0.0 and c["c2I"] == 0.0 and c["c3I"] == 0.0


# --- tortoise coordinate ------------------------------------------------------------
def test_tortoise_closed_form_schwarzschild(oracle_mod):
    """a = 0: r* = r + 2M ln(r/2M - 1)."""
    for r in (2.0001, 2.5, 3.0, 10.0, 700.0):
        x = r - 2.0
        want = r + 2.0 * math.log(r / 2.0 - 1.0)
        assert abs(oracle_mod.tortoise_x(1.0, 0.0, x) - want) <= 1e-13 * max(1.0, abs(want))


@pytest.mark.parametrize("a", [0.0, 0.5, 0.9, 0.99])
def test_tortoise_derivative_is_varpi_over_delta(oracle_mod, a):
    """d r*/dr = (r^2 + a^2)/Delta, the defining property of r*."""
    M = 1.0
    rp, rm = oracle_mod.horizons(M, a)
    for x in (0.05, 0.7, 3.0, 40.0):
        h = 1e-4 * x
        num = (oracle_mod.tortoise_x(M, a, x + h) - oracle_mod.tortoise_x(M, a, x - h)) / (2 * h)
        r = rp + x
        want = (r * r + a * a) / ((r - rp) * (r - rm))
        assert abs(num - want) < 1e-6 * want


@pytest.mark.parametrize("a", [0.0, 0.5, 0.9, 0.99])
def test_tortoise_inverse_round_trip(oracle_mod, a):
    M = 1.0
    for rs in (-100.0, -50.0, -3.3, 0.0, 1.6, 20.0, 500.0, 700.0):
        x = oracle_mod.x_of_rstar(M, a, rs)
        assert x > 0
        back = oracle_mod.tortoise_x(M, a, x)
        assert abs(back - rs) <= 4e-14 * max(1.0, abs(rs)), (a, rs, x, back)


def test_tortoise_near_horizon_asymptotics(oracle_mod):
    """Near the horizon x = r - r+ ~ C exp(2 kappa r*) with surface gravity
    kappa = (r+ - r-)/(2 (r+^2 + a^2)); the ratio x(r*)/exp(2 kappa r*) is constant."""
    for a in (0.0, 0.9):
        rp, rm = oracle_mod.horizons(1.0, a)
        kappa = (rp - rm) / (2 * (rp * rp + a * a))
        ratios = [oracle_mod.x_of_rstar(1.0, a, rs) / math.exp(2 * kappa * rs) for rs in (-100.0, -90.0, -80.0)]
        assert abs(ratios[0] / ratios[2] - 1.0) < 1e-9
