"""The oracle's coefficient tables evaluated in a wider floating-point type.

TEST INFRASTRUCTURE ONLY, like the rest of this package: only the tests and the
script that writes the stored full-length runs use it.

The FP64 evaluation of the first-order system's coefficients (``tko_coeffs_point``
in ``tk_oracle.c``, derived from Eq. 1 with the m-mode ansatz of Eq. 2) loses
digits where terms of order one cancel.  The worst case is c1R near the horizon:
as Delta -> 0 the O(1) parts of b C_t and E0 cancel exactly, leaving

    c1R = (Delta / Sigma^2) [2 s b r + 2 r + 2 s r
                             - 2 s M a^2 (r^2 - a^2) sin^2 / (Sigma (Sigma + varpi))]
          + 2 b^2 f_*/f - b b_*,

so at r* = -100 (Delta ~ 1e-13) an FP64 evaluation keeps only two or three
digits of it.  c1R is also small far out, where b C_t, E0 and b b_* nearly
cancel as well.  Any FP64 implementation of the formulas carries an error of
this kind, and two implementations that order the operations differently carry
different errors.

``tables`` evaluates the same formulas, in the same order, at the same FP64
grid points (r*_a = rs_min + a drs, r*_{a-1/2} = rs_min + (a - 1/2) drs,
theta_b = (b + 1/2) pi / Ntheta, each formed in FP64 as the oracle forms it)
with numpy's ``longdouble`` (x87 80-bit extended precision on x86-64, 11 more
bits than FP64; IEEE binary128 on aarch64) and rounds every value to FP64 only
at the end.  The tortoise inversion x(r*) is done in the same wider type by
bisection in ln x, as in the C oracle.  The run that starts from these tables
instead of the oracle's own differs from the plain run by the effect of the
FP64 evaluation error of the coefficient formulas: one of the sensitivity runs
that set the parity bar of the full-length test.
"""
from __future__ import annotations

import numpy as np

NCOEF = 9
_L = np.longdouble


def _horizons(M, a):
    d = np.sqrt(M * M - a * a)
    return M + d, M - d


def _tortoise_x(M, a, x):
    """r*(x), x = r - r+, the oracle's closed form in the wider type."""
    rp, rm = _horizons(M, a)
    r = rp + x
    Ap = 2 * M * rp / (rp - rm)
    Am = 2 * M * rm / (rp - rm)
    return r + Ap * np.log(x / (2 * M)) - Am * np.log((r - rm) / (2 * M))


def x_of_rstar(M, a, rstar):
    """x = r - r+ for each r* (array), by bisection in y = ln x in the wider
    type: r*(e^y) is strictly increasing in y."""
    M, a = _L(M), _L(a)
    rs = np.asarray(rstar, dtype=np.float64).astype(_L)
    ylo = np.full(rs.shape, _L(-700))
    yhi = np.full(rs.shape, _L(1))
    while True:
        low = _tortoise_x(M, a, np.exp(yhi)) < rs
        if not low.any():
            break
        yhi = np.where(low, yhi + 1, yhi)
    for _ in range(400):
        ym = (ylo + yhi) / 2
        if not np.any((ym > ylo) & (ym < yhi)):
            break
        below = _tortoise_x(M, a, np.exp(ym)) < rs
        ylo = np.where(below, ym, ylo)
        yhi = np.where(below, yhi, ym)
    xlo, xhi = np.exp(ylo), np.exp(yhi)
    elo = np.abs(_tortoise_x(M, a, xlo) - rs)
    ehi = np.abs(_tortoise_x(M, a, xhi) - rs)
    return np.where(elo <= ehi, xlo, xhi)


def coeffs(M, a, s, m, variable, x, theta):
    """The nine coefficients b, c1R, c1I, c2R, c2I, c3R, c3I, c4, c5 at every
    (theta, x) pair of the two 1-D arrays (x = r - r+ in the wider type, theta
    in FP64), as an array [9][len(theta)][len(x)] of the wider type.  The same
    expressions as ``tko_coeffs_point``."""
    M, a = _L(M), _L(a)
    rp, rm = _horizons(M, a)
    x = np.asarray(x, dtype=_L)[None, :]
    th = np.asarray(theta, dtype=np.float64).astype(_L)[:, None]
    r = rp + x
    varpi = r * r + a * a
    Delta = x * (r - rm)
    dDelta = 2 * (r - M)
    sn, cs = np.sin(th), np.cos(th)
    sn2 = sn * sn
    Sig2 = varpi * varpi - a * a * Delta * sn2
    Sig = np.sqrt(Sig2)
    b = varpi / Sig
    db_dr = 2 * r / Sig - varpi * (4 * r * varpi - a * a * dDelta * sn2) / (2 * Sig2 * Sig)
    b_s = (Delta / varpi) * db_dr
    fs = 3 * Delta / (r * varpi)
    d_3r2D = (6 * r * Delta + 3 * r * r * dDelta) / varpi - 6 * r * r * r * Delta / (varpi * varpi)
    fss = (Delta / varpi) * d_3r2D / (r * r * r)
    CtR = 2 * s * (r * Delta - M * (r * r - a * a)) / Sig2
    CtI = (4 * M * a * m * r + 2 * s * a * Delta * cs) / Sig2
    E0 = (2 * r * Delta + s * dDelta * varpi) / Sig2
    E = 2 * b * b * fs + E0
    QR = _L(m * m) * a * a / Sig2
    QI = 2 * m * s * a * (r - M) / Sig2
    c4 = Delta / Sig2
    if variable == 0:
        g = cs / sn
        V = -(m + s * cs) * (m + s * cs) / (sn * sn) + s
    else:
        al = _L(abs(m + s)) / 2
        be = _L(abs(m - s)) / 2
        l0 = max(abs(m), abs(s))
        V = -_L((l0 - s) * (l0 + s + 1))
        g = cs / sn + 2 * (al / np.tan(th / 2) - be * np.tan(th / 2))
    one = np.ones_like(b)
    return np.stack([b, b * CtR + E - b * b_s, b * CtI, -CtR, -CtI,
                     b * b * fss + E0 * fs + QR + c4 * V, QI * one, c4, c4 * g * one])


def tables(M, a, s, m, variable, rs_min, drs, Nr, Ntheta):
    """(node, half) tables in the layout of ``oracle.Solver.coeffs()``: each
    [9][Ntheta][Nr] FP64, the half table's column a >= 1 holding the values at
    r*_{a-1/2} and column 0 zero.  Every value is evaluated in the wider type
    and rounded to FP64 once."""
    ia = np.arange(Nr, dtype=np.float64)
    rs_node = rs_min + ia * drs
    rs_half = rs_min + (ia[1:] - 0.5) * drs
    theta = (np.arange(Ntheta, dtype=np.float64) + 0.5) * (np.pi / Ntheta)
    node = coeffs(M, a, s, m, variable, x_of_rstar(M, a, rs_node), theta).astype(np.float64)
    half = np.zeros_like(node)
    half[:, :, 1:] = coeffs(M, a, s, m, variable, x_of_rstar(M, a, rs_half), theta).astype(np.float64)
    return node, half
