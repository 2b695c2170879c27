"""Pins of oracle.coeffs_ext, the oracle's coefficient formulas evaluated in
numpy's longdouble, which supplies the extended-precision coefficient run of
the full-length sensitivity study.

(1) Where the formulas do not cancel, it equals the FP64 oracle's tables to
FP64 rounding.  (2) Near the horizon, where the FP64 value of c1R keeps only a
few digits, it equals a rearrangement of c1R (worked out by hand from the
oracle's expressions) from which the O(1) terms that cancel have been removed
analytically; evaluated in FP64 that form keeps full precision there.  (3) Its
tortoise inversion agrees with the oracle's.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import coeffs_ext

M, A, S, MM = 1.0, 0.9, -2, 2

pytestmark = pytest.mark.skipif(np.finfo(np.longdouble).eps >= np.finfo(np.float64).eps,
                                reason="numpy's longdouble is no wider than FP64 here")


def _c1R_rearranged(x, th):
    """c1R = b C_tR + E0 + 2 b^2 f_*/f - b b_* with the cancellations done by
    hand (FP64, x = r - r+ the independent variable):
      b C_tR + E0 = (Delta/Sigma^2) [2 s b r + 2 r + 2 s r
                                     - 2 s M a^2 (r^2 - a^2) sin^2 / (Sigma (Sigma + varpi))]
    using (r - M) varpi - M (r^2 - a^2) = r Delta and
    1 - b = -a^2 Delta sin^2 / (Sigma (Sigma + varpi)), and
      d_r b = a^2 sin^2 (varpi Delta' - 4 r Delta) / (2 Sigma^3)
    using 1 - varpi^2/Sigma^2 = -a^2 Delta sin^2 / Sigma^2."""
    d = math.sqrt(M * M - A * A)
    rp, rm = M + d, M - d
    r = rp + x
    varpi = r * r + A * A
    Delta = x * (r - rm)
    dDelta = 2.0 * (r - M)
    sn2 = math.sin(th) ** 2
    Sig2 = varpi * varpi - A * A * Delta * sn2
    Sig = math.sqrt(Sig2)
    b = varpi / Sig
    bC_E0 = (Delta / Sig2) * (2 * S * b * r + 2 * r + 2 * S * r
                              - 2 * S * M * A * A * (r * r - A * A) * sn2 / (Sig * (Sig + varpi)))
    db_dr = A * A * sn2 * (varpi * dDelta - 4 * r * Delta) / (2 * Sig2 * Sig)
    return bC_E0 + 2 * b * b * 3 * Delta / (r * varpi) - b * (Delta / varpi) * db_dr


@pytest.mark.parametrize("variable", [0, 1])
def test_equals_the_fp64_oracle_where_nothing_cancels(variable):
    Nr, Nth = 801, 16
    sol = oracle.Solver(M=M, a=A, s=S, m=MM, rs_min=-100.0, rs_max=700.0, Nr=Nr, Ntheta=Nth,
                        dt=0.5, variable=variable)
    on, oh = sol.coeffs()
    en, eh = coeffs_ext.tables(M, A, S, MM, variable, -100.0, sol.drs, Nr, Nth)
    rs = -100.0 + np.arange(Nr) * sol.drs
    assert np.all(eh[:, :, 0] == 0)
    for E, O in ((en, on), (eh, oh)):
        for q, name in enumerate(oracle.COEF_NAMES):
            colmax = np.abs(O[q]).max(axis=0, keepdims=True)
            d = np.abs(E[q] - O[q]) / np.where(colmax > 0, colmax, 1.0)
            if name == "c1R":
                # cancels near the horizon and far out: compare where it does not
                mid = (rs > -30.0) & (rs < 60.0)
                assert d[:, mid].max() < 1e-9, name
            elif name == "c3R":
                assert d.max() < 1e-10, name       # b^2 f_** + E0 f_* + Q + c4 V cancel partly
            else:
                assert d.max() < 1e-13, (name, d.max())


@pytest.mark.parametrize("x", [1e-14, 6e-14, 1e-12, 1e-10, 1e-8, 1e-6, 1e-4, 1e-2, 1.0])
def test_c1R_near_the_horizon_matches_the_cancellation_free_form(x):
    """Away from the horizon (x >= 1e-2) the two forms agree to FP64 rounding,
    which pins the rearrangement.  Closer in, the wider type's evaluation of
    the cancelling form keeps about 2^11 times more of c1R's digits than the
    FP64 one (the longdouble has 11 more bits on x86-64): its distance to the
    cancellation-free value is at most 1/200 of the FP64 evaluation's."""
    th = (np.arange(16) + 0.5) * (math.pi / 16)
    ext = coeffs_ext.coeffs(M, A, S, MM, 1, np.array([x]), th)[1, :, 0].astype(np.float64)
    fp64 = np.array([oracle.coeffs_point(M, A, S, MM, 1, x, t)["c1R"] for t in th])
    want = np.array([_c1R_rearranged(x, t) for t in th])
    rel_ext = (np.abs(ext - want) / np.abs(want)).max()
    rel_fp64 = (np.abs(fp64 - want) / np.abs(want)).max()
    assert rel_ext <= max(1e-14, 5e-3 * rel_fp64), (rel_ext, rel_fp64)
    if x <= 1e-12:
        # the FP64 evaluation of the oracle's expression is far off there:
        # the reason for the extended-precision tables
        assert rel_fp64 > 1e-6


def test_tortoise_inversion_agrees_with_the_oracle():
    rs = np.array([-100.0, -99.96875, -60.0, -10.0, 0.0, 3.5, 50.0, 699.96875, 700.0])
    x = coeffs_ext.x_of_rstar(M, A, rs)
    for r, xe in zip(rs, x):
        xo = oracle.x_of_rstar(M, A, float(r))
        assert abs(float(xe) / xo - 1.0) < 1e-13, (r, float(xe), xo)
        # and the wider-type inversion hits r* to far better than FP64 resolution
        assert abs(float(coeffs_ext._tortoise_x(np.longdouble(M), np.longdouble(A), xe)
                         - np.longdouble(r))) <= 4 * np.finfo(np.longdouble).eps * max(1.0, abs(r))
