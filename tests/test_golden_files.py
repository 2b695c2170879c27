"""The stored full-length oracle runs (tests/golden/kerr_25601x64_oracle*.npz,
written by tests/golden/make_kerr_golden.py, which calls only the oracle) are
what the committed oracle computes: their first waveform samples equal a
fresh oracle run of the same workload bit for bit (the FMA-contracted run
against a fresh run of the FMA-contracted build), and the runs that differ
from the plain one only by rounding -- FMA contraction, a one-ulp change of
the initial data, a one-ulp random walk of the state, two-ulp changes of the
coefficients, the coefficients evaluated in extended precision -- differ from
it by the small amounts their definitions imply (rounding amplified by the
run), nothing more."""
import os

import numpy as np
import pytest

from inputs import KERR_25601x64, initial_planes

HERE = os.path.dirname(os.path.abspath(__file__))
PLAIN = "kerr_25601x64_oracle.npz"
OTHERS = ("kerr_25601x64_oracle_fma.npz", "kerr_25601x64_oracle_perturbed.npz",
          "kerr_25601x64_oracle_noisy.npz", "kerr_25601x64_oracle_coeffs.npz",
          "kerr_25601x64_oracle_extcoeffs.npz")
NAMES = (PLAIN,) + OTHERS
PREFIX = 12   # outer steps re-run here


def _load(name):
    return np.load(os.path.join(HERE, "golden", name))


def _sub(d, rows, cols):
    ri = np.searchsorted(d["rows"], rows)
    ci = np.searchsorted(d["cols"], cols)
    assert np.array_equal(d["rows"][ri], rows) and np.array_equal(d["cols"][ci], cols)
    return d["state_sub"][:, ri][:, :, ci]


@pytest.mark.parametrize("name", NAMES)
def test_golden_file_layout(name):
    w = KERR_25601x64
    d = _load(name)
    assert d["wave0"].shape == (w.steps,) and d["wave1"].shape == (w.steps,)
    assert np.iscomplexobj(d["wave0"])
    rows, cols = d["rows"], d["cols"]
    assert d["state_sub"].shape == (4, len(rows), len(cols))
    assert d["plane_norms"].shape == (4,)
    for k in ("wave0", "wave1", "state_sub", "plane_norms"):
        assert np.isfinite(d[k]).all()


def test_plain_and_fma_runs_store_every_row_and_every_4th_column():
    for name in (PLAIN, OTHERS[0]):
        d = _load(name)
        assert np.array_equal(d["rows"], np.arange(KERR_25601x64.Ntheta))
        assert np.array_equal(d["cols"], np.arange(0, KERR_25601x64.Nr, 4))


@pytest.mark.parametrize("build,name", [("plain", PLAIN), ("fma", OTHERS[0])])
def test_golden_prefix_is_the_oracle(build, name):
    import oracle
    w = KERR_25601x64
    sol = oracle.Solver(M=w.M, a=w.a, s=w.s, m=w.m, rs_min=w.rs_min, rs_max=w.rs_max, Nr=w.Nr,
                        Ntheta=w.Ntheta, dt=w.dt, substeps=w.substeps, variable=w.variable,
                        build=build)
    ids = [sol.add_observer(r, t) for r, t in w.observers]
    re, im = initial_planes(w)
    sol.set_initial(re, im)
    sol.run(PREFIX)
    d = _load(name)
    for k, key in zip(ids, ("wave0", "wave1")):
        assert np.array_equal(sol.waveform(k), d[key][:PREFIX])
    if build == "plain":
        # the noisy run is perturbed only after its first 16 outer steps
        assert np.array_equal(_load(OTHERS[2])["wave0"][:PREFIX], d["wave0"][:PREFIX])


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name", OTHERS)
def test_rounding_runs_differ_by_rounding_sized_amounts(name):
    ref, p = _load(PLAIN), _load(name)
    for key in ("wave0", "wave1"):
        assert 0.0 < _rel(p[key], ref[key]) < 1e-13
    base = _sub(ref, p["rows"], p["cols"])
    for c in range(4):
        assert 0.0 < _rel(p["state_sub"][c], base[c]) < 1e-11
        assert abs(p["plane_norms"][c] / ref["plane_norms"][c] - 1.0) < 1e-11
