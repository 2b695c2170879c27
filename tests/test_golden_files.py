"""The stored full-length oracle runs (tests/golden/kerr_25601x64_oracle*.npz,
written by tests/golden/make_kerr_golden.py, which calls only the oracle) are
what the committed oracle computes: their first waveform samples equal a
fresh oracle run of the same workload bit for bit, and the perturbed and
noisy runs differ from the plain one by the small amounts their definitions
imply (about one ulp per outer step amplified by the run), nothing more."""
import os

import numpy as np
import pytest

from inputs import KERR_25601x64, initial_planes

HERE = os.path.dirname(os.path.abspath(__file__))
NAMES = ("kerr_25601x64_oracle.npz", "kerr_25601x64_oracle_perturbed.npz",
         "kerr_25601x64_oracle_noisy.npz")
PREFIX = 12   # outer steps re-run here


def _load(name):
    return np.load(os.path.join(HERE, "golden", name))


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


def test_golden_prefix_is_the_oracle():
    import oracle
    w = KERR_25601x64
    sol = oracle.Solver(M=w.M, a=w.a, s=w.s, m=w.m, rs_min=w.rs_min, rs_max=w.rs_max, Nr=w.Nr,
                        Ntheta=w.Ntheta, dt=w.dt, substeps=w.substeps, variable=w.variable)
    ids = [sol.add_observer(r, t) for r, t in w.observers]
    re, im = initial_planes(w)
    sol.set_initial(re, im)
    sol.run(PREFIX)
    d = _load(NAMES[0])
    for k, key in zip(ids, ("wave0", "wave1")):
        assert np.array_equal(sol.waveform(k), d[key][:PREFIX])
    # the noisy run is perturbed only after its first 16 outer steps
    assert np.array_equal(_load(NAMES[2])["wave0"][:PREFIX], d["wave0"][:PREFIX])


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name", NAMES[1:])
def test_perturbed_runs_differ_by_rounding_sized_amounts(name):
    ref, p = _load(NAMES[0]), _load(name)
    for key in ("wave0", "wave1"):
        assert 0.0 < _rel(p[key], ref[key]) < 1e-13
    for c in range(4):
        assert 0.0 < _rel(p["state_sub"][c], ref["state_sub"][c]) < 5e-12
        assert abs(p["plane_norms"][c] / ref["plane_norms"][c] - 1.0) < 1e-12
