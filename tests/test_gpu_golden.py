"""The benchmark workload at full length against the oracle's full run.

`tests/golden/make_kerr_golden.py` stores the CPU oracle's run of all 38400
outer steps (76800 Lax-Wendroff steps, t = 600 M) of the Kerr a = 0.9,
25601 x 64 workload: both waveforms, the physical state on every 8th theta
row and every 16th r* column, and the L2 norm of every physical plane.  It
also stores two perturbed runs: one from initial data changed by about one
ulp (--perturbed), and one whose state takes a random walk of about one ulp
per outer step (--noisy), the size of the rounding differences between two
correct implementations.  Their differences from the plain run (kappa) are the
run's own conditioning: no other rounding order can be held closer.

The GPU runs the workload in the launch configuration the benchmark times
(graph replay, one block per SM).  Bars: waveforms max(1e-12, 10 kappa),
sampled state per plane and plane norms max(1e-12, 10 kappa), kappa the larger
of the two runs' differences.  The FP32 path is compared with the same stored
FP64 run: its waveform error is the one stated for the FP32 variant.
"""
import os

import numpy as np
import pytest

from inputs import KERR_25601x64

from _parity import rel_l2, row_weights, run_gpu

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "kerr_25601x64_oracle.npz")
PERTURBED = os.path.join(HERE, "golden", "kerr_25601x64_oracle_perturbed.npz")
NOISY = os.path.join(HERE, "golden", "kerr_25601x64_oracle_noisy.npz")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1010_3816_gb300 as tk
    tk.load_library()


def _stored():
    ref = np.load(GOLDEN)
    perts = [np.load(PERTURBED), np.load(NOISY)]
    rows, cols = ref["rows"], ref["cols"]
    return ref, perts, rows, cols


def _kappa(perts, ref, get):
    return max(rel_l2(get(p), get(ref)) for p in perts)


def _physical_sub(w, state, rows, cols):
    wt = row_weights(w)[None, :, None]
    phys = state * wt
    return phys[:, rows][:, :, cols], np.linalg.norm(phys.reshape(4, -1), axis=1)


def test_kerr_25601x64_full_length_parity():
    w = KERR_25601x64
    ref, perts, rows, cols = _stored()
    state, waves = run_gpu(w)
    assert np.isfinite(state).all()
    sub, norms = _physical_sub(w, state, rows, cols)
    report = {}
    for k, key in enumerate(("wave0", "wave1")):
        kappa = _kappa(perts, ref, lambda d: d[key])
        err = rel_l2(waves[k], ref[key])
        report[key] = (err, kappa)
        assert err <= max(1e-12, 10 * kappa), (key, err, kappa)
    for c, name in enumerate(("PhiR", "PhiI", "PiR", "PiI")):
        kappa = _kappa(perts, ref, lambda d: d["state_sub"][c])
        err = rel_l2(sub[c], ref["state_sub"][c])
        en = abs(norms[c] / ref["plane_norms"][c] - 1.0)
        report[name] = (err, kappa, en)
        assert err <= max(1e-12, 10 * kappa), (name, err, kappa)
        assert en <= max(1e-12, 10 * kappa), (name, en, kappa)
    print(report)


def test_kerr_25601x64_fp32_error_against_fp64_oracle():
    """FP32 planes, tables and arithmetic over the full run: the waveform
    error against the FP64 oracle at t = 600 M (stated as the FP32 variant's
    accuracy) stays below 1e-3 relative L2."""
    w = KERR_25601x64
    ref = np.load(GOLDEN)
    state, waves = run_gpu(w, precision=1)
    assert np.isfinite(state).all()
    errs = [rel_l2(waves[k], ref[key]) for k, key in enumerate(("wave0", "wave1"))]
    print({"fp32_wave_rel_l2": errs})
    assert max(errs) <= 1e-3, errs
