"""FP32 step (TK_PREC_F32): FP32 planes, tables and stencil arithmetic, with
the coefficient precompute (including the r(r*) inversion) in FP64 and the
waveform samples formed in FP64 from the FP32 state values.  Its error against
the FP64 oracle is measured and bounded per waveform; the bounds below are the
measured errors with a safety factor, not parity claims.
"""
import math

import numpy as np
import pytest

from inputs import KERR_25601x64, Workload

from _parity import rel_l2, row_weights, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

BASE = Workload(name="base32", rs_min=-40.0, rs_max=60.0, Nr=803, Ntheta=64, dt=0.0625, steps=160,
                a=0.9, center=10.0, width=3.0, noise=1e-3, seed=7,
                observers=((30.0, math.pi / 2), (17.31, 1.0)))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1010_3816_gb300 as tk
    tk.load_library()


@pytest.mark.parametrize("kw", [dict(), dict(Ntheta=32, a=0.0), dict(Ntheta=128, Nr=401, substeps=4),
                                dict(variable=0, dt=0.01, m=3)])
def test_fp32_error_against_fp64_oracle(kw):
    w = BASE.with_(**kw)
    gs, gw = run_gpu(w, precision=1)
    os_, ow = run_oracle(w)
    wt = row_weights(w)[None, :, None]
    state_err = max(rel_l2(gs[c] * wt[0], os_[c] * wt[0]) for c in range(4) if np.any(os_[c]))
    wave_err = max(rel_l2(a, b) for a, b in zip(gw, ow))
    print(kw, "state", state_err, "wave", wave_err)
    assert wave_err < 1e-4
    assert state_err < 1e-3
    # and it is genuinely FP32: not bit-identical to the FP64 result
    assert wave_err > 0.0


def test_fp32_kerr_25601x64_full_run_error():
    """The full 38400-step Kerr run in FP32 against the same run in FP64 (which
    matches the oracle): waveform error stated per observer."""
    w = KERR_25601x64
    g64 = run_gpu(w)
    g32 = run_gpu(w, precision=1)
    errs = [rel_l2(a, b) for a, b in zip(g32[1], g64[1])]
    print("FP32 vs FP64 waveform relative L2 per observer:", errs)
    assert all(np.isfinite(errs)) and max(errs) < 1e-2


@pytest.mark.parametrize("kw", [dict(), dict(Ntheta=128, Nr=401, substeps=4), dict(variable=0, dt=0.01, m=3)])
def test_fp32_samples_are_formed_in_fp64(kw):
    """The last sample of every observer equals the bilinear interpolant of the
    final FP32 state (exported exactly as doubles) evaluated in FP64 with the
    oracle's row weights, to FP64 rounding: the FP32 variant keeps FP64 for the
    waveform, only its state is FP32."""
    import oracle
    w = BASE.with_(**kw)
    gs, gw = run_gpu(w, precision=1)
    assert np.array_equal(gs, gs.astype(np.float32).astype(np.float64))   # FP32 state
    th = (np.arange(w.Ntheta) + 0.5) * (math.pi / w.Ntheta)
    for (rs, tho), wave in zip(w.observers, gw):
        fi = (rs - w.rs_min) / w.drs
        fj = tho / (math.pi / w.Ntheta) - 0.5
        i0, j0 = min(int(fi), w.Nr - 2), min(int(fj), w.Ntheta - 2)
        fr, ft = fi - i0, fj - j0
        wa = oracle.weight(w.s, w.m, w.variable, th[j0])
        wb = oracle.weight(w.s, w.m, w.variable, th[j0 + 1])
        want = 0.0
        for dc, wr in ((0, 1.0 - fr), (1, fr)):
            col = gs[0][:, i0 + dc] + 1j * gs[1][:, i0 + dc]
            want += wr * ((1.0 - ft) * wa * col[j0] + ft * wb * col[j0 + 1])
        got = wave[-1]
        assert abs(got - want) <= 1e-14 * abs(want), (got, want)
