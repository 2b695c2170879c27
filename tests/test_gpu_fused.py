"""Launch structures of tk_step (tk_set_steps_per_launch): two Lax-Wendroff
steps per launch, and every step of a call in one persistent launch.

The two-step kernel does, per node and half node, the arithmetic of the
one-step kernel on the same operands, so a solve with pairs of steps per
launch must be bit-identical to the same solve one step per launch: state and
waveforms, for every theta packing, both launch shapes (one block per SM on
large grids, small blocks on small ones), odd and even numbers of substeps
(an outer step may end inside a pair), odd step counts (a single launch ends
the call), observers on the radial edge columns, and graph replay.
"""
import math

import numpy as np
import pytest

from inputs import Workload, initial_planes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1010_3816_gb300 as tk
    tk.load_library()


def _run(w, precision, steps_per_launch, calls, chunk=-1):
    import paper_1010_3816_gb300 as tk
    g = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt,
                  substeps=w.substeps, variable=w.variable, precision=precision)
    g.precompute(w.a, w.M, w.s, w.m)
    g.set_steps_per_launch(steps_per_launch)
    g.set_graph_chunk(chunk)
    re, im = initial_planes(w)
    g.set_initial(re, im)
    ids = [g.add_observer(r, t) for r, t in w.observers]
    for n in calls:
        g.step(n)
    out = g.state(), [g.waveform(k) for k in ids]
    g.close()
    return out


def _grid(Nr, Ntheta, **kw):
    drs = 1.0 / 16.0
    rs_min = -30.0
    rs_max = rs_min + (Nr - 1) * drs
    base = dict(name=f"f{Nr}x{Ntheta}", a=0.9, m=2, rs_min=rs_min, rs_max=rs_max, Nr=Nr,
                Ntheta=Ntheta, dt=drs / 2, center=5.0, width=3.0, noise=1e-3, seed=7,
                observers=((rs_min, math.pi / 2), (rs_max, 1.0), (rs_min + 17.3 * drs * 16, 2.0)))
    base.update(kw)
    return Workload(**base)


CASES = [
    # precision, workload (sizes pick the launch shape), calls of tk_step
    (1, _grid(3001, 64, substeps=2), (7, 10, 1)),          # FP32 K=2, one block per SM
    (1, _grid(3001, 64, substeps=1), (9, 4)),              # an outer step ends inside every pair
    (1, _grid(5003, 32, substeps=3), (5, 6)),              # FP32 K=1, pairs straddle outer steps
    (1, _grid(1301, 128, substeps=4), (3, 8)),             # FP32 K=4
    (1, _grid(401, 64, substeps=2), (13,)),                # small grid: small blocks
    (0, _grid(1301, 64, substeps=2), (7, 6)),              # FP64 K=2 one block per SM
    (0, _grid(3101, 32, substeps=3, variable=0, dt=0.01), (5, 4)),  # FP64 K=1, literal
    (0, _grid(700, 128, substeps=1), (11,)),               # FP64 K=4
]


@pytest.mark.parametrize("precision,w,calls", CASES, ids=[f"case{k}" for k in range(len(CASES))])
def test_two_steps_per_launch_bit_identical(precision, w, calls):
    s1, w1 = _run(w, precision, 1, calls)
    s2, w2 = _run(w, precision, 2, calls)
    assert np.isfinite(s1).all()
    assert np.array_equal(s1, s2)
    assert all(np.array_equal(a, b) for a, b in zip(w1, w2))
    # graph chunks of other lengths (direct launches for the remainder)
    s3, w3 = _run(w, precision, 2, calls, chunk=3)
    assert np.array_equal(s1, s3)
    assert all(np.array_equal(a, b) for a, b in zip(w1, w3))


def test_fp32_pairs_steps_by_default():
    w = _grid(3001, 64, substeps=2)
    s0, w0 = _run(w, 1, 0, (6,))
    s2, w2 = _run(w, 1, 2, (6,))
    assert np.array_equal(s0, s2) and all(np.array_equal(a, b) for a, b in zip(w0, w2))


def test_steps_per_launch_argument():
    import paper_1010_3816_gb300 as tk
    w = _grid(401, 32)
    g = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt)
    for bad in (-2, 3):
        with pytest.raises(tk.TkError):
            g.set_steps_per_launch(bad)
    g.close()


@pytest.mark.parametrize("precision,Nr,want", [(0, 1601, -1), (0, 25601, -1), (1, 1601, -1), (1, 25601, -1)])
def test_get_steps_per_launch_reports_the_default_choice(precision, Nr, want):
    """The default resolved for the grid: every step of a call in one
    persistent launch, for both precisions and grid sizes.  An explicit choice
    reads back as set."""
    import paper_1010_3816_gb300 as tk
    w = _grid(Nr, 64 if Nr > 2000 else 32)
    g = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt,
                  precision=precision)
    assert tk.tk_get_steps_per_launch(g.h) == want
    g.set_steps_per_launch(2)
    assert tk.tk_get_steps_per_launch(g.h) == 2
    g.set_steps_per_launch(1)
    assert tk.tk_get_steps_per_launch(g.h) == 1
    g.set_steps_per_launch(0)
    assert tk.tk_get_steps_per_launch(g.h) == want
    g.close()


PERSISTENT_CASES = [
    (0, _grid(1601, 32, substeps=1), (17, 1, 40)),         # the 1601 x 32 workload's shape
    (0, _grid(803, 64, substeps=2), (9, 11)),
    (0, _grid(401, 128, substeps=3), (5,)),
    (0, _grid(997, 40, substeps=1, variable=0, dt=0.01), (25,)),   # literal, padded rows
    (1, _grid(1601, 32, substeps=2), (13, 8)),
    (0, _grid(23, 8, substeps=1, observers=((-30.0, 1.5), (-29.0, 0.5))), (31,)),  # few columns
    (0, _grid(2501, 64, substeps=2), (6, 3)),               # FP64, one 16-warp block per SM
    (0, _grid(3701, 32, substeps=1), (7, 2)),               # FP64, one 24-warp block per SM (K = 1)
    (0, _grid(1301, 128, substeps=4), (3, 1)),              # FP64, one 8-warp block per SM (K = 4)
    (0, _grid(25601, 64, substeps=2), (2,)),                # FP64, the benchmark's grid
    (1, _grid(3001, 64, substeps=2), (7, 1, 4)),            # FP32 pairs, one 12-warp block per SM
    (1, _grid(3001, 64, substeps=3), (5,)),                 # FP32, an odd last step
    (1, _grid(5003, 32, substeps=1), (9,)),                 # FP32 K = 1
    (1, _grid(1301, 128, substeps=4), (3,)),                # FP32 K = 4
    # FP32 grids with at least 4 columns per warp of one block per SM: sweeps
    # of four steps, ending on outer step boundaries; the rest as pairs and a
    # single step
    (1, _grid(4901, 64, substeps=2), (7, 1, 4)),            # K = 2: 3 sweeps + 1 pair; a pair; 2 sweeps
    (1, _grid(4901, 64, substeps=3), (5, 4)),               # k = 3: 3 sweeps + a pair + a single step
    (1, _grid(9800, 32, substeps=1), (9, 2)),               # K = 1: 2 sweeps + a single step
    (1, _grid(2500, 128, substeps=4), (3, 1)),              # K = 4: 3 sweeps; 1 sweep
    (1, _grid(5000, 64, substeps=8), (2, 3)),               # k = 8: 4 sweeps; 6 sweeps
    # observers at one r* and several theta share their two columns (the sweep's samples)
    (1, _grid(4901, 64, substeps=2, observers=((100.0, 0.7), (100.0, 1.6), (100.0, 2.5))), (6,)),
    # four r* two columns apart put seven observer columns in one warp's range:
    # those calls run in pairs of steps
    (1, _grid(9801, 64, substeps=2, observers=((100.0, 0.7), (100.125, 1.6), (100.25, 2.5),
                                               (100.375, 1.1))), (6, 3)),
]


@pytest.mark.parametrize("precision,w,calls", PERSISTENT_CASES,
                         ids=[f"case{k}" for k in range(len(PERSISTENT_CASES))])
def test_persistent_launch_bit_identical(precision, w, calls):
    """All inner steps of each tk_step call in one cooperative launch (FP64:
    single steps, each warp waiting only for the warps it depends on; FP32:
    sweeps of four steps on large grids, then pairs of steps, blocks waiting on
    their neighbours in between): the same bits as one launch per step,
    waveforms included."""
    s1, w1 = _run(w, precision, 1, calls)
    sp, wp = _run(w, precision, -1, calls)
    assert np.isfinite(s1).all()
    assert np.array_equal(s1, sp)
    assert all(np.array_equal(a, b) for a, b in zip(w1, wp))
    # and the automatic choice
    s0, w0 = _run(w, precision, 0, calls)
    assert np.array_equal(s0, sp) and all(np.array_equal(a, b) for a, b in zip(w0, wp))


# grid sizes around the launch-shape switches (narrow 4-warp blocks below
# 152 x the wide warp count, one wide block per SM from there), grids that
# barely give every warp of a narrow launch one column, and uneven splits
SHAPES = [(64, 32), (607, 32), (1215, 32), (3647, 32), (3648, 32), (3649, 32), (5000, 32),
          (2431, 64), (2432, 64), (2433, 64), (1215, 128), (1216, 128), (1217, 128), (611, 40)]


@pytest.mark.parametrize("Nr,Ntheta", SHAPES, ids=[f"{a}x{b}" for a, b in SHAPES])
def test_persistent_fp64_dataflow_across_launch_shapes(Nr, Ntheta):
    """The persistent FP64 sweep (each warp waiting only for the warps it
    depends on) against one launch per step, bit for bit, on grid sizes
    around the launch-shape switches."""
    w = _grid(Nr, Ntheta, substeps=2, observers=((-30.0, 1.5), (-30.0 + (Nr - 1) / 32.0, 1.0)))
    s1, w1 = _run(w, 0, 1, (5, 2))
    sp, wp = _run(w, 0, -1, (5, 2))
    assert np.isfinite(s1).all() and np.abs(s1).max() > 0
    assert np.array_equal(s1, sp)
    assert all(np.array_equal(a, b) for a, b in zip(w1, wp))
