"""Batches (tk_batch_*): many uneven solvers advanced by one kernel launch per
inner tick (its warps take work items from a queue in device memory),
replayed from a CUDA graph, segment length and grid size chosen by the
autotuner.  The batched results must be bit-identical to stepping every
member alone (same arithmetic per half node and node), and so inherit the
members' parity with the oracle, which one member re-checks directly."""
import math

import numpy as np
import pytest

from inputs import Workload, initial_planes

from _parity import compare, run_oracle

pytestmark = pytest.mark.gpu

DT = 0.0625
MEMBERS = [
    Workload(name="b0", a=0.0, m=2, rs_min=-30.0, rs_max=45.0, Nr=601, Ntheta=32, dt=DT,
             center=8.0, width=2.5, observers=((30.0, math.pi / 2),)),
    Workload(name="b1", a=0.9, m=2, rs_min=-40.0, rs_max=60.0, Nr=803, Ntheta=64, dt=DT,
             substeps=2, noise=1e-3, seed=3, observers=((40.0, math.pi / 4), (40.0, math.pi / 2))),
    Workload(name="b2", a=0.99, m=3, rs_min=-20.0, rs_max=80.0, Nr=401, Ntheta=128, dt=DT,
             substeps=4, center=15.0, observers=((50.0, 1.0),)),
    Workload(name="b3", a=0.5, m=0, s=0, rs_min=-10.0, rs_max=27.375, Nr=300, Ntheta=33, dt=DT,
             center=5.0, width=2.0, observers=()),
    Workload(name="b4", a=0.7, m=-1, rs_min=-25.0, rs_max=35.0, Nr=481, Ntheta=16, dt=DT,
             variable=0, substeps=4, center=3.0, observers=((10.0, 2.0),)),
]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1010_3816_gb300 as tk
    tk.load_library()


def _solver(w):
    import paper_1010_3816_gb300 as tk
    g = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt,
                  substeps=w.substeps, variable=w.variable)
    g.precompute(w.a, w.M, w.s, w.m)
    re, im = initial_planes(w)
    g.set_initial(re, im)
    ids = [g.add_observer(r, t) for r, t in w.observers]
    return g, ids


def _results(solvers):
    return [(g.state(), [g.waveform(k) for k in ids]) for g, ids in solvers]


def _same(a, b):
    for (s1, w1), (s2, w2) in zip(a, b):
        assert np.array_equal(s1, s2)
        assert len(w1) == len(w2) and all(np.array_equal(x, y) for x, y in zip(w1, w2))


@pytest.mark.parametrize("chunk,seg", [(-1, None), (0, 16), (3, 5), (-1, 0)])
def test_batch_is_bit_identical_to_members_alone(chunk, seg):
    import paper_1010_3816_gb300 as tk
    alone = [_solver(w) for w in MEMBERS]
    for g, _ in alone:
        g.step(23)
        g.step(14)
    ref = _results(alone)
    batched = [_solver(w) for w in MEMBERS]
    b = tk.Batch([g for g, _ in batched])
    assert b.info()["kmax"] == 4
    b.set_graph_chunk(chunk)
    if seg:
        b.set_segment(seg)
    b.step(23)
    b.step(14)
    _same(_results(batched), ref)
    for g, _ in batched:
        assert g.steps_done() == 37
    b.close()


def test_autotuner_keeps_state_and_results():
    import paper_1010_3816_gb300 as tk
    alone = [_solver(w) for w in MEMBERS]
    for g, _ in alone:
        g.step(10)
    batched = [_solver(w) for w in MEMBERS]
    b = tk.Batch([g for g, _ in batched])
    b.step(5)
    before = _results(batched)
    seg, ms = b.tune(trial_steps=2)
    assert seg in (0, 4, 8, 12, 16, 24, 32, 48, 64, 96, 128) and ms > 0
    assert b.info()["seg"] == seg
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    if seg:                                    # the tuned work-queue grid
        assert b.info()["blocks"] % sms == 0 and b.info()["blocks"] >= sms
    else:                                      # the members one after another
        assert b.info()["blocks"] == 0
    _same(_results(batched), before)          # tuning left every member untouched
    b.step(5)
    for g, _ in alone:
        pass
    _same(_results(batched), _results(alone))
    b.close()


def test_batched_member_matches_oracle():
    import paper_1010_3816_gb300 as tk
    batched = [_solver(w) for w in MEMBERS]
    b = tk.Batch([g for g, _ in batched])
    b.step(40)
    w = MEMBERS[1].with_(steps=40)
    g, ids = batched[1]
    compare(w, (g.state(), [g.waveform(k) for k in ids]), run_oracle(w))
    b.close()


def test_batch_rejects_mismatched_members():
    import paper_1010_3816_gb300 as tk
    g1, _ = _solver(MEMBERS[0])
    g2, _ = _solver(MEMBERS[1].with_(dt=DT / 2))
    with pytest.raises(tk.TkError):
        tk.Batch([g1, g2])


def test_full_batched_set_is_bit_identical_to_members_alone():
    """All 24 instances of the batched workload at full size (16x spread in
    size, three theta packings, k = 2, 4, 8) for 12 outer steps, in the
    launch configuration the benchmark times (the autotuner's choice: for
    this set the members one after another), and through the work queue."""
    import paper_1010_3816_gb300 as tk
    from inputs import batched_instances
    inst = batched_instances()
    alone = [_solver(w) for w in inst]
    for g, _ in alone:
        g.step(12)
    ref = _results(alone)
    for g, _ in alone:
        g.close()
    for tuned in (True, False):   # the tuner's choice, then the work queue itself
        batched = [_solver(w) for w in inst]
        b = tk.Batch([g for g, _ in batched])
        assert b.info()["kmax"] == 8
        if tuned:
            b.tune(2)
        else:
            b.set_segment(12)
            assert b.info()["seg"] == 12
        b.step(12)
        _same(_results(batched), ref)
        b.close()
        for g, _ in batched:
            g.close()
