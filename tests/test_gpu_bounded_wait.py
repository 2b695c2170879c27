"""Failure detection of the persistent launches without a GPU fault: their
blocks (or, in the one-step sweep, the warps at a block's two edges) wait for
their neighbours with a bounded number of polls, after which the wait sets
the launch's error flag and returns (tk_step then reports TK_ERR_INTERNAL).
tk_check_bounded_wait runs every kind of wait with one block that never
publishes its flag and itself waits on a shared-memory counter that nothing
sets: its neighbours' waits on the global flags and its own wait must all run
out, each must raise its flag, every block must return, and the context must
stay usable.  Nothing here faults, traps or hangs the GPU: every wait ends by
itself."""
import math
import time

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


@pytest.mark.parametrize("n_blocks,silent", [(8, 3), (8, 0), (8, 7), (2, 1)])
def test_wait_runs_out_and_raises_the_flag(n_blocks, silent):
    import paper_1010_3816_gb300 as tk
    assert tk.tk_check_bounded_wait(n_blocks, silent, 1 << 16) is True


def test_no_silent_block_no_timeout():
    import paper_1010_3816_gb300 as tk
    assert tk.tk_check_bounded_wait(8, -1, 1 << 16) is False


def test_production_limit_ends_and_context_stays_usable():
    import paper_1010_3816_gb300 as tk
    t0 = time.time()
    assert tk.tk_check_bounded_wait(4, 1) is True          # 2^24 polls, as in the step kernels
    elapsed = time.time() - t0
    print({"seconds_to_time_out": elapsed})
    assert elapsed < 120.0
    # a persistent solve right after: same bits as one launch per step
    w = Workload(name="bw", a=0.9, m=2, rs_min=-30.0, rs_max=70.0, Nr=1601, Ntheta=32, dt=1 / 32,
                 substeps=1, center=5.0, width=3.0, noise=1e-3, seed=7,
                 observers=((10.0, math.pi / 2),))
    out = []
    for spl in (1, -1):
        g = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt,
                      substeps=w.substeps)
        g.precompute(w.a, w.M, w.s, w.m)
        g.set_steps_per_launch(spl)
        g.set_initial(*initial_planes(w))
        k = g.add_observer(*w.observers[0])
        g.step(40)
        out.append((g.state(), g.waveform(k)))
        g.close()
    assert np.isfinite(out[0][0]).all()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_argument_errors():
    import paper_1010_3816_gb300 as tk
    for args in ((1, 0), (65, 0), (8, 8), (8, -2)):
        with pytest.raises(tk.TkError):
            tk.tk_check_bounded_wait(*args)


@pytest.mark.parametrize("precision", [0, 1])
def test_timed_out_step_invalidates_the_state_until_it_is_set_again(precision):
    """A persistent launch whose waits ran out (injected on the host after the
    launch ran normally) leaves the step and sample counts where the call
    found them and the samples taken before it readable; every call that
    would read the state refuses (TK_ERR_STATE) until tk_set_state sets it
    again, and stepping on from the restored state gives the bits of the
    uninterrupted run."""
    import paper_1010_3816_gb300 as tk
    w = Workload(name="bw2", a=0.7, m=2, rs_min=-30.0, rs_max=70.0, Nr=1601, Ntheta=32, dt=1 / 32,
                 substeps=2, center=5.0, width=3.0, noise=1e-3, seed=8,
                 observers=((10.0, math.pi / 2),))

    def solver():
        g = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt,
                      substeps=w.substeps, precision=precision)
        g.precompute(w.a, w.M, w.s, w.m)
        g.set_steps_per_launch(-1)
        g.set_initial(*initial_planes(w))
        return g, g.add_observer(*w.observers[0])

    ref, kr = solver()
    ref.step(30)
    ref.step(30)
    want_state, want_wave = ref.state(), ref.waveform(kr)
    ref.close()

    g, k = solver()
    g.step(30)
    checkpoint, wave30 = g.state(), g.waveform(k)
    tk.tk_inject_wait_timeout(g.h)
    with pytest.raises(tk.TkError) as e:
        g.step(30)
    assert e.value.status == tk.TK_ERR_INTERNAL
    assert tk.tk_steps_done(g.h) == 30
    assert np.array_equal(g.waveform(k), wave30)
    for call in (lambda: g.step(1), g.state, lambda: tk.tk_check_finite(g.h)):
        with pytest.raises(tk.TkError) as e:
            call()
        assert e.value.status == tk.TK_ERR_STATE
    tk.tk_set_state(g.h, checkpoint)
    g.step(30)
    assert np.array_equal(g.state(), want_state)
    assert np.array_equal(g.waveform(k), want_wave)
    g.close()
