"""tk_extract_noalloc: the allocation-free waveform read-out, for callers that
must not allocate device memory (code running while a CUDA graph is being
captured, loops whose memory is fixed in advance, hosts with their own memory
pool).  It must return what tk_extract returns, on consecutive calls that
reuse its fixed scratch array, and refuse requests larger than that array.
Collected last on purpose: it needs nothing from the other tests and passes
alone in a fresh process as well as after them."""
import ctypes as C
import math

import numpy as np
import pytest

from inputs import Workload

pytestmark = pytest.mark.gpu

W = Workload(name="noalloc", a=0.9, rs_min=-40.0, rs_max=60.0, Nr=803, Ntheta=64, dt=0.0625,
             steps=300, center=10.0, width=3.0, noise=1e-3, seed=9,
             observers=((30.0, math.pi / 2), (17.31, 1.0), (45.5, 2.2)))


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_noalloc_extract_matches_extract_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1010_3816_gb300 as tk
    from inputs import initial_planes
    lib = tk.load_library()
    g = tk.Solver(rstar_min=W.rs_min, rstar_max=W.rs_max, Nr=W.Nr, Ntheta=W.Ntheta, dt=W.dt)
    g.precompute(W.a, W.M, W.s, W.m)
    re0, im0 = initial_planes(W)
    g.set_initial(re0, im0)
    ids = [g.add_observer(r, t) for r, t in W.observers]
    g.step(W.steps)
    ref = [tk.tk_extract(g.h, k) for k in ids]
    dp = C.POINTER(C.c_double)

    def call(k, first, count):
        re = np.full(count, np.nan)
        im = np.full(count, np.nan)
        st = lib.tk_extract_noalloc(g.h, k, first, count, re.ctypes.data_as(dp), im.ctypes.data_as(dp))
        return st, re + 1j * im

    for _ in range(2):                       # two rounds of calls in a row
        for k, r in zip(ids, ref):
            st, got = call(k, 0, W.steps)
            assert st == tk.TK_OK, tk.tk_last_error(g.h)
            assert _rel(got, r) <= 1e-12
    st, part = call(ids[1], 37, 100)         # a window
    assert st == tk.TK_OK and _rel(part, ref[1][37:137]) <= 1e-12
    st, _ = call(ids[0], 0, 65537)           # beyond the fixed array
    assert st == tk.TK_ERR_ARG and "65536" in tk.tk_last_error(g.h)
    st, _ = call(ids[0], 250, 51)            # beyond the samples taken
    assert st == tk.TK_ERR_ARG
    g.close()
