"""tk_extract_noalloc: the allocation-free waveform read-out.

Some callers must not allocate device memory once they are set up: hosts that
hand all device memory to their own pool and treat any other allocation as a
failure, and loops with a device-memory budget fixed in advance.  For them the
library reads waveforms out through a fixed array compiled into it instead of
a buffer it allocates.  The read-out must return exactly what tk_extract
returns (both run the same read-out kernel), on consecutive calls that reuse
the fixed array, for FP64 and FP32 solvers; it must leave the device's free
memory unchanged; and it must refuse requests larger than the array.
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


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_extract_matches_extract_on_consecutive_calls(precision):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1010_3816_gb300 as tk
    from inputs import initial_planes
    lib = tk.load_library()
    g = tk.Solver(rstar_min=W.rs_min, rstar_max=W.rs_max, Nr=W.Nr, Ntheta=W.Ntheta, dt=W.dt,
                  precision=precision)
    g.precompute(W.a, W.M, W.s, W.m)
    re0, im0 = initial_planes(W)
    g.set_initial(re0, im0)
    ids = [g.add_observer(r, t) for r, t in W.observers]
    g.step(W.steps)
    ref = [tk.tk_extract(g.h, k) for k in ids]
    assert all(np.isfinite(r).all() and np.abs(r).max() > 0 for r in ref)
    dp = C.POINTER(C.c_double)

    def call(k, first, count):
        re = np.full(count, np.nan)
        im = np.full(count, np.nan)
        st = lib.tk_extract_noalloc(g.h, k, first, count, re.ctypes.data_as(dp), im.ctypes.data_as(dp))
        return st, re + 1j * im

    st, _ = call(ids[0], 0, W.steps)          # first call on the device: the symbol lookup
    assert st == tk.TK_OK, tk.tk_last_error(g.h)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):                       # two rounds of calls in a row
        for k, r in zip(ids, ref):
            st, got = call(k, 0, W.steps)
            assert st == tk.TK_OK, tk.tk_last_error(g.h)
            assert np.array_equal(got, r)
    st, part = call(ids[1], 37, 100)         # a window
    assert st == tk.TK_OK and np.array_equal(part, ref[1][37:137])
    assert torch.cuda.mem_get_info()[0] == free0     # nothing was allocated
    st, _ = call(ids[0], 0, 65537)           # beyond the fixed array
    assert st == tk.TK_ERR_ARG and "65536" in tk.tk_last_error(g.h)
    st, _ = call(ids[0], 250, 51)            # beyond the samples taken
    assert st == tk.TK_ERR_ARG
    g.close()
