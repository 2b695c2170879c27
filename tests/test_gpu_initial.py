"""Initial data generated on the device (tk_set_initial_gaussian) and the
automatic number of Lax-Wendroff substeps (substeps = 0).

* The generated planes equal the host planes of the shared input generator:
  the noise (SplitMix64) bit for bit, the Gaussian and sin^2 profile to the
  last bits of exp and sin; the momentum derived from them then agrees to
  rounding.
* substeps = 0 picks the count tk_stability_bound reports for a growth of
  2.5e-5 per step, is re-chosen at every precompute, and a solve with it is
  bit-identical to one made with that count given explicitly (the captured
  graphs follow the change).
"""
import math

import numpy as np
import pytest

from inputs import KERR_25601x64, SCHWARZSCHILD_1601x32, Workload, initial_planes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1010_3816_gb300 as tk
    tk.load_library()


def _solver(w, substeps=None):
    import paper_1010_3816_gb300 as tk
    g = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt,
                  substeps=w.substeps if substeps is None else substeps, variable=w.variable)
    g.precompute(w.a, w.M, w.s, w.m)
    return g


CASES = [
    SCHWARZSCHILD_1601x32,
    KERR_25601x64.with_(Nr=3001, rs_max=-100.0 + 3000 / 32.0, center=-50.0),
    Workload(name="odd", a=0.5, m=-1, rs_min=-13.0, rs_max=29.0, Nr=337, Ntheta=45, dt=0.05,
             center=3.0, width=2.5, amp=-0.7, noise=0.25, seed=2 ** 64 - 5),
]


@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
def test_gaussian_matches_host_planes(w):
    g_dev = _solver(w)
    g_dev.set_initial_gaussian(w.amp, w.center, w.width, w.noise, w.seed)
    dev = g_dev.state()
    g_host = _solver(w)
    re, im = initial_planes(w)
    g_host.set_initial(re, im)
    host = g_host.state()
    edge = np.ones(w.Nr, bool)
    edge[0] = edge[-1] = False
    # Phi: to a few ulps of the pulse's size (exp and sin differ in the last bits)
    scale = max(abs(w.amp), w.noise, 1e-300)
    for c in (0, 1):
        assert np.max(np.abs(dev[c] - host[c])) <= 8 * np.finfo(float).eps * scale
        assert np.all(dev[c][:, ~edge] == 0.0)
    # Pi = b dPhi/dr*: the same few ulps, divided by 2 dr*
    for c in (2, 3):
        assert np.max(np.abs(dev[c] - host[c])) <= 64 * np.finfo(float).eps * scale / w.drs
    g_dev.close()
    g_host.close()


def test_gaussian_noise_is_bit_exact():
    """With amp = 0 only the SplitMix64 noise remains: identical to the host's."""
    w = KERR_25601x64.with_(Nr=2049, amp=0.0)
    g = _solver(w)
    g.set_initial_gaussian(0.0, w.center, w.width, w.noise, w.seed)
    re, im = initial_planes(w)
    st = g.state()
    re[:, 0] = re[:, -1] = 0.0
    im[:, 0] = im[:, -1] = 0.0
    assert np.array_equal(st[0], re) and np.array_equal(st[1], im)
    g.close()


def test_gaussian_argument_errors():
    import paper_1010_3816_gb300 as tk
    w = SCHWARZSCHILD_1601x32.with_(Nr=101, rs_max=-50.0 + 100 / 8.0)
    g = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt)
    with pytest.raises(tk.TkError):
        g.set_initial_gaussian(1.0, 0.0, 1.0)          # before precompute
    g.precompute(w.a, w.M, w.s, w.m)
    for bad in [(1.0, 0.0, 0.0), (1.0, 0.0, -1.0), (float("nan"), 0.0, 1.0),
                (1.0, float("inf"), 1.0), (1.0, 0.0, 1.0, -1e-3)]:
        with pytest.raises(tk.TkError):
            g.set_initial_gaussian(*bad)
    g.close()


@pytest.mark.parametrize("w", [
    Workload(name="s128", a=0.0, m=2, rs_min=-30.0, rs_max=30.0, Nr=961, Ntheta=128, dt=1 / 32.0,
             steps=30, observers=((10.0, math.pi / 2),)),
    Workload(name="k64", a=0.9, m=2, rs_min=-30.0, rs_max=30.0, Nr=481, Ntheta=64, dt=1 / 16.0,
             steps=25, observers=((5.0, math.pi / 4),)),
], ids=lambda w: w.name)
def test_auto_substeps(w):
    probe = _solver(w, substeps=1)
    dt_max, k = probe.stability_bound(2.5e-5)
    probe.close()
    auto = _solver(w, substeps=0)
    assert auto.substeps == k >= 1
    explicit = _solver(w, substeps=k)
    for g in (auto, explicit):
        g.set_initial_gaussian(1.0, 2.0, 3.0)
        g.add_observer(*w.observers[0])
        g.step(w.steps)
    assert np.array_equal(auto.state(), explicit.state())
    assert np.array_equal(auto.waveform(0), explicit.waveform(0))
    # a new precompute re-chooses k, and stepping follows it
    auto.precompute(0.99, 1.0, -2, 3)
    k2 = auto.substeps
    probe = _solver(w.with_(a=0.99, m=3), substeps=1)
    assert probe.stability_bound(2.5e-5)[1] == k2
    probe.close()
    ref = _solver(w.with_(a=0.99, m=3), substeps=k2)
    for g in (auto, ref):
        g.set_initial_gaussian(1.0, 2.0, 3.0)
        g.step(w.steps)
    assert np.array_equal(auto.state(), ref.state())
    for g in (auto, explicit, ref):
        g.close()
