"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module holds workload shapes and random numbers only: it contains none of
the method's arithmetic (no coefficients, no stencil, no boundary rule).  Both
sides receive the arrays it returns as plain inputs.

Random numbers come from SplitMix64 (G. L. Steele, D. Lea, C. H. Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), the
counter-based form: the k-th output (k = 0, 1, ...) of seed S is
``mix(S + (k+1) * 0x9E3779B97F4A7C15)`` with the 64-bit finaliser
``z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB;
z ^= z >> 31``.  A uniform double in [0, 1) is ``(z >> 11) * 2^-53``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Tuple

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+n-1`` of SplitMix64 seeded with ``seed``."""
    k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from SplitMix64."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclass(frozen=True)
class Workload:
    """One Teukolsky m-mode evolution: black hole, mode, grid, initial pulse,
    observers and run length."""
    name: str
    M: float = 1.0
    a: float = 0.0
    s: int = -2
    m: int = 2
    rs_min: float = -50.0
    rs_max: float = 150.0
    Nr: int = 1601
    Ntheta: int = 32
    dt: float = 1.0 / 16.0
    substeps: int = 1
    variable: int = 1                 # 1: evolve Phi^ = Phi / w, 0: literal Phi
    steps: int = 2000                 # outer steps
    amp: float = 1.0                  # Gaussian amplitude
    center: float = 20.0              # Gaussian centre in r*
    width: float = 4.0                # Gaussian standard deviation in r*
    angular: str = "sin2"             # angular profile of the initial data
    noise: float = 0.0                # half-width of the uniform noise
    seed: int = 0
    observers: Tuple[Tuple[float, float], ...] = ((100.0, math.pi / 2),)

    @property
    def drs(self) -> float:
        return (self.rs_max - self.rs_min) / (self.Nr - 1)

    @property
    def points(self) -> int:
        return self.Nr * self.Ntheta

    @property
    def updates(self) -> int:
        """Grid-point updates of a full run (inner steps counted)."""
        return self.points * self.steps * self.substeps

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def initial_planes(w: Workload) -> Tuple[np.ndarray, np.ndarray]:
    """Real and imaginary planes [Ntheta][Nr] of the evolved field at t = 0:
    amp * exp(-(r* - center)^2 / (2 width^2)) * A(theta) + noise, with the
    noise ~ U[-noise, noise) drawn from SplitMix64(seed) for the real plane
    (outputs 0 .. P-1) then the imaginary plane (outputs P .. 2P-1), P = Nr*Ntheta,
    both in row-major [theta][r*] order."""
    rs = w.rs_min + np.arange(w.Nr) * w.drs
    th = (np.arange(w.Ntheta) + 0.5) * (math.pi / w.Ntheta)
    g = w.amp * np.exp(-((rs - w.center) ** 2) / (2.0 * w.width ** 2))
    if w.angular == "sin2":
        ang = np.sin(th) ** 2
    elif w.angular == "one":
        ang = np.ones_like(th)
    elif w.angular == "cos":
        ang = np.cos(th)
    else:
        raise ValueError(w.angular)
    re = ang[:, None] * g[None, :]
    im = np.zeros_like(re)
    if w.noise > 0.0:
        P = w.Nr * w.Ntheta
        u = uniform01(w.seed, 2 * P)
        re = re + w.noise * (2.0 * u[:P] - 1.0).reshape(w.Ntheta, w.Nr)
        im = im + w.noise * (2.0 * u[P:] - 1.0).reshape(w.Ntheta, w.Nr)
    return np.ascontiguousarray(re), np.ascontiguousarray(im)


# --- the workloads ---------------------------------------------------------------
# Schwarzschild, L2-resident: 1601 x 32, 2000 steps of dt = dr*/2.
SCHWARZSCHILD_1601x32 = Workload(name="schwarzschild_a0_1601x32_2000steps")

# Kerr a = 0.9, 25601 x 64, 38400 steps (t = 600 M), noisy pulse, two observers.
# The outer step dt = dr*/2 is the sampling cadence; each outer step is two
# Lax-Wendroff steps of dt/2, which keeps the growth factor of the stiffest
# angular mode, exp(N (omega dt_inner)^4 / 8), near 3 over the whole run
# (about 1e4 with one step), so the 1e-3 noise cannot seed a spurious mode.
KERR_25601x64 = Workload(
    name="kerr_a0.9_25601x64_38400steps", a=0.9, rs_min=-100.0, rs_max=700.0, Nr=25601,
    Ntheta=64, dt=1.0 / 64.0, steps=38400, substeps=2, center=50.0, width=6.0, noise=1e-3, seed=1,
    observers=((500.0, math.pi / 4), (500.0, math.pi / 2)))


# Lax-Wendroff steps per outer step of the batched instances, by Ntheta: the
# angular stiffness grows like Ntheta^2, and k keeps the growth factor of the
# stiffest angular mode over 5000 outer steps of dt = 1/32 near e.
BATCH_SUBSTEPS = {32: 2, 64: 4, 128: 8}


def batched_instances(seed: int = 2) -> List[Workload]:
    """24 independent solves: a in {0, .5, .9, .99} x m in {0,1,2,3,4,-2}, s = -2,
    dr* = 1/16, Nr and Ntheta cycling through {4001, 8001, 16001} and
    {32, 64, 128}, centre ~ U[10, 60), width ~ U[2, 8) from SplitMix64(seed),
    5000 outer steps of dt = 1/32 (BATCH_SUBSTEPS inner steps each), observer
    at (r*_max - 50, pi/2)."""
    avals = (0.0, 0.5, 0.9, 0.99)
    mvals = (0, 1, 2, 3, 4, -2)
    nrs = (4001, 8001, 16001)
    nths = (32, 64, 128)
    u = uniform01(seed, 2 * len(avals) * len(mvals))
    out = []
    k = 0
    for ia, a in enumerate(avals):
        for im, m in enumerate(mvals):
            Nr = nrs[(im + ia) % 3]
            Nth = nths[(im + 2 * ia) % 3]
            rs_min = -50.0
            rs_max = rs_min + (Nr - 1) / 16.0
            center = 10.0 + 50.0 * u[2 * k]
            width = 2.0 + 6.0 * u[2 * k + 1]
            out.append(Workload(name=f"batch_a{a}_m{m}_{Nr}x{Nth}", a=a, m=m, rs_min=rs_min,
                                rs_max=rs_max, Nr=Nr, Ntheta=Nth, dt=1.0 / 32.0, steps=5000,
                                substeps=BATCH_SUBSTEPS[Nth],
                                center=float(center), width=float(width),
                                observers=((rs_max - 50.0, math.pi / 2),)))
            k += 1
    return out


# Adjoint workload: Kerr a = 0.7, 16001 x 128, dr* = 1/16, 20000 outer steps of
# dt = 1/32 (8 Lax-Wendroff steps each), observer at (400, pi/2); the target
# waveform comes from a Gaussian whose amplitude, centre and width are
# perturbed by SplitMix64(seed 4) draws.
ADJOINT_16001x128 = Workload(
    name="adjoint_kerr_a0.7_16001x128_20000steps", a=0.7, rs_min=-100.0, rs_max=900.0,
    Nr=16001, Ntheta=128, dt=1.0 / 32.0, substeps=8, steps=20000, center=50.0, width=6.0,
    observers=((400.0, math.pi / 2),))


def adjoint_target_params(seed: int = 4):
    """(amplitude, centre, width) of the target pulse: the workload's values
    times 1 + U[-5%, 5%) each."""
    u = uniform01(seed, 3)
    w = ADJOINT_16001x128
    f = 1.0 + 0.1 * (u - 0.5)
    return w.amp * f[0], w.center * f[1], w.width * f[2]
