"""CPU oracle for the Teukolsky Lax-Wendroff step (arXiv 1010.3816, Sec. 3).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It wraps the plain C
implementation in ``tk_oracle.c`` (FP64, no FMA contraction, no fast-math),
which shares no code with the CUDA path.

The same unchanged source is also built a second time with FMA contraction
(``build(fma=True)``, selected per solver by ``Solver(..., build="fma")``): a
different, equally correct rounding order of the same scheme.  The distance
between the two builds' runs is the size of the rounding differences any two
correct implementations of the scheme accumulate over a run.

The state layout is the paper's (Sec. 4): four planes ``qre, qim, pre, pim``,
each ``[Ntheta][Nr]`` with the r* index fastest.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tk_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libtk_oracle.so")
_SO_FMA = os.path.join(_BUILD, "libtk_oracle_fma.so")
_lock = threading.Lock()
_lib_handles = {}

NCOEF = 9
COEF_NAMES = ("b", "c1R", "c1I", "c2R", "c2I", "c3R", "c3I", "c4", "c5")


def _fma_flags():
    """Flags that let gcc contract a*b + c into fused multiply-adds.  aarch64
    has FMA in its base instruction set; x86-64 needs -mfma to emit one."""
    import platform
    flags = ["-ffp-contract=fast"]
    if platform.machine().lower() in ("x86_64", "amd64"):
        flags.append("-mfma")
    return flags


def build(force: bool = False, fma: bool = False) -> str:
    """Compile ``tk_oracle.c`` into ``_build/libtk_oracle.so`` (with OpenMP if
    the compiler supports it).  Returns the path of the shared library.

    With ``fma`` the same source is compiled into ``libtk_oracle_fma.so`` with
    FMA contraction on (the only change); it serves as a second rounding order
    of the same arithmetic."""
    os.makedirs(_BUILD, exist_ok=True)
    so = _SO_FMA if fma else _SO
    if not force and os.path.exists(so) and os.path.getmtime(so) >= os.path.getmtime(_SRC):
        return so
    contract = _fma_flags() if fma else ["-ffp-contract=off"]
    tmp = so + ".%d.tmp" % os.getpid()
    base = ["gcc", "-std=gnu11", "-O2"] + contract + ["-fno-fast-math",
            "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, so)
    return so


class Params(C.Structure):
    _fields_ = [("M", C.c_double), ("a", C.c_double), ("s", C.c_int), ("m", C.c_int),
                ("rs_min", C.c_double), ("drs", C.c_double), ("Nr", C.c_int), ("Ntheta", C.c_int),
                ("dt", C.c_double), ("substeps", C.c_int), ("variable", C.c_int)]


_dp = C.POINTER(C.c_double)


def _lib(variant: str = "plain"):
    """The loaded oracle library: ``"plain"`` (no contraction) or ``"fma"``."""
    if variant not in ("plain", "fma"):
        raise ValueError(variant)
    with _lock:
        if variant not in _lib_handles:
            if variant == "fma":
                path = build(fma=True)
            else:
                # TKO_SO names an alternative build of tk_oracle.c (used to check
                # that the pins catch deliberately planted mistakes).
                path = os.environ.get("TKO_SO") or build()
            lib = C.CDLL(path)
            lib.tko_tortoise_x.restype = C.c_double
            lib.tko_tortoise_x.argtypes = [C.c_double, C.c_double, C.c_double]
            lib.tko_x_of_rstar.restype = C.c_double
            lib.tko_x_of_rstar.argtypes = [C.c_double, C.c_double, C.c_double]
            lib.tko_weight.restype = C.c_double
            lib.tko_weight.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double]
            lib.tko_parity.restype = C.c_int
            lib.tko_parity.argtypes = [C.c_int, C.c_int]
            lib.tko_coeffs_point.restype = None
            lib.tko_coeffs_point.argtypes = [C.c_double, C.c_double, C.c_int, C.c_int, C.c_int,
                                             C.c_double, C.c_double, _dp]
            lib.tko_angular_apply.restype = None
            lib.tko_angular_apply.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _dp, _dp]
            lib.tko_angular_apply_many.restype = None
            lib.tko_angular_apply_many.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _dp, _dp]
            lib.tko_regular_stencil.restype = None
            lib.tko_regular_stencil.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp]
            lib.tko_average.restype = None
            lib.tko_average.argtypes = [_dp, _dp, C.c_int, C.c_int]
            lib.tko_new.restype = C.c_void_p
            lib.tko_new.argtypes = [C.POINTER(Params)]
            lib.tko_free.restype = None
            lib.tko_free.argtypes = [C.c_void_p]
            lib.tko_get_coeffs.restype = None
            lib.tko_get_coeffs.argtypes = [C.c_void_p, _dp, _dp]
            lib.tko_set_initial.restype = None
            lib.tko_set_initial.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
            lib.tko_get_state.restype = None
            lib.tko_get_state.argtypes = [C.c_void_p, _dp]
            lib.tko_replace_state.restype = None
            lib.tko_replace_state.argtypes = [C.c_void_p, _dp]
            lib.tko_replace_coeffs.restype = None
            lib.tko_replace_coeffs.argtypes = [C.c_void_p, _dp, _dp]
            lib.tko_add_observer.restype = C.c_int
            lib.tko_add_observer.argtypes = [C.c_void_p, C.c_double, C.c_double]
            lib.tko_run.restype = None
            lib.tko_run.argtypes = [C.c_void_p, C.c_int]
            lib.tko_waveform.restype = C.c_int
            lib.tko_waveform.argtypes = [C.c_void_p, C.c_int, _dp, _dp]
            lib.tko_set_threads.restype = None
            lib.tko_set_threads.argtypes = [C.c_int]
            lib.tko_get_threads.restype = C.c_int
            lib.tko_get_threads.argtypes = []
            _lib_handles[variant] = lib
        return _lib_handles[variant]


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


# --- point functions ---------------------------------------------------------
def tortoise_x(M: float, a: float, x: float) -> float:
    """r*(r) with x = r - r_+ (Kerr tortoise coordinate)."""
    return _lib().tko_tortoise_x(M, a, x)


def x_of_rstar(M: float, a: float, rstar: float) -> float:
    """Inverse tortoise map: x = r - r_+ at a given r*."""
    return _lib().tko_x_of_rstar(M, a, rstar)


def horizons(M: float, a: float):
    d = (M * M - a * a) ** 0.5
    return M + d, M - d


def weight(s: int, m: int, variable: int, theta: float) -> float:
    return _lib().tko_weight(s, m, variable, theta)


def parity(m: int, variable: int) -> int:
    return _lib().tko_parity(m, variable)


def coeffs_point(M, a, s, m, variable, x, theta) -> dict:
    out = np.zeros(NCOEF)
    _lib().tko_coeffs_point(M, a, s, m, variable, x, theta, _ptr(out))
    return dict(zip(COEF_NAMES, out.tolist()))


def angular_apply(s: int, m: int, variable: int, F: np.ndarray) -> np.ndarray:
    F = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros_like(F)
    _lib().tko_angular_apply(s, m, variable, F.shape[0], _ptr(F), _ptr(out))
    return out


def angular_matrix(s: int, m: int, variable: int, Ntheta: int) -> np.ndarray:
    """Matrix of the discrete angular operator, column k = operator applied to
    the k-th unit vector."""
    eye = np.ascontiguousarray(np.eye(Ntheta))
    out = np.zeros_like(eye)
    _lib().tko_angular_apply_many(s, m, variable, Ntheta, Ntheta, _ptr(eye), _ptr(out))
    return out.T.copy()


def regular_stencil(s: int, m: int, Ntheta: int):
    """(Ap, Am): the self-adjoint angular stencil of the regularised variable."""
    Ap = np.zeros(Ntheta)
    Am = np.zeros(Ntheta)
    _lib().tko_regular_stencil(s, m, Ntheta, _ptr(Ap), _ptr(Am))
    return Ap, Am


def average(q: np.ndarray) -> np.ndarray:
    """The paper's kernel_average1 on one plane [Ntheta][Nr]; column 0 of the
    result is left at zero."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    out = np.zeros_like(q)
    _lib().tko_average(_ptr(q), _ptr(out), q.shape[1], q.shape[0])
    return out


def set_threads(n: int) -> None:
    _lib().tko_set_threads(int(n))


def get_threads() -> int:
    return _lib().tko_get_threads()


# --- solver --------------------------------------------------------------------
class Solver:
    """One Teukolsky m-mode evolution on the CPU.

    Parameters mirror the CUDA library's make_grid/precompute calls: the radial
    grid is ``rs_min + a*drs`` for ``a < Nr``, the angular grid is
    ``(b + 1/2) pi / Ntheta``; ``dt`` is the outer step, split into
    ``substeps`` Lax-Wendroff steps; ``variable`` 0 evolves the literal
    field, 1 the pole-regularised one.  ``build`` picks the library:
    ``"plain"`` (no FMA contraction) or ``"fma"`` (the same source contracted).
    """

    def __init__(self, *, M=1.0, a=0.0, s=-2, m=2, rs_min, rs_max, Nr, Ntheta, dt,
                 substeps=1, variable=1, build="plain"):
        self.Nr, self.Ntheta = int(Nr), int(Ntheta)
        drs = (rs_max - rs_min) / (Nr - 1)
        self.params = Params(M, a, s, m, rs_min, drs, Nr, Ntheta, dt, substeps, variable)
        self._lib = _lib(build)
        self._h = self._lib.tko_new(C.byref(self.params))
        if not self._h:
            raise ValueError("oracle rejected the parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.tko_free(h)
            self._h = None

    @property
    def drs(self) -> float:
        return self.params.drs

    def set_initial(self, phi_re, phi_im, pi_re=None, pi_im=None):
        shp = (self.Ntheta, self.Nr)
        pr = np.ascontiguousarray(phi_re, dtype=np.float64).reshape(shp)
        pi = np.ascontiguousarray(phi_im, dtype=np.float64).reshape(shp)
        if pi_re is None:
            self._lib.tko_set_initial(self._h, _ptr(pr), _ptr(pi), None, None)
        else:
            qr = np.ascontiguousarray(pi_re, dtype=np.float64).reshape(shp)
            qi = np.ascontiguousarray(pi_im, dtype=np.float64).reshape(shp)
            self._lib.tko_set_initial(self._h, _ptr(pr), _ptr(pi), _ptr(qr), _ptr(qi))

    def add_observer(self, rstar: float, theta: float) -> int:
        k = self._lib.tko_add_observer(self._h, rstar, theta)
        if k < 0:
            raise ValueError("observer outside the grid")
        return k

    def run(self, n: int) -> None:
        self._lib.tko_run(self._h, int(n))

    def state(self) -> np.ndarray:
        out = np.zeros((4, self.Ntheta, self.Nr))
        self._lib.tko_get_state(self._h, _ptr(out))
        return out

    def replace_state(self, planes4) -> None:
        """Overwrite the state (4 planes), keeping steps and samples."""
        a = np.ascontiguousarray(planes4, dtype=np.float64).reshape(4, self.Ntheta, self.Nr)
        self._lib.tko_replace_state(self._h, _ptr(a))

    def replace_coeffs(self, node, half) -> None:
        """Overwrite the coefficient tables (layout of ``coeffs()``)."""
        shp = (NCOEF, self.Ntheta, self.Nr)
        n = np.ascontiguousarray(node, dtype=np.float64).reshape(shp)
        h = np.ascontiguousarray(half, dtype=np.float64).reshape(shp)
        self._lib.tko_replace_coeffs(self._h, _ptr(n), _ptr(h))

    def coeffs(self):
        """(node, half) coefficient tables, each [NCOEF][Ntheta][Nr]; the half
        table's column a >= 1 holds the values at r*_{a-1/2}."""
        node = np.zeros((NCOEF, self.Ntheta, self.Nr))
        half = np.zeros((NCOEF, self.Ntheta, self.Nr))
        self._lib.tko_get_coeffs(self._h, _ptr(node), _ptr(half))
        return node, half

    def waveform(self, obs_id: int) -> np.ndarray:
        n = self._lib.tko_waveform(self._h, obs_id, None, None)
        if n < 0:
            raise ValueError("bad observer id")
        re = np.zeros(max(n, 1))
        im = np.zeros(max(n, 1))
        self._lib.tko_waveform(self._h, obs_id, _ptr(re), _ptr(im))
        return (re + 1j * im)[:n]
