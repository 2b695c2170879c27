"""Python binding of libtk, the GB300 (sm_103a) Teukolsky Lax-Wendroff solver.

The functions below carry the names of the C ABI in ``include/tk.h`` and only
marshal arguments: every step of the computation runs in the library's CUDA
kernels.  Arrays are numpy arrays (host memory, ``on_device=0``) or CUDA
torch tensors (device memory, ``on_device=1``); PyTorch supplies device memory
and the CUDA stream.  If ``libtk.so`` has not been built the import of the
library fails loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtk.so")

TK_OK, TK_ERR_ARG, TK_ERR_STATE, TK_ERR_CUDA, TK_ERR_OOM, TK_ERR_UNSTABLE, TK_ERR_INTERNAL = range(7)
TK_VAR_LITERAL, TK_VAR_REGULARISED = 0, 1
TK_PREC_F64, TK_PREC_F32 = 0, 1
_STATUS = {0: "TK_OK", 1: "TK_ERR_ARG", 2: "TK_ERR_STATE", 3: "TK_ERR_CUDA", 4: "TK_ERR_OOM",
           5: "TK_ERR_UNSTABLE", 6: "TK_ERR_INTERNAL"}

# every symbol declared in include/tk.h
EXPORTS = ("tk_make_grid", "tk_precompute_coeffs", "tk_set_initial_data", "tk_add_observer",
           "tk_step", "tk_extract", "tk_get_state", "tk_set_state", "tk_stability_bound", "tk_steps_done",
           "tk_check_finite", "tk_synchronize", "tk_last_error", "tk_destroy", "tk_set_graph_chunk",
           "tk_batch_create", "tk_batch_step", "tk_batch_tune", "tk_batch_set_segment",
           "tk_batch_set_graph_chunk", "tk_batch_info", "tk_batch_last_error", "tk_batch_destroy",
           "tk_extract_noalloc", "tk_adjoint", "tk_set_initial_gaussian", "tk_get_substeps",
           "tk_set_steps_per_launch", "tk_param_gradient", "tk_check_bounded_wait",
           "tk_inject_wait_timeout", "tk_probe_fp64_fma", "tk_set_coefficients",
           "tk_get_coefficients", "tk_get_steps_per_launch")


class TkError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib_handle = None
_vp, _dp, _ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)


def load_library(path: str = LIB_PATH):
    """Load libtk.so and declare its signatures (raises if it is missing)."""
    global _lib_handle
    with _lock:
        if _lib_handle is not None:
            return _lib_handle
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = C.CDLL(path)
        sig = {
            "tk_make_grid": (C.c_int, [C.POINTER(_vp), C.c_double, C.c_double, C.c_int, C.c_int,
                                       C.c_double, C.c_int, C.c_int, C.c_int, _vp]),
            "tk_precompute_coeffs": (C.c_int, [_vp, C.c_double, C.c_double, C.c_int, C.c_int]),
            "tk_set_initial_data": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_int]),
            "tk_add_observer": (C.c_int, [_vp, C.c_double, C.c_double, _ip]),
            "tk_step": (C.c_int, [_vp, C.c_int]),
            "tk_extract": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int, _ip, C.c_int]),
            "tk_get_state": (C.c_int, [_vp, _vp, C.c_int]),
            "tk_set_state": (C.c_int, [_vp, _vp, C.c_int]),
            "tk_stability_bound": (C.c_int, [_vp, C.c_double, C.POINTER(C.c_double), _ip]),
            "tk_steps_done": (C.c_int, [_vp, C.POINTER(C.c_int64)]),
            "tk_check_finite": (C.c_int, [_vp]),
            "tk_set_graph_chunk": (C.c_int, [_vp, C.c_int]),
            "tk_synchronize": (C.c_int, [_vp]),
            "tk_last_error": (C.c_char_p, [_vp]),
            "tk_destroy": (None, [_vp]),
            "tk_batch_create": (C.c_int, [C.POINTER(_vp), C.POINTER(_vp), C.c_int]),
            "tk_batch_step": (C.c_int, [_vp, C.c_int]),
            "tk_batch_tune": (C.c_int, [_vp, C.c_int, _ip, C.POINTER(C.c_double)]),
            "tk_batch_set_segment": (C.c_int, [_vp, C.c_int]),
            "tk_batch_set_graph_chunk": (C.c_int, [_vp, C.c_int]),
            "tk_batch_info": (C.c_int, [_vp, _ip, _ip, _ip]),
            "tk_batch_last_error": (C.c_char_p, [_vp]),
            "tk_batch_destroy": (None, [_vp]),
            "tk_extract_noalloc": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, _vp, _vp]),
            "tk_adjoint": (C.c_int, [_vp, _vp, _vp, C.c_int, _vp, C.c_int, C.c_int]),
            "tk_set_initial_gaussian": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double,
                                                  C.c_double, C.c_uint64]),
            "tk_get_substeps": (C.c_int, [_vp, _ip]),
            "tk_get_steps_per_launch": (C.c_int, [_vp, _ip]),
            "tk_set_steps_per_launch": (C.c_int, [_vp, C.c_int]),
            "tk_param_gradient": (C.c_int, [_vp, C.c_int, _vp, C.c_int, C.c_int,
                                            C.POINTER(C.c_double)]),
            "tk_check_bounded_wait": (C.c_int, [C.c_int, C.c_int, C.c_int64, _ip]),
            "tk_inject_wait_timeout": (C.c_int, [_vp]),
            "tk_set_coefficients": (C.c_int, [_vp, C.c_double, C.c_double, C.c_int, C.c_int, _vp, _vp,
                                              _vp, C.c_int]),
            "tk_get_coefficients": (C.c_int, [_vp, _vp, _vp, C.c_int]),
            "tk_probe_fp64_fma": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double),
                                            C.POINTER(C.c_double)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib_handle = lib
        return lib


def _check(h, status: int):
    if status != TK_OK:
        raise TkError(status, load_library().tk_last_error(h).decode())


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


def _arg(x, n: Optional[int] = None):
    """(pointer, on_device, keepalive) for a numpy array or a CUDA torch tensor."""
    if x is None:
        return None, None, None
    if isinstance(x, np.ndarray):
        a = np.ascontiguousarray(x, dtype=np.float64)
        if n is not None and a.size < n:
            raise ValueError(f"array has {a.size} elements, need {n}")
        return a.ctypes.data, 0, a
    import torch
    if isinstance(x, torch.Tensor):
        if not x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous():
            raise ValueError("device arrays must be contiguous float64 CUDA tensors")
        if n is not None and x.numel() < n:
            raise ValueError(f"tensor has {x.numel()} elements, need {n}")
        return x.data_ptr(), 1, x
    raise TypeError(f"unsupported array type {type(x)}")


# --- the C ABI, one function per entry point --------------------------------------
def tk_make_grid(rstar_min: float, rstar_max: float, Nr: int, Ntheta: int, dt: float,
                 substeps: int = 1, angular_variable: int = TK_VAR_REGULARISED,
                 precision: int = TK_PREC_F64, stream=None):
    lib = load_library()
    h = _vp()
    st = _current_stream() if stream is None else stream
    status = lib.tk_make_grid(C.byref(h), rstar_min, rstar_max, Nr, Ntheta, dt, substeps,
                              angular_variable, precision, _vp(st))
    _check(None, status)
    return h


def tk_precompute_coeffs(h, a: float, M: float, s: int, m: int) -> None:
    _check(h, load_library().tk_precompute_coeffs(h, a, M, s, m))


def tk_set_coefficients(h, a: float, M: float, s: int, m: int, node9, half9, ang2=None) -> None:
    """Raw coefficients [9][Ntheta][Nr] at nodes and half nodes (half node i at
    r*_{i+1/2}) and optionally the regularised stencil [2][Ntheta]; numpy
    arrays or CUDA tensors (all on the same side)."""
    p = [_arg(x) for x in (node9, half9, ang2)]
    dev = {q[1] for q in p if q[1] is not None}
    if len(dev) != 1:
        raise ValueError("all arrays must be on the host or all on the device")
    _check(h, load_library().tk_set_coefficients(h, a, M, int(s), int(m), p[0][0], p[1][0], p[2][0],
                                                 dev.pop()))


def tk_get_coefficients(h, shape):
    """(node9, half9): the precompute's raw coefficients, numpy [9][Ntheta][Nr]."""
    node = np.zeros((9,) + tuple(shape))
    half = np.zeros((9,) + tuple(shape))
    _check(h, load_library().tk_get_coefficients(h, node.ctypes.data, half.ctypes.data, 0))
    return node, half


def tk_set_initial_data(h, phi_re, phi_im, pi_re=None, pi_im=None) -> None:
    p = [_arg(x) for x in (phi_re, phi_im, pi_re, pi_im)]
    dev = {q[1] for q in p if q[1] is not None}
    if len(dev) != 1:
        raise ValueError("all arrays must be on the host or all on the device")
    _check(h, load_library().tk_set_initial_data(h, p[0][0], p[1][0], p[2][0], p[3][0], dev.pop()))


def tk_set_initial_gaussian(h, amp: float, center: float, width: float, noise_amp: float = 0.0,
                            seed: int = 0) -> None:
    _check(h, load_library().tk_set_initial_gaussian(h, amp, center, width, noise_amp,
                                                     int(seed) & 0xFFFFFFFFFFFFFFFF))


def tk_add_observer(h, rstar_obs: float, theta_obs: float) -> int:
    k = C.c_int(-1)
    _check(h, load_library().tk_add_observer(h, rstar_obs, theta_obs, C.byref(k)))
    return k.value


def tk_step(h, n: int) -> None:
    _check(h, load_library().tk_step(h, int(n)))


def tk_extract(h, obs_id: int, re=None, im=None):
    """Without re/im: returns the waveform as a complex numpy array.  With two
    CUDA tensors (or numpy arrays): fills them and returns the sample count."""
    lib = load_library()
    cnt = C.c_int(0)
    if re is None:
        _check(h, lib.tk_extract(h, obs_id, None, None, 0, C.byref(cnt), 0))
        n = cnt.value
        r = np.zeros(max(n, 1))
        i = np.zeros(max(n, 1))
        _check(h, lib.tk_extract(h, obs_id, r.ctypes.data, i.ctypes.data, n, C.byref(cnt), 0))
        return (r + 1j * i)[:n]
    pr, dr, kr = _arg(re)
    pi, di, ki = _arg(im)
    cap = min(int(np.prod(getattr(re, "shape", (0,)))), int(np.prod(getattr(im, "shape", (0,)))))
    _check(h, lib.tk_extract(h, obs_id, pr, pi, cap, C.byref(cnt), dr))
    if dr == 0 and isinstance(re, np.ndarray) and kr is not re:
        re[...] = kr
        im[...] = ki
    return cnt.value


def tk_get_state(h, out=None, shape=None):
    """State as planes4 [4, Ntheta, Nr]: a new numpy array, or written into a
    CUDA tensor ``out``."""
    lib = load_library()
    if out is None:
        if shape is None:
            raise ValueError("shape (Ntheta, Nr) is needed to allocate the host result")
        a = np.zeros((4,) + tuple(shape))
        _check(h, lib.tk_get_state(h, a.ctypes.data, 0))
        return a
    p, d, _ = _arg(out)
    _check(h, lib.tk_get_state(h, p, d))
    return out


def tk_set_state(h, planes4) -> None:
    p, d, _k = _arg(planes4)
    _check(h, load_library().tk_set_state(h, p, d))


def tk_stability_bound(h, growth_per_step: float = 2.5e-5):
    """(dt_max, substeps_needed) for the current coefficients and dt."""
    d = C.c_double(0.0)
    k = C.c_int(0)
    _check(h, load_library().tk_stability_bound(h, growth_per_step, C.byref(d), C.byref(k)))
    return d.value, k.value


def tk_adjoint(h, grad, dL_dwave=None, dL_dfinal=None, independent_pi: bool = False) -> None:
    """dL/d(initial data) into ``grad`` (numpy array or CUDA tensor of 2 or 4
    planes [Ntheta][Nr]); dL_dwave is [nobs][count][2], dL_dfinal planes4."""
    pw, dw, kw = _arg(dL_dwave)
    pf, df, kf = _arg(dL_dfinal)
    locs = {d for d in (dw, df) if d is not None}
    if len(locs) != 1:
        raise ValueError("give dL_dwave and/or dL_dfinal, both on the host or both on the device")
    pg, dg, kg = _arg(grad)
    _check(h, load_library().tk_adjoint(h, pw, pf, locs.pop(), pg, dg, 1 if independent_pi else 0))
    if dg == 0 and isinstance(grad, np.ndarray) and kg is not grad:
        grad[...] = kg


def tk_param_gradient(h, param: int, dL_dwave, checkpoint_every: int = 0) -> float:
    """dL/da (param 0) or dL/dM (param 1) for the waveform-loss gradient dL_dwave
    [obs][samples][2] (numpy or CUDA tensor), by checkpointed recomputation."""
    p, dev, _keep = _arg(dL_dwave)
    g = C.c_double(0.0)
    _check(h, load_library().tk_param_gradient(h, int(param), p, dev, int(checkpoint_every),
                                               C.byref(g)))
    return g.value


def tk_check_bounded_wait(n_blocks: int, silent: int, max_polls: int = 1 << 24) -> bool:
    """Run the persistent launches' neighbour wait with block `silent` never
    publishing; True if the waits ran out and raised the error flag."""
    t = C.c_int(0)
    _check(None, load_library().tk_check_bounded_wait(int(n_blocks), int(silent), int(max_polls),
                                                      C.byref(t)))
    return bool(t.value)


def tk_probe_fp64_fma(blocks_per_sm: int = 4, threads: int = 256, iters: int = 1 << 16):
    """(seconds, flop) of the FP64 FMA-pipe microbenchmark (tk_probe_fp64_fma)."""
    s = C.c_double(0.0)
    f = C.c_double(0.0)
    _check(None, load_library().tk_probe_fp64_fma(int(blocks_per_sm), int(threads), int(iters),
                                                  C.byref(s), C.byref(f)))
    return s.value, f.value


def tk_inject_wait_timeout(h) -> None:
    _check(h, load_library().tk_inject_wait_timeout(h))


def tk_steps_done(h) -> int:
    v = C.c_int64(0)
    _check(h, load_library().tk_steps_done(h, C.byref(v)))
    return v.value


def tk_get_substeps(h) -> int:
    v = C.c_int(0)
    _check(h, load_library().tk_get_substeps(h, C.byref(v)))
    return v.value


def tk_set_steps_per_launch(h, steps: int) -> None:
    _check(h, load_library().tk_set_steps_per_launch(h, int(steps)))


def tk_get_steps_per_launch(h) -> int:
    """-1 (persistent), 1 or 2: the launch structure tk_step uses now."""
    v = C.c_int(0)
    _check(h, load_library().tk_get_steps_per_launch(h, C.byref(v)))
    return v.value


def tk_set_graph_chunk(h, outer_steps: int) -> None:
    _check(h, load_library().tk_set_graph_chunk(h, int(outer_steps)))


def tk_check_finite(h) -> None:
    _check(h, load_library().tk_check_finite(h))


def tk_synchronize(h) -> None:
    _check(h, load_library().tk_synchronize(h))


def tk_last_error(h) -> str:
    return load_library().tk_last_error(h).decode()


def tk_destroy(h) -> None:
    if h:
        load_library().tk_destroy(h)


def _bcheck(b, status: int):
    if status != TK_OK:
        msg = load_library().tk_batch_last_error(b).decode() if b else "tk_batch_create failed"
        raise TkError(status, msg)


def tk_batch_create(solvers) -> C.c_void_p:
    hs = [s.h if isinstance(s, Solver) else s for s in solvers]
    arr = (_vp * len(hs))(*[h.value if isinstance(h, C.c_void_p) else h for h in hs])
    b = _vp()
    _bcheck(None, load_library().tk_batch_create(C.byref(b), arr, len(hs)))
    return b


def tk_batch_step(b, n: int) -> None:
    _bcheck(b, load_library().tk_batch_step(b, int(n)))


def tk_batch_tune(b, trial_steps: int = 3):
    seg = C.c_int(0)
    ms = C.c_double(0.0)
    _bcheck(b, load_library().tk_batch_tune(b, int(trial_steps), C.byref(seg), C.byref(ms)))
    return seg.value, ms.value


def tk_batch_set_segment(b, seg: int) -> None:
    _bcheck(b, load_library().tk_batch_set_segment(b, int(seg)))


def tk_batch_set_graph_chunk(b, outer_steps: int) -> None:
    _bcheck(b, load_library().tk_batch_set_graph_chunk(b, int(outer_steps)))


def tk_batch_info(b):
    k, s, bl = C.c_int(0), C.c_int(0), C.c_int(0)
    _bcheck(b, load_library().tk_batch_info(b, C.byref(k), C.byref(s), C.byref(bl)))
    return {"kmax": k.value, "seg": s.value, "blocks": bl.value}


def tk_batch_last_error(b) -> str:
    return load_library().tk_batch_last_error(b).decode()


def tk_batch_destroy(b) -> None:
    if b:
        load_library().tk_batch_destroy(b)


# --- convenience object --------------------------------------------------------------
class Solver:
    """One m-mode evolution on the GPU, owning a tk_solver handle."""

    def __init__(self, *, rstar_min, rstar_max, Nr, Ntheta, dt, substeps=1,
                 variable=TK_VAR_REGULARISED, precision=TK_PREC_F64, stream=None):
        self.Nr, self.Ntheta = int(Nr), int(Ntheta)
        self.h = tk_make_grid(rstar_min, rstar_max, Nr, Ntheta, dt, substeps, variable,
                              precision, stream)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            tk_destroy(h)
            self.h = None

    def close(self):
        self.__del__()

    def precompute(self, a, M, s, m):
        tk_precompute_coeffs(self.h, a, M, s, m)
        return self

    def set_initial(self, phi_re, phi_im, pi_re=None, pi_im=None):
        tk_set_initial_data(self.h, phi_re, phi_im, pi_re, pi_im)
        return self

    def set_initial_gaussian(self, amp, center, width, noise=0.0, seed=0):
        tk_set_initial_gaussian(self.h, amp, center, width, noise, seed)
        return self

    @property
    def substeps(self) -> int:
        return tk_get_substeps(self.h)

    def add_observer(self, rstar, theta) -> int:
        k = tk_add_observer(self.h, rstar, theta)
        self._observers = getattr(self, "_observers", []) + [(rstar, theta)]
        return k

    def step(self, n: int):
        tk_step(self.h, n)
        return self

    def waveform(self, obs_id: int) -> np.ndarray:
        return tk_extract(self.h, obs_id)

    def state(self, out=None):
        return tk_get_state(self.h, out, (self.Ntheta, self.Nr))

    def set_state(self, planes4):
        tk_set_state(self.h, planes4)

    def set_graph_chunk(self, outer_steps: int):
        tk_set_graph_chunk(self.h, outer_steps)
        return self

    def set_steps_per_launch(self, steps: int):
        tk_set_steps_per_launch(self.h, steps)
        return self

    def stability_bound(self, growth_per_step: float = 2.5e-5):
        return tk_stability_bound(self.h, growth_per_step)

    def adjoint(self, grad, dL_dwave=None, dL_dfinal=None, independent_pi=False):
        tk_adjoint(self.h, grad, dL_dwave, dL_dfinal, independent_pi)
        return grad

    def steps_done(self) -> int:
        return tk_steps_done(self.h)

    def param_gradient(self, param, dL_dwave, checkpoint_every=0) -> float:
        """param: "a" or "M" (or 0, 1)."""
        idx = {"a": 0, "M": 1}.get(param, param)
        return tk_param_gradient(self.h, idx, dL_dwave, checkpoint_every)

    def check_finite(self):
        tk_check_finite(self.h)

    def synchronize(self):
        tk_synchronize(self.h)


class Batch:
    """Several Solver objects advanced together (tk_batch_*).  Keeps its
    members alive."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        self.b = tk_batch_create(self.solvers)

    def __del__(self):
        b = getattr(self, "b", None)
        if b:
            tk_batch_destroy(b)
            self.b = None

    def close(self):
        self.__del__()

    def step(self, n: int):
        tk_batch_step(self.b, n)
        return self

    def tune(self, trial_steps: int = 3):
        return tk_batch_tune(self.b, trial_steps)

    def set_segment(self, seg: int):
        tk_batch_set_segment(self.b, seg)
        return self

    def set_graph_chunk(self, outer_steps: int):
        tk_batch_set_graph_chunk(self.b, outer_steps)
        return self

    def info(self):
        return tk_batch_info(self.b)


def waveforms_with_params(solver: "Solver", a, M, s: int, m: int, phi_re, phi_im, n_steps: int):
    """Like waveforms(), and also differentiable in the black-hole spin a and
    mass M (0-dim float64 tensors): the forward pass runs the precompute at
    (a, M, s, m), the initial data and the steps; the backward pass gives the
    planes' gradient through tk_adjoint and dL/da, dL/dM through
    tk_param_gradient (checkpointed recomputation of the trajectory), each
    only when it is needed."""
    import torch

    class _WaveformsParams(torch.autograd.Function):
        @staticmethod
        def forward(ctx, a_, M_, pr, pi):
            solver.precompute(float(a_), float(M_), s, m)
            solver.set_initial(pr.detach().contiguous(), pi.detach().contiguous())
            solver.step(n_steps)
            out = []
            for k in range(len(solver._observers)):
                re = torch.empty(n_steps, dtype=torch.float64, device=pr.device)
                im = torch.empty(n_steps, dtype=torch.float64, device=pr.device)
                tk_extract(solver.h, k, re, im)
                out.append(torch.stack([re, im], dim=1))
            return torch.stack(out, dim=0)

        @staticmethod
        def backward(ctx, g):
            g = g.detach().contiguous()
            ga = gM = gpr = gpi = None
            if ctx.needs_input_grad[2] or ctx.needs_input_grad[3]:
                grad = torch.empty((2, solver.Ntheta, solver.Nr), dtype=torch.float64, device=g.device)
                tk_adjoint(solver.h, grad, dL_dwave=g)
                gpr, gpi = grad[0], grad[1]
            if ctx.needs_input_grad[0]:
                ga = torch.tensor(tk_param_gradient(solver.h, 0, g), dtype=torch.float64,
                                  device=g.device)
            if ctx.needs_input_grad[1]:
                gM = torch.tensor(tk_param_gradient(solver.h, 1, g), dtype=torch.float64,
                                  device=g.device)
            return ga, gM, gpr, gpi

    return _WaveformsParams.apply(a, M, phi_re, phi_im)


def waveforms(solver: "Solver", phi_re, phi_im, n_steps: int):
    """Differentiable map from the initial planes (CUDA float64 tensors
    [Ntheta][Nr], momentum for zero time derivative) to the waveforms of the
    solver's observers, a tensor [nobs, n_steps, 2] (real, imaginary).  The
    solver must be precomputed and have its observers; its state is
    overwritten.  The backward pass runs the adjoint kernel (tk_adjoint)."""
    import torch

    class _Waveforms(torch.autograd.Function):
        @staticmethod
        def forward(ctx, pr, pi):
            solver.set_initial(pr.detach().contiguous(), pi.detach().contiguous())
            solver.step(n_steps)
            nobs = len(solver._observers) if hasattr(solver, "_observers") else None
            out = []
            for k in range(nobs):
                re = torch.empty(n_steps, dtype=torch.float64, device=pr.device)
                im = torch.empty(n_steps, dtype=torch.float64, device=pr.device)
                tk_extract(solver.h, k, re, im)
                out.append(torch.stack([re, im], dim=1))
            return torch.stack(out, dim=0)

        @staticmethod
        def backward(ctx, g):
            grad = torch.empty((2, solver.Ntheta, solver.Nr), dtype=torch.float64, device=g.device)
            tk_adjoint(solver.h, grad, dL_dwave=g.detach().contiguous())
            return grad[0], grad[1]

    return _Waveforms.apply(phi_re, phi_im)
