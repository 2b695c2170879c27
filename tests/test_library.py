"""Host-side checks of the C-ABI library that need no GPU: it builds, loads,
exports every entry point that include/tk.h declares, and rejects bad
arguments before touching the device."""
import ctypes as C
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tk_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1010_3816_gb300 import build
    path = build.build()
    import paper_1010_3816_gb300 as tk
    return tk.load_library(path)


def test_exports_every_declared_symbol(lib):
    import paper_1010_3816_gb300 as tk
    decl = _declared()
    assert len(decl) >= 13
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(tk.EXPORTS) == decl


def test_argument_validation_without_gpu(lib):
    import paper_1010_3816_gb300 as tk
    h = C.c_void_p()
    for args in [(1.0, 0.0, 10, 8, 0.1, 1, 1, 0), (0.0, 1.0, 2, 8, 0.1, 1, 1, 0),
                 (0.0, 1.0, 10, 1, 0.1, 1, 1, 0), (0.0, 1.0, 10, 129, 0.1, 1, 1, 0),
                 (0.0, 1.0, 10, 8, 0.0, 1, 1, 0), (0.0, 1.0, 10, 8, 0.1, -1, 1, 0),
                 (0.0, 1.0, 10, 8, 0.1, 1, 2, 0), (0.0, 1.0, 10, 8, 0.1, 1, 1, 5)]:
        st = lib.tk_make_grid(C.byref(h), *args, None)
        assert st == tk.TK_ERR_ARG, args
        assert h.value is None
        assert len(lib.tk_last_error(None)) > 0
    assert lib.tk_make_grid(None, 0.0, 1.0, 10, 8, 0.1, 1, 1, 0, None) == tk.TK_ERR_ARG
    # calls on a NULL solver fail cleanly
    assert lib.tk_step(None, 1) == tk.TK_ERR_ARG
    assert lib.tk_check_finite(None) == tk.TK_ERR_ARG
    v = C.c_int(7)
    assert lib.tk_get_steps_per_launch(None, C.byref(v)) == tk.TK_ERR_ARG and v.value == 7
    assert lib.tk_get_substeps(None, C.byref(v)) == tk.TK_ERR_ARG
    assert lib.tk_get_coefficients(None, None, None, 0) == tk.TK_ERR_ARG
    assert lib.tk_set_coefficients(None, 0.0, 1.0, -2, 2, None, None, None, 0) == tk.TK_ERR_ARG
    lib.tk_destroy(None)


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_1010_3816_gb300 as tk
    saved = tk._lib_handle
    tk._lib_handle = None
    try:
        with pytest.raises(RuntimeError):
            tk.load_library(str(tmp_path / "missing.so"))
    finally:
        tk._lib_handle = saved
