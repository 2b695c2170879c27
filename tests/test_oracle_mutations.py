"""The oracle's pins are strong enough to catch plausible mistakes: each case
below plants one (a dropped term, a wrong sign, a wrong index, transposed
operands) in a copy of oracle/tk_oracle.c, builds it, and runs the pin tests
against that build (the oracle loads the library named by TKO_SO); at least
one pin must fail.  The unmodified source, built the same way, must pass.
Everything runs on the CPU; nothing here touches the CUDA path."""
import os
import shutil
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
ORACLE_C = os.path.join(ROOT, "oracle", "tk_oracle.c")
PINS = ["tests/test_oracle_step.py", "tests/test_oracle_coeffs.py", "tests/test_oracle_angular.py",
        "tests/test_oracle_physics.py"]   # fastest first: a failure stops the run (-x)

# (what the mistake is, text in tk_oracle.c, replacement)
MUTANTS = [
    ("c1_sign_of_b_bstar", "out[K_C1R] = b * CtR + E - b * b_s;", "out[K_C1R] = b * CtR + E + b * b_s;"),
    ("c3_drops_Q", "out[K_C3R] = b * b * fss + E0 * fs + QR + c4 * V;",
     "out[K_C3R] = b * b * fss + E0 * fs + c4 * V;"),
    ("c2_imaginary_sign", "out[K_C2I] = -CtI;", "out[K_C2I] = CtI;"),
    ("D_c1_block_transposed", "{ -cf[K_C1R], cf[K_C1I], -bb, 0.0 },", "{ -cf[K_C1I], cf[K_C1R], -bb, 0.0 },"),
    ("S_c2_wrong_component", "Svec[3] = cf[K_C2R] * u0[3] + cf[K_C2I] * u0[2]",
     "Svec[3] = cf[K_C2R] * u0[3] + cf[K_C2I] * u0[3]"),
    ("average_wrong_index", "0.5 * (q[IDX(b, a)] + q[IDX(b, a - 1)]);", "0.5 * (q[IDX(b, a)] + q[IDX(b, a)]);"),
    ("lw1_full_instead_of_half_step", "- 0.5 * dt * S->rhs[k][IDX(b, a)];", "- dt * S->rhs[k][IDX(b, a)];"),
    ("lw2_average_one_sided", "0.5 * (S->q_h[k][IDX(b, a + 1)] + S->q_h[k][IDX(b, a)]);",
     "0.5 * (S->q_h[k][IDX(b, a + 1)] + S->q_h[k][IDX(b, a + 1)]);"),
    ("ghost_parity_inverted", "return (abs(m) % 2 == 0) ? 1 : -1;", "return (abs(m) % 2 == 0) ? -1 : 1;"),
    ("tortoise_inner_log_sign", "- Am * log((r - rm) / (2.0 * M));", "+ Am * log((r - rm) / (2.0 * M));"),
    ("stencil_wrong_face", "Am[j] = Plo / (Q * dth * dth);", "Am[j] = Phi / (Q * dth * dth);"),
    ("c5_term_sign", "+ cf[K_C5] * (up[k] - um[k]) / (2.0 * dth);", "+ cf[K_C5] * (um[k] - up[k]) / (2.0 * dth);"),
    ("extraction_theta_weights_swapped",
     "double lo = (1.0 - o->fth) * o->w0 * q[IDX(o->j0, o->i0)] + o->fth * o->w1 * q[IDX(o->j0 + 1, o->i0)];",
     "double lo = o->fth * o->w0 * q[IDX(o->j0, o->i0)] + (1.0 - o->fth) * o->w1 * q[IDX(o->j0 + 1, o->i0)];"),
    ("initial_momentum_without_b", "S->q[2][IDX(b, a)] = bb * (", "S->q[2][IDX(b, a)] = ("),
]


def _build(tmp_path, src, name):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    c = tmp_path / f"{name}.c"
    c.write_text(src)
    so = tmp_path / f"lib{name}.so"
    base = [cc, "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", str(c),
            "-o", str(so), "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(base, check=True, capture_output=True, text=True)
    return str(so)


def _pins(so):
    env = dict(os.environ, TKO_SO=so)
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)


def test_unmodified_oracle_passes_the_pins(tmp_path):
    r = _pins(_build(tmp_path, open(ORACLE_C).read(), "orig"))
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("what,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_a_planted_mistake(tmp_path, what, old, new):
    src = open(ORACLE_C).read()
    assert src.count(old) == 1, f"{what}: the text to change is not unique in tk_oracle.c"
    r = _pins(_build(tmp_path, src.replace(old, new), what))
    assert r.returncode == 1, (what, r.stdout[-3000:])
