"""Plant plausible mistakes in copies of oracle.c (on the CPU) and check that the
pins of test_oracle_pins.py catch every one of them.  Each mutant is compiled
into a temporary library and the pin suite is run against it in a child
process; the suite must fail."""
import os
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

# (name, original text, mutated text): each a single plausible slip.
MUTANTS = [
    ("x_sign", "U[0] = s; U[1] = I * s; U[2] = I * s; U[3] = s;",
     "U[0] = s; U[1] = -I * s; U[2] = -I * s; U[3] = s;"),
    ("y_transposed", "U[0] = s; U[1] = s; U[2] = -s; U[3] = s;",
     "U[0] = s; U[1] = -s; U[2] = s; U[3] = s;"),
    ("h_sign", "U[0] = s; U[1] = s; U[2] = s; U[3] = -s;",
     "U[0] = s; U[1] = s; U[2] = -s; U[3] = s;"),
    ("phase_sign", "U[3] = cexp(I * p[0]); return 0;", "U[3] = cexp(-I * p[0]); return 0;"),
    ("v_dropped_term", "U[0] = 0.5 * (1 + e); U[1] = 0.5 * (1 - e);",
     "U[0] = 0.5 * (1 + e); U[1] = 0.5 * (0 - e);"),
    ("su2_sign", "U[2] = -p[2] + I * p[3];", "U[2] = p[2] + I * p[3];"),
    ("apply_transposed", "a[i] = U[0] * a0 + U[1] * a1;\n        a[j] = U[2] * a0 + U[3] * a1;",
     "a[i] = U[0] * a0 + U[2] * a1;\n        a[j] = U[1] * a0 + U[3] * a1;"),
    ("control_ignored", "        if ((i & cmask) != cmask) continue;\n        uint64_t j = i | bt;",
     "        uint64_t j = i | bt;"),
    ("swap_gate_partner", "uint64_t j = (i & ~b0) | b1;", "uint64_t j = i | b1;"),
    ("dense_transposed", "s += U[r * K + c] * v[c];", "s += U[c * K + r] * v[c];"),
    ("permute_wrong_bit", "j |= (bl << h[m]) | (bh << l[m]);", "j |= (bl << h[m]) | (bl << l[m]);"),
    ("norm_dropped_im", "        s += re * re + im * im;\n    }\n    return s;",
     "        s += re * re;\n    }\n    return s;"),
    ("qubit_probs_inverted", "if (!(i & bq)) continue;", "if (i & bq) continue;"),
    ("sample_off_by_one", "if (target < c) { x = i; break; }", "if (target < c) { x = i + 1 < D ? i + 1 : i; break; }"),
]


def _run_mutant(tmp, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor not unique: %s" % name
    path = os.path.join(tmp, name + ".c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    lib = os.path.join(tmp, name + ".so")
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", lib, path, "-lm"])
    env = dict(os.environ, QSIM_ORACLE_LIB=lib, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        "-x", "-q", "-p", "no:cacheprovider"], cwd=ROOT, env=env,
                       stdout=subprocess.PIPE, stderr=subprocess.STDOUT, timeout=600)
    return name, r.returncode, r.stdout.decode()[-400:]


def test_every_planted_mistake_fails_a_pin():
    with tempfile.TemporaryDirectory() as tmp:
        with ThreadPoolExecutor(max_workers=4) as ex:
            results = list(ex.map(lambda m: _run_mutant(tmp, *m), MUTANTS))
    survivors = [(n, out) for n, rc, out in results if rc == 0]
    assert not survivors, "mutants not caught by any pin: %s" % [n for n, _ in survivors]
    assert all(rc == 1 for _, rc, _ in results), results
