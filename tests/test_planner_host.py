"""The tile planner's programs, executed on the host (no GPU).

``tests/host/plan_emu.cpp`` links the library's planner (planner.cpp), plans a
circuit exactly as the C ABI does (tile geometry, pass capacity cuts, register
phases, and for complex128 plans the butterfly and per-tile-factor
transforms), and runs the resulting tile programs in FP64 with the meaning of
each tile op.  The result must equal the oracle's: a wrong commutation in the
scheduler, a lost gate at a pass cut, a wrong phase permutation or a wrong
folded factor shows up here without a GPU.
"""
import math
import os
import shutil
import struct
import subprocess
import tempfile

import numpy as np
import pytest

import inputs
import oracle
from inputs import Gate
from paper_quant_ph_0608239_gb300._capi import gate_array

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"
PARAMS = {"R": (0.7,), "V": (2 * math.pi / 8,), "SU2": (0.5, -0.1, 0.7, math.sqrt(1 - 0.25 - 0.01 - 0.49))}


@pytest.fixture(scope="module")
def emu():
    cxx = shutil.which("g++")
    if not cxx or not os.path.isdir(CUDA_INC):
        pytest.skip("needs g++ and the CUDA headers")
    d = tempfile.mkdtemp(prefix="plan_emu_")
    exe = os.path.join(d, "plan_emu")
    src = [os.path.join(ROOT, "tests", "host", "plan_emu.cpp"),
           os.path.join(ROOT, "paper_quant_ph_0608239_gb300", "csrc", "planner.cpp")]
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CUDA_INC, "-I", os.path.join(ROOT, "include"), "-o", exe] + src,
                   check=True)
    yield exe
    shutil.rmtree(d, ignore_errors=True)


def run_emu(exe, n, gates, psi, T, RB=0, c128=True, max_ops=0, max_phases=0):
    arr = gate_array(gates)
    blob = struct.pack("<iiiiiiQ", n, T, RB, int(c128), max_ops, max_phases, len(gates))
    blob += bytes(memoryview(arr).cast("B")) + np.ascontiguousarray(psi, dtype=np.complex128).tobytes()
    r = subprocess.run([exe], input=blob, capture_output=True)
    assert r.returncode == 0, r.stderr.decode()
    out = np.frombuffer(r.stdout[:16 << n], dtype=np.complex128)
    stats = struct.unpack("<6i", r.stdout[16 << n:])
    return out, dict(zip(["passes", "ops", "phases", "nglob", "absorbers", "butterflies"], stats))


def rand_state(n, seed):
    rng = np.random.default_rng(seed)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return psi / np.linalg.norm(psi)


def g1(kind, t, ctrl=(), params=()):
    return Gate(kind, (int(t),), tuple(int(c) for c in ctrl), tuple(params))


def mixed_circuit(n, count, seed):
    # every gate kind, 0-3 controls, SWAP gates with and without controls
    rng = np.random.default_rng(seed)
    kinds = ["H", "R", "SU2", "NOT", "V", "X", "YB", "SWAP"]
    out = []
    for _ in range(count):
        k = kinds[int(rng.integers(len(kinds)))]
        qs = [int(x) for x in rng.permutation(n)]
        nc = int(rng.integers(0, 4))
        if k == "SWAP":
            out.append(Gate("SWAP", (qs[0], qs[1]), tuple(qs[2:2 + nc]), ()))
        else:
            out.append(g1(k, qs[0], qs[1:1 + nc], PARAMS.get(k, ())))
    return out


def layered_circuit(n, layers, seed, dense=True):
    # the random-circuit shape with extra Hadamards and phases: many
    # butterflies, phases on bits outside the tile, controlled phases
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(layers):
        for t in range(n):
            k = int(rng.integers(3))
            if k == 1:
                out.append(g1("R", t, (), (float(rng.uniform(0, 2 * math.pi)),)))
            elif k == 2 and dense:
                out.append(g1("SU2", t, (), PARAMS["SU2"]))
            else:
                out.append(g1("H", t))
        for _ in range(3):
            a, b = (int(x) for x in rng.choice(n, 2, replace=False))
            out.append(g1("R", a, (b,), (float(rng.uniform(0, 2 * math.pi)),)))
        p = [int(x) for x in rng.permutation(n)]
        for i in range(0, n - 1, 2):
            out.append(g1("NOT", p[i + 1], (p[i],)))
    return out


def check(exe, n, gates, T, **kw):
    psi = rand_state(n, n + T)
    ref = oracle.run(n, gates, state=psi.copy())
    got, stats = run_emu(exe, n, gates, psi, T, **kw)
    assert float(np.max(np.abs(got - ref))) < 1e-12, stats
    return stats


@pytest.mark.parametrize("n,T", [(6, 4), (9, 6), (11, 8), (13, 10), (14, 12)])
def test_complex128_plans(emu, n, T):
    check(emu, n, mixed_circuit(n, 120, 10 + n), T)
    s = check(emu, n, layered_circuit(n, 5, 20 + n), T)
    assert s["butterflies"] > 0
    if n > T:
        assert s["nglob"] > 0 and s["absorbers"] > 0
    # only Hadamards, phases and CNOTs: no op can take the per-tile factor
    s = check(emu, n, layered_circuit(n, 4, 30 + n, dense=False), T)
    if n > T:
        assert s["nglob"] > 0


@pytest.mark.parametrize("n,T", [(12, 12), (14, 12), (15, 13)])
def test_register_plans_with_capacity_cuts(emu, n, T):
    RB = T - 8
    gates = mixed_circuit(n, 150, 40 + n) + layered_circuit(n, 3, 50 + n)
    full = check(emu, n, gates, T, RB=RB, c128=False, max_ops=64, max_phases=32)
    # a tiny capacity forces many cuts: every gate must still run once, in order
    cut = check(emu, n, gates, T, RB=RB, c128=False, max_ops=5, max_phases=2)
    assert cut["passes"] > full["passes"]
    assert full["phases"] > 0


def test_paper_circuits_exact(emu):
    # QFT of a basis state against its closed form; the adder's sum basis state
    n = 10
    x, gates = inputs.qft_circuit(n, seed=1)
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[x] = 1.0
    got, _ = run_emu(emu, n, gates, psi, 6)
    k = np.arange(1 << n)
    closed = np.exp(2j * np.pi * x * k / (1 << n)) / math.sqrt(1 << n)
    assert np.max(np.abs(got - closed)) < 1e-12
    values, m = [1365, 682], 11
    gates = inputs.adder_circuit(values, m)
    psi = np.zeros(1 << (2 * m), dtype=np.complex128)
    psi[0] = 1.0
    got, _ = run_emu(emu, 2 * m, gates, psi, 12)
    assert int(np.argmax(np.abs(got))) == inputs.adder_expected_index(values, m)
    assert abs(np.max(np.abs(got)) - 1.0) < 1e-12


# Plausible slips planted in a copy of the planner: each must make the
# emulated programs disagree with the oracle (so the checks above can see them).
PLANNER_MUTANTS = {
    "absorber not scaled": ("            scale_op(ops[absorber], S);\n", "\n"),
    "pass cut reorders gates": (
        "std::merge(sched.begin() + take, sched.end(), rest.begin(), rest.end(), std::back_inserter(merged));",
        "merged.insert(merged.end(), rest.begin(), rest.end()); "
        "merged.insert(merged.end(), sched.begin() + take, sched.end());"),
    "controlled phase hoisted": ("if (ops[i].kind == TOP_DIAG_G && ops[i].lcmask == 0) glob.push_back(ops[i]);",
                                 "if (ops[i].kind == TOP_DIAG_G) glob.push_back(ops[i]);"),
    "merged phase on the wrong side": ("if (after) mat2_mul(d.u, x.u, M);", "if (!after) mat2_mul(d.u, x.u, M);"),
    "phase merged across a mixing op": ("after = true;\n                    break;\n                }\n"
                                        "                if (mixes_bit(ops[j], b)) break;",
                                        "after = true;\n                    break;\n                }"),
}


@pytest.mark.parametrize("name", sorted(PLANNER_MUTANTS))
def test_planner_mutants_are_caught(emu, name, tmp_path):
    old, new = PLANNER_MUTANTS[name]
    src = open(os.path.join(ROOT, "paper_quant_ph_0608239_gb300", "csrc", "planner.cpp")).read()
    assert src.count(old) == 1, name
    d = tmp_path / "pkg" / "csrc"  # the same relative layout as the package
    d.mkdir(parents=True)
    (tmp_path / "include").mkdir()
    shutil.copy(os.path.join(ROOT, "include", "qsim.h"), tmp_path / "include" / "qsim.h")
    for f in ("planner.hpp", "kernels.hpp", "perm_layout.hpp"):
        shutil.copy(os.path.join(ROOT, "paper_quant_ph_0608239_gb300", "csrc", f), d / f)
    (d / "planner.cpp").write_text(src.replace(old, new))
    emu_src = open(os.path.join(ROOT, "tests", "host", "plan_emu.cpp")).read().replace(
        "../../paper_quant_ph_0608239_gb300/csrc/planner.hpp", str(d / "planner.hpp"))
    (tmp_path / "plan_emu.cpp").write_text(emu_src)
    exe = str(tmp_path / "mutant")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CUDA_INC, "-I", os.path.join(ROOT, "include"), "-o", exe,
                    str(tmp_path / "plan_emu.cpp"), str(d / "planner.cpp")], check=True)
    n = 14
    cases = [(layered_circuit(n, 5, 77), dict(T=10)),
             (mixed_circuit(n, 150, 78) + layered_circuit(n, 3, 79),
              dict(T=12, RB=4, c128=False, max_ops=5, max_phases=2))]
    caught = False
    for gates, kw in cases:
        psi = rand_state(n, 5)
        ref = oracle.run(n, gates, state=psi.copy())
        got, _ = run_emu(exe, n, gates, psi, **kw)
        caught |= float(np.max(np.abs(got - ref))) > 1e-9
    assert caught, name
