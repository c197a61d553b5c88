"""Phase passes of the complex64 tensor-core plans, on the host.

tests/host/phase_emu.cpp links the planner (planner.cpp), plans a circuit with
plan_fused_phases and applies the result the way the kernels do: dense blocks
as their FP64 matrices, phase passes as sums of the planner's tables (fixed-
point turns mod 2^32, the evaluation of k_phase.cu).  Against the oracle:

  * the QFT register adder of Sec. V.A (the controlled phases between the two
    registers become one phase pass, and the plan has fewer passes in all),
    with the complex64 (32-bit turns) and complex128 (64-bit turns) tables;
  * the adder's phase shifts interleaved with Hadamards on other qubits and
    controlled NOTs whose controls share their bits (they commute);
  * circuits without long runs keep the plain block plan.
"""
import ctypes
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


@pytest.fixture(scope="module")
def emu():
    cxx = shutil.which("g++")
    if not cxx or not os.path.isdir(CUDA_INC):
        pytest.skip("needs g++ and the CUDA headers")
    d = tempfile.mkdtemp(prefix="phase_emu_")
    exe = os.path.join(d, "phase_emu")
    src = [os.path.join(ROOT, "tests", "host", "phase_emu.cpp"),
           os.path.join(ROOT, "paper_quant_ph_0608239_gb300", "csrc", "planner.cpp")]
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CUDA_INC, "-I", os.path.join(ROOT, "include"), "-o", exe] + src,
                   check=True)
    yield exe
    shutil.rmtree(d, ignore_errors=True)


def run_emu(exe, n, k, gates, psi, minrun=24, wide=False):
    arr = gate_array(gates)
    blob = struct.pack("<iiiiQ", n, k, minrun, int(wide), len(gates)) + bytes(memoryview(arr).cast("B"))[:len(gates) * ctypes.sizeof(arr._type_)]
    blob += np.ascontiguousarray(psi, dtype=np.complex128).tobytes()
    r = subprocess.run([exe], input=blob, capture_output=True)
    assert r.returncode == 0, (r.returncode, r.stderr.decode())
    out = np.frombuffer(r.stdout[:16 << n], dtype=np.complex128)
    return out, dict(zip(["blocks", "phase_passes", "phase_gates", "plain_blocks"],
                         struct.unpack("<4i", r.stdout[16 << n:])))


@pytest.mark.parametrize("k,m,wide", [(5, 7, False), (6, 10, False), (5, 7, True), (5, 10, True)])
def test_adder_phase_pass(emu, k, m, wide):
    vals = (37, 98)
    gates = inputs.adder_circuit(vals, m)
    n = 2 * m
    psi = oracle.basis(n, 0)
    got, st = run_emu(emu, n, k, gates, psi, wide=wide)
    ref = oracle.run(n, gates, x0=0)
    assert st["phase_passes"] >= 1 and st["phase_gates"] >= m * (m + 1) // 2, st
    assert st["blocks"] < st["plain_blocks"], st
    # 64-bit turns (complex128): within the complex128 tolerance; 32-bit
    # turns: within 2^-32 turns per table entry
    assert np.max(np.abs(got - ref)) < (1e-13 if wide else 1e-8)
    assert int(np.argmax(np.abs(got))) == inputs.adder_expected_index(vals, m)


def test_commuting_gates_between_phases(emu):
    # controlled phases among 12 qubits, with Hadamards on 3 other qubits and
    # CNOTs whose controls (not targets) are phase bits in between: they
    # commute with the phases, so one run of 40 phases remains
    n = 15
    rng = np.random.default_rng(5)
    gates = [Gate("H", (q,), (), ()) for q in range(n)]
    for i in range(40):
        a, b = (int(x) for x in rng.choice(12, 2, replace=False))
        gates.append(Gate("R", (a,), (b,), (float(rng.uniform(0, 2 * math.pi)),)))
        if i % 7 == 3:
            gates.append(Gate("H", (12 + i % 3,), (), ()))
        if i % 11 == 5:
            gates.append(Gate("NOT", (13,), (int(rng.integers(12)),), ()))
    gates += [Gate("H", (q,), (), ()) for q in range(n)]
    psi = oracle.basis(n, 0)
    got, st = run_emu(emu, n, 5, gates, psi)
    ref = oracle.run(n, gates, x0=0)
    assert st["phase_passes"] == 1 and st["phase_gates"] == 40, st
    assert np.max(np.abs(got - ref)) < 1e-8


def test_random_circuit_keeps_plain_blocks(emu):
    n = 12
    gates = inputs.random_circuit(n, 8, seed=3)
    rng = np.random.default_rng(1)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi /= np.linalg.norm(psi)
    got, st = run_emu(emu, n, 5, gates, psi)
    assert st["phase_passes"] == 0 and st["blocks"] == st["plain_blocks"], st
    assert np.max(np.abs(got - oracle.run(n, gates, state=psi.copy()))) < 1e-10
