"""The App. A command format: parsing on the CPU, execution on the GPU."""
import math
import os

import numpy as np
import pytest

import inputs
import oracle
from inputs import Gate
from paper_quant_ph_0608239_gb300 import program

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROG_H = """
# Hadamard on every qubit of a 12-qubit register, with interchanges
QUBITS 12
INITIAL STATE 0
MPIPROCESSES 8        ! ignored on one GPU
H 0
H 1
H 2
H 3
H 4
H 5
H 6
H 7
H 8
SWAP 1 0 9            ! bring qubit 9 to where qubit 0 was
H 9
SWAP 2 1 2 10 11
H 10
H 11
BEGIN MEASUREMENT
DO MEASUREMENT 0 1 2 3 4 5
DO MEASUREMENT 6 7 8 9 10 11
END MEASUREMENT
"""


def test_parse_structure():
    L, x0, steps = program.parse(PROG_H)
    assert L == 12 and x0 == 0
    kinds = [s.kind for s in steps]
    assert kinds == ["gates", "swap", "gates", "swap", "gates", "measure", "measure"]
    assert steps[1].args == ([0], [9]) and steps[3].args == ([1, 2], [10, 11])
    assert steps[0].args[0] == Gate("H", (0,), (), ())
    assert steps[5].args == [0, 1, 2, 3, 4, 5]


def test_parse_gate_keywords():
    text = ("QUBITS 4\nINITIAL STATE 5\nR 1 3\nCNOT 2 0\nCR 3 1 4\nCV 0 2 2\nTOFFOLI 3 0 1\nSWAPGATE 0 3\nXB 2\n"
            "RB 0 2\nCRB 1 3 5\n")
    L, x0, steps = program.parse(text)
    g = steps[0].args
    assert (L, x0) == (4, 5)
    assert g[0] == Gate("R", (1,), (), (2 * math.pi / 8,))
    assert g[1] == Gate("NOT", (2,), (0,), ())
    assert g[2] == Gate("R", (3,), (1,), (2 * math.pi / 16,))
    assert g[3] == Gate("V", (0,), (2,), (2 * math.pi / 4,))
    assert g[4] == Gate("NOT", (3,), (0, 1), ())
    assert g[5] == Gate("SWAP", (0, 3), (), ())
    assert g[6] == Gate("XB", (2,), (), ())
    assert g[7] == Gate("R", (0,), (), (-2 * math.pi / 4,))
    assert g[8] == Gate("R", (1,), (3,), (-2 * math.pi / 32,))


@pytest.mark.parametrize("bad", [
    "H 0\n",                                    # no QUBITS
    "QUBITS 3\nH 3\n",                          # qubit out of range
    "QUBITS 3\nSWAP 2 0 1 2\n",                 # too few labels
    "QUBITS 3\nSWAP 1 0 0\n",                   # repeated label
    "QUBITS 3\nDO MEASUREMENT 0\n",             # outside a block
    "QUBITS 3\nFOO 1\n",                        # unknown command
    "QUBITS 3\nINITIAL STATE 8\n",              # basis state out of range
])
def test_parse_errors(bad):
    with pytest.raises(program.ProgramError):
        program.parse(bad)


def _render(gates):
    """gate list -> program lines (phases as 2 pi / 2^k where exact)."""
    out = []
    for g in gates:
        if g.kind in ("H", "X", "Y", "XB", "YB") and not g.controls:
            out.append("%s %d" % (g.kind, g.targets[0]))
        elif g.kind == "R":
            phi = g.params[0]
            k = round(math.log2(2 * math.pi / abs(phi)))
            assert abs(2 * math.pi / (1 << k) - abs(phi)) < 1e-15
            bar = "" if phi > 0 else "B"
            if g.controls:
                out.append("CR%s %d %d %d" % (bar, g.targets[0], g.controls[0], k))
            else:
                out.append("R%s %d %d" % (bar, g.targets[0], k))
        else:
            raise ValueError(g)
    return "\n".join(out)


@pytest.mark.gpu
def test_run_programs_on_gpu():
    import torch
    torch.cuda.set_device(0)
    st, res = program.run(PROG_H, "c128")
    assert len(res) == 2
    for d in res:
        for v in d.values():
            assert abs(v - 0.5) < 1e-12
    a = st.get_state()
    assert np.max(np.abs(a - 2.0 ** -6)) < 1e-13
    st.free()
    # a QFT adder written as a program: the sum appears bit-exact
    values, m = [13, 22], 5
    text = "QUBITS %d\nINITIAL STATE 0\n" % (2 * m)
    loads = []
    for r, v in enumerate(values):
        for b in range(m):
            if (v >> b) & 1:
                loads += ["X %d" % (r * m + b)] * 2
    gates = inputs.adder_circuit([0, 0], m)  # the QFT/add/IQFT part (no loading gates)
    text += "\n".join(loads) + "\n" + _render(gates) + "\nBEGIN MEASUREMENT\nDO MEASUREMENT %s\nEND MEASUREMENT\n" % (
        " ".join(str(i) for i in range(2 * m)))
    st, res = program.run(text, "c64")
    want = inputs.adder_expected_index(values, m)
    got = sum(1 << qb for qb, v in res[0].items() if v > 0.5)
    assert got == want
    st.free()


def test_package_does_not_need_the_input_generators():
    # the product (binding and program front-end) must import and parse without
    # the repository's test-input package on the path
    import subprocess
    import sys
    code = ("import sys; sys.modules['inputs'] = None\n"
            "import paper_quant_ph_0608239_gb300.program as p\n"
            "L, x0, steps = p.parse('QUBITS 3\\nH 0\\nCNOT 1 0\\n')\n"
            "assert L == 3 and steps[0].args[0].kind == 'H'\n")
    subprocess.check_call([sys.executable, "-c", code], cwd=ROOT)
