"""Text programs in the command format of App. A.

A program is a list of lines ``KEYWORD values...``; text after ``!`` and lines
starting with ``#`` are comments.  Commands:

    QUBITS L                    size of the register
    INITIAL STATE x             start from basis state |x>
    MPIPROCESSES N              accepted for compatibility; one GPU holds the state
    <gate> ...                  a gate (below)
    SWAP K a1 .. aK b1 .. bK    the SWAP *command* of Sec. III.B: interchange
                                qubits a_i and b_i in memory (one pass, the
                                qubit-to-bit map follows; the logical state
                                does not change)
    BEGIN MEASUREMENT           starts the measurement block
    DO MEASUREMENT q1 q2 ...    report <Q_q> = P(qubit q = 1) (Eq. Shor7)
    END MEASUREMENT

App. A prints only ``H q``; the other gate keywords are this library's:

    H q  X q  Y q  XB q  YB q       single-qubit gates of Sec. II.B
    R q k                           phase shift R(2 pi / 2^k) (Eq. singlephase)
    RB q k                          its inverse R(-2 pi / 2^k) (the bar of Sec. II.B)
    CNOT t c                        target t, control c (Eq. CNOT2)
    CR t c k                        controlled phase shift R_tc(2 pi / 2^k) (Eq. COMM5)
    CRB t c k                       its inverse
    CV t c k                        controlled V(2 pi / 2^k) (Eq. COMM4)
    TOFFOLI t c1 c2                 (Eq. Toffoli)
    SWAPGATE a b                    the quantum SWAP gate

Parsing is plain host code; execution goes through the C ABI.
"""
from __future__ import annotations

import math
from collections import namedtuple

from .gate import Gate

Step = namedtuple("Step", ["kind", "args"])  # kind: "gates", "swap", "measure"


class ProgramError(ValueError):
    pass


def _ints(tok, lineno, count=None):
    try:
        vals = [int(t) for t in tok]
    except ValueError:
        raise ProgramError("line %d: expected integers, got %s" % (lineno, " ".join(tok)))
    if count is not None and len(vals) != count:
        raise ProgramError("line %d: expected %d values" % (lineno, count))
    return vals


def parse(text):
    """Parse a program.  Returns (L, x0, steps)."""
    L, x0 = None, 0
    steps = []
    pending = []
    in_meas = False

    def flush():
        if pending:
            steps.append(Step("gates", list(pending)))
            pending.clear()

    for lineno, raw in enumerate(text.splitlines(), 1):
        line = raw.split("!", 1)[0].strip()
        if not line or line.startswith("#"):
            continue
        tok = line.split()
        key = tok[0].upper()
        if key == "QUBITS":
            (L,) = _ints(tok[1:], lineno, 1)
            continue
        if key == "INITIAL" and len(tok) >= 2 and tok[1].upper() == "STATE":
            (x0,) = _ints(tok[2:], lineno, 1)
            continue
        if key == "MPIPROCESSES":
            _ints(tok[1:], lineno, 1)
            continue
        if L is None:
            raise ProgramError("line %d: QUBITS must come first" % lineno)
        if key == "BEGIN" and len(tok) > 1 and tok[1].upper() == "MEASUREMENT":
            flush()
            in_meas = True
            continue
        if key == "END" and len(tok) > 1 and tok[1].upper() == "MEASUREMENT":
            in_meas = False
            continue
        if key == "DO" and len(tok) > 1 and tok[1].upper() == "MEASUREMENT":
            if not in_meas:
                raise ProgramError("line %d: DO MEASUREMENT outside a measurement block" % lineno)
            qs = _ints(tok[2:], lineno)
            for qb in qs:
                if not 0 <= qb < L:
                    raise ProgramError("line %d: qubit %d out of range" % (lineno, qb))
            steps.append(Step("measure", qs))
            continue
        if key == "SWAP":
            v = _ints(tok[1:], lineno)
            if not v or len(v) != 1 + 2 * v[0]:
                raise ProgramError("line %d: SWAP K needs 2K qubit labels" % lineno)
            K = v[0]
            a, b = v[1:1 + K], v[1 + K:]
            if len(set(a + b)) != 2 * K or any(not 0 <= x < L for x in a + b):
                raise ProgramError("line %d: SWAP labels must be 2K distinct qubits" % lineno)
            flush()
            steps.append(Step("swap", (a, b)))
            continue
        if in_meas:
            raise ProgramError("line %d: gate inside a measurement block" % lineno)
        pending.append(_gate(key, tok[1:], lineno, L))
    flush()
    if L is None:
        raise ProgramError("no QUBITS command")
    if not 0 <= x0 < (1 << L):
        raise ProgramError("INITIAL STATE out of range")
    return L, x0, steps


def _gate(key, args, lineno, L):
    def qb(v):
        if not 0 <= v < L:
            raise ProgramError("line %d: qubit %d out of range" % (lineno, v))
        return v

    single = {"H": "H", "X": "X", "Y": "Y", "XB": "XB", "YB": "YB", "NOT": "NOT"}
    if key in single:
        (t,) = _ints(args, lineno, 1)
        return Gate(single[key], (qb(t),), (), ())
    if key in ("R", "RB"):
        t, k = _ints(args, lineno, 2)
        sign = 1.0 if key == "R" else -1.0
        return Gate("R", (qb(t),), (), (sign * 2 * math.pi / (1 << k),))
    if key == "CNOT":
        t, c = _ints(args, lineno, 2)
        return Gate("NOT", (qb(t),), (qb(c),), ())
    if key in ("CR", "CV", "CRB"):
        t, c, k = _ints(args, lineno, 3)
        sign = -1.0 if key == "CRB" else 1.0
        return Gate("V" if key == "CV" else "R", (qb(t),), (qb(c),), (sign * 2 * math.pi / (1 << k),))
    if key == "TOFFOLI":
        t, c1, c2 = _ints(args, lineno, 3)
        return Gate("NOT", (qb(t),), (qb(c1), qb(c2)), ())
    if key == "SWAPGATE":
        a, b = _ints(args, lineno, 2)
        return Gate("SWAP", (qb(a), qb(b)), (), ())
    raise ProgramError("line %d: unknown command %s" % (lineno, key))


def run(text, dtype="c128"):
    """Parse and execute a program on the current CUDA device.

    Returns (state, measurements): measurements is a list with one dict
    {qubit: <Q_qubit>} per DO MEASUREMENT command."""
    from . import State
    L, x0, steps = parse(text)
    st = State(L, dtype)
    st.set_basis(x0)
    results = []
    for step in steps:
        if step.kind == "gates":
            st.run(step.args)
        elif step.kind == "swap":
            st.swap_qubits(*step.args)
        else:
            qp = st.qubit_probs()
            results.append({qb: float(qp[qb]) for qb in step.args})
    return st, results
