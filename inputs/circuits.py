"""Symbolic, seeded circuit generators (no simulation arithmetic in here).

A circuit is a list of :class:`Gate`.  Qubit q is bit q of the amplitude index,
qubit 0 the least significant bit (Sec. II.A, Eq. STAT2).  A gate names its
target qubit(s), its control qubits and its parameters; each consumer builds the
matrix itself.

Gate kinds and the passage that defines them:

=======  ================================================================
kind     meaning
=======  ================================================================
H        Hadamard (Eq. Hadamard)
X, Y     pi/2 rotations about x / y (Eqs. Xoperation, Yoperation)
XB, YB   their inverses (Sec. II.B, "inverse ... denoted by a bar")
NOT      bit flip; with one control it is CNOT (Eq. CNOT2, Eq. NUM6),
         with two controls the Toffoli gate (Eq. Toffoli, Eq. NUM8)
R        phase shift R(phi) (Eq. singlephase); with a control it is the
         controlled phase shift (Eq. COMM5)
V        V(phi); with a control it is controlled-V (Eq. COMM4, Eq. NUM7)
SU2      2x2 special unitary from a unit quaternion (a, b, c, d):
         [[a+ib, c+id], [-c+id, a-ib]]  (random test circuits only)
U        explicit 2x2 complex matrix, params = 8 floats, row-major
         (re, im) pairs
SWAP     quantum swap gate of two qubits (final reversal of the QFT); not
         the SWAP *command* of App. A, which only relabels qubits
=======  ================================================================

Random draws (angles, quaternions, basis states, qubit pairings) come from
``numpy.random.default_rng(seed)`` so the oracle and the GPU path see the same
gate list.
"""
from __future__ import annotations

import math
from collections import namedtuple

import numpy as np

Gate = namedtuple("Gate", ["kind", "targets", "controls", "params"])

GATE_KINDS = ("H", "X", "Y", "XB", "YB", "NOT", "R", "V", "SU2", "U", "SWAP")

TWO_PI = 2.0 * math.pi


def _g(kind, target, controls=(), params=()):
    return Gate(kind, (int(target),), tuple(int(c) for c in controls),
                tuple(float(p) for p in params))


def hadamard_all(n):
    """Hadamard on every qubit of an n-qubit register (the scaling test of Sec. V)."""
    return [_g("H", q) for q in range(n)]


def qft(qubits, swaps=False):
    """Quantum Fourier transform network on ``qubits`` (LSB first).

    The network of Fig. QFT (Nielsen & Chuang form): for j from the most
    significant qubit down, a Hadamard on qubit j followed by controlled phase
    shifts R(2*pi/2^(j-l+1)) with target j and control l for every lower qubit
    l.  Without the final swaps the output register is bit-reversed; with
    ``swaps=True`` floor(m/2) quantum SWAP gates restore the standard order so
    that QFT|x> = 2^(-m/2) sum_k exp(+2 pi i x k / 2^m) |k>.
    """
    q = [int(x) for x in qubits]
    m = len(q)
    out = []
    for j in range(m - 1, -1, -1):
        out.append(_g("H", q[j]))
        for l in range(j - 1, -1, -1):
            out.append(_g("R", q[j], (q[l],), (TWO_PI / float(1 << (j - l + 1)),)))
    if swaps:
        for i in range(m // 2):
            out.append(Gate("SWAP", (q[i], q[m - 1 - i]), (), ()))
    return out


def _inverse_gate(g):
    """Symbolic inverse of a gate used by the QFT networks (H, R, SWAP)."""
    if g.kind in ("H", "SWAP", "NOT"):
        return g
    if g.kind in ("R", "V"):
        return Gate(g.kind, g.targets, g.controls, (-g.params[0],))
    raise ValueError("no symbolic inverse for %s" % g.kind)


def iqft(qubits, swaps=False):
    """Inverse QFT: the QFT network reversed with conjugated phases."""
    return [_inverse_gate(g) for g in reversed(qft(qubits, swaps))]


def qft_circuit(n, seed=1, swaps=True):
    """Config: n-qubit QFT on a seeded random basis state.

    Returns (x, gates) where x is the initial basis-state index.
    """
    rng = np.random.default_rng(seed)
    x = int(rng.integers(0, 1 << n))
    return x, qft(range(n), swaps=swaps)


_INIT_PAIRS = ("X", "Y", "XB", "YB")


def adder_circuit(values, m):
    """QFT register adder of Sec. V.A (Fig. adder): n registers of m qubits.

    Register r holds qubits r*m .. r*m+m-1 (LSB first).  Each set bit of the
    initial values is loaded with a pair of equal pi/2 rotations (XX, YY,
    XbarXbar, YbarYbar in turn), each pair counting as two operations.  The
    last register is Fourier transformed (no bit-reversal swaps), every other
    register is added into it with controlled phase shifts, and the inverse QFT
    brings the sum back: the last register ends up holding the sum of all
    registers modulo 2^m, the others are unchanged.

    In the QFT output without swaps, the qubit at position m-1-j of the
    accumulator carries the phase of Fourier bit k_j; adding register a needs a
    controlled phase 2*pi/2^(m-i-j) from a_i onto that qubit for every
    i + j <= m - 1.
    """
    values = [int(v) for v in values]
    nreg = len(values)
    gates = []
    kind_i = 0
    for r, v in enumerate(values):
        for b in range(m):
            if (v >> b) & 1:
                k = _INIT_PAIRS[kind_i % 4]
                kind_i += 1
                gates.append(_g(k, r * m + b))
                gates.append(_g(k, r * m + b))
    acc = list(range((nreg - 1) * m, nreg * m))
    gates += qft(acc, swaps=False)
    for r in range(nreg - 1):
        src = list(range(r * m, r * m + m))
        for i in range(m):
            for j in range(m - i):
                phi = TWO_PI / float(1 << (m - i - j))
                gates.append(_g("R", acc[m - 1 - j], (src[i],), (phi,)))
    gates += iqft(acc, swaps=False)
    return gates


def adder_gate_count(values, m):
    """Number of operations N_O of the adder (the count Table App. B prints)."""
    nreg = len(values)
    set_bits = sum(bin(int(v) % (1 << m)).count("1") for v in values)
    qft_ops = m + m * (m - 1) // 2
    return 2 * set_bits + 2 * qft_ops + (nreg - 1) * (m * (m + 1) // 2)


def adder_expected_index(values, m):
    """Basis-state index the adder must produce (registers LSB first)."""
    values = [int(v) % (1 << m) for v in values]
    total = sum(values) % (1 << m)
    idx = 0
    for r, v in enumerate(values[:-1]):
        idx |= v << (r * m)
    idx |= total << ((len(values) - 1) * m)
    return idx


def adder_pairs(m=15, count=8, seed=3):
    """Seeded register values for the two-register adder: ``count`` pairs
    (a, b) drawn as ``default_rng(seed).integers(0, 2^m, (count, 2))``; the
    first pair is the one the single-pair workload draws."""
    rng = np.random.default_rng(seed)
    return [(int(a), int(b)) for a, b in rng.integers(0, 1 << m, (count, 2))]


def _random_layers(rng, n, depth):
    gates = []
    for _ in range(depth):
        for q in range(n):
            kind = int(rng.integers(0, 3))
            if kind == 0:
                gates.append(_g("H", q))
            elif kind == 1:
                gates.append(_g("R", q, (), (rng.uniform(0.0, TWO_PI),)))
            else:
                v = rng.standard_normal(4)
                v = v / np.sqrt(np.dot(v, v))  # uniform point on S^3 (a draw, not a gate rule)
                gates.append(_g("SU2", q, (), tuple(v)))
        p = rng.permutation(n)
        for i in range(n // 2):
            gates.append(_g("NOT", int(p[2 * i + 1]), (int(p[2 * i]),)))
    return gates


def random_circuit(n, depth, seed):
    """Seeded random circuit: per layer a random 1-qubit gate on every qubit
    (H, R(theta) with theta ~ U[0, 2pi), or a Haar-random SU(2)), then CNOTs on
    disjoint random qubit pairs (control p[2i], target p[2i+1])."""
    rng = np.random.default_rng(seed)
    return _random_layers(rng, n, depth)


def batch_circuits(count=512, seed0=1000, nmin=12, nmax=24, dmin=10, dmax=60):
    """Batch of independent random circuits with uneven sizes.

    Circuit i uses seed seed0+i, n ~ U{nmin..nmax}, depth ~ U{dmin..dmax}.
    Returns a list of (n, gates).
    """
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        n = int(rng.integers(nmin, nmax + 1))
        d = int(rng.integers(dmin, dmax + 1))
        out.append((n, _random_layers(rng, n, d)))
    return out


def random_basis(n, seed):
    """Seeded random basis-state index in [0, 2^n)."""
    return int(np.random.default_rng(seed).integers(0, 1 << n))


def shor_initial_support(X, G, y):
    """Support of the state of Eq. Shor2: for each x in [0, 2^X) the value
    f(x) = y^x mod G held by the f-register.  The paper gives no gate network
    for this step, so it enters the simulation as an initial state: amplitude
    2^(-X/2) at index x + 2^X * f(x)."""
    f = np.empty(1 << X, dtype=np.int64)
    v = 1
    for x in range(1 << X):
        f[x] = v
        v = (v * y) % G
    return f


def logical_gate_count(gates):
    """Gates counted as operations (N_O excludes only SWAP *commands*, which
    never appear in a gate list; quantum SWAP gates are counted)."""
    return len(gates)
