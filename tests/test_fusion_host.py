"""The dense-fusion planner on the host (qsim_fuse_blocks, no device).

A block may take a gate past earlier gates on other qubits (they commute), so
the blocks applied in order must equal the circuit exactly (up to rounding):
checked against the oracle's gate-by-gate run for random circuits, the QFT with
its reversal swaps, the register adder (Sec. V.A) and multi-controlled gates
(Toffoli, controlled-V, controlled phase, controlled SWAP)."""
import math

import numpy as np
import pytest

import inputs
import oracle
from inputs import Gate

PARAMS = {"R": (1.1,), "V": (2 * math.pi / 16,), "SU2": (0.5, -0.1, 0.7, math.sqrt(1 - 0.25 - 0.01 - 0.49))}


@pytest.fixture(scope="module")
def q():
    from paper_quant_ph_0608239_gb300 import build
    build.build()  # host entry point only: no device work
    import paper_quant_ph_0608239_gb300 as q
    return q


def controlled_mix(rng, n, count, kmax):
    out = []
    kinds = ["NOT", "R", "V", "SU2", "H", "SWAP"]
    while len(out) < count:
        kind = kinds[int(rng.integers(len(kinds)))]
        qs = [int(x) for x in rng.permutation(n)]
        nc = int(rng.integers(0, 3))
        if kind == "SWAP":
            if 2 + nc <= kmax:
                out.append(Gate("SWAP", (qs[0], qs[1]), tuple(qs[2:2 + nc]), ()))
        elif 1 + nc <= kmax:
            out.append(Gate(kind, (qs[0],), tuple(qs[1:1 + nc]), tuple(float(p) for p in PARAMS.get(kind, ()))))
    return out


def apply_blocks(n, blocks, x0):
    psi = oracle.basis(n, x0)
    for qubits, U in blocks:
        oracle.apply_dense(psi, n, qubits, U)
    return psi


def consecutive_count(gates, k):
    """Blocks of the plain grouping of consecutive gates (no reordering)."""
    count, cur = 0, set()
    for g in gates:
        m = set(g.targets) | set(g.controls)
        if len(cur | m) > k:
            count, cur = count + 1, set(m)
        else:
            cur |= m
    return count + (1 if cur else 0)


@pytest.mark.parametrize("k", [2, 3, 4, 5, 6])
@pytest.mark.parametrize("n", [7, 10])
def test_blocks_equal_the_circuit(q, n, k):
    gates = inputs.random_circuit(n, 6, seed=40 + n + k)
    rng = np.random.default_rng(n * 10 + k)
    mix = controlled_mix(rng, n, 30, k)
    for g in mix:  # scatter the controlled gates through the layers
        gates.insert(int(rng.integers(len(gates) + 1)), g)
    x0 = inputs.random_basis(n, seed=k)
    ref = oracle.run(n, gates, x0=x0)
    blocks = q.fuse_blocks(n, gates, k)
    got = apply_blocks(n, blocks, x0)
    assert np.max(np.abs(got - ref)) < 1e-12
    for qubits, U in blocks:
        assert len(qubits) == k and len(set(qubits)) == k and all(0 <= b < n for b in qubits)
        assert np.max(np.abs(U @ U.conj().T - np.eye(1 << k))) < 1e-12


def test_single_qubit_blocks(q):
    n = 6
    gates = [g for g in inputs.random_circuit(n, 4, seed=3) if not g.controls]
    blocks = q.fuse_blocks(n, gates, 1)
    assert len(blocks) == n  # every qubit's gates commute past the other qubits' gates
    ref = oracle.run(n, gates, x0=5)
    assert np.max(np.abs(apply_blocks(n, blocks, 5) - ref)) < 1e-12


def test_qft_with_swaps_and_inverse(q):
    n = 9
    x0, gates = inputs.qft_circuit(n, seed=5)
    gates = list(gates) + list(inputs.iqft(range(n), swaps=True))
    for k in (2, 4, 6):
        got = apply_blocks(n, q.fuse_blocks(n, gates, k), x0)
        # QFT followed by its inverse is the identity: back to |x0>
        want = np.zeros(1 << n, dtype=complex)
        want[x0] = 1.0
        assert np.max(np.abs(got - want)) < 1e-12


def test_adder_blocks_give_the_sum(q):
    values, m = [45, 17, 99], 7
    n = 3 * m
    gates = inputs.adder_circuit(values, m)
    ref_index = inputs.adder_expected_index(values, m)
    blocks = q.fuse_blocks(n, gates, 5)
    psi = apply_blocks(n, blocks, 0)
    assert int(np.argmax(np.abs(psi))) == ref_index
    assert abs(abs(psi[ref_index]) - 1.0) < 1e-12


def test_reordering_saves_blocks(q):
    # 30 qubits, depth 40: a layer's 1-qubit gates and CNOTs on random pairs
    # leave much to gain by taking gates out of order
    gates = inputs.random_circuit(30, 40, seed=11)
    for k in (4, 5, 6):
        nb = len(q.fuse_blocks(30, gates, k))
        assert nb <= 0.4 * consecutive_count(gates, k), (k, nb)
    # and no more blocks than consecutive grouping on circuits with controlled gates
    rng = np.random.default_rng(2)
    for n, k in [(8, 3), (12, 5)]:
        g2 = inputs.random_circuit(n, 10, seed=n) + controlled_mix(rng, n, 20, k)
        assert len(q.fuse_blocks(n, g2, k)) <= consecutive_count(g2, k)


def test_gate_wider_than_k_is_rejected(q):
    from paper_quant_ph_0608239_gb300 import QsimError, QSIM_EINVAL
    cnot = [Gate("NOT", (1,), (0,), ())]
    toffoli = [Gate("NOT", (2,), (0, 1), ())]
    for gates, k in [(cnot, 1), (toffoli, 2)]:
        with pytest.raises(QsimError) as e:
            q.fuse_blocks(4, gates, k)
        assert e.value.status == QSIM_EINVAL
    for bad_k in (0, 7):
        with pytest.raises(QsimError):
            q.fuse_blocks(8, cnot, bad_k)
    assert q.fuse_blocks(4, [], 3) == []


@pytest.mark.parametrize("seed", range(8))
def test_searched_blocks_equal_the_circuit(q, seed):
    """The grouping the beam search may pick (plan_fused keeps whichever of
    the greedy and the searched grouping has fewer blocks): deep random
    circuits with controlled gates and SWAP gates, where the search changes
    the blocks, applied block by block against the oracle."""
    rng = np.random.default_rng(500 + seed)
    n = 11
    k = 3 + seed % 4
    gates = inputs.random_circuit(n, 12, seed=600 + seed)
    for g in controlled_mix(rng, n, 40, k):
        gates.insert(int(rng.integers(len(gates) + 1)), g)
    x0 = inputs.random_basis(n, seed=seed)
    ref = oracle.run(n, gates, x0=x0)
    blocks = q.fuse_blocks(n, gates, k)
    assert np.max(np.abs(apply_blocks(n, blocks, x0) - ref)) < 1e-12
    assert len(blocks) <= consecutive_count(gates, k)


def test_search_saves_blocks_on_the_bench_circuit(q):
    """On the 30-qubit depth-40 bench circuit the searched grouping needs
    fewer 5-qubit blocks than the greedy one alone (145)."""
    gates = inputs.random_circuit(30, 40, seed=2)
    assert len(q.fuse_blocks(30, gates, 5)) <= 140


@pytest.mark.parametrize("k", [4, 5, 6])
def test_bench_generators_blocks_equal_the_circuit(q, k):
    """The bench circuits' generators (depth 40 seed 2, depth 20 seed 4) at 16
    qubits, grouped as the GPU plans group them, against the oracle."""
    n = 16
    for depth, seed in ((40, 2), (20, 4)):
        gates = inputs.random_circuit(n, depth, seed=seed)
        x0 = inputs.random_basis(n, seed=seed)
        got = apply_blocks(n, q.fuse_blocks(n, gates, k), x0)
        assert np.max(np.abs(got - oracle.run(n, gates, x0=x0))) < 1e-12
