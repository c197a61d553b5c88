"""Seeded, synthetic circuit generators shared by the oracle and the CUDA path.

This package holds no arithmetic of the simulation method: it only draws random
numbers and lists gates symbolically (kind, qubits, parameters).  Both the
oracle (``oracle/``) and the product (``paper_quant_ph_0608239_gb300``, fed by
the tests and ``bench.py``) turn these symbolic gates into matrices with their
own, separate code; the product does not import this package.
"""
from .circuits import (  # noqa: F401
    Gate, GATE_KINDS, hadamard_all, qft, iqft, qft_circuit, adder_circuit,
    adder_expected_index, adder_gate_count, adder_pairs, random_circuit, batch_circuits,
    random_basis, shor_initial_support, logical_gate_count,
)
