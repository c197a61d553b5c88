"""Pins for the CPU oracle: values the paper prints, closed forms, textbook
identities, library routines for special cases and brute force on small
registers.  None of these re-types the oracle's own formulas; a dropped term, a
wrong sign, a swapped index or a transposed operand in oracle.c fails at least
one of them (tests/test_oracle_mutants.py checks that claim)."""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
import inputs
from inputs import Gate
import golden_io

SX = np.array([[0, 1], [1, 0]], dtype=complex)
SY = np.array([[0, -1j], [1j, 0]], dtype=complex)
SZ = np.array([[1, 0], [0, -1]], dtype=complex)
I2 = np.eye(2, dtype=complex)
P1 = np.array([[0, 0], [0, 1]], dtype=complex)


def g1(kind, t, ctrl=(), params=()):
    return Gate(kind, (t,), tuple(ctrl), tuple(params))


# ---------------------------------------------------------------------------
# Gate matrices: the rotations of Sec. II.B as matrix exponentials of the
# spin-1/2 operators S = sigma/2 (scipy.linalg.expm), not re-typed entries.
# ---------------------------------------------------------------------------
def test_matrix_hadamard_textbook():
    # Textbook: H = (sigma_x + sigma_z)/sqrt(2).
    np.testing.assert_allclose(oracle.gate_matrix(g1("H", 0)), (SX + SZ) / math.sqrt(2), atol=1e-15)


def test_matrix_rotations_are_exponentials():
    X = scipy.linalg.expm(1j * math.pi / 2 * SX / 2)     # e^{i pi S^x / 2}
    Y = scipy.linalg.expm(1j * math.pi / 2 * SY / 2)     # e^{i pi S^y / 2}
    np.testing.assert_allclose(oracle.gate_matrix(g1("X", 0)), X, atol=1e-15)
    np.testing.assert_allclose(oracle.gate_matrix(g1("Y", 0)), Y, atol=1e-15)
    np.testing.assert_allclose(oracle.gate_matrix(g1("XB", 0)), np.linalg.inv(X), atol=1e-15)
    np.testing.assert_allclose(oracle.gate_matrix(g1("YB", 0)), np.linalg.inv(Y), atol=1e-15)


@pytest.mark.parametrize("phi", [0.3, 2 * math.pi / 8, -1.7, math.pi])
def test_matrix_phase_shift_exponential(phi):
    # R(phi) = e^{i phi/2} e^{-i phi S^z} (Eq. singlephase).
    R = np.exp(1j * phi / 2) * scipy.linalg.expm(-1j * phi * SZ / 2)
    np.testing.assert_allclose(oracle.gate_matrix(g1("R", 0, (), (phi,))), R, atol=1e-15)


@pytest.mark.parametrize("phi", [0.3, 2 * math.pi / 16, -2.2])
def test_matrix_controlled_v_is_conjugated_phase(phi):
    # V(phi) = H R(phi) H, and V(pi) is the bit flip, so CNOT is a special case
    # of controlled-V (Sec. II.C).
    H = (SX + SZ) / math.sqrt(2)
    R = np.diag([1, np.exp(1j * phi)])
    np.testing.assert_allclose(oracle.gate_matrix(g1("V", 0, (), (phi,))), H @ R @ H, atol=1e-15)
    np.testing.assert_allclose(oracle.gate_matrix(g1("V", 0, (), (math.pi,))), SX, atol=1e-15)
    np.testing.assert_allclose(oracle.gate_matrix(g1("NOT", 0)), SX, atol=0)


def test_matrix_su2_quaternion():
    rng = np.random.default_rng(5)
    v = rng.standard_normal(4)
    v /= np.linalg.norm(v)
    U = oracle.gate_matrix(g1("SU2", 0, (), tuple(v)))
    # U = a I + i (d X + c Y + b Z): an element of SU(2), det 1 and unitary,
    # and equal to exp of i theta n.sigma for the quaternion's axis.
    np.testing.assert_allclose(U @ U.conj().T, I2, atol=1e-15)
    assert abs(np.linalg.det(U) - 1) < 1e-15
    theta = math.acos(max(-1.0, min(1.0, v[0])))
    axis = np.array([v[3], v[2], v[1]]) / math.sin(theta)   # (x, y, z) weights
    gen = axis[0] * SX + axis[1] * SY + axis[2] * SZ
    np.testing.assert_allclose(scipy.linalg.expm(1j * theta * gen), U, atol=1e-14)


def test_paper_loading_ops_bring_zero_to_one():
    # Sec. V.A: XX, YY, XbarXbar and YbarYbar each bring a qubit from |0> to |1>
    # (up to a phase).
    for k in ("X", "Y", "XB", "YB"):
        a = oracle.run(1, [g1(k, 0), g1(k, 0)])
        assert abs(abs(a[1]) - 1.0) < 1e-15 and abs(a[0]) < 1e-15


# ---------------------------------------------------------------------------
# Worked examples of Sec. II (tests/golden/worked_examples.txt).
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("ex", golden_io.worked_examples(), ids=lambda e: e["name"])
def test_worked_examples(ex):
    n = ex["n"]
    a = np.arange(1, (1 << n) + 1, dtype=np.complex128) * (1 + 0.5j)
    before = a.copy()
    phi = 0.7
    if ex["what"] == "perm":
        oracle.run(n, [g1("NOT", ex["target"], ex["controls"])], state=a)
        np.testing.assert_array_equal(a, before[ex["vals"]])
    else:
        oracle.run(n, [g1("R", ex["target"], ex["controls"], (phi,))], state=a)
        expect = before.copy()
        for i in ex["vals"]:
            expect[i] *= np.exp(1j * phi)
        np.testing.assert_allclose(a, expect, atol=1e-13)


# ---------------------------------------------------------------------------
# Brute force: the full 2^n x 2^n matrix from Kronecker products.
# ---------------------------------------------------------------------------
def embed(n, ops):
    """Kronecker product with ops[q] on qubit q (identity elsewhere); the
    leftmost factor is the most significant qubit."""
    M = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        M = np.kron(M, ops.get(q, I2))
    return M


def dense_gate(n, g):
    if g.kind == "SWAP":
        a, b = g.targets
        # SWAP = (I + XX + YY + ZZ) / 2 on the two qubits.
        S = sum(embed(n, {a: P, b: P}) for P in (I2, SX, SY, SZ)) / 2
        if g.controls:
            proj = {c: P1 for c in g.controls}
            return embed(n, {}) + (embed(n, proj) @ (S - embed(n, {})))
        return S
    U = oracle.gate_matrix(g)
    ops = {c: P1 for c in g.controls}
    ops[g.targets[0]] = U - I2
    return embed(n, {}) + embed(n, ops)


def random_gates(rng, n, count):
    kinds = ["H", "X", "Y", "XB", "YB", "NOT", "R", "V", "SU2", "SWAP"]
    out = []
    for _ in range(count):
        k = kinds[int(rng.integers(len(kinds)))]
        qs = rng.permutation(n)
        nc = int(rng.integers(0, 3))
        if k == "SWAP":
            out.append(Gate("SWAP", (int(qs[0]), int(qs[1])), tuple(int(c) for c in qs[2:2 + nc]), ()))
            continue
        params = ()
        if k in ("R", "V"):
            params = (float(rng.uniform(-math.pi, math.pi)),)
        if k == "SU2":
            v = rng.standard_normal(4)
            params = tuple(v / np.linalg.norm(v))
        out.append(g1(k, int(qs[0]), [int(c) for c in qs[1:1 + nc]], params))
    return out


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_circuit_matches_dense_kronecker(n):
    rng = np.random.default_rng(100 + n)
    gates = random_gates(rng, n, 40) if n > 2 else [g for g in random_gates(rng, 3, 60)
                                                    if max(g.targets + g.controls) < n]
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi /= np.linalg.norm(psi)
    M = np.eye(1 << n, dtype=complex)
    for g in gates:
        M = dense_gate(n, g) @ M
    got = oracle.run(n, gates, state=psi.copy())
    np.testing.assert_allclose(got, M @ psi, atol=1e-13)


def test_dense_kq_matches_einsum_and_sequence():
    rng = np.random.default_rng(7)
    n = 8
    for k in (1, 2, 3, 4):
        q = [int(x) for x in rng.permutation(n)[:k]]
        Z = rng.standard_normal((1 << k, 1 << k)) + 1j * rng.standard_normal((1 << k, 1 << k))
        U, _ = np.linalg.qr(Z)
        psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
        got = oracle.apply_dense(psi.copy(), n, q, U)
        # Independent route: view the state as an n-index tensor (axis 0 = qubit
        # n-1) and contract U's column index bits with the chosen axes.
        T = psi.reshape((2,) * n)
        Ut = U.reshape((2,) * (2 * k))          # row bits k-1..0, column bits k-1..0
        axes_state = [n - 1 - q[j] for j in range(k - 1, -1, -1)]
        out = np.tensordot(Ut, T, axes=(list(range(k, 2 * k)), axes_state))
        # out has axes (row bits k-1..0, remaining state axes in order)
        rest = [ax for ax in range(n) if ax not in axes_state]
        perm = [None] * n
        for j, ax in enumerate(axes_state):
            perm[ax] = j
        for j, ax in enumerate(rest):
            perm[ax] = k + j
        expect = np.transpose(out, perm).reshape(-1)
        np.testing.assert_allclose(got, expect, atol=1e-12)
    # A tensor product of two single-qubit gates applied densely equals the
    # two gates applied one after the other.
    A = oracle.gate_matrix(g1("SU2", 0, (), (0.5, 0.5, 0.5, 0.5)))
    B = oracle.gate_matrix(g1("H", 0))
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    seq = oracle.run(n, [g1("U", 2, (), _u8(A)), g1("U", 5, (), _u8(B))], state=psi.copy())
    dense = oracle.apply_dense(psi.copy(), n, [2, 5], np.kron(B, A))
    np.testing.assert_allclose(dense, seq, atol=1e-13)


def _u8(U):
    return tuple(x for z in U.reshape(-1) for x in (z.real, z.imag))


# ---------------------------------------------------------------------------
# Closed forms.
# ---------------------------------------------------------------------------
def test_hadamard_all_uniform():
    n = 14
    a = oracle.run(n, inputs.hadamard_all(n))
    np.testing.assert_allclose(a, np.full(1 << n, 2.0 ** (-n / 2)), atol=1e-15)


@pytest.mark.parametrize("n,seed", [(10, 1), (7, 3)])
def test_qft_closed_form(n, seed):
    x, gates = inputs.qft_circuit(n, seed=seed)
    a = oracle.run(n, gates, x0=x)
    k = np.arange(1 << n)
    expect = np.exp(2j * np.pi * x * k / (1 << n)) / math.sqrt(1 << n)
    np.testing.assert_allclose(a, expect, atol=1e-13)


def test_qft_matches_numpy_fft():
    # QFT with e^{+2 pi i xk/N} / sqrt(N) is N * ifft / sqrt(N) in numpy's convention.
    n = 9
    rng = np.random.default_rng(11)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    got = oracle.run(n, inputs.qft(range(n), swaps=True), state=psi.copy())
    np.testing.assert_allclose(got, np.fft.ifft(psi) * math.sqrt(1 << n), atol=1e-12)


def test_qft_then_inverse_is_identity():
    n = 11
    rng = np.random.default_rng(12)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi /= np.linalg.norm(psi)
    for swaps in (True, False):
        got = oracle.run(n, inputs.qft(range(n), swaps) + inputs.iqft(range(n), swaps), state=psi.copy())
        np.testing.assert_allclose(got, psi, atol=1e-13)


def test_norm_conserved_random_circuit():
    n = 12
    a = oracle.run(n, inputs.random_circuit(n, 20, seed=2))
    assert abs(oracle.norm(a, n) - 1.0) < 1e-13


# ---------------------------------------------------------------------------
# Adders (Sec. V.A, Fig. adder, App. B).
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("ad", [a for a in golden_io.adders() if a["n_ops"]], ids=lambda a: a["name"])
def test_adder_operation_counts_match_paper(ad):
    gates = inputs.adder_circuit(ad["values"], ad["m"])
    assert len(gates) == ad["n_ops"] == inputs.adder_gate_count(ad["values"], ad["m"])


def test_fig_adder_sum_exact():
    ad = golden_io.adders()[0]
    assert ad["values"] == [1365, 682] and ad["m"] == 11
    n = 22
    gates = inputs.adder_circuit(ad["values"], ad["m"])
    # 22 loading operations, then QFT (66), 66 controlled phases, inverse QFT (66)
    assert len(gates) == 22 + 66 + 66 + 66
    p = oracle.probs(oracle.run(n, gates), n)
    want = inputs.adder_expected_index(ad["values"], ad["m"])
    assert want == 1365 | (2047 << 11)
    assert int(np.argmax(p)) == want and abs(p[want] - 1.0) < 1e-12


@pytest.mark.parametrize("values,m", [([3, 5, 9], 4), ([15, 15, 15], 4), ([7, 9, 19, 35, 65], 3), ([100, 200], 8)])
def test_small_adders_exact(values, m):
    n = len(values) * m
    p = oracle.probs(oracle.run(n, inputs.adder_circuit(values, m)), n)
    want = inputs.adder_expected_index(values, m)
    assert int(np.argmax(p)) == want and abs(p[want] - 1.0) < 1e-12


# ---------------------------------------------------------------------------
# Shor (Sec. V.B, Table Shortab, Eq. Shor7).
# ---------------------------------------------------------------------------
def test_shor_table_L24():
    t = golden_io.shor_table()
    X, L, G, y = t["X"], t["L"], t["G"], t["y"]
    f = inputs.shor_initial_support(X, G, y)
    # the period printed in the table is the order of y mod G
    assert np.flatnonzero(f[1:] == 1)[0] + 1 == t["r"]
    a = np.zeros(1 << L, dtype=np.complex128)
    a[np.arange(1 << X) + (f << X)] = 2.0 ** (-X / 2)
    oracle.run(L, inputs.qft(range(X), swaps=True), state=a)
    q = oracle.qubit_probs(a, L)
    np.testing.assert_allclose(q[:X], t["Q"], atol=5e-4 + 1e-12)


def shor_closed_form_Q(X, r):
    """<Q_i>, i < X, after the QFT of the x-register of the Eq. Shor2 state,
    from the period alone: the x in each residue class mod r (s or s + 1 of
    them, s = floor(2^X / r)) add up to a geometric sum, so
    p_k = [(r - t) |S_s(k)|^2 + t |S_(s+1)(k)|^2] / 2^(2X),  t = 2^X mod r,
    S_m(k) = sum_{j<m} exp(2 pi i k r j / 2^X); then <Q_i> = sum_k p_k bit_i(k)."""
    N = 1 << X
    k = np.arange(N, dtype=np.float64)
    theta = 2 * np.pi * ((k * r) % N) / N
    s, t = N // r, N % r

    def S2(m):
        num = np.abs(np.sin(theta * m / 2)) ** 2
        den = np.abs(np.sin(theta / 2)) ** 2
        out = np.full(N, float(m * m))
        nz = den > 1e-300
        out[nz] = num[nz] / den[nz]
        return out

    p = ((r - t) * S2(s) + t * S2(s + 1)) / float(N) ** 2
    ki = np.arange(N, dtype=np.int64)
    return np.array([p[(ki >> i) & 1 == 1].sum() for i in range(X)]), p.sum()


@pytest.mark.parametrize("name", ["shortab_L24.txt", "shortab_L33_G1961.txt", "shortab_L33_G2047.txt"])
def test_shor_table_columns_closed_form(name):
    # The L = 33 columns are beyond the oracle's host memory; their printed
    # values are pinned here by the closed form (and the L = 24 column, which
    # the oracle reproduces above, by both).
    t = golden_io.shor_table(name)
    X, G, y, r = t["X"], t["G"], t["y"], t["r"]
    assert pow(y, r, G) == 1 and all(pow(y, d, G) != 1 for d in range(1, r))  # r = order of y mod G
    assert (1 << (t["L"] - X)) >= G
    Q, tot = shor_closed_form_Q(X, r)
    assert abs(tot - 1) < 1e-9
    np.testing.assert_allclose(Q, t["Q"], atol=5e-4 + 1e-9)


# ---------------------------------------------------------------------------
# Qubit interchange layouts (Tables onequbittab, twoqubittab).
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("table", ["onequbittab.txt", "twoqubittab.txt"])
def test_permute_bits_tables(table):
    steps, body = golden_io.layout_table_steps(table)
    for sig, seq in steps.items():
        a = np.arange(16, dtype=np.complex128)
        for pairs in seq:
            a = oracle.permute_bits(a, 4, pairs)
        for phys, logical in body[sig].items():
            assert a[phys].real == logical, (table, sig, phys)


def test_permute_bits_k_pairs_is_composition_of_single_swaps():
    # K disjoint pairs at once = the K single interchanges one after another.
    rng = np.random.default_rng(3)
    n = 10
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    pairs = [(0, 7), (2, 9), (3, 5)]
    one = oracle.permute_bits(psi, n, pairs)
    seq = psi
    for p in pairs:
        seq = oracle.permute_bits(seq, n, [p])
    np.testing.assert_array_equal(one, seq)
    # and it moves exactly the amplitudes whose paired bits differ: (2^K-1)/2^K
    moved = np.count_nonzero(one != psi)
    assert moved == (1 << n) - (1 << n) // 8


# ---------------------------------------------------------------------------
# Reductions and sampling.
# ---------------------------------------------------------------------------
def test_probs_and_qubit_probs_brute_force():
    rng = np.random.default_rng(4)
    n = 9
    a = oracle.run(n, inputs.random_circuit(n, 6, seed=9))
    p = oracle.probs(a, n)
    np.testing.assert_allclose(p, np.abs(a) ** 2, rtol=1e-15, atol=0)
    idx = np.arange(1 << n)
    qp = oracle.qubit_probs(a, n)
    for q in range(n):
        assert abs(qp[q] - p[(idx >> q) & 1 == 1].sum()) < 1e-14
    # basis state: <Q_q> are the bits of x
    x = 0b101100101
    b = oracle.basis(n, x)
    assert list(oracle.qubit_probs(b, n)) == [float((x >> q) & 1) for q in range(n)]
    assert oracle.norm(b, n) == 1.0


def test_sample_inverse_cdf():
    a = np.sqrt(np.array([0.1, 0.2, 0.3, 0.4])).astype(np.complex128)
    u = np.array([0.0, 0.05, 0.0999, 0.1001, 0.29, 0.31, 0.59, 0.61, 0.999])
    got = oracle.sample(a, 2, u)
    assert list(got) == [0, 0, 0, 1, 1, 2, 2, 3, 3]
    # unnormalised state samples its normalised distribution
    got2 = oracle.sample(2 * a, 2, u)
    assert list(got2) == list(got)
