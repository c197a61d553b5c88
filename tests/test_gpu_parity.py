"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (max-abs amplitude error): 1e-12 for complex128, 2e-5 for
complex64.  Basis-state outcomes (adder sums, argmax) must match exactly.
"""
import math

import numpy as np
import pytest

import inputs
import oracle
from inputs import Gate

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 2e-5}
DTYPES = ["c128", "c64"]


@pytest.fixture(scope="module")
def q():
    import torch
    torch.cuda.set_device(0)
    import paper_quant_ph_0608239_gb300 as qq
    qq._capi.load()
    return qq


def rand_state(n, seed):
    rng = np.random.default_rng(seed)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return psi / np.linalg.norm(psi)


def g1(kind, t, ctrl=(), params=()):
    return Gate(kind, (int(t),), tuple(int(c) for c in ctrl), tuple(params))


def run_gpu(q, n, dt, gates, psi=None, x0=0, mode=None, tile_bits=0):
    st = q.State(n, dt)
    if psi is not None:
        st.set_state(psi)
    else:
        st.set_basis(x0)
    st.run(gates, mode=q.MODE_FUSED if mode is None else mode, tile_bits=tile_bits)
    out = st.get_state()
    st.free()
    return out


def err(a, b):
    return float(np.max(np.abs(np.asarray(a, dtype=np.complex128) - b)))


PARAMS = {"R": (0.7,), "V": (2 * math.pi / 8,), "SU2": (0.5, -0.1, 0.7, math.sqrt(1 - 0.25 - 0.01 - 0.49))}


# ---------------------------------------------------------------- state init
@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("n", [1, 5, 13])
def test_basis_state_and_norm(q, dt, n):
    st = q.State(n, dt)
    x = (1 << n) - 3 if n > 2 else 1
    st.set_basis(x)
    a = st.get_state()
    expect = np.zeros(1 << n)
    expect[x] = 1
    assert np.array_equal(a, expect.astype(a.dtype))
    assert st.norm() == 1.0
    assert list(st.qubit_probs()) == [float((x >> b) & 1) for b in range(n)]
    st.free()


# ------------------------------------------------------- single-qubit sweeps
@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("mode", ["pergate", "fused"])
def test_every_kind_every_target(q, dt, mode):
    n = 12
    psi = rand_state(n, 1)
    m = q.MODE_PERGATE if mode == "pergate" else q.MODE_FUSED
    for kind in ["H", "X", "Y", "XB", "YB", "NOT", "R", "V", "SU2"]:
        for t in range(n):
            g = g1(kind, t, (), PARAMS.get(kind, ()))
            ref = oracle.run(n, [g], state=psi.copy())
            got = run_gpu(q, n, dt, [g], psi=psi, mode=m, tile_bits=8)
            assert err(got, ref) < TOL[dt], (kind, t)


@pytest.mark.parametrize("dt", DTYPES)
def test_apply_1q_and_ctrl_entry_points(q, dt):
    n = 11
    rng = np.random.default_rng(2)
    psi = rand_state(n, 2)
    st = q.State(n, dt)
    st.set_state(psi)
    ref = psi.copy()
    for _ in range(30):
        Z = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
        U, _ = np.linalg.qr(Z)
        t = int(rng.integers(n))
        others = [b for b in range(n) if b != t]
        ctrl = [int(c) for c in rng.choice(others, size=int(rng.integers(0, 4)), replace=False)]
        mask = sum(1 << c for c in ctrl)
        if ctrl:
            st.apply_ctrl(mask, t, U)
        else:
            st.apply_1q(t, U)
        oracle.run(n, [g1("U", t, ctrl, tuple(x for z in U.reshape(-1) for x in (z.real, z.imag)))], state=ref)
    assert err(st.get_state(), ref) < TOL[dt]
    st.free()


# ---------------------------------------------------- controlled, Toffoli, swap
def controlled_gates(rng, n, count):
    out = []
    kinds = ["NOT", "R", "V", "SU2", "H", "SWAP"]
    for _ in range(count):
        k = kinds[int(rng.integers(len(kinds)))]
        qs = [int(x) for x in rng.permutation(n)]
        nc = int(rng.integers(1, 4))
        if k == "SWAP":
            out.append(Gate("SWAP", (qs[0], qs[1]), tuple(qs[2:2 + nc - 1]), ()))
            continue
        out.append(g1(k, qs[0], qs[1:1 + nc], PARAMS.get(k, ())))
    return out


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("mode", ["pergate", "fused"])
def test_controlled_gates(q, dt, mode):
    n = 13
    rng = np.random.default_rng(3)
    gates = controlled_gates(rng, n, 60)
    psi = rand_state(n, 3)
    ref = oracle.run(n, gates, state=psi.copy())
    m = q.MODE_PERGATE if mode == "pergate" else q.MODE_FUSED
    assert err(run_gpu(q, n, dt, gates, psi=psi, mode=m, tile_bits=9), ref) < TOL[dt]


def test_worked_examples_on_gpu(q):
    # Eqs. CNOT2, Toffoli: pure data movement, bit-exact in both precisions.
    for dt in DTYPES:
        a = (np.arange(1, 9) * (1 + 0.5j)).astype(np.complex128)
        got = run_gpu(q, 3, dt, [g1("NOT", 2, (0, 1))], psi=a, mode=q.MODE_PERGATE)
        assert np.array_equal(got, a[[0, 1, 2, 7, 4, 5, 6, 3]].astype(got.dtype))
        b = a[:4].copy()
        got = run_gpu(q, 2, dt, [g1("NOT", 1, (0,))], psi=b, mode=q.MODE_FUSED)
        assert np.array_equal(got, b[[0, 3, 2, 1]].astype(got.dtype))


# ------------------------------------------------------- circuits, both paths
@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("n,depth,tile", [(4, 6, 0), (9, 8, 6), (14, 10, 0), (14, 10, 8), (18, 6, 0), (20, 4, 10)])
def test_random_circuit_both_paths(q, dt, n, depth, tile):
    gates = inputs.random_circuit(n, depth, seed=100 + n)
    rng = np.random.default_rng(n)
    gates += controlled_gates(rng, n, 10)
    x0 = inputs.random_basis(n, seed=n)
    ref = oracle.run(n, gates, x0=x0)
    for m in (q.MODE_PERGATE, q.MODE_FUSED):
        got = run_gpu(q, n, dt, gates, x0=x0, mode=m, tile_bits=tile)
        e = err(got, ref)
        assert e < TOL[dt], (m, e)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("n", [1, 2, 3])
def test_tiny_registers(q, dt, n):
    # registers of one to three qubits: the tile is the whole register
    rng = np.random.default_rng(40 + n)
    gates = inputs.random_circuit(n, 8, seed=40 + n)
    if n >= 2:
        gates += [g for g in controlled_gates(rng, n, 12) if len(g.controls) + len(g.targets) <= n]
    psi = rand_state(n, 41 + n)
    ref = oracle.run(n, gates, state=psi.copy())
    for m in (q.MODE_PERGATE, q.MODE_FUSED):
        assert err(run_gpu(q, n, dt, gates, psi=psi, mode=m), ref) < TOL[dt]


@pytest.mark.parametrize("dt", DTYPES)
def test_long_pass_many_ops(q, dt):
    # one tile holds the whole 10-qubit register, so all 300 gates land in one
    # pass: several staging chunks of ops, controls, SWAP gates
    n = 10
    rng = np.random.default_rng(77)
    kinds = ["H", "R", "SU2", "NOT", "V", "X", "YB"]
    gates = []
    for i in range(300):
        k = kinds[int(rng.integers(len(kinds)))]
        qs = [int(x) for x in rng.permutation(n)]
        nc = int(rng.integers(0, 3))
        if i % 37 == 0:
            gates.append(Gate("SWAP", (qs[0], qs[1]), (), ()))
            continue
        gates.append(g1(k, qs[0], qs[1:1 + nc], PARAMS.get(k, ())))
    psi = rand_state(n, 78)
    ref = oracle.run(n, gates, state=psi.copy())
    st = q.State(n, dt)
    st.set_state(psi)
    plan = st.plan(gates)
    assert plan.stats()["passes"] == 1
    plan.run()
    assert err(st.get_state(), ref) < TOL[dt] * 4
    plan.free()
    st.free()


@pytest.mark.parametrize("absorber", [True, False])
def test_c128_tile_pass_factor_folding(q, absorber):
    # complex128 tile passes fold the factors of uncontrolled Hadamard gates
    # and of phases on bits outside the tile into one op per pass: passes with
    # such an op (dense SU(2) gates present) and without it (only H, phases and
    # CNOTs), phases with controls inside and outside the tile
    n, tile = 16, 8
    rng = np.random.default_rng(2024 + absorber)
    gates = []
    for _layer in range(6):
        for t in range(n):
            k = int(rng.integers(3))
            if k == 1:
                gates.append(g1("R", t, (), (float(rng.uniform(0, 2 * math.pi)),)))
            elif k == 2 and absorber:
                gates.append(g1("SU2", t, (), PARAMS["SU2"]))
            else:
                gates.append(g1("H", t))
        for _ in range(6):
            a, b = (int(x) for x in rng.choice(n, 2, replace=False))
            gates.append(g1("R", a, (b,), (float(rng.uniform(0, 2 * math.pi)),)))
        p = [int(x) for x in rng.permutation(n)]
        for i in range(0, n, 2):
            gates.append(g1("NOT", p[i + 1], (p[i],)))
    psi = rand_state(n, 7 + absorber)
    ref = oracle.run(n, gates, state=psi.copy())
    got = run_gpu(q, n, "c128", gates, psi=psi, tile_bits=tile)
    assert err(got, ref) < TOL["c128"]
    # the same through a plan run twice (the state returns to IEEE doubles
    # after every run)
    st = q.State(n, "c128")
    plan = st.plan(gates, tile_bits=tile)
    for _ in range(2):
        st.set_state(psi)
        plan.run()
        assert err(st.get_state(), ref) < TOL["c128"]
    plan.free()
    st.free()


@pytest.mark.parametrize("dt", DTYPES)
def test_autotuned_plan(q, dt):
    # QSIM_MODE_AUTO: each of the first runs uses another candidate (tile size,
    # fusion width); every run applies the whole circuit, so every run must
    # match the oracle, and afterwards the fastest candidate is in use
    n = 18
    gates = inputs.random_circuit(n, 8, seed=91)
    x0 = inputs.random_basis(n, seed=91)
    ref = oracle.run(n, gates, x0=x0)
    st = q.State(n, dt)
    plan = st.plan(gates, mode=q.MODE_AUTO)
    s0 = plan.stats()
    assert s0["candidates"] >= 2 and s0["chosen"] == -1
    tol = TOL[dt] * (1 if dt == "c128" else 2)  # fused 3xTF32 blocks round a little more
    for _ in range(s0["candidates"] + 1):
        st.set_basis(x0)
        plan.run()
        assert err(st.get_state(), ref) < tol
    s1 = plan.stats()
    assert 0 <= s1["chosen"] < s1["candidates"]
    ms = [c["ms"] for c in s1["autotune"]]
    assert all(m > 0 for m in ms) and ms[s1["chosen"]] == min(ms)
    if dt == "c64":
        assert any(c["fuse_k"] for c in s1["autotune"])  # tensor-core widths are candidates
    plan.free()
    st.free()


def test_autotune_drops_fusion_narrower_than_a_gate(q):
    # a NOT with four controls acts on 5 qubits: the k = 4 candidate cannot
    # hold it and is left out, k = 5 stays; a plain fused plan that is too
    # narrow is rejected before any work
    n = 16
    gates = inputs.random_circuit(n, 4, seed=17)
    gates.insert(40, Gate("NOT", (3,), (0, 7, 11, 15), ()))
    x0 = inputs.random_basis(n, seed=17)
    ref = oracle.run(n, gates, x0=x0)
    st = q.State(n, "c64")
    plan = st.plan(gates, mode=q.MODE_AUTO)
    ks = [c["fuse_k"] for c in plan.stats()["autotune"]]
    assert 5 in ks and 4 not in ks, ks
    for _ in range(len(ks) + 1):
        st.set_basis(x0)
        plan.run()
        assert err(st.get_state(), ref) < 2 * TOL["c64"]
    plan.free()
    st.set_basis(x0)
    with pytest.raises(q.QsimError) as e:
        st.run(gates, fuse_k=4)
    assert e.value.status == q.QSIM_EINVAL
    assert err(st.get_state(), oracle.basis(n, x0)) == 0.0  # nothing applied
    st.free()


def test_qft_config_c128_and_closed_form(q):
    n = 10
    x, gates = inputs.qft_circuit(n, seed=1)
    assert len(gates) == 55 + 5
    ref = oracle.run(n, gates, x0=x)
    got = run_gpu(q, n, "c128", gates, x0=x)
    assert err(got, ref) < 1e-12
    k = np.arange(1 << n)
    assert err(got, np.exp(2j * np.pi * x * k / (1 << n)) / math.sqrt(1 << n)) < 1e-12


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("values,m", [([1365, 682], 11), ([45, 17, 60], 6), ([7, 9, 19, 35, 65], 3)])
def test_adder_exact(q, dt, values, m):
    n = len(values) * m
    gates = inputs.adder_circuit(values, m)
    want = inputs.adder_expected_index(values, m)
    st = q.State(n, dt)
    st.run(gates)
    qp = st.qubit_probs()
    got_idx = sum(1 << b for b in range(n) if qp[b] > 0.5)
    assert got_idx == want
    assert np.max(np.minimum(qp, 1 - qp)) < TOL[dt]
    p = st.probs()
    assert int(np.argmax(p)) == want and p[want] > 1 - 10 * TOL[dt]
    st.free()


# ---------------------------------------------- register-blocked tile kernel
# Default tiles (T = 12, or 13 for complex64) on n >= T run the register
# kernel: lane bits 0..4 by warp shuffles, register bits in registers, warp
# bits through shared-memory phases; complex128 in double-float.
REG_TILES = [("c128", 12), ("c64", 12), ("c64", 13)]


@pytest.mark.parametrize("dt,tile", REG_TILES)
def test_register_tile_every_kind_every_target(q, dt, tile):
    n = 15
    psi = rand_state(n, 4)
    for kind in ["H", "X", "Y", "XB", "YB", "NOT", "R", "V", "SU2"]:
        for t in range(n):
            g = g1(kind, t, (), PARAMS.get(kind, ()))
            ref = oracle.run(n, [g], state=psi.copy())
            got = run_gpu(q, n, dt, [g], psi=psi, tile_bits=tile)
            assert err(got, ref) < TOL[dt], (kind, t)


@pytest.mark.parametrize("dt,tile", REG_TILES)
@pytest.mark.parametrize("n", [13, 16, 21])
def test_register_tile_circuits_with_controls_and_swaps(q, dt, tile, n):
    rng = np.random.default_rng(40 + n)
    gates = inputs.random_circuit(n, 5, seed=n)
    gates += controlled_gates(rng, n, 40)
    # uncontrolled quantum SWAPs (applied as store permutations) between layers
    for _ in range(6):
        a, b = (int(x) for x in rng.permutation(n)[:2])
        gates.insert(int(rng.integers(len(gates))), Gate("SWAP", (a, b), (), ()))
    gates += inputs.random_circuit(n, 3, seed=n + 1)
    x0 = inputs.random_basis(n, seed=n)
    ref = oracle.run(n, gates, x0=x0)
    got = run_gpu(q, n, dt, gates, x0=x0, tile_bits=tile)
    assert err(got, ref) < TOL[dt]


@pytest.mark.parametrize("dt,tile", REG_TILES)
def test_register_tile_qft_and_inverse(q, dt, tile):
    n = 17
    x, gates = inputs.qft_circuit(n, seed=9)
    ref = oracle.run(n, gates, x0=x)
    got = run_gpu(q, n, dt, gates, x0=x, tile_bits=tile)
    assert err(got, ref) < TOL[dt]
    back = run_gpu(q, n, dt, gates + inputs.iqft(range(n), swaps=True), x0=x, tile_bits=tile)
    expect = np.zeros(1 << n)
    expect[x] = 1
    assert err(back, expect) < TOL[dt]


# ------------------------------------------------------------ interchanges
@pytest.mark.parametrize("table", ["onequbittab.txt", "twoqubittab.txt"])
def test_permute_bits_matches_paper_tables(q, table):
    import golden_io
    steps, body = golden_io.layout_table_steps(table)
    for dt in DTYPES:
        for sig, seq in steps.items():
            st = q.State(4, dt)
            st.set_state(np.arange(16).astype(np.complex128))
            for pairs in seq:
                st.permute_bits([p[0] for p in pairs], [p[1] for p in pairs])
            a = st.get_state()
            for phys, logical in body[sig].items():
                assert a[phys].real == logical
            st.free()


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("pairs", [[(0, 13)], [(2, 9), (4, 15)], [(0, 10), (1, 11), (3, 16)], [(5, 6), (7, 8)]])
def test_permute_bits_vs_oracle(q, dt, pairs):
    n = 17
    psi = rand_state(n, 7).astype(np.complex128)
    st = q.State(n, dt)
    st.set_state(psi)
    st.permute_bits([p[0] for p in pairs], [p[1] for p in pairs])
    expect = oracle.permute_bits(psi.astype(np.complex64).astype(np.complex128) if dt == "c64" else psi, n, pairs)
    got = st.get_state()
    assert np.array_equal(got, expect.astype(got.dtype))  # pure data movement: bit-exact
    st.free()


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("kind,K", [("cross", 2), ("cross", 3), ("cross", 6), ("any", 4), ("any", 5), ("low", 2)])
def test_permute_bits_random_pairs_many_tiles(q, dt, kind, K):
    """The interchange pass at 22 qubits (1024 to 4096 tiles, several laps of
    each CTA's four-stage ring): pairs from the low bits to high ones at random
    places ("cross"), anywhere ("any") or all among the lowest 11 bits ("low",
    the slow in-run layout).  Bit-exact against the oracle's permutation."""
    n = 22
    rng = np.random.default_rng(100 * K + len(kind))
    if kind == "cross":
        lo = rng.choice(np.arange(0, 8), K, replace=False)
        hi = rng.choice(np.arange(12, n), K, replace=False)
    elif kind == "low":
        b = rng.choice(np.arange(0, 11), 2 * K, replace=False)
        lo, hi = b[:K], b[K:]
    else:
        b = rng.choice(np.arange(n), 2 * K, replace=False)
        lo, hi = b[:K], b[K:]
    pairs = [(int(a), int(c)) for a, c in zip(lo, hi)]
    psi = rand_state(n, 11).astype(np.complex128)
    if dt == "c64":
        psi = psi.astype(np.complex64).astype(np.complex128)
    st = q.State(n, dt)
    st.set_state(psi)
    st.permute_bits([p[0] for p in pairs], [p[1] for p in pairs])
    got = st.get_state()
    assert np.array_equal(got, oracle.permute_bits(psi, n, pairs).astype(got.dtype)), pairs
    st.permute_bits([p[0] for p in pairs], [p[1] for p in pairs])  # an involution: back to the start
    assert np.array_equal(st.get_state(), psi.astype(got.dtype))
    st.free()


@pytest.mark.parametrize("dt", DTYPES)
def test_swap_qubits_keeps_logical_state(q, dt):
    n = 15
    gates = inputs.random_circuit(n, 6, seed=5)
    ref = oracle.run(n, gates)
    st = q.State(n, dt)
    st.run(gates[: len(gates) // 2])
    st.swap_qubits([0, 3], [12, 14])
    assert st.layout()[0] == 12 and st.layout()[12] == 0 and st.layout()[3] == 14
    st.swap_qubits([5], [13])
    st.run(gates[len(gates) // 2:])
    assert err(st.get_state(), ref) < TOL[dt]
    assert abs(st.norm() - 1) < 10 * TOL[dt]
    np.testing.assert_allclose(st.qubit_probs(), oracle.qubit_probs(ref, n), atol=10 * TOL[dt])
    np.testing.assert_allclose(st.probs(), oracle.probs(ref, n), atol=10 * TOL[dt])
    st.free()


# ----------------------------------------------------------------- fusion
@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_apply_fused_dense(q, dt, k):
    n = 14
    rng = np.random.default_rng(20 + k)
    qs = [int(x) for x in rng.permutation(n)[:k]]
    Z = rng.standard_normal((1 << k, 1 << k)) + 1j * rng.standard_normal((1 << k, 1 << k))
    U, _ = np.linalg.qr(Z)
    psi = rand_state(n, 9)
    ref = oracle.apply_dense(psi.copy(), n, qs, U)
    st = q.State(n, dt)
    st.set_state(psi)
    st.apply_fused(qs, U)
    assert err(st.get_state(), ref) < TOL[dt] * (4 if dt == "c64" else 1)
    st.free()


# ---------------------------------------- fused gates on the tensor cores
@pytest.mark.parametrize("k", [4, 5])
@pytest.mark.parametrize("n,where", [(12, "low"), (16, "high"), (16, "mixed"), (20, "mixed"), (22, "high")])
def test_fused_tensor_cores_c64(q, k, n, where):
    rng = np.random.default_rng(70 + 10 * k + n)
    if where == "low":
        qs = list(rng.permutation(k))
    elif where == "high":
        qs = [int(x) for x in rng.permutation(np.arange(n - k, n))]
    else:
        qs = [int(x) for x in rng.permutation(n)[:k]]
    Z = rng.standard_normal((1 << k, 1 << k)) + 1j * rng.standard_normal((1 << k, 1 << k))
    U, _ = np.linalg.qr(Z)
    psi = rand_state(n, 90 + n)
    ref = oracle.apply_dense(psi.astype(np.complex64).astype(np.complex128), n, qs, U)
    st = q.State(n, "c64")
    st.set_state(psi)
    st.profile(True)
    st.apply_fused(qs, U)
    prof = st.profile_read()
    assert "fused_tensor_core" in prof, prof  # the tcgen05 kernel ran
    e = err(st.get_state(), ref)
    # 3xTF32 keeps about 2^-21 relative per product; amplitudes are <= 1
    assert e < 2e-5, e
    st.free()


@pytest.mark.parametrize("k", [4, 5])
@pytest.mark.parametrize("n", [13, 18])
def test_fused_blocks_circuit_c64(q, k, n):
    gates = inputs.random_circuit(n, 6, seed=200 + n)
    rng = np.random.default_rng(n)
    gates += [g for g in controlled_gates(rng, n, 12) if len(g.controls) + len(g.targets) <= k]
    x0 = inputs.random_basis(n, seed=n + 1)
    ref = oracle.run(n, gates, x0=x0)
    st = q.State(n, "c64")
    st.set_basis(x0)
    st.profile(True)
    st.run(gates, fuse_k=k)
    prof = st.profile_read()
    assert "fused_tensor_core" in prof and "tile_pass" not in prof
    e = err(st.get_state(), ref)
    assert e < 2e-5, e
    st.free()


# ------------------------- complex128 fused gates on the tensor cores (digits)
@pytest.mark.parametrize("n,where", [(12, "low"), (12, "mixed"), (16, "high"), (16, "mixed"), (20, "mixed"),
                                     (22, "high"), (22, "low")])
def test_fused_tensor_cores_c128(q, n, where):
    k = 5
    rng = np.random.default_rng(170 + n + len(where))
    if where == "low":
        qs = list(rng.permutation(k))
    elif where == "high":
        qs = [int(x) for x in rng.permutation(np.arange(n - k, n))]
    else:
        qs = [int(x) for x in rng.permutation(n)[:k]]
    Z = rng.standard_normal((1 << k, 1 << k)) + 1j * rng.standard_normal((1 << k, 1 << k))
    U, _ = np.linalg.qr(Z)
    psi = rand_state(n, 190 + n)
    ref = oracle.apply_dense(psi.copy(), n, qs, U)
    st = q.State(n, "c128")
    st.set_state(psi)
    st.profile(True)
    st.apply_fused(qs, U)
    prof = st.profile_read()
    assert "fused_tc_digits" in prof, prof  # the tcgen05 digit-slice kernel ran
    e = err(st.get_state(), ref)
    # the digit slices keep about 2^-47 of a group's largest magnitude
    assert e < 1e-14, e
    st.free()


def test_fused_tensor_cores_c128_wide_range_and_zeros(q):
    # groups with one large amplitude and the rest 2^-60 smaller, all-zero
    # groups and exact zeros: every output against the oracle to 1e-12
    # relative to its group's largest magnitude
    n, k = 13, 5
    rng = np.random.default_rng(5)
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[::7] = rng.standard_normal(psi[::7].size) * 2.0 ** -60
    psi[::97] = rng.standard_normal(psi[::97].size) + 1j * rng.standard_normal(psi[::97].size)
    psi[1 << 12:(1 << 12) + 512] = 0.0
    psi /= np.linalg.norm(psi)
    qs = [0, 3, 7, 9, 12]
    Z = rng.standard_normal((32, 32)) + 1j * rng.standard_normal((32, 32))
    U, _ = np.linalg.qr(Z)
    ref = oracle.apply_dense(psi.copy(), n, qs, U)
    st = q.State(n, "c128")
    st.set_state(psi)
    st.profile(True)
    st.apply_fused(qs, U)
    assert "fused_tc_digits" in st.profile_read()
    got = st.get_state()
    assert err(got, ref) < 1e-14
    zero = ref == 0
    assert np.all(got[zero] == 0)
    st.free()


def test_fused_c128_non_unitary_falls_back(q):
    # an entry outside (-2, 2) is beyond the digit scheme: the gate runs on
    # the CUDA cores in FP64 instead, with the same result
    n, k = 12, 5
    rng = np.random.default_rng(9)
    U = rng.standard_normal((32, 32)) + 1j * rng.standard_normal((32, 32))
    U[3, 4] = 3.5
    psi = rand_state(n, 4)
    ref = oracle.apply_dense(psi.copy(), n, list(range(k)), U)
    st = q.State(n, "c128")
    st.set_state(psi)
    st.profile(True)
    st.apply_fused(list(range(k)), U)
    prof = st.profile_read()
    assert "dense_cuda_core" in prof and "fused_tc_digits" not in prof, prof
    assert err(st.get_state(), ref) < 1e-12 * float(np.max(np.abs(ref)))
    st.free()


@pytest.mark.parametrize("n", [12, 13, 18, 21])
def test_fused_blocks_circuit_c128_tensor_cores(q, n):
    gates = inputs.random_circuit(n, 8, seed=400 + n)
    rng = np.random.default_rng(n + 40)
    gates += [g for g in controlled_gates(rng, n, 12) if len(g.controls) + len(g.targets) <= 5]
    x0 = inputs.random_basis(n, seed=n + 3)
    ref = oracle.run(n, gates, x0=x0)
    st = q.State(n, "c128")
    st.set_basis(x0)
    st.profile(True)
    plan = st.plan(gates, fuse_k=5)
    plan.run()
    prof = st.profile_read()
    assert "fused_tc_digits" in prof and "tile_pass" not in prof and "dense_cuda_core" not in prof, prof
    assert err(st.get_state(), ref) < 1e-12
    assert abs(st.norm() - 1) < 1e-12
    # the one-shot path (gate list in host memory) gives the same state
    st.set_basis(x0)
    st.run(gates, fuse_k=5)
    assert err(st.get_state(), ref) < 1e-12
    plan.free()
    st.free()


@pytest.mark.parametrize("n,where", [(13, "low"), (16, "high"), (16, "mixed"), (20, "mixed"), (22, "high")])
def test_fused_tensor_cores_c64_k6(q, n, where):
    # 6-qubit blocks: bf16 hi/mid/lo slices, six products on the tensor cores
    k = 6
    rng = np.random.default_rng(270 + n + len(where))
    if where == "low":
        qs = list(rng.permutation(k))
    elif where == "high":
        qs = [int(x) for x in rng.permutation(np.arange(n - k, n))]
    else:
        qs = [int(x) for x in rng.permutation(n)[:k]]
    Z = rng.standard_normal((1 << k, 1 << k)) + 1j * rng.standard_normal((1 << k, 1 << k))
    U, _ = np.linalg.qr(Z)
    psi = rand_state(n, 290 + n)
    ref = oracle.apply_dense(psi.astype(np.complex64).astype(np.complex128), n, qs, U)
    st = q.State(n, "c64")
    st.set_state(psi)
    st.profile(True)
    st.apply_fused(qs, U)
    prof = st.profile_read()
    assert "fused_tc_bf16x3" in prof, prof
    e = err(st.get_state(), ref)
    # bf16x3 keeps about 2^-24 relative per product and FP32 sums of 128 terms
    assert e < 2e-5, e
    st.free()


@pytest.mark.parametrize("n", [13, 18])
def test_fused_blocks_circuit_c64_k6(q, n):
    gates = inputs.random_circuit(n, 6, seed=600 + n)
    rng = np.random.default_rng(n + 60)
    gates += [g for g in controlled_gates(rng, n, 12) if len(g.controls) + len(g.targets) <= 6]
    x0 = inputs.random_basis(n, seed=n + 7)
    ref = oracle.run(n, gates, x0=x0)
    st = q.State(n, "c64")
    st.set_basis(x0)
    st.profile(True)
    st.run(gates, fuse_k=6)
    prof = st.profile_read()
    assert "fused_tc_bf16x3" in prof and "tile_pass" not in prof and "dense_cuda_core" not in prof, prof
    e = err(st.get_state(), ref)
    assert e < 2e-5, e
    st.free()


@pytest.mark.parametrize("dt,k", [("c128", 3), ("c128", 6), ("c64", 3)])
def test_fused_blocks_cuda_cores(q, dt, k):
    # fusion widths and precisions the tensor-core kernel does not take run
    # as dense blocks on the CUDA cores (FP64 for complex128)
    n = 13
    gates = inputs.random_circuit(n, 5, seed=300 + k)
    rng = np.random.default_rng(k)
    gates += [g for g in controlled_gates(rng, n, 10) if len(g.controls) + len(g.targets) <= k]
    x0 = inputs.random_basis(n, seed=k)
    ref = oracle.run(n, gates, x0=x0)
    st = q.State(n, dt)
    st.set_basis(x0)
    st.profile(True)
    plan = st.plan(gates, fuse_k=k)
    assert plan.stats()["fuse_k"] == k
    plan.run()
    prof = st.profile_read()
    assert "dense_cuda_core" in prof and "tile_pass" not in prof, prof
    assert err(st.get_state(), ref) < TOL[dt]
    # the one-shot path (gate list in host memory) gives the same state
    st.set_basis(x0)
    st.run(gates, fuse_k=k)
    assert err(st.get_state(), ref) < TOL[dt]
    plan.free()
    st.free()


def test_fused_blocks_adder_exact(q):
    values, m = [45, 17], 7
    n = 2 * m
    gates = inputs.adder_circuit(values, m)
    st = q.State(n, "c64")
    st.run(gates, fuse_k=5)
    qp = st.qubit_probs()
    want = inputs.adder_expected_index(values, m)
    assert sum(1 << b for b in range(n) if qp[b] > 0.5) == want
    assert np.max(np.minimum(qp, 1 - qp)) < 1e-4
    st.free()


@pytest.mark.parametrize("k,m", [(4, 7), (5, 7), (6, 10)])
def test_phase_pass_adder(q, k, m):
    """The controlled phases between the adder's registers (Sec. V.A) as one
    phase pass among the tensor-core blocks: the state against the oracle,
    the sum bit-exact, and the pass in the launch profile."""
    values = (37, 98)
    n = 2 * m
    gates = inputs.adder_circuit(values, m)
    st = q.State(n, "c64")
    st.set_basis(0)
    st.profile(True)
    st.run(gates, fuse_k=k)
    prof = st.profile_read()
    assert "phase_pass" in prof, prof
    got = st.get_state()
    ref = oracle.run(n, gates, x0=0)
    assert err(got, ref) < TOL["c64"], err(got, ref)
    assert int(np.argmax(np.abs(got))) == inputs.adder_expected_index(values, m)
    plan = st.plan(gates, fuse_k=k)
    st.set_basis(0)
    plan.run()
    assert err(st.get_state(), ref) < TOL["c64"]  # plans upload the tables themselves
    plan.free()
    st.free()


@pytest.mark.parametrize("m", [7, 11])
def test_phase_pass_adder_c128(q, m):
    """complex128 phase pass (64-bit turns) between the 5-qubit tensor-core
    blocks of the adder (Sec. V.A): the blocks around it hand IEEE doubles
    to it and take them back; within the complex128 tolerance, the sum
    bit-exact."""
    values = (37, 98)
    n = 2 * m
    gates = inputs.adder_circuit(values, m)
    st = q.State(n, "c128")
    st.set_basis(0)
    st.profile(True)
    st.run(gates, fuse_k=5)
    prof = st.profile_read()
    assert "phase_pass" in prof, prof
    got = st.get_state()
    ref = oracle.run(n, gates, x0=0)
    assert err(got, ref) < TOL["c128"], err(got, ref)
    assert int(np.argmax(np.abs(got))) == inputs.adder_expected_index(values, m)
    st.free()


@pytest.mark.parametrize("shape", ["alone", "first", "last"])
@pytest.mark.parametrize("pairs", ["separable", "chunk01"])
def test_phase_pass_c128_ends(q, shape, pairs):
    """complex128 phase pass as the whole plan (IEEE doubles in and out), as
    its first step (IEEE in, double-float out to the blocks) and as its last
    (double-float in, IEEE out), with the factor split into lane and loop
    parts (no gate pairs index bits 0..4 with bits 5..9) and without, on a
    random state, against the oracle."""
    n = 16
    rng = np.random.default_rng(3 * ["alone", "first", "last"].index(shape) + (pairs == "chunk01"))
    phases = []
    while len(phases) < 40:
        a, b = (int(x) for x in rng.choice(n, 2, replace=False))
        if pairs == "separable" and {a // 5, b // 5} == {0, 1}:
            continue
        phases.append(g1("R", a, (b,), (float(rng.uniform(0, 2 * np.pi)),)))
    if pairs == "chunk01":
        phases.append(g1("R", 2, (7,), (0.3,)))
    layer = [g1("H", t) for t in range(n)]
    gates = {"alone": phases, "first": phases + layer, "last": layer + phases}[shape]
    psi = rand_state(n, 5)
    ref = oracle.run(n, gates, state=psi.copy())
    st = q.State(n, "c128")
    st.set_state(psi)
    st.profile(True)
    st.run(gates, fuse_k=5)
    assert "phase_pass" in st.profile_read()
    assert err(st.get_state(), ref) < TOL["c128"], err(st.get_state(), ref)
    st.free()


@pytest.mark.parametrize("n", [12, 13, 22])
def test_phase_pass_random_phases(q, n):
    """A long run of controlled phases on random qubit pairs (every chunk
    pair of the tables), Hadamards around it, on 4-, 5- and 6-qubit block
    plans (complex64) and 5-qubit ones (complex128), against the oracle."""
    rng = np.random.default_rng(n)
    gates = [g1("H", t) for t in range(n)]
    for _ in range(60):
        a, b = (int(x) for x in rng.choice(n, 2, replace=False))
        gates.append(g1("R", a, (b,), (float(rng.uniform(0, 2 * np.pi)),)))
    gates += [g1("R", int(t), (), (float(rng.uniform(0, 2 * np.pi)),)) for t in rng.choice(n, 6, replace=False)]
    gates += [g1("H", t) for t in range(n)]
    ref = oracle.run(n, gates, x0=0)
    for dt, k in (("c64", 4), ("c64", 5), ("c64", 6), ("c128", 5)):
        if (k == 6 and n < 13) or (k < 6 and n < 12):
            continue
        st = q.State(n, dt)
        st.set_basis(0)
        st.profile(True)
        st.run(gates, fuse_k=k)
        assert "phase_pass" in st.profile_read()
        assert err(st.get_state(), ref) < TOL[dt], (n, dt, k, err(st.get_state(), ref))
        st.free()


# ------------------------------------------------------------- reductions
@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("n", [3, 9, 10, 13, 16, 21])
def test_reductions(q, dt, n):
    psi = rand_state(n, 11 + n)
    st = q.State(n, dt)
    st.set_state(psi)
    a = psi.astype(np.complex64).astype(np.complex128) if dt == "c64" else psi
    tol = 1e-13 if dt == "c128" else 1e-6
    assert abs(st.norm() - oracle.norm(a, n)) < tol
    np.testing.assert_allclose(st.qubit_probs(), oracle.qubit_probs(a, n), atol=tol)
    np.testing.assert_allclose(st.probs(), oracle.probs(a, n), atol=tol * 1e-3, rtol=1e-6 if dt == "c64" else 1e-12)
    st.free()


@pytest.mark.parametrize("n", [13, 15, 20])
def test_bit_marginals_c128_wide_magnitudes(q, n):
    """complex128 per-bit marginals (the double-float reduction for n >= 13)
    on a state that is not normalised: exact zeros, magnitudes far below the
    float range (1e-40, 1e-300), and chunks holding magnitudes >= 2 (the FP64
    branch), against the oracle's FP64 sums, relative to the total."""
    rng = np.random.default_rng(40 + n)
    psi = rand_state(n, 90 + n)
    D = 1 << n
    psi[rng.choice(D, D // 4, replace=False)] = 0.0
    psi[rng.choice(D, 64, replace=False)] *= 1e-40
    psi[rng.choice(D, 64, replace=False)] = 1e-300 * (1 + 1j)
    psi[rng.choice(D, 5, replace=False)] = 3.0 - 2.5j
    st = q.State(n, "c128")
    st.set_state(psi)
    got = st.qubit_probs()
    ref = oracle.qubit_probs(psi, n)
    tot = float(np.sum(np.abs(psi) ** 2))
    assert np.max(np.abs(got - ref)) < 1e-13 * tot, (np.max(np.abs(got - ref)), tot)
    st.free()


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("n", [1, 3, 8, 14])
def test_sampling_matches_oracle(q, dt, n):
    psi = rand_state(n, 30 + n) * (1.0 + np.arange(1 << n) / (1 << n))  # uneven weights
    psi /= np.linalg.norm(psi)
    a = psi.astype(np.complex64).astype(np.complex128) if dt == "c64" else psi
    u = np.random.default_rng(5).random(1001)
    st = q.State(n, dt)
    st.set_state(psi)
    got = st.sample(u)
    ref = oracle.sample(a, n, u)
    # samples may differ only where u * norm lies within rounding of a CDF step
    cdf = np.cumsum(oracle.probs(a, n))
    tot = cdf[-1]
    near = np.min(np.abs(cdf[None, :] - (u * tot)[:, None]), axis=1) < 1e-9
    assert np.all((got == ref) | near)
    assert np.mean(got == ref) > 0.99
    st.free()


@pytest.mark.parametrize("dt", DTYPES)
def test_sampling_distribution_chi2(q, dt):
    # the sampled histogram against the oracle's probabilities (Pearson chi^2
    # over cells with at least 5 expected counts; fixed seeds, so the outcome
    # is deterministic)
    scipy_stats = pytest.importorskip("scipy.stats")
    n, S = 10, 200000
    psi = rand_state(n, 61) * (1.0 + 3.0 * np.arange(1 << n) / (1 << n))
    psi /= np.linalg.norm(psi)
    st = q.State(n, dt)
    st.set_state(psi)
    got = st.sample(np.random.default_rng(62).random(S))
    st.free()
    p = oracle.probs(psi, n)
    counts = np.bincount(got, minlength=1 << n)
    exp = S * p / p.sum()
    keep = exp >= 5
    chi2 = float(np.sum((counts[keep] - exp[keep]) ** 2 / exp[keep]))
    dof = int(keep.sum()) - 1
    assert scipy_stats.chi2.sf(chi2, dof) > 1e-4, (chi2, dof)
    assert counts[~keep].sum() <= max(20, 3 * exp[~keep].sum())


# ------------------------------------- complex64: relative error and fidelity
def rel_and_fidelity(got, ref):
    got = np.asarray(got, dtype=np.complex128)
    rel = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    fid = float(abs(np.vdot(ref, got)) ** 2 / (np.vdot(ref, ref).real * np.vdot(got, got).real))
    return rel, fid


@pytest.mark.parametrize("n,depth,seed", [(20, 20, 7), (24, 20, 4)])
def test_c64_relative_error_and_fidelity(q, n, depth, seed):
    # At n qubits a random state's amplitudes are ~2^(-n/2), so the absolute
    # 2e-5 bound says little; the relative error max|da| / max|a_ref| and the
    # fidelity |<ref|got>|^2 are checked as well.  (24, 20, 4) is the 34-qubit
    # configuration's generator (depth 20, seed 4) at 24 qubits, where the
    # oracle still runs.  Bound: FP32 rounds each amplitude by <= 2^-23
    # relative per gate; over G gates the error walks as ~2^-23 sqrt(G) times a
    # few roundings per update (G = 600-720: ~1e-5); 1e-4 leaves a margin and
    # still fails any wrong gate.
    gates = inputs.random_circuit(n, depth, seed=seed)
    x0 = inputs.random_basis(n, seed=seed)
    ref = oracle.run(n, gates, x0=x0)
    got = run_gpu(q, n, "c64", gates, x0=x0)
    assert err(got, ref) < TOL["c64"]
    rel, fid = rel_and_fidelity(got, ref)
    print("n=%d gates=%d  max-abs %.3g  relative %.3g  1-fidelity %.3g" % (n, len(gates), err(got, ref), rel, 1 - fid))
    assert rel < 1e-4, rel
    assert 1 - fid < 1e-8, fid


# ------------------------------------------------------------- edge cases
def test_invalid_arguments_change_nothing(q):
    n = 6
    psi = rand_state(n, 1)
    st = q.State(n, "c128")
    st.set_state(psi)
    bad = [
        lambda: st.apply_1q(n, np.eye(2)),
        lambda: st.apply_ctrl(1 << 2, 2, np.eye(2)),
        lambda: st.apply_ctrl(1 << n, 1, np.eye(2)),
        lambda: st.apply_fused([1, 1], np.eye(4)),
        lambda: st.apply_fused([0, 1, 2, 3, 4, 5, 6][:7], np.eye(128)),
        lambda: st.swap_qubits([0, 1, 2, 3], [4, 5, 0, 1]),
        lambda: st.swap_qubits([0], [0]),
        lambda: st.run([g1("H", 0), g1("H", 9)]),
        lambda: st.run([g1("NOT", 1, (1,))]),
        lambda: st.run([Gate("SWAP", (2, 2), (), ())]),
        lambda: st.run([g1("R", 0, (), (float("nan"),))]),
        lambda: st.set_basis(1 << n),
        lambda: st.sample(np.array([1.5])),
    ]
    for f in bad:
        with pytest.raises(q.QsimError) as ei:
            f()
        assert ei.value.status == q.QSIM_EINVAL
    assert np.array_equal(st.get_state(), psi)
    st.free()


def test_empty_circuit_and_one_qubit(q):
    st = q.State(1, "c64")
    st.run([])
    assert np.array_equal(st.get_state(), np.array([1, 0], dtype=np.complex64))
    st.run([g1("H", 0)])
    assert err(st.get_state(), np.array([1, 1]) / math.sqrt(2)) < 1e-7
    st.free()


# ------------------------------------------- full-size checks (any-size properties)
def _inverse(gates):
    inv = []
    for g in reversed(gates):
        if g.kind == "R":
            inv.append(Gate("R", g.targets, g.controls, (-g.params[0],)))
        elif g.kind == "SU2":
            a, b, c, d = g.params
            inv.append(Gate("SU2", g.targets, g.controls, (a, -b, -c, -d)))
        elif g.kind in ("H", "NOT", "SWAP"):
            inv.append(g)
        else:
            raise ValueError(g.kind)
    return inv


def test_full_size_qft_sampled_amplitudes_c128(q):
    # 30-qubit QFT (480 gates) on a basis state: every amplitude has a closed
    # form, so a sample of 4096 of them is checked one by one (16 GiB state).
    n = 30
    x, gates = inputs.qft_circuit(n, seed=7)
    st = q.State(n, "c128")
    st.set_basis(x)
    st.run(gates)
    import torch
    torch.cuda.synchronize()
    idx = np.random.default_rng(1).integers(0, 1 << n, 4096)
    got = st.tensor[torch.as_tensor(idx, device="cuda")].cpu().numpy()
    expect = np.exp(2j * np.pi * ((x * idx) % (1 << n)) / (1 << n)) / math.sqrt(1 << n)
    assert err(got, expect) < 1e-12
    assert abs(st.norm() - 1) < 1e-12
    st.free()


@pytest.mark.parametrize("n,depth,dt", [(30, 40, "c128"), (30, 40, "c64"), (34, 20, "c64")])
def test_full_size_random_circuit_then_inverse(q, n, depth, dt):
    # The bench circuits at full size: circuit then its inverse must return
    # |x0> exactly (to the dtype's tolerance), and the norm must be conserved.
    gates = inputs.random_circuit(n, depth, seed=2 if n == 30 else 4)
    x0 = inputs.random_basis(n, seed=2)
    st = q.State(n, dt)
    st.set_basis(x0)
    st.run(gates)
    # FP32 rounds every output amplitude with relative error <= ~2^-23 per
    # gate; G gates move the norm by about 2^-23 * sqrt(G) typically and
    # 2^-23 * G at worst (2.1e-4 for G = 1800).  1e-4 sits between the two.
    assert abs(st.norm() - 1) < (1e-12 if dt == "c128" else 1e-4)
    st.run(_inverse(gates))
    import torch
    t = st.tensor
    torch.cuda.synchronize()
    a0 = complex(t[x0].item())
    t[x0] = 0
    # max |a_i| over i != x0, in chunks (no full-size temporaries)
    rest = max(float(t[i:i + (1 << 26)].abs().max().item()) for i in range(0, t.numel(), 1 << 26))
    tol = TOL[dt] * (1 if dt == "c128" else 2.5)
    assert abs(a0 - 1) < tol and rest < tol, (a0, rest)
    st.free()


# ------------------------------------------------ Shor, Table Shortab (L = 24)
@pytest.mark.parametrize("dt", DTYPES)
def test_shor_table_L24_on_gpu(q, dt):
    import golden_io
    t = golden_io.shor_table()
    X, L, G, y = t["X"], t["L"], t["G"], t["y"]
    f = inputs.shor_initial_support(X, G, y)
    a = np.zeros(1 << L, dtype=np.complex128)
    a[np.arange(1 << X) + (f << X)] = 2.0 ** (-X / 2)   # Eq. Shor2
    st = q.State(L, dt)
    st.set_state(a)
    st.run(inputs.qft(range(X), swaps=True))             # QFT on the x-register
    qp = st.qubit_probs()                                # Eq. Shor7
    np.testing.assert_allclose(qp[:X], t["Q"], atol=5e-4 + 1e-12)
    ref = oracle.qubit_probs(oracle.run(L, inputs.qft(range(X), swaps=True), state=a.copy()), L)
    np.testing.assert_allclose(qp, ref, atol=1e-12 if dt == "c128" else 1e-5)
    # the device-written Eq. Shor2 state equals the host-built one exactly
    st.set_shor_state(X, y, G)
    assert np.array_equal(st.get_state(), a.astype(st.get_state().dtype))
    st.free()


# ------------------------------------------------ Shor, Table Shortab (L = 33)
@pytest.mark.parametrize("name,dt", [("shortab_L33_G1961.txt", "c64"), ("shortab_L33_G2047.txt", "c64"),
                                     ("shortab_L33_G2047.txt", "c128")])
def test_shor_table_L33_on_gpu(q, name, dt):
    # 33 qubits: 64 GiB (complex64) / 128 GiB (complex128), beyond the
    # oracle's host memory; checked against the paper's column and against
    # the closed form of the QFT'd Eq. Shor2 state
    import golden_io
    from test_oracle_pins import shor_closed_form_Q
    t = golden_io.shor_table(name)
    X, L, G, y, r = t["X"], t["L"], t["G"], t["y"], t["r"]
    st = q.State(L, dt)
    st.set_shor_state(X, y, G)
    st.run(inputs.qft(range(X), swaps=True))
    qp = st.qubit_probs()
    st.free()
    np.testing.assert_allclose(qp[:X], t["Q"], atol=5e-4 + 1e-9)
    Q, _ = shor_closed_form_Q(X, r)
    np.testing.assert_allclose(qp[:X], Q, atol=1e-10 if dt == "c128" else 5e-5)
    # the f-register: y^x mod G over a whole number of periods and a remainder,
    # <Q_i> for i >= X follow from the values f(x) directly
    f = inputs.shor_initial_support(X, G, y)
    fb = np.array([np.mean((f >> (i - X)) & 1) for i in range(X, L)])
    np.testing.assert_allclose(qp[X:], fb, atol=1e-10 if dt == "c128" else 5e-5)
    st.free()
