"""GPU parity at the sizes of the benchmark configurations, on the paths the
planner's autotuner actually picks there (tile passes and tensor-core blocks).

* 30-qubit random circuit (depth 40, seed 2; the headline configuration): the
  first 8 layers (360 gates) through every candidate of an autotuned plan, in
  complex128 and complex64, element by element against the CPU oracle at 30
  qubits.  Unlike a circuit followed by its inverse, this catches a kernel
  that applies U^T or conj(U).
* 34-qubit generator (depth 20, seed 4) on its 24-qubit slice: every candidate
  of the autotuned complex64 plan against the oracle (max-abs, relative error,
  fidelity).
* 34 qubits (128 GiB complex64) on the tensor-core blocks: sampled amplitudes
  of a QFT against the closed form, and the random circuit followed by its
  inverse.
* Register adder of two 15-qubit registers (Sec. V.A, Fig. adder), 8 seeded
  pairs, on the tensor-core blocks: bit-exact output index.
* The paper's own adder runs (App. B): 3-11QBA at L = 33 (complex128) gives
  292 + 585 + 1170 = 2047 and 2-17QBA at L = 34 (complex64) gives
  26214 + 104857 = 131071, read bit-exact from <Q_q>.
"""
import math

import numpy as np
import pytest

import inputs
import oracle
from inputs import Gate

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 2e-5}
CHUNK = 1 << 24


@pytest.fixture(scope="module")
def q():
    import torch
    torch.cuda.set_device(0)
    import paper_quant_ph_0608239_gb300 as qq
    qq._capi.load()
    return qq


@pytest.fixture(autouse=True)
def _release_cached_memory():
    yield
    import torch
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def compare(got, ref):
    """max |got - ref|, max |ref| and |<ref|got>|^2 / (|ref|^2 |got|^2), in
    chunks (no full-size temporaries)."""
    err = amax = 0.0
    dot = 0j
    nr = ng = 0.0
    for i in range(0, ref.size, CHUNK):
        g = got[i:i + CHUNK].astype(np.complex128)
        r = ref[i:i + CHUNK]
        err = max(err, float(np.max(np.abs(g - r))))
        amax = max(amax, float(np.max(np.abs(r))))
        dot += np.vdot(r, g)
        nr += float(np.vdot(r, r).real)
        ng += float(np.vdot(g, g).real)
    return err, err / amax, abs(dot) ** 2 / (nr * ng)


def run_candidates(q, st, plan, x0, check):
    """Run an autotuned plan once per candidate (each run applies the whole
    circuit with the next candidate) and check the state after every run."""
    stats = plan.stats()
    seen = []
    for i in range(max(1, stats["candidates"])):
        st.set_basis(x0)
        st.profile(True)
        plan.run()
        prof = st.profile_read()
        st.profile(False)
        c = stats["autotune"][i] if stats["candidates"] else {"tile_bits": stats["tile_bits"],
                                                              "fuse_k": stats["fuse_k"]}
        check(c, prof)
        seen.append(c)
    return seen


# ------------------------------------ 30 qubits, depth 40, seed 2: a prefix
@pytest.fixture(scope="module")
def c2_prefix():
    n, layers = 30, 8
    gates = inputs.random_circuit(n, 40, seed=2)[: layers * (n + n // 2)]
    x0 = inputs.random_basis(n, seed=2)
    ref = oracle.run(n, gates, x0=x0)  # 16 GiB of host memory, ~1 min on 16 threads
    return n, gates, x0, ref


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_c2_prefix_elementwise_every_autotune_candidate(q, c2_prefix, dt):
    n, gates, x0, ref = c2_prefix
    st = q.State(n, dt)
    plan = st.plan(gates, mode=q.MODE_AUTO)

    def check(c, prof):
        if c["fuse_k"]:
            assert "fused_tensor_core" in prof or "fused_tc_digits" in prof or "fused_tc_bf16x3" in prof, prof
        else:
            assert "tile_pass" in prof, prof
        e, rel, fid = compare(st.get_state(), ref)
        print("%s %s: max-abs %.3g relative %.3g 1-fidelity %.3g" % (dt, c, e, rel, 1 - fid))
        assert e < TOL[dt], (c, e)
        if dt == "c64":
            assert rel < 1e-4, (c, rel)
            assert 1 - fid < 1e-8, (c, fid)
        else:
            assert abs(st.norm() - 1) < 1e-12

    seen = run_candidates(q, st, plan, x0, check)
    # the tensor-core widths are among the candidates
    assert ({4, 5, 6} if dt == "c64" else {5}) <= {c["fuse_k"] for c in seen}, seen
    plan.free()
    st.free()


# --------------------------------- the 34-qubit generator at 24 qubits
def test_c4_slice_every_autotune_candidate(q):
    n = 24
    gates = inputs.random_circuit(n, 20, seed=4)
    x0 = inputs.random_basis(n, seed=4)
    ref = oracle.run(n, gates, x0=x0)
    st = q.State(n, "c64")
    plan = st.plan(gates, mode=q.MODE_AUTO)

    def check(c, prof):
        e, rel, fid = compare(st.get_state(), ref)
        print("%s: max-abs %.3g relative %.3g 1-fidelity %.3g" % (c, e, rel, 1 - fid))
        assert e < TOL["c64"] and rel < 1e-4 and 1 - fid < 1e-8, (c, e, rel, fid)
        if c["fuse_k"] in (4, 5):
            assert "fused_tensor_core" in prof and "tile_pass" not in prof, prof
        if c["fuse_k"] == 6:
            assert "fused_tc_bf16x3" in prof and "tile_pass" not in prof, prof

    seen = run_candidates(q, st, plan, x0, check)
    assert {4, 5, 6} <= {c["fuse_k"] for c in seen}
    plan.free()
    st.free()


# ----------------------------------- 34 qubits on the tensor-core blocks
FAMILY = {5: "fused_tensor_core", 6: "fused_tc_bf16x3"}


@pytest.mark.parametrize("k", [5, 6])
def test_34q_qft_tensor_cores_sampled_amplitudes(q, k):
    # QFT|x> has a closed form at every index; the fused blocks of the QFT
    # network are not symmetric, so a transposed block would show here
    import torch
    n = 34
    x, gates = inputs.qft_circuit(n, seed=11)
    st = q.State(n, "c64")
    st.set_basis(x)
    st.profile(True)
    st.run(gates, fuse_k=k)
    prof = st.profile_read()
    assert FAMILY[k] in prof, prof
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.integers(0, 1 << n, 8192), [0, 1, (1 << n) - 1, 1 << 32, (1 << 32) - 1]])
    got = st.tensor[torch.as_tensor(idx, device="cuda")].cpu().numpy().astype(np.complex128)
    expect = np.exp(2j * np.pi * ((x * idx) % (1 << n)) / (1 << n)) / math.sqrt(1 << n)
    rel = float(np.max(np.abs(got - expect))) / (2.0 ** (-n / 2))
    print("34-qubit QFT, %d-qubit tensor-core blocks: relative error %.3g" % (k, rel))
    assert rel < 1e-4, rel
    assert abs(st.norm() - 1) < 1e-4
    st.free()


def _inverse(gates):
    inv = []
    for g in reversed(gates):
        if g.kind == "R":
            inv.append(Gate("R", g.targets, g.controls, (-g.params[0],)))
        elif g.kind == "SU2":
            a, b, c, d = g.params
            inv.append(Gate("SU2", g.targets, g.controls, (a, -b, -c, -d)))
        else:
            assert g.kind in ("H", "NOT", "SWAP")
            inv.append(g)
    return inv


@pytest.mark.parametrize("k", [5, 6])
def test_34q_random_circuit_tensor_cores_then_inverse(q, k):
    import torch
    n = 34
    gates = inputs.random_circuit(n, 20, seed=4)
    x0 = inputs.random_basis(n, seed=4)
    st = q.State(n, "c64")
    st.set_basis(x0)
    st.profile(True)
    st.run(gates, fuse_k=k)
    assert abs(st.norm() - 1) < 1e-4
    st.run(_inverse(gates), fuse_k=k)
    prof = st.profile_read()
    assert FAMILY[k] in prof and "tile_pass" not in prof, prof
    t = st.tensor
    torch.cuda.synchronize()
    a0 = complex(t[x0].item())
    t[x0] = 0
    rest = max(float(t[i:i + (1 << 26)].abs().max().item()) for i in range(0, t.numel(), 1 << 26))
    assert abs(a0 - 1) < 5e-5 and rest < 5e-5, (a0, rest)
    st.free()


# ------------------------------------------ adder of two 15-qubit registers
def _outcome(qp):
    return sum(1 << b for b in range(qp.size) if qp[b] > 0.5), float(np.max(np.minimum(qp, 1 - qp)))


@pytest.mark.parametrize("k", [5, 6])
def test_adder_2x15_eight_pairs_tensor_cores(q, k):
    m = 15
    st = q.State(2 * m, "c64")
    for a, b in inputs.adder_pairs(m, 8, seed=3):
        gates = inputs.adder_circuit([a, b], m)
        st.set_basis(0)
        st.profile(True)
        st.run(gates, fuse_k=k)
        prof = st.profile_read()
        assert ("fused_tensor_core" if k < 6 else "fused_tc_bf16x3") in prof and "tile_pass" not in prof, prof
        got, spread = _outcome(st.qubit_probs())
        assert got == inputs.adder_expected_index([a, b], m), (a, b, got)
        assert spread < 1e-4, (a, b, spread)
    st.free()


# ------------------------------------------------- the paper's own adders
@pytest.mark.parametrize("values,m,dt,fuse_k", [((292, 585, 1170), 11, "c128", 0),
                                                ((26214, 104857), 17, "c64", 5)])
def test_paper_adders_app_b(q, values, m, dt, fuse_k):
    n = len(values) * m
    gates = inputs.adder_circuit(list(values), m)
    assert len(gates) == {11: 286, 17: 493}[m]  # N_O of App. B
    st = q.State(n, dt)
    st.run(gates, fuse_k=fuse_k)
    got, spread = _outcome(st.qubit_probs())
    want = inputs.adder_expected_index(list(values), m)
    assert got == want and (want >> (n - m)) == {11: 2047, 17: 131071}[m], (got, want)
    assert spread < (1e-10 if dt == "c128" else 1e-4), spread
    st.free()
