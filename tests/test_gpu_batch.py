"""Batches of independent circuits (qsim_run_batch, qsim_batch_*): one
persistent launch plus the tensor-core lane for circuits of 20 qubits or more;
parity with the oracle, CUDA-graph replay, and the bounded wait between passes
(forced to expire: an error status, not a fault)."""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch
    torch.cuda.set_device(0)
    import paper_quant_ph_0608239_gb300 as qq
    qq._capi.load()
    return qq


def _err(a, b):
    return float(np.max(np.abs(np.asarray(a, dtype=np.complex128) - b)))


def test_batch_matches_oracle(q):
    circs = inputs.batch_circuits(count=40, seed0=500, nmin=3, nmax=17, dmin=1, dmax=14)
    states, x0s, gls = [], [], []
    for i, (n, gates) in enumerate(circs):
        states.append(q.State(n, "c64"))
        x0s.append(inputs.random_basis(n, seed=700 + i))
        gls.append(gates)
    gls[3] = []  # an empty circuit must still leave |x0>
    q.run_batch(states, x0s, gls)
    for st, x0, (n, _), gl in zip(states, x0s, circs, gls):
        ref = oracle.run(n, gl, x0=x0)
        assert _err(st.get_state(), ref) < 2e-5, n
        st.free()


def test_batch_long_passes_with_controls_and_swaps(q):
    # one 12-qubit tile per circuit, so every gate lands in one pass: more ops
    # and phases than a block keeps in shared memory (read from global memory
    # instead), controlled gates and SWAP gates; plus a 14-qubit circuit that
    # needs several passes of the same shape
    from inputs import Gate
    rng = np.random.default_rng(11)
    kinds = ["H", "R", "SU2", "NOT", "V", "X", "YB"]
    params = {"R": (0.7,), "V": (0.785398,), "SU2": (0.5, -0.1, 0.7, (1 - 0.25 - 0.01 - 0.49) ** 0.5)}
    circs = []
    for n in (12, 12, 14):
        gl = []
        for i in range(220):
            qs = [int(x) for x in rng.permutation(n)]
            if i % 29 == 0:
                gl.append(Gate("SWAP", (qs[0], qs[1]), tuple(qs[2:2 + int(rng.integers(0, 2))]), ()))
                continue
            k = kinds[int(rng.integers(len(kinds)))]
            gl.append(Gate(k, (qs[0],), tuple(qs[1:1 + int(rng.integers(0, 3))]), params.get(k, ())))
        circs.append((n, gl))
    states = [q.State(n, "c64") for n, _ in circs]
    x0s = [inputs.random_basis(n, seed=40 + i) for i, (n, _) in enumerate(circs)]
    q.run_batch(states, x0s, [g for _, g in circs])
    for st, x0, (n, gl) in zip(states, x0s, circs):
        ref = oracle.run(n, gl, x0=x0)
        assert _err(st.get_state(), ref) < 4e-5, n
        st.free()


def test_batch_graph_replay_is_repeatable(q):
    circs = inputs.batch_circuits(count=12, seed0=900, nmin=12, nmax=19, dmin=4, dmax=10)
    states = [q.State(n, "c64") for n, _ in circs]
    x0s = [inputs.random_basis(n, seed=i) for i, (n, _) in enumerate(circs)]
    b = q.Batch(states, x0s, [g for _, g in circs])
    stats = b.stats()
    assert stats["circuits"] == 12 and stats["items"] >= stats["passes"] >= 12
    assert stats["graph"], "the persistent launch was not captured in a CUDA graph"
    first = None
    for rep in range(3):
        b.run()
        b.sync()
        got = [st.get_state() for st in states]
        if first is None:
            first = got
        else:
            for a, c in zip(first, got):
                assert np.array_equal(a, c)
    for st, x0, (n, g) in zip(states, x0s, circs):
        assert _err(first[states.index(st)], oracle.run(n, g, x0=x0)) < 2e-5
    b.free()
    for st in states:
        st.free()


def test_batch_wait_budget_expiry_is_reported(q):
    # 20-qubit circuits kept in the persistent launch (fuse_k = -1) need many
    # passes of 256 tiles; with a 1 microsecond budget the waits between
    # passes must expire.  The call returns QSIM_ETIMEOUT, the device stays
    # usable, and a normal run afterwards is correct.
    circs = inputs.batch_circuits(count=4, seed0=50, nmin=20, nmax=20, dmin=12, dmax=12)
    states = [q.State(n, "c64") for n, _ in circs]
    x0s = [0] * len(states)
    with pytest.raises(q.QsimError) as ei:
        q.run_batch(states, x0s, [g for _, g in circs], wait_budget_us=1, fuse_k=-1)
    assert ei.value.status == q.QSIM_ETIMEOUT
    q.run_batch(states, x0s, [g for _, g in circs])
    n, g = circs[0]
    assert _err(states[0].get_state(), oracle.run(n, g, x0=0)) < 2e-5
    for st in states:
        st.free()


def test_batch_tensor_core_lane(q):
    """Circuits of 20 qubits or more run as 6-qubit tensor-core blocks after
    the persistent launch (the others in it), in one captured graph: every
    state against the oracle, twice in a row; the same with 5-qubit blocks
    (fuse_k = 5) and with every circuit kept in the persistent launch
    (fuse_k = -1)."""
    circs = (inputs.batch_circuits(count=3, seed0=70, nmin=12, nmax=16, dmin=6, dmax=12) +
             inputs.batch_circuits(count=3, seed0=80, nmin=20, nmax=21, dmin=8, dmax=14))
    states = [q.State(n, "c64") for n, _ in circs]
    x0s = [inputs.random_basis(n, seed=90 + i) for i, (n, _) in enumerate(circs)]
    b = q.Batch(states, x0s, [g for _, g in circs])
    st = b.stats()
    assert st["fused"] == sum(1 for n, _ in circs if n >= 20) == 3
    assert st["graph"]
    refs = [oracle.run(n, g, x0=x0) for (n, g), x0 in zip(circs, x0s)]
    for rep in range(2):
        b.run()
        b.sync()
        for s_, ref, (n, _) in zip(states, refs, circs):
            assert _err(s_.get_state(), ref) < 2e-5, (rep, n)
    b.free()
    q.run_batch(states, x0s, [g for _, g in circs], fuse_k=5)  # 5-qubit blocks (3xTF32) on the lane
    for s_, ref, (n, _) in zip(states, refs, circs):
        assert _err(s_.get_state(), ref) < 2e-5, n
    q.run_batch(states, x0s, [g for _, g in circs], fuse_k=-1)
    for s_, ref, (n, _) in zip(states, refs, circs):
        assert _err(s_.get_state(), ref) < 2e-5, n
        s_.free()


def test_batch_config_512_sampled(q):
    # the batch workload at full size: 512 circuits, n ~ U{12..24}, depth ~
    # U{10..60}; every norm is conserved and a sample of the smaller circuits
    # matches the oracle amplitude by amplitude
    circs = inputs.batch_circuits()
    states = [q.State(n, "c64") for n, _ in circs]
    x0s = [inputs.random_basis(n, seed=3000 + i) for i, (n, _) in enumerate(circs)]
    b = q.Batch(states, x0s, [g for _, g in circs])
    assert b.stats()["graph"], "the persistent launch was not captured in a CUDA graph"
    b.run()
    b.sync()
    for st, (n, g) in zip(states, circs):
        assert abs(st.norm() - 1) < 1e-4
    picked = [i for i, (n, _) in enumerate(circs) if n <= 15][:6]
    picked += [i for i, (n, _) in enumerate(circs) if n == 20][:2]  # the tensor-core lane
    for i in picked:
        n, g = circs[i]
        assert _err(states[i].get_state(), oracle.run(n, g, x0=x0s[i])) < 2e-5
    b.free()
    for st in states:
        st.free()
