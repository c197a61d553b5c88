"""bench.py's host-side bookkeeping on the CPU, with the device calls faked:
the interchange sweep's algorithmic bytes, fractions and its error reporting
(a failing K is reported in place of its figure and the run goes on)."""
import types

import pytest


class _Event:
    def __init__(self, enable_timing=False):
        pass

    def record(self, stream):
        pass

    def elapsed_time(self, other):
        return 40.0  # ms for the 4 timed passes: 10 ms per pass


class _State:
    freed = []

    def __init__(self, n, dt):
        self.dt = dt

    def permute_bits(self, lo, hi):
        assert len(lo) == len(hi) and not set(lo) & set(hi)
        if self.dt == "c128" and len(lo) == 4:
            raise RuntimeError("refused")

    def free(self):
        _State.freed.append(self.dt)


def test_interchange_sweeps_bookkeeping(monkeypatch):
    import torch
    import bench
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    monkeypatch.setattr(torch.cuda, "empty_cache", lambda: None)
    monkeypatch.setattr(bench, "peaks", lambda: (1000.0, "test"))
    _State.freed = []
    out = bench.qubit_interchange_sweeps(types.SimpleNamespace(State=_State), n=30)
    # K = 1 counts half the state (the amplitudes whose two bits differ), K >= 2 all of it
    half64 = 2 * 8 * 0.5 * (1 << 30) / 10e-3 / 1e9
    assert out["c64"]["1"]["GBs"] == pytest.approx(half64, rel=1e-3)
    assert out["c64"]["2"]["GBs"] == pytest.approx(2 * half64, rel=1e-3)
    assert out["c128"]["2"]["GBs"] == pytest.approx(4 * half64, rel=1e-3)
    assert out["c64"]["2"]["frac"] == pytest.approx(out["c64"]["2"]["GBs"] / 1000.0, rel=1e-2)
    assert out["c128"]["4"] == {"error": "refused"}
    assert _State.freed == ["c64", "c128"]


# ---------------------------------------------------------------- config lines
class _Plan:
    def __init__(self, st, gates, mode=1, tile_bits=0, fuse_k=0):
        self.st, self.gates, self.mode, self.fuse_k = st, gates, mode, fuse_k
        _Dev.planned.append((st.n, st.dt, mode, tile_bits, fuse_k))

    def run(self):
        _Dev.runs += 1

    def stats(self):
        S = 8 if self.st.dt == "c64" else 16
        passes = 7
        return {"passes": passes, "sweeps": len(self.gates), "fuse_k": self.fuse_k, "mode": self.mode,
                "candidates": 3 if self.mode == _Dev.MODE_AUTO else 0,
                "alg_bytes": passes * 2.0 * S * (1 << self.st.n)}

    def free(self):
        pass


class _CState:
    def __init__(self, n, dt):
        self.n, self.dt = n, dt

    def plan(self, gates, **kw):
        return _Plan(self, gates, **kw)

    def set_basis(self, x):
        pass

    def run(self, gates, fuse_k=0):
        pass

    def qubit_probs(self):
        return [float((_Dev.expect >> i) & 1) for i in range(self.n)]

    def free(self):
        pass


class _Batch:
    def __init__(self, states, x0s, gates):
        self.ng = sum(len(g) for g in gates)

    def run(self):
        pass

    def sync(self):
        pass

    def stats(self):
        return {"gates": self.ng, "graph": True, "fused": 2, "alg_bytes": 5e9}

    def free(self):
        pass


class _Dev:
    MODE_PERGATE, MODE_FUSED, MODE_AUTO = 0, 1, 2
    State, Batch = _CState, _Batch
    planned, runs, expect = [], 0, 0


def test_config_lines_bookkeeping(monkeypatch):
    """Every configuration line is there, with gates/s and the HBM fraction
    from the plan's algorithmic bytes over the event-timed median, the
    fused-over-per-gate ratio taken from the faster complex64 fused path, the
    adder's output index read from <Q_q>, and the autotuned lines planned with
    the autotuning mode."""
    import torch
    import bench
    import inputs
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    monkeypatch.setattr(torch.cuda, "empty_cache", lambda: None)
    monkeypatch.setattr(bench, "peaks", lambda: (1000.0, "test"))
    # every run 40 ms, except the per-gate complex128 arm (400 ms) and the
    # 6-qubit complex64 arm (20 ms)
    def fake_runs(fn, reps):
        for _ in range(reps):
            fn()
        last = _Dev.planned[-1]
        ms = 400.0 if last[2] == _Dev.MODE_PERGATE and last[1] == "c128" and last[0] == 30 else \
            20.0 if last[4] == 6 else 40.0
        return [ms] * reps
    monkeypatch.setattr(bench, "_event_runs", fake_runs)
    a, b = inputs.adder_pairs(15, 8, seed=3)[0]
    _Dev.expect = inputs.adder_expected_index([a, b], 15)
    _Dev.planned = []
    args = types.SimpleNamespace(steps=4)
    main = {"gates_per_s": 1.0}
    res = bench.config_lines(_Dev, main, args)
    c2 = res["random30"]
    assert c2["c128_autotuned"] is main
    for k in ("c64_autotuned", "c64_tile_passes", "c64_tensor_cores_k5", "c64_tensor_cores_k6",
              "c128_tensor_cores_k5", "c128_tile_passes", "c128_pergate"):
        assert c2[k]["ms_per_run"] > 0, k
    assert c2["c64_tensor_cores_k5"]["gates_per_s"] == pytest.approx(1800 / 0.040)
    assert c2["c64_tensor_cores_k6"]["hbm_frac"] == pytest.approx(7 * 2 * 8 * 2 ** 30 / 0.020 / 1e9 / 1000.0)
    assert c2["fused_c64_over_pergate_c128"] == pytest.approx(400.0 / 20.0)
    assert c2["c64_tensor_cores_k6"]["path"] == "planner (fused 6-qubit blocks on the tensor cores, bf16x3)"
    assert c2["c128_pergate"]["path"] == "one sweep per gate"
    ad = res["adder2x15_c64"]
    assert set(ad) == {"autotuned", "tile_passes", "tensor_cores_k5", "tensor_cores_k6", "output_index_exact"}
    assert ad["output_index_exact"] is True
    assert (30, "c64", _Dev.MODE_AUTO, 0, 0) in _Dev.planned
    assert res["batch512_c64"]["cuda_graph"] is True
    bms = res["batch512_c64"]["ms_per_run"]
    assert res["batch512_c64"]["eff_hbm_frac"] == pytest.approx(5e9 / (bms / 1e3) / 1e9 / 1000.0)
    assert set(res["random34_c64"]) == {"tensor_cores_k5", "tensor_cores_k6"}
    assert "random34_c64" in res and "qft10_c128" in res


def test_resize_workload():
    """--n: the random circuit and the Hadamard replay at n qubits, the seeded
    adder as two registers of n / 2 qubits (its gate list on exactly n
    qubits, its operation count the adder's N_O); the paper's fixed adders,
    the batch and an odd adder size refuse it."""
    import numpy as np

    import bench
    import inputs

    w, name = bench.resize_workload("random30_c128", 24)
    assert (w["n"], name) == (24, "random30_c128_n24") and "24 qubits" in w["text"]
    assert bench.WORKLOADS["random30_c128"]["n"] == 30  # the table itself is left alone
    w, name = bench.resize_workload("hadamard30_c128", 27)
    assert w["n"] == 27 and len(bench.workload_gates(w)[0]) == 27
    w, name = bench.resize_workload("adder30_c64", 26)
    assert (w["n"], w["m"], name) == (26, 13, "adder30_c64_n26")
    assert "two 13-qubit registers" in w["text"] and "26 qubits" in w["text"]
    gates, x0 = bench.workload_gates(w)
    used = {q for g in gates for q in tuple(g.targets) + tuple(g.controls)}
    values = [int(v) for v in np.random.default_rng(w["seed"]).integers(0, 1 << 13, 2)]
    assert x0 == 0 and max(used) == 25 and len(gates) == inputs.adder_gate_count(values, 13)
    for bad, n in (("adder3x11_c128", 30), ("batch512_c64", 20), ("adder30_c64", 25)):
        with pytest.raises(ValueError):
            bench.resize_workload(bad, n)
