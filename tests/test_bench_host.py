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
