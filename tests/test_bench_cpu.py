"""Host arithmetic of the bench's side measurements (no GPU: the creates are
replaced by a fake whose duration is known)."""

from types import SimpleNamespace

import pytest


def test_power_spmv_timing_arithmetic(monkeypatch):
    import torch
    import bench
    from paper_2303_14495_gb300 import binding as B
    clock = [0.0]
    per_iter, fixed = 128e-6, 0.035

    class FakeProblem:
        def __init__(self, row_ptr, col, w, K, fid_mask, fid_labels, prm, device=None):
            # a create costs a fixed part plus its power iterations; the first
            # of each pair is slower (as a cold create would be)
            clock[0] += fixed + per_iter * prm.power_iters + (0.002 if FakeProblem.first else 0.0)
            FakeProblem.first = False

        def close(self):
            pass

    FakeProblem.first = True
    monkeypatch.setattr(B, "Problem", FakeProblem)
    monkeypatch.setattr(bench.time, "perf_counter", lambda: clock[0])
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    wl = SimpleNamespace(row_ptr=None, col=None, w=None, K=4, fid_mask=None, fid_labels=None, n=1000, nnz=16000,
                         params={"eps": 1.0, "c": 502.0, "eta": 500.0, "precond": 2})
    r = bench.power_spmv_timing(wl, {}, "cpu", 6651.7, extra=400, reps=2)
    assert r["us_per_iteration"] == pytest.approx(128.0, rel=1e-9)   # the cold first create is not the best
    assert r["bytes_per_iteration"] == 8 * 16000 + 8 * 1000
    assert r["achieved"] == pytest.approx((8 * 16000 + 8 * 1000) / 128e-6 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6651.7)
    assert r["unit"] == "GB/s" and r["peak"] == 6651.7
