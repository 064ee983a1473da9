"""The continuous-batching loop's host logic on the CPU: the binding's
Problem and Batch and the CUDA events are replaced by fakes that count
passes, so admission by slots and memory, retiring and the pipelined and
waiting forms can be checked without a GPU."""

import contextlib
from types import SimpleNamespace

import numpy as np
import pytest


class _FakeEvent:
    recorded = 0

    def record(self, stream=None):
        _FakeEvent.recorded += 1

    def synchronize(self):
        pass


class _FakeProblem:
    live = {}

    @classmethod
    def like(cls, base, K, fid_mask, fid_labels, params, wait=True):
        p = cls()
        p.h = SimpleNamespace(value=id(p))
        p.n, p.K, p.wait = base.n, int(K), wait
        p.labels_in = np.asarray(fid_labels)
        p.passes = 0
        p.ended = None
        cls.live[id(p)] = p
        return p

    def _result(self):
        # a function of the inputs and of the passes made, like a real solve
        return ((self.labels_in + self.passes) % self.K).astype(np.int32)

    def labels(self):
        return self._result()

    def labels_async(self, out, status):
        import torch
        out.copy_(torch.from_numpy(self._result()))
        status[0] = 0
        return out

    def get_u(self):
        return np.full((self.n, self.K), float(self.passes), np.float32)

    def release(self):
        self.ended = "release"

    def close(self):
        self.ended = "close"


class _FakeBatch:
    def __init__(self, max_problems, stream=None):
        self.max_problems = max_problems
        self.members = []
        self.done = []
        self.most = 0

    def add(self, prob, outer, inner):
        assert len(self.members) < self.max_problems
        self.members.append([prob, outer * inner])
        self.most = max(self.most, len(self.members))

    def step(self, passes):
        keep = []
        for m in self.members:
            n = min(passes, m[1])
            m[0].passes += n
            m[1] -= n
            (self.done if m[1] == 0 else keep).append(m[0] if m[1] == 0 else m)
        self.members = keep
        return len(keep)

    def poll(self):
        out, self.done = self.done, []
        return out

    def close(self):
        pass


@pytest.fixture
def fakes(monkeypatch):
    import torch
    from paper_2303_14495_gb300 import binding as B
    _FakeProblem.live = {}
    batches = []

    def make_batch(max_problems, stream=None):
        b = _FakeBatch(max_problems, stream)
        batches.append(b)
        return b

    monkeypatch.setattr(B.Problem, "like", _FakeProblem.like)
    monkeypatch.setattr(B, "Batch", make_batch)
    monkeypatch.setattr(B, "workspace_size_like", lambda base, K, prm: 1000 * int(K))
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "Event", _FakeEvent)
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self: self)
    real_empty, real_zeros = torch.empty, torch.zeros
    monkeypatch.setattr(torch, "empty", lambda *a, pin_memory=False, **k: real_empty(*a, **k))
    monkeypatch.setattr(torch, "zeros", lambda *a, pin_memory=False, **k: real_zeros(*a, **k))
    return batches


def _requests(n_req, seed=0):
    rng = np.random.default_rng(seed)
    reqs = []
    for rid in range(n_req):
        K = int(rng.choice([2, 5, 10]))
        reqs.append(SimpleNamespace(
            rid=rid, arrival=0.0, template=int(rng.integers(0, 2)), K=K,
            fid_mask=(rng.random(50) < 0.2).astype(np.uint8), fid_labels=rng.integers(0, K, 50).astype(np.int32),
            params={"eps": 1.0, "c": 502.0, "eta": 500.0, "precond": 2, "damping": 0.5, "delta0": 1e-6,
                    "power_iters": 150},
            outer=int(rng.integers(1, 6)), inner=int(rng.integers(1, 6))))
    return reqs


@pytest.mark.parametrize("pipelined", [True, False])
def test_every_request_served_with_its_own_passes(fakes, pipelined):
    from paper_2303_14495_gb300 import serving
    bases = [SimpleNamespace(n=50, stream=None), SimpleNamespace(n=50, stream=None)]
    reqs = _requests(40)
    stats, res = serving.serve_batched(bases, reqs, max_slots=6, passes_per_tick=3, keep_results=True,
                                       pipelined=pipelined)
    s = stats.summary()
    assert s["requests"] == len(reqs) and sorted(res) == [r.rid for r in reqs]
    assert fakes[0].most == 6                       # the slot limit was reached, never passed
    for r in reqs:
        lab, u = res[r.rid]
        assert np.all(u == r.outer * r.inner)         # exactly outer x inner passes, no more
        np.testing.assert_array_equal(lab, (r.fid_labels + r.outer * r.inner) % r.K)
    ended = {p.ended for p in _FakeProblem.live.values()}
    assert ended == {"release" if pipelined else "close"}
    assert all(p.wait is (not pipelined) for p in _FakeProblem.live.values())


def test_memory_budget_bounds_the_resident_workspace(fakes):
    from paper_2303_14495_gb300 import serving
    bases = [SimpleNamespace(n=50, stream=None), SimpleNamespace(n=50, stream=None)]
    reqs = _requests(30, seed=3)
    budget = 12000                                   # room for a few problems (1000 x K bytes each)
    stats, _ = serving.serve_batched(bases, reqs, max_slots=64, passes_per_tick=2, mem_budget=budget)
    assert stats.summary()["requests"] == len(reqs)
    assert stats.peak_mem <= budget
    assert stats.admitted_while_busy > 0


def test_pipelined_and_waiting_loops_agree(fakes):
    from paper_2303_14495_gb300 import serving
    bases = [SimpleNamespace(n=50, stream=None), SimpleNamespace(n=50, stream=None)]
    reqs = _requests(25, seed=5)
    _, a = serving.serve_batched(bases, reqs, max_slots=4, passes_per_tick=2, keep_results=True)
    _, b = serving.serve_batched(bases, reqs, max_slots=4, passes_per_tick=2, keep_results=True, pipelined=False)
    for r in reqs:
        np.testing.assert_array_equal(a[r.rid][0], b[r.rid][0])
        np.testing.assert_array_equal(a[r.rid][1], b[r.rid][1])
