"""The serving autotuner's choice rule on the CPU, with the batching loop
replaced by a fake that returns fixed statistics per (slots, passes) pair:
the lowest p99 among the pairs within 5% of the best throughput."""

import pytest


class _Stats:
    def __init__(self, tp, p99):
        self.tp, self.p99 = tp, p99

    def summary(self):
        return {"requests": 10, "problems_per_s": self.tp, "p50_ms": self.p99 / 2, "p99_ms": self.p99}


def test_tune_serving_rule(monkeypatch):
    from paper_2303_14495_gb300 import autotune, serving
    table = {(16, 1): (100.0, 5.0),    # lowest p99 but too slow
             (16, 4): (980.0, 40.0),
             (32, 1): (990.0, 30.0),   # within 5% of the best, lowest p99 there
             (32, 4): (1000.0, 35.0)}
    calls = []

    def fake(bases, requests, precision, mem_budget, max_slots, passes_per_tick):
        calls.append((max_slots, passes_per_tick))
        return _Stats(*table[(max_slots, passes_per_tick)]), {}

    monkeypatch.setattr(serving, "serve_batched", fake)
    pick, rows = autotune.tune_serving([None], [], slots=(16, 32), passes=(1, 4))
    assert sorted(calls) == sorted(table)
    assert pick == {"max_slots": 32, "passes_per_tick": 1}
    assert len(rows) == 4 and all("max_slots" in r and "passes_per_tick" in r for r in rows)


def test_tune_serving_tie_prefers_throughput(monkeypatch):
    from paper_2303_14495_gb300 import autotune, serving
    table = {(8, 2): (950.0, 30.0), (8, 4): (1000.0, 30.0)}
    monkeypatch.setattr(serving, "serve_batched",
                        lambda bases, requests, precision, mem_budget, max_slots, passes_per_tick:
                        (_Stats(*table[(max_slots, passes_per_tick)]), {}))
    pick, _ = autotune.tune_serving([None], [], slots=(8,), passes=(2, 4))
    assert pick == {"max_slots": 8, "passes_per_tick": 4}
