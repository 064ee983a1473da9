"""Continuous-batching serving loop over the C interface.

Graphs are prepared once (``prepare``: one base problem per graph holding
the renumbered sliced-ELL operator and its lambda_max estimate) and stay
resident.  Requests (graph, K, fidelity, parameters, outer/inner counts,
arrival time) are admitted while the device-memory budget and the slot count
allow: each admitted request gets its own workspace (PyTorch-owned) for its
per-problem state, is created on the graph's shared operator
(pdca_create_like) and joins the batch.  Every tick advances all resident
problems by a few passes in shared launches (pdca_batch_step); finished
problems are polled, their labels read, their memory released, and waiting
requests take the freed slots while the others keep running.  The graph and
the iterate of a problem stay resident on the device from admission to
completion.

``serve_sequential`` is the comparison: one problem at a time (FP32 by
default), pdca_solve per request in arrival order, on the same prepared
operators.
"""

from __future__ import annotations

import time
from typing import Dict, List

import numpy as np

from . import binding as B


def _params(req, precision):
    p = dict(req.params)
    return B.make_params(eps=p["eps"], c=p["c"], eta=p["eta"], precond=p["precond"], damping=p["damping"],
                         delta0=p["delta0"], power_iters=p["power_iters"], precision=precision)


class Stats:
    def __init__(self, latencies: Dict[int, float], makespan: float, peak_mem: int, admitted_while_busy: int):
        self.latencies = latencies
        self.makespan = makespan
        self.peak_mem = peak_mem
        self.admitted_while_busy = admitted_while_busy

    def summary(self) -> dict:
        lat = np.array(sorted(self.latencies.values()))
        return {"requests": int(lat.size), "problems_per_s": float(lat.size / self.makespan),
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3), "makespan_s": float(self.makespan),
                "peak_workspace_bytes": int(self.peak_mem),
                "admitted_while_others_ran": int(self.admitted_while_busy)}


def prepare(pool, precision: int, stream):
    """One base problem per graph (operator prepared once, kept resident)."""
    import torch
    bases = []
    with torch.cuda.stream(stream):
        for t in pool:
            prm = B.make_params(eps=1.0, c=502.0, eta=500.0, precond=B.PDCA_RICHARDSON, precision=precision)
            bases.append(B.Problem(t.row_ptr, t.col, t.w, 1, np.zeros(t.n, np.uint8), np.zeros(t.n, np.int32),
                                   prm, stream=stream))
    torch.cuda.synchronize()
    return bases


def serve_batched(bases, requests, precision: int = B.PDCA_MIXED_BF16W_FP16U, mem_budget: int = 64 << 30,
                  max_slots: int = 64, passes_per_tick: int = 4, keep_results: bool = False,
                  time_scale: float = 1.0):
    """Continuous batching on prepared operators (``bases`` of the matching
    precision family).  Returns (Stats, {rid: (labels, u)} if keep_results)."""
    import torch
    stream = bases[0].stream
    batch = B.Batch(max_problems=max_slots, stream=stream)
    pending = sorted(requests, key=lambda r: r.arrival)
    active = {}                       # handle value -> (request, problem, ws bytes)
    used = peak = busy_admits = 0
    lat: Dict[int, float] = {}
    results = {}
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        while pending or active:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival * time_scale <= now and len(active) < max_slots:
                req = pending[0]
                base = bases[req.template]
                prm = _params(req, precision)
                ws = B.workspace_size_like(base, req.K, prm)
                if used + ws > mem_budget and active:
                    break
                prob = B.Problem.like(base, req.K, req.fid_mask, req.fid_labels, prm)
                batch.add(prob, req.outer, req.inner)
                busy_admits += 1 if active else 0
                active[prob.h.value] = (req, prob, ws)
                used += ws
                peak = max(peak, used)
                pending.pop(0)
            if not active:
                wait = pending[0].arrival * time_scale - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
                continue
            batch.step(passes_per_tick)
            for prob in batch.poll():
                req, p, ws = active.pop(prob.h.value)
                lab = prob.labels()               # synchronises the serving stream
                lat[req.rid] = time.perf_counter() - t0 - req.arrival * time_scale
                if keep_results:
                    results[req.rid] = (lab, prob.get_u())
                prob.close()
                del prob, p
                used -= ws
    makespan = time.perf_counter() - t0
    batch.close()
    return Stats(lat, makespan, peak, busy_admits), results


def serve_sequential(bases, requests, precision: int = B.PDCA_FP32, keep_results: bool = False,
                     time_scale: float = 1.0):
    """One problem at a time in arrival order: create on the prepared
    operator, pdca_solve, labels."""
    import torch
    lat: Dict[int, float] = {}
    results = {}
    t0 = time.perf_counter()
    with torch.cuda.stream(bases[0].stream):
        for req in sorted(requests, key=lambda r: r.arrival):
            wait = req.arrival * time_scale - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            prob = B.Problem.like(bases[req.template], req.K, req.fid_mask, req.fid_labels,
                                  _params(req, precision))
            prob.solve(req.outer, req.inner)
            lab = prob.labels()
            lat[req.rid] = time.perf_counter() - t0 - req.arrival * time_scale
            if keep_results:
                results[req.rid] = (lab, prob.get_u())
            prob.close()
    return Stats(lat, time.perf_counter() - t0, 0, 0), results
