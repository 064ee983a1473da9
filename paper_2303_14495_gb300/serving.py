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
completion.  The loop is pipelined: admission, the labels read and the
release are enqueued without waiting for the stream, and the host waits only
for the tick before the newest, so host work overlaps the device's.

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
                  time_scale: float = 1.0, pipelined: bool = True):
    """Continuous batching on prepared operators (``bases`` of the matching
    precision family).  Returns (Stats, {rid: (labels, u)} if keep_results).

    pipelined=True keeps the stream busy while the host works: requests are
    admitted with pdca_create_like_async (fidelity arrays staged in pinned
    host memory), a finished problem's labels are enqueued with
    pdca_labels_async into pinned memory, and the host waits only for the
    tick before the one it has just enqueued, so that the device runs tick t
    while the host retires tick t - 1 and admits for tick t + 1.  A finished
    problem is released (pdca_release) once its labels have arrived; its
    workspace returns to PyTorch's allocator on the serving stream.
    pipelined=False waits for the stream at every admission and every
    finished problem (pdca_create_like, pdca_labels, pdca_destroy)."""
    import collections
    import torch
    stream = bases[0].stream
    batch = B.Batch(max_problems=max_slots, stream=stream)
    pending = sorted(requests, key=lambda r: r.arrival)
    nxt = 0                           # next pending request
    active = {}                       # handle value -> (request, problem, ws bytes)
    inflight = collections.deque()    # (event after a tick, [(request, problem, ws, labels, status)])
    used = peak = busy_admits = 0
    lat: Dict[int, float] = {}
    results = {}
    t0 = time.perf_counter()

    def retire(entries):
        nonlocal used
        now = time.perf_counter() - t0
        for req, prob, ws, lab, st in entries:
            if st is not None and int(st[0]) != 0:
                raise B.PdcaError(B.PDCA_ERR_BAD_GRAPH, f"pdca_create_like_async (request {req.rid})")
            lat[req.rid] = now - req.arrival * time_scale
            if keep_results:
                host = lab.numpy() if hasattr(lab, "numpy") else lab    # pinned tensor or numpy array
                results[req.rid] = (np.array(host, dtype=np.int32), prob.get_u())
            if pipelined:
                prob.release()
            else:
                prob.close()
            used -= ws

    with torch.cuda.stream(stream):
        while nxt < len(pending) or active or inflight:
            now = time.perf_counter() - t0
            while nxt < len(pending) and pending[nxt].arrival * time_scale <= now and len(active) < max_slots:
                req = pending[nxt]
                base = bases[req.template]
                prm = _params(req, precision)
                ws = B.workspace_size_like(base, req.K, prm)
                if used + ws > mem_budget and (active or inflight):
                    break
                if pipelined:
                    mask = torch.from_numpy(np.ascontiguousarray(req.fid_mask)).pin_memory()
                    labs = torch.from_numpy(np.ascontiguousarray(req.fid_labels)).pin_memory()
                    prob = B.Problem.like(base, req.K, mask, labs, prm, wait=False)
                else:
                    prob = B.Problem.like(base, req.K, req.fid_mask, req.fid_labels, prm)
                batch.add(prob, req.outer, req.inner)
                busy_admits += 1 if active else 0
                active[prob.h.value] = (req, prob, ws)
                used += ws
                peak = max(peak, used)
                nxt += 1
            if active:
                batch.step(passes_per_tick)
                done = []
                for prob in batch.poll():
                    req, p, ws = active.pop(prob.h.value)
                    if pipelined:
                        lab = torch.empty(prob.n, dtype=torch.int32, pin_memory=True)
                        st = torch.zeros(1, dtype=torch.int32, pin_memory=True)
                        prob.labels_async(lab, st)
                        done.append((req, prob, ws, lab, st))
                    else:
                        done.append((req, prob, ws, prob.labels(), None))   # synchronises the stream
                    del p
                if not pipelined:
                    retire(done)
                    continue
                ev = torch.cuda.Event()
                ev.record(stream)
                inflight.append((ev, done))
                while len(inflight) > 1:      # the device keeps the newest tick
                    ev_old, entries = inflight.popleft()
                    ev_old.synchronize()
                    retire(entries)
                continue
            while inflight:                   # nothing resident: drain
                ev_old, entries = inflight.popleft()
                ev_old.synchronize()
                retire(entries)
            if nxt < len(pending) and not active:
                wait = pending[nxt].arrival * time_scale - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
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
