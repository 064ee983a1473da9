"""Choices made by measurement on the caller's own graph and request mix.

``tune_layout`` times the fused sweep under each candidate layout (node
renumbering, degree-sort window, entry order, shared-memory tiles) with the
library's sweep profiler (CUDA events around every sweep launch) and returns
the fastest parameters.  Layouts change the order of the floating-point sums
only, so every candidate solves the same problem.

``tune_shape`` then times the kernels' own shape on the chosen layout: the
column format (16-bit where it fits, or int32), the slices one block takes
from its queue (8, 16 or 32) and the split length of long rows.

``tune_sweeps`` picks the number of inner sweeps per outer step: for each
candidate it finds the number of outer steps that brings the iterate within
a relative distance of a long reference solve, times that solve, and keeps
the candidate that gets there first.

``tune_serving`` replays a sample of a request mix through the continuous
batching loop for each (slot count, passes per tick) pair and returns the
pair with the lowest p99 latency among those within 5% of the best
throughput.

Both run through the C interface only; they measure, they compute nothing of
the method themselves.
"""

from __future__ import annotations

import itertools
import time
from typing import Dict, List, Optional, Sequence, Tuple

from . import binding as B

# (name, pdca_params overrides)
DEFAULT_LAYOUTS: List[Tuple[str, dict]] = [
    ("bfs, window 1024, spread", dict(reorder=B.PDCA_REORDER_BFS, sort_window=0, tiling=B.PDCA_TILING_OFF,
                                      entry_order=B.PDCA_ENTRIES_SPREAD)),
    ("bfs, window 1024, csr order", dict(reorder=B.PDCA_REORDER_BFS, sort_window=0, tiling=B.PDCA_TILING_OFF,
                                         entry_order=B.PDCA_ENTRIES_CSR)),
    ("bfs, window 256, spread", dict(reorder=B.PDCA_REORDER_BFS, sort_window=256, tiling=B.PDCA_TILING_OFF,
                                     entry_order=B.PDCA_ENTRIES_SPREAD)),
    ("bfs, tiles", dict(reorder=B.PDCA_REORDER_BFS, sort_window=0, tiling=B.PDCA_TILING_ON,
                        entry_order=B.PDCA_ENTRIES_SPREAD)),
    ("caller order, auto window", dict(reorder=B.PDCA_REORDER_NONE, sort_window=0, tiling=B.PDCA_TILING_OFF,
                                       entry_order=B.PDCA_ENTRIES_SPREAD)),
]


def shape_candidates(max_degree: int) -> List[Tuple[str, dict]]:
    """Kernel-shape candidates: column format x slices per block range, and,
    on graphs with rows longer than 64 entries, a split length of 64."""
    out = []
    for cols, cname in ((B.PDCA_COLUMNS_AUTO, "16-bit columns"), (B.PDCA_COLUMNS_32, "int32 columns")):
        for bs in (32, 16, 8):
            out.append((f"{cname}, {bs} slices per block", dict(columns=cols, block_slices=bs)))
    if max_degree > 64:
        out.append(("16-bit columns, 32 slices per block, split at 64",
                    dict(columns=B.PDCA_COLUMNS_AUTO, block_slices=32, row_split=64)))
    return out


def tune_layout(row_ptr, col, w, K, fid_mask, fid_labels, base: dict,
                candidates: Optional[Sequence[Tuple[str, dict]]] = None, sweeps: int = 8, repeats: int = 3,
                device="cuda"):
    """Fastest layout for this graph.

    ``base``: keyword arguments of ``binding.make_params`` (eps, c, eta,
    precond, ...); each candidate overrides some of them.  Returns
    (params_kwargs of the fastest candidate, table), the table a list of
    dicts (name, ms_per_sweep, create_ms) sorted by ms_per_sweep; candidates
    the library refuses for these parameters (e.g. tiles with the
    unnormalized Laplacian) are listed with the refusal instead of a time.
    """
    import torch
    rows = []
    for name, over in (candidates or DEFAULT_LAYOUTS):
        kw = dict(base)
        kw.update(over)
        prm = B.make_params(**kw)
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g = B.Problem(row_ptr, col, w, K, fid_mask, fid_labels, prm, device=device)
            torch.cuda.synchronize()
            create_ms = (time.perf_counter() - t0) * 1e3
        except B.PdcaError as e:
            rows.append({"name": name, "params": kw, "refused": str(e)})
            continue
        g.step(sweeps)                      # warm-up
        g.profile(True)
        for _ in range(repeats):
            g.set_u(None)
            g.step(sweeps)
        torch.cuda.synchronize()
        ms, cnt = g.profile_read()
        g.profile(False)
        g.close()
        rows.append({"name": name, "params": kw, "ms_per_sweep": ms / max(cnt, 1), "create_ms": create_ms,
                     "sweeps_timed": int(cnt)})
    timed = sorted((r for r in rows if "ms_per_sweep" in r), key=lambda r: r["ms_per_sweep"])
    if not timed:
        raise ValueError("tune_layout: the library refused every candidate layout for these parameters")
    return timed[0]["params"], timed + [r for r in rows if "refused" in r]


def tune_shape(row_ptr, col, w, K, fid_mask, fid_labels, base: dict, sweeps: int = 8, repeats: int = 3,
               device="cuda"):
    """Fastest kernel shape for this graph on the layout in ``base``; same
    return form as ``tune_layout``."""
    import numpy as np
    max_degree = int(np.max(np.diff(np.asarray(row_ptr)))) if len(row_ptr) > 1 else 0
    return tune_layout(row_ptr, col, w, K, fid_mask, fid_labels, base, candidates=shape_candidates(max_degree),
                       sweeps=sweeps, repeats=repeats, device=device)


def tune_sweeps(make_problem, candidates: Sequence[int] = (2, 4, 8), tol: float = 1e-4, max_outer: int = 64):
    """Inner sweeps per outer step by time to a fixed point.

    The outer pDCA iteration has converged when a step moves the iterate
    little: d_t = ||u^t - u^{t-1}|| / ||u^t|| <= ``tol``.  More sweeps per
    outer step solve each linear system (Sec. 3) more exactly; whether that
    saves outer steps depends on the problem: with a large c the system is
    solved in two sweeps and the outer steps take the same course for every
    count, with a small c and a large eps extra sweeps shorten the outer
    course.  ``make_problem()`` returns a fresh ``binding.Problem``.  For
    each m the problem runs from u^0 one outer step at a time (each step
    timed with CUDA events on the problem's stream; the norms are taken
    between steps, outside the timed region) until d_t <= ``tol`` or
    ``max_outer`` steps.  Returns (m, table): the fastest m among those that
    reached ``tol``, else the m that reduced d by the most decades per
    millisecond; the table has, per m, the outer steps, the milliseconds,
    the last d_t, whether ``tol`` was reached and the decades per ms."""
    import math
    import torch
    table = []
    for m in candidates:
        g = make_problem()
        shape = (g.n,) if g.K == 1 else (g.n, g.K)
        prev = torch.empty(shape, dtype=torch.float32, device=g.device)
        cur = torch.empty_like(prev)
        g.solve(1, m)                       # warm-up (kernels, graphs)
        g.set_u(None)
        g.get_u(prev)
        torch.cuda.synchronize()
        ms, d, d1, T = 0.0, float("inf"), None, 0
        while T < max_outer:
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(g.stream)
            g.solve(1, m)
            b.record(g.stream)
            torch.cuda.synchronize()
            ms += a.elapsed_time(b)
            T += 1
            g.get_u(cur)
            torch.cuda.synchronize()
            nrm = float(torch.linalg.vector_norm(cur.double()))
            d = float(torch.linalg.vector_norm((cur - prev).double())) / max(nrm, 1e-300)
            d1 = d if d1 is None else d1
            prev, cur = cur, prev
            if d <= tol:
                break
        g.close()
        table.append({"inner": int(m), "outer_steps": T, "ms": ms, "step_change": d, "reached": bool(d <= tol),
                      "ms_per_outer": ms / max(T, 1),
                      "decades_per_ms": math.log10(max(d1, 1e-300) / max(d, 1e-300)) / max(ms, 1e-9)})
    hit = [t for t in table if t["reached"]]
    best = min(hit, key=lambda t: t["ms"]) if hit else max(table, key=lambda t: t["decades_per_ms"])
    return best["inner"], table


def tune_serving(bases, requests, precision: int = B.PDCA_MIXED_BF16W_FP16U,
                 slots: Sequence[int] = (16, 32, 64), passes: Sequence[int] = (1, 2, 4, 8),
                 mem_budget: int = 64 << 30):
    """(max_slots, passes_per_tick) for the continuous-batching loop.

    Replays ``requests`` (a sample of the mix, arrival times included)
    through ``serving.serve_batched`` once per pair.  Returns
    (dict(max_slots=..., passes_per_tick=...), table of summaries)."""
    from . import serving
    table: List[Dict] = []
    for s, p in itertools.product(slots, passes):
        st, _ = serving.serve_batched(bases, requests, precision=precision, mem_budget=mem_budget, max_slots=s,
                                      passes_per_tick=p)
        row = dict(st.summary())
        row.update(max_slots=int(s), passes_per_tick=int(p))
        table.append(row)
    best_tp = max(r["problems_per_s"] for r in table)
    ok = [r for r in table if r["problems_per_s"] >= 0.95 * best_tp]
    pick = min(ok, key=lambda r: (r["p99_ms"], -r["problems_per_s"]))
    return {"max_slots": pick["max_slots"], "passes_per_tick": pick["passes_per_tick"]}, table
