"""Choices made by measurement on the caller's own graph and request mix.

``tune_layout`` times the fused sweep under each candidate layout (node
renumbering, degree-sort window, entry order, shared-memory tiles) with the
library's sweep profiler (CUDA events around every sweep launch) and returns
the fastest parameters.  Layouts change the order of the floating-point sums
only, so every candidate solves the same problem.

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
