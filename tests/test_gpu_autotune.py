"""Autotuning (autotune.py) on the GPU: the layout tuner times every
candidate, picks the fastest, and the tuned problem iterates exactly like a
problem created directly with the chosen parameters; the serving tuner
returns a pair from its grid that keeps within 5% of the best throughput."""

import numpy as np
import pytest

from gen import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(cuda_lib):
    from paper_2303_14495_gb300 import binding
    return binding


def test_tune_layout(B):
    from paper_2303_14495_gb300 import autotune
    wl = make_workload("voronoi2048", size=256)
    p = wl.params
    base = dict(eps=p["eps"], c=p["c"], eta=p["eta"], precond=p["precond"], lambda_max=1.99)
    best, table = autotune.tune_layout(wl.row_ptr, wl.col, wl.w, wl.K, wl.fid_mask, wl.fid_labels, base,
                                       sweeps=4, repeats=2)
    timed = [r for r in table if "ms_per_sweep" in r]
    assert len(timed) == len(autotune.DEFAULT_LAYOUTS)
    assert best == timed[0]["params"]
    assert all(timed[0]["ms_per_sweep"] <= r["ms_per_sweep"] for r in timed)
    assert all(r["sweeps_timed"] == 2 * 4 for r in timed)
    # the chosen layout is an ordinary parameter set
    a = B.Problem(wl.row_ptr, wl.col, wl.w, wl.K, wl.fid_mask, wl.fid_labels, B.make_params(**best))
    b = B.Problem(wl.row_ptr, wl.col, wl.w, wl.K, wl.fid_mask, wl.fid_labels, B.make_params(**best))
    a.solve(2, 4)
    b.solve(2, 4)
    np.testing.assert_array_equal(a.get_u(), b.get_u())


def test_tune_layout_refusals_listed(B):
    from paper_2303_14495_gb300 import autotune
    wl = make_workload("voronoi2048", size=128)
    p = wl.params
    base = dict(eps=p["eps"], c=p["c"], eta=p["eta"], precond=B.PDCA_JACOBI_PERTURBED,
                laplacian=B.PDCA_LAP_UNNORMALIZED)
    best, table = autotune.tune_layout(wl.row_ptr, wl.col, wl.w, wl.K, wl.fid_mask, wl.fid_labels, base,
                                       sweeps=2, repeats=1)
    refused = [r for r in table if "refused" in r]
    assert [r["name"] for r in refused] == ["bfs, tiles"]     # tiles take the normalized Laplacian only
    assert best["tiling"] != B.PDCA_TILING_ON


def test_tune_serving(B):
    import torch
    from gen import serving_mix
    from paper_2303_14495_gb300 import autotune, serving
    pool = serving_mix.templates(device="cuda", max_n=1 << 16)
    reqs = serving_mix.requests(pool, n_requests=48, rate=2000.0, n_max=1 << 16)
    stream = torch.cuda.current_stream()
    bases = serving.prepare(pool, B.PDCA_MIXED_BF16W_FP16U, stream)
    pick, table = autotune.tune_serving(bases, reqs, slots=(8, 32), passes=(2, 8))
    assert len(table) == 4 and all(r["requests"] == 48 for r in table)
    best_tp = max(r["problems_per_s"] for r in table)
    row = next(r for r in table if (r["max_slots"], r["passes_per_tick"]) == (pick["max_slots"],
                                                                              pick["passes_per_tick"]))
    assert row["problems_per_s"] >= 0.95 * best_tp


def test_tune_shape_and_block_ranges(B):
    """The shape tuner times every candidate; slices per block range change
    the launch only, so the iterates are the same bits for 8, 16 and 32."""
    from paper_2303_14495_gb300 import autotune
    wl = make_workload("gmm70k", n_per=2000, dim=64)      # hub rows: the split candidate is offered
    p = wl.params
    base = dict(eps=p["eps"], c=p["c"], eta=p["eta"], precond=p["precond"], damping=p["damping"] or 0.5)
    best, table = autotune.tune_shape(wl.row_ptr, wl.col, wl.w, wl.K, wl.fid_mask, wl.fid_labels, base,
                                      sweeps=4, repeats=2)
    timed = [r for r in table if "ms_per_sweep" in r]
    maxdeg = int(np.max(np.diff(wl.row_ptr)))
    assert len(timed) == len(autotune.shape_candidates(maxdeg))
    assert best == timed[0]["params"]
    us = []
    for bs in (8, 16, 32):
        g = B.Problem(wl.row_ptr, wl.col, wl.w, wl.K, wl.fid_mask, wl.fid_labels,
                      B.params_from_workload(p, block_slices=bs))
        g.solve(3, 5)
        us.append(g.get_u())
    np.testing.assert_array_equal(us[0], us[1])
    np.testing.assert_array_equal(us[0], us[2])
    with pytest.raises(B.PdcaError, match="INVALID_ARG"):
        B.Problem(wl.row_ptr, wl.col, wl.w, wl.K, wl.fid_mask, wl.fid_labels,
                  B.params_from_workload(p, block_slices=12))


def test_tune_sweeps(B):
    """Inner sweep counts by time to a fixed point of the outer iteration.
    With c = 2/eps + eta = 502 two sweeps solve each system (on the 128 x 128
    image the oracle's outer steps agree to 1e-8 for 2, 4 and 8 sweeps):
    every count stops at the same outer step and the cheapest count wins."""
    from paper_2303_14495_gb300 import autotune
    wl = make_workload("voronoi2048", size=256)
    prm = B.params_from_workload(wl.params)
    make = lambda: B.Problem(wl.row_ptr, wl.col, wl.w, wl.K, wl.fid_mask, wl.fid_labels, prm)
    m, table = autotune.tune_sweeps(make, candidates=(2, 4, 8), tol=1e-4, max_outer=32)
    assert [t["inner"] for t in table] == [2, 4, 8]
    assert all(t["reached"] and t["step_change"] <= 1e-4 and t["ms"] > 0 for t in table), table
    steps = [t["outer_steps"] for t in table]
    assert max(steps) - min(steps) <= 1, table
    assert m == 2, table


def test_tune_sweeps_small_c(B):
    """The setting of the preconditioner study (eps = 100, c = 11,
    eta = 100): extra sweeps shorten the outer course.  The pick is the
    fastest count that reached the tolerance, and each row's flag agrees
    with its last step change."""
    from paper_2303_14495_gb300 import autotune
    wl = make_workload("ellipses256", size=96)
    prm = B.params_from_workload(dict(wl.params, eps=100.0, c=11.0, eta=100.0))
    make = lambda: B.Problem(wl.row_ptr, wl.col, wl.w, wl.K, wl.fid_mask, wl.fid_labels, prm)
    m, table = autotune.tune_sweeps(make, candidates=(2, 4, 8), tol=2e-2, max_outer=96)
    assert [t["inner"] for t in table] == [2, 4, 8]
    for t in table:
        assert t["ms"] > 0 and t["reached"] == (t["step_change"] <= 2e-2), t
    hit = [t for t in table if t["reached"]]
    assert hit, table
    row = next(t for t in table if t["inner"] == m)
    assert row["ms"] == min(t["ms"] for t in hit)
    # more sweeps per outer step: fewer outer steps to the tolerance
    assert table[2]["outer_steps"] <= table[0]["outer_steps"], table
