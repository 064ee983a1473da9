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
