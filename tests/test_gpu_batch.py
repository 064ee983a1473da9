"""Batched passes (pdca_batch_*): problems of different sizes, K classes,
precisions and inner-sweep counts advanced together must produce exactly the
iterates they produce alone, including when they join while others run."""

import numpy as np
import pytest

from gen import make_workload, random_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(cuda_lib):
    from paper_2303_14495_gb300 import binding
    return binding


def problem_specs():
    specs = []
    for i, (n, K, prec, inner) in enumerate([(300, 1, 0, 3), (1031, 4, 0, 2), (2050, 4, 1, 4),
                                             (777, 10, 2, 1), (4096, 3, 0, 5), (65, 2, 1, 2),
                                             (5000, 4, 2, 3), (33, 1, 1, 1)]):
        rp, col, w = random_graph(n, 8, seed=100 + i)
        rng = np.random.default_rng(i)
        mask = (rng.uniform(size=n) < 0.1).astype(np.uint8)
        lab = rng.integers(0, max(K, 2), size=n).astype(np.int32)
        specs.append(dict(rp=rp, col=col, w=w, K=K, mask=mask, lab=lab, prec=prec, inner=inner, outer=2 + i % 3))
    return specs


def make(B, sp):
    prm = B.make_params(eps=1.0, eta=20.0, c=22.0, precond=1, precision=sp["prec"])
    return B.Problem(sp["rp"], sp["col"], sp["w"], sp["K"], sp["mask"], sp["lab"], prm)


def test_batch_equals_alone(B):
    specs = problem_specs()
    alone = []
    for sp in specs:
        g = make(B, sp)
        g.solve(sp["outer"], sp["inner"])
        alone.append((g.get_u(), g.energy()[0]))
    batch = B.Batch()
    probs = [make(B, sp) for sp in specs]
    for g, sp in zip(probs, specs):
        batch.add(g, sp["outer"], sp["inner"])
    done = []
    while True:
        active = batch.step(3)
        done += batch.poll()
        if active == 0:
            break
    done += batch.poll()
    assert len(done) == len(specs)
    for g, sp, (u, F) in zip(probs, specs, alone):
        np.testing.assert_array_equal(g.get_u(), u)
        assert g.energy()[0] == F


def test_continuous_joining(B):
    """Members join while others are mid-step; each result equals its solo run."""
    specs = problem_specs()
    solo = []
    for sp in specs:
        g = make(B, sp)
        g.solve(sp["outer"], sp["inner"])
        solo.append(g.get_u())
    batch = B.Batch(max_problems=3)
    pending = list(range(len(specs)))
    probs = {}
    finished = {}
    steps = 0
    while pending or len(finished) < len(specs):
        while pending and len(probs) - len(finished) < 3:
            i = pending.pop(0)
            probs[i] = make(B, specs[i])
            batch.add(probs[i], specs[i]["outer"], specs[i]["inner"])
        batch.step(1 + steps % 2)
        steps += 1
        for g in batch.poll():
            i = next(k for k, v in probs.items() if v is g)
            finished[i] = g.get_u()
        assert steps < 1000
    for i in range(len(specs)):
        np.testing.assert_array_equal(finished[i], solo[i])


def test_batch_workload_mix(B):
    """Real graphs of the serving mix: image and point-cloud graphs, K in {1, 4, 10}."""
    wls = [make_workload("ellipses256", size=96), make_workload("voronoi2048", size=128),
           make_workload("gmm70k", n_per=400, dim=32), make_workload("moons2k", n=500)]
    solo, probs = [], []
    batch = B.Batch()
    for j, wl in enumerate(wls):
        for prec in (0, 1):
            prm = B.params_from_workload(wl.params, precision=prec)
            a = B.Problem(wl.row_ptr, wl.col, wl.w, wl.K, wl.fid_mask, wl.fid_labels, prm)
            a.solve(wl.params["outer"], wl.params["inner"])
            solo.append(a.get_u())
            g = B.Problem(wl.row_ptr, wl.col, wl.w, wl.K, wl.fid_mask, wl.fid_labels, prm)
            batch.add(g, wl.params["outer"], wl.params["inner"])
            probs.append(g)
    while batch.step(4):
        pass
    assert len(batch.poll()) == len(probs)
    for g, u in zip(probs, solo):
        np.testing.assert_array_equal(g.get_u(), u)


def test_batch_argument_checks(B):
    import torch
    sp = problem_specs()[0]
    batch = B.Batch(max_problems=1)
    g = make(B, sp)
    batch.add(g, 2, 2)
    with pytest.raises(B.PdcaError):
        batch.add(g, 2, 2)                       # twice
    with pytest.raises(B.PdcaError):
        batch.add(make(B, sp), 2, 2)             # full
    other = B.Batch(stream=torch.cuda.Stream())
    with pytest.raises(B.PdcaError):
        other.add(make(B, sp), 2, 2)             # different stream
    with pytest.raises(B.PdcaError):
        B.Batch().add(make(B, sp), 0, 2)
    batch.remove(g)
    assert batch.step(5) == 0
