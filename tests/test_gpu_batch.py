"""Batched passes (pdca_batch_*): problems of different sizes, K classes,
Laplacians, step sizes, precisions and inner-sweep counts advanced together.

Two bars.  Against the FP64 oracle, every member after every outer step:
FP32 members within 1e-5 relative L2 of u with labels identical except at
ties (gap < 1e-6); mixed-precision members within 1e-4 relative L2, labels
agreeing on 99.9% of the non-tie rows (one row allowed on graphs of fewer
than 1000 rows) and the energy within 1e-3.  Against the solo path:
bit-identical iterates, including when members join while others run."""

import numpy as np
import pytest

import oracle
from gen import make_workload, random_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(cuda_lib):
    from paper_2303_14495_gb300 import binding
    return binding


EPS, ETA, C = 1.0, 20.0, 22.0
TIE = 1e-6


def problem_specs(variants=False):
    """Random graphs of mixed sizes; with ``variants`` also members on the
    unnormalized Laplacian (lap = 1) and with a finite step size k."""
    rows = [(300, 1, 0, 3, 0, 0.0), (1031, 4, 0, 2, 0, 0.0), (2050, 4, 1, 4, 0, 0.0),
            (777, 10, 2, 1, 0, 0.0), (4096, 3, 0, 5, 0, 0.0), (65, 2, 1, 2, 0, 0.0),
            (5000, 4, 2, 3, 0, 0.0), (33, 1, 1, 1, 0, 0.0)]
    if variants:
        rows += [(1500, 4, 0, 3, 1, 0.0), (900, 2, 0, 2, 0, 0.5), (1200, 5, 1, 3, 1, 0.0),
                 (800, 1, 0, 4, 1, 2.0), (2600, 10, 0, 2, 0, 0.05)]
    splits = {9: 8, 10: 12, 11: 8, 12: 4}     # members whose long rows continue in the overflow CSR
    specs = []
    for i, (n, K, prec, inner, lap, k) in enumerate(rows):
        rp, col, w = random_graph(n, 8, seed=100 + i)
        rng = np.random.default_rng(i)
        mask = (rng.uniform(size=n) < 0.1).astype(np.uint8)
        lab = rng.integers(0, max(K, 2), size=n).astype(np.int32)
        specs.append(dict(rp=rp, col=col, w=w, K=K, mask=mask, lab=lab, prec=prec, inner=inner, outer=2 + i % 3,
                          lap=lap, k=k, split=splits.get(i, 0) if variants else 0))
    return specs


def make(B, sp):
    prm = B.make_params(eps=EPS, eta=ETA, c=C, precond=1, precision=sp["prec"], laplacian=sp.get("lap", 0),
                        step_k=sp.get("k", 0.0), row_split=sp.get("split", 0))
    return B.Problem(sp["rp"], sp["col"], sp["w"], sp["K"], sp["mask"], sp["lab"], prm)


def oracle_of(sp):
    return oracle.Problem(sp["rp"], sp["col"], sp["w"], sp["K"], sp["mask"], sp["lab"], EPS, ETA, C, precond=1,
                          laplacian=sp.get("lap", 0), step_k=sp.get("k", 0.0))


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def check_member(g, ref, u_ref, prec, K, what, F_ref=None):
    """One member's iterate against the oracle's after the same outer steps."""
    u = g.get_u()
    err = rel_l2(u, u_ref)
    lab = g.labels()
    lab_ref = ref.labels_of(u_ref)
    if K == 1:
        margin = np.abs(u_ref)
    else:
        srt = np.sort(u_ref, axis=1)
        margin = srt[:, -1] - srt[:, -2]
    nontie = margin >= TIE
    if prec == 0:
        assert err <= 1e-5, (what, err)
        assert np.all(lab[nontie] == lab_ref[nontie]), what
    else:
        assert err <= 1e-4, (what, err)
        mism = int(np.sum(lab[nontie] != lab_ref[nontie]))
        assert mism <= max(1, 0.001 * nontie.sum()), (what, mism, int(nontie.sum()))
    if F_ref is not None:
        F, _ = g.energy()
        tol = 1e-5 if prec == 0 else 1e-3
        assert abs(F - F_ref) <= tol * abs(F_ref), (what, F, F_ref)
    return err


def test_batch_vs_oracle_every_outer_step(B):
    """Every member joins the batch for one outer step at a time; after each
    step its iterate is compared with the oracle's."""
    specs = problem_specs(variants=True)
    probs = [make(B, sp) for sp in specs]
    refs = [oracle_of(sp) for sp in specs]
    u_ref = [r.init_u() for r in refs]
    batch = B.Batch()
    worst = [0.0, 0.0]
    for t in range(max(sp["outer"] for sp in specs)):
        live = [i for i, sp in enumerate(specs) if t < sp["outer"]]
        for i in live:
            batch.add(probs[i], 1, specs[i]["inner"])
        while batch.step(2):
            pass
        assert len(batch.poll()) == len(live)
        for i in live:
            sp = specs[i]
            u_ref[i], e_ref, _ = refs[i].solve(1, sp["inner"], u_ref[i])
            err = check_member(probs[i], refs[i], u_ref[i], sp["prec"], sp["K"], (i, t), F_ref=e_ref[0])
            worst[sp["prec"] != 0] = max(worst[sp["prec"] != 0], err)
    print(f"worst rel L2 vs oracle: fp32 {worst[0]:.2e}, mixed {worst[1]:.2e}")


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
    # and the batched results against the oracle's
    for i, (g, sp) in enumerate(zip(probs, specs)):
        ref = oracle_of(sp)
        u_ref, e_ref, _ = ref.solve(sp["outer"], sp["inner"])
        check_member(g, ref, u_ref, sp["prec"], sp["K"], i, F_ref=e_ref[-1])


def test_continuous_joining(B):
    """Members join while others are mid-step; each result equals its solo run
    and agrees with the oracle's."""
    specs = problem_specs(variants=True)
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
        sp = specs[i]
        ref = oracle_of(sp)
        u_ref, e_ref, _ = ref.solve(sp["outer"], sp["inner"])
        check_member(probs[i], ref, u_ref, sp["prec"], sp["K"], i, F_ref=e_ref[-1])


def test_batch_workload_mix(B):
    """Real graphs of the serving mix: image and point-cloud graphs, K in {1, 4, 10}."""
    wls = [make_workload("ellipses256", size=96), make_workload("voronoi2048", size=128),
           make_workload("gmm70k", n_per=400, dim=32), make_workload("moons2k", n=500)]
    solo, probs, refs = [], [], []
    batch = B.Batch()
    for j, wl in enumerate(wls):
        p = wl.params
        ref = oracle.Problem(wl.row_ptr, wl.col, wl.w, wl.K, wl.fid_mask, wl.fid_labels, p["eps"], p["eta"], p["c"],
                             precond=p["precond"], damping=p.get("damping") or 0.5)
        lam = oracle.safe_lambda(ref.power_max_eig(150)) if p["precond"] == 2 else 0.0
        ref.set_lambda_max(lam)
        u_ref, e_ref, _ = ref.solve(p["outer"], p["inner"])
        for prec in (0, 1):
            prm = B.params_from_workload(p, precision=prec, lambda_max=lam)
            a = B.Problem(wl.row_ptr, wl.col, wl.w, wl.K, wl.fid_mask, wl.fid_labels, prm)
            a.solve(p["outer"], p["inner"])
            solo.append(a.get_u())
            g = B.Problem(wl.row_ptr, wl.col, wl.w, wl.K, wl.fid_mask, wl.fid_labels, prm)
            batch.add(g, p["outer"], p["inner"])
            probs.append(g)
            refs.append((ref, u_ref, e_ref[-1], prec, wl.K, wl.name))
    while batch.step(4):
        pass
    assert len(batch.poll()) == len(probs)
    for g, u, (ref, u_ref, F_ref, prec, K, name) in zip(probs, solo, refs):
        np.testing.assert_array_equal(g.get_u(), u)
        check_member(g, ref, u_ref, prec, K, (name, prec), F_ref=F_ref)


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
