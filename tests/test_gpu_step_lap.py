"""Unnormalized Laplacian L = D - W and finite step size k on the GPU, against
the FP64 oracle (which runs the step-size-k system I + kT, u^t + k b^t, G_k
literally, while the CUDA path runs the equivalent c + 1/k, delta0/k form).

Bar as in the FP32 parity tests: relative L2 error of u at most 1e-5 after
every outer step, energies within 1e-5, identical labels except at ties.  The
mixed-precision form keeps its own bar (decided-row label agreement >= 0.999,
energy within 1e-3).
"""

import numpy as np
import pytest

import oracle
from gen import make_workload, random_graph

pytestmark = pytest.mark.gpu

TOL_U = 1e-5
TOL_F = 1e-5
UN = 1


@pytest.fixture(scope="module")
def B(cuda_lib):
    from paper_2303_14495_gb300 import binding
    return binding


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def graph_case(n, K, seed, deg=8):
    rp, col, w = random_graph(n, deg, seed=seed)
    rng = np.random.default_rng(seed)
    mask = (rng.uniform(size=n) < 0.15).astype(np.uint8)
    lab = rng.integers(0, max(K, 2), size=n).astype(np.int32)
    return rp, col, w, mask, lab


def lam_dense_free(rp, col, w, lap):
    """lambda_max from the oracle's power method (then the safe reading)."""
    P = oracle.Problem(rp, col, w, 1, np.zeros(rp.shape[0] - 1, np.uint8), np.zeros(rp.shape[0] - 1, np.int32),
                       1.0, 0.0, 1.0, laplacian=lap)
    d, _ = oracle.degrees(rp, col, w)
    return oracle.safe_lambda(P.power_max_eig(150), lap, d.max())


def pair(B, rp, col, w, K, mask, lab, lap, k, precond, eps=1.0, eta=20.0, c=40.0, damping=0.8, lam=0.0,
         precision=0, omp=False):
    prm = B.make_params(eps=eps, eta=eta, c=c, precond=precond, damping=damping, lambda_max=lam,
                        laplacian=lap, step_k=k, precision=precision)
    gpu = B.Problem(rp, col, w, K, mask, lab, prm)
    ref = oracle.Problem(rp, col, w, K, mask, lab, eps, eta, c, precond=precond, damping=damping,
                         lambda_max=lam, laplacian=lap, step_k=k, omp=omp)
    return gpu, ref


def label_mismatch(lab_gpu, u_ref, K):
    if K == 1:
        ref = (u_ref >= 0).astype(np.int32)
        tie = np.abs(u_ref) < 1e-6
    else:
        ref = np.argmax(u_ref, axis=1).astype(np.int32)
        srt = np.sort(u_ref, axis=1)
        tie = (srt[:, -1] - srt[:, -2]) < 1e-6
    return np.nonzero((lab_gpu != ref) & ~tie)[0]


def run(gpu, ref, outer, inner):
    u_ref = ref.init_u()
    errs = []
    for t in range(outer):
        gpu.step(inner)
        u_ref, e_ref, r_ref = ref.solve(1, inner, u_ref)
        err = rel_l2(gpu.get_u(), u_ref)
        errs.append(err)
        assert err <= TOL_U, f"step {t}: rel L2 {err:.3e}"
        F, rel = gpu.energy()
        assert abs(F - e_ref[0]) <= TOL_F * abs(e_ref[0]), (t, F, e_ref[0])
        assert abs(rel - r_ref[0]) <= 1e-3 * abs(r_ref[0]) + 1e-7, (t, rel, r_ref[0])
    bad = label_mismatch(gpu.labels(), u_ref, gpu.K)
    assert bad.size == 0, f"{bad.size} label mismatches"
    return errs


@pytest.mark.parametrize("precond", [0, 1, 2])
@pytest.mark.parametrize("K", [1, 3, 4])
@pytest.mark.parametrize("n", [33, 1031, 3000])
def test_unnormalized_parity(B, precond, K, n):
    rp, col, w, mask, lab = graph_case(n, K, seed=n + 10 * K + precond)
    lam = lam_dense_free(rp, col, w, UN) if precond == 2 else 0.0
    d, _ = oracle.degrees(rp, col, w)
    c = max(40.0, 3.0 * d.max() + 1.0)     # damped Jacobi, omega = 0.8 on L needs c > 3 eps d_max
    gpu, ref = pair(B, rp, col, w, K, mask, lab, UN, 0.0, precond, c=c, lam=lam)
    run(gpu, ref, 4, 3)


@pytest.mark.parametrize("lap", [0, 1])
@pytest.mark.parametrize("precond", [0, 1, 2])
@pytest.mark.parametrize("k", [0.01, 0.1, 1.0, 5.0])
def test_finite_step_parity(B, lap, precond, k):
    n, K = 1500, 3
    rp, col, w, mask, lab = graph_case(n, K, seed=int(k * 100) + 3 * precond + lap)
    lam = lam_dense_free(rp, col, w, lap) if precond == 2 else 0.0
    gpu, ref = pair(B, rp, col, w, K, mask, lab, lap, k, precond, c=40.0 if lap == 0 else 80.0, lam=lam)
    run(gpu, ref, 4, 3)


def test_power_method_unnormalized(B):
    """The GPU power method on L against the oracle's (same start vector and
    iteration count), and the safe value min(2 d_max, 1.001 estimate)."""
    n = 4000
    rp, col, w, mask, lab = graph_case(n, 1, seed=77)
    d, _ = oracle.degrees(rp, col, w)
    P = oracle.Problem(rp, col, w, 1, mask, lab, 1.0, 20.0, 40.0, laplacian=UN)
    est = P.power_max_eig(150)
    prm = B.make_params(eps=1.0, eta=20.0, c=40.0, precond=B.PDCA_RICHARDSON, laplacian=UN)
    g = B.Problem(rp, col, w, 1, mask, lab, prm)
    used, est_gpu = g.lambda_max()
    assert abs(est_gpu - est) <= 1e-4 * est, (est_gpu, est)
    assert used == pytest.approx(min(2 * d.max(), 1.001 * est_gpu), rel=1e-12)


def test_unnormalized_damped_feasibility(B):
    """create refuses damped Jacobi on L unless c + 1/k > eps d_max (2w-1)/(1-w)."""
    n = 500
    rp, col, w, mask, lab = graph_case(n, 1, seed=5)
    d, _ = oracle.degrees(rp, col, w)
    bound = 1.0 * d.max() * (2 * 0.8 - 1) / (1 - 0.8)
    mk = lambda c, k=0.0: B.make_params(eps=1.0, eta=5.0, c=c, precond=0, damping=0.8, laplacian=UN, step_k=k)
    with pytest.raises(B.PdcaError, match="INFEASIBLE"):
        B.Problem(rp, col, w, 1, mask, lab, mk(bound * 0.99))
    B.Problem(rp, col, w, 1, mask, lab, mk(bound * 1.01)).close()
    # a finite step size adds 1/k to c
    B.Problem(rp, col, w, 1, mask, lab, mk(bound * 0.99, k=10.0 / bound)).close()
    # the normalized rule stays c > eps (2w-1)/(1-w) = 3
    B.Problem(rp, col, w, 1, mask, lab, B.make_params(eps=1.0, eta=5.0, c=3.1, precond=0, damping=0.8)).close()


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("lap,k", [(1, 0.0), (0, 0.5), (1, 0.5)])
def test_mixed_unnormalized_and_step(B, prec, lap, k):
    n, K = 6000, 4
    rp, col, w, mask, lab = graph_case(n, K, seed=31 + prec)
    gpu, ref = pair(B, rp, col, w, K, mask, lab, lap, k, 1, c=60.0, precision=prec)
    u_ref = ref.init_u()
    for _ in range(5):
        gpu.step(4)
        u_ref, e_ref, _ = ref.solve(1, 4, u_ref)
    F, _ = gpu.energy()
    assert abs(F - e_ref[0]) <= 1e-3 * abs(e_ref[0]), (F, e_ref[0])
    srt = np.sort(u_ref, axis=1)
    decided = (srt[:, -1] - srt[:, -2]) >= 1e-4
    agree = np.mean(gpu.labels()[decided] == np.argmax(u_ref, axis=1)[decided])
    assert agree >= 0.999, agree
    assert rel_l2(gpu.get_u(), u_ref) <= 1e-4


def test_batch_mixes_laplacians(B):
    """Problems on L and on L_s, with and without a step size, advance together
    in one batch exactly as alone."""
    specs = []
    for i, (n, K, lap, k, prec) in enumerate([(700, 1, 1, 0.0, 0), (1300, 4, 0, 0.2, 0), (900, 4, 1, 0.2, 0),
                                              (2100, 3, 1, 0.0, 1), (500, 3, 0, 0.0, 2), (64, 2, 1, 1.0, 0)]):
        rp, col, w, mask, lab = graph_case(n, K, seed=200 + i)
        specs.append((rp, col, w, K, mask, lab, B.make_params(eps=1.0, eta=20.0, c=60.0, precond=1, laplacian=lap,
                                                               step_k=k, precision=prec)))
    alone = []
    for rp, col, w, K, mask, lab, prm in specs:
        g = B.Problem(rp, col, w, K, mask, lab, prm)
        g.solve(3, 2)
        alone.append(g.get_u())
    batch = B.Batch()
    probs = [B.Problem(rp, col, w, K, mask, lab, prm) for rp, col, w, K, mask, lab, prm in specs]
    for g in probs:
        batch.add(g, 3, 2)
    while batch.step(2):
        pass
    assert len(batch.poll()) == len(specs)
    for g, u in zip(probs, alone):
        np.testing.assert_array_equal(g.get_u(), u)


def test_create_like_unnormalized(B):
    n, K = 2000, 3
    rp, col, w, mask, lab = graph_case(n, K, seed=9)
    prm = B.make_params(eps=1.0, eta=20.0, c=60.0, precond=2, laplacian=UN)
    base = B.Problem(rp, col, w, K, mask, lab, prm)
    rng = np.random.default_rng(1)
    mask2 = (rng.uniform(size=n) < 0.2).astype(np.uint8)
    lab2 = rng.integers(0, 5, size=n).astype(np.int32)
    prm2 = B.make_params(eps=1.0, eta=30.0, c=70.0, precond=2, laplacian=UN, step_k=0.3)
    like = B.Problem.like(base, 5, mask2, lab2, prm2)
    fresh = B.Problem(rp, col, w, 5, mask2, lab2, prm2)
    assert like.lambda_max() == fresh.lambda_max()
    like.solve(3, 3)
    fresh.solve(3, 3)
    np.testing.assert_array_equal(like.get_u(), fresh.get_u())
    with pytest.raises(B.PdcaError, match="INVALID_ARG"):
        B.Problem.like(base, 5, mask2, lab2, B.make_params(eps=1.0, eta=30.0, c=70.0, precond=2))


def test_moons_unnormalized_full_run(B):
    """The two-moons workload on L with a step size, its configured schedule."""
    wl = make_workload("moons2k")
    p = wl.params
    d, _ = oracle.degrees(wl.row_ptr, wl.col, wl.w)
    c = max(p["c"], 3.0 * p["eps"] * d.max() + 1.0)
    gpu, ref = pair(B, wl.row_ptr, wl.col, wl.w, wl.K, wl.fid_mask, wl.fid_labels, UN, 1.0, p["precond"],
                    eps=p["eps"], eta=p["eta"], c=c, damping=p["damping"])
    run(gpu, ref, p["outer"], p["inner"])
