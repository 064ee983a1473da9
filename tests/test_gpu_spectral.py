"""Spectral initial iterate (pdca_spectral_init) against the oracle's second
eigenpair, and the unsupervised model run from it (GPU required).

Bars: lambda_2 within 1e-5 absolute (+ 1e-4 relative) of the oracle's; the
initial iterate u^0 = v_2 / max |v_2| within 10 x (tol / spectral gap) of the
oracle's (the eigenvector error of a residual-tol Ritz vector is bounded by
residual / gap); the unsupervised pDCA run from it within 10 x the initial
difference (+ 1e-5), and identical labels on rows the oracle decides by a
margin of 1e-3.
"""

import numpy as np
import pytest

import oracle
from gen import csr_from_pairs, make_workload, random_graph

pytestmark = pytest.mark.gpu

TOL = 2e-6


@pytest.fixture(scope="module")
def B(cuda_lib):
    from paper_2303_14495_gb300 import binding
    return binding


def gap_of(rp, col, w, lap):
    """lambda_3 - lambda_2 from a dense eigh (small graphs) for the error bound."""
    n = rp.shape[0] - 1
    if n > 3000:
        return None
    W = np.zeros((n, n))
    for i in range(n):
        W[i, col[rp[i]:rp[i + 1]]] = w[rp[i]:rp[i + 1]]
    d = W.sum(1)
    M = np.eye(n) - W / np.sqrt(np.outer(d, d)) if lap == 0 else np.diag(d) - W
    ev = np.linalg.eigvalsh(M)
    return ev[2] - ev[1]


def two_cliques(m=40, bridge=0.05):
    pairs = [(i, j) for c in (0, m) for i in range(c, c + m) for j in range(i + 1, c + m)] + [(m - 1, m), (0, m + 1)]
    i, j = np.array(pairs).T
    wt = np.ones(len(pairs), np.float32)
    wt[-2:] = bridge
    return csr_from_pairs(2 * m, i, j, wt)


def assert_same_init(u0, u_ref, bound):
    """u0 == u_ref within bound.  The sign convention (largest-magnitude entry
    positive) can only flip where the largest positive and the largest
    negative entry of the oracle's vector tie within the error bound (e.g. a
    symmetric graph); the unsupervised model is odd-symmetric in u, so u and
    -u are equally valid there."""
    err_same = np.abs(u0 - u_ref).max()
    err_flip = np.abs(u0 + u_ref).max()
    if err_same <= bound:
        return
    assert err_flip <= bound, (err_same, err_flip, bound)
    assert abs(u_ref.max() + u_ref.min()) <= 2 * bound, "sign flipped without a tie"


CASES = {
    "random500": lambda: random_graph(500, 6, seed=41),
    "random3000": lambda: random_graph(3000, 8, seed=42),
    "cliques": lambda: two_cliques(),
    "moons2k": lambda: (lambda wl: (wl.row_ptr, wl.col, wl.w))(make_workload("moons2k")),
}


def unsup_problem(B, rp, col, w, lap=0, precision=0, eps=100.0, c=11.0, **kw):
    n = rp.shape[0] - 1
    prm = B.make_params(eps=eps, eta=100.0, c=c, precond=B.PDCA_JACOBI_PERTURBED, laplacian=lap,
                        precision=precision, **kw)
    return B.Problem(rp, col, w, 1, np.zeros(n, np.uint8), np.zeros(n, np.int32), prm)


@pytest.mark.parametrize("lap", [0, 1])
@pytest.mark.parametrize("case", list(CASES))
def test_second_eigenpair(B, case, lap):
    rp, col, w = CASES[case]()
    lam_ref, v_ref = oracle.second_eigenpair(rp, col, w, lap)
    u_ref = oracle.spectral_init(v_ref)
    g = unsup_problem(B, rp, col, w, lap=lap)
    lam, u0, its = g.spectral_init(max_iters=3000, tol=TOL)
    print(f"{case} lap={lap}: lambda2 {lam:.8g} vs {lam_ref:.8g}, {its} iterations")
    assert abs(lam - lam_ref) <= 1e-5 + 1e-4 * abs(lam_ref)
    gap = gap_of(rp, col, w, lap)
    d, _ = oracle.degrees(rp, col, w)
    spec = 2.0 if lap == 0 else 2.0 * d.max()      # the residual tolerance is TOL x spec
    bound = max(10 * TOL * spec / gap if gap else 1e-3, 1e-5)
    assert_same_init(u0, u_ref, bound)
    # the iterate the handle holds is u0
    np.testing.assert_array_equal(g.get_u(), u0)


@pytest.mark.parametrize("lap", [0, 1])
def test_second_eigenpair_split_rows(B, lap):
    """Rows longer than 8 entries continue in the overflow CSR (forced split
    length): the block SpMM adds their pre-pass sums."""
    rp, col, w = random_graph(3000, 14, seed=43)
    lam_ref, v_ref = oracle.second_eigenpair(rp, col, w, lap)
    g = unsup_problem(B, rp, col, w, lap=lap, row_split=8)
    assert g.layout()["split_rows"] > 0
    lam, u0, its = g.spectral_init(max_iters=3000, tol=TOL)
    assert abs(lam - lam_ref) <= 1e-5 + 1e-4 * abs(lam_ref)
    gap = gap_of(rp, col, w, lap)
    d, _ = oracle.degrees(rp, col, w)
    spec = 2.0 if lap == 0 else 2.0 * d.max()
    assert_same_init(u0, oracle.spectral_init(v_ref), max(10 * TOL * spec / gap, 1e-5))


def test_two_cliques_unsupervised_split(B):
    """The unsupervised model started from u^0 separates two weakly joined
    cliques exactly."""
    rp, col, w = two_cliques()
    g = unsup_problem(B, rp, col, w)
    g.spectral_init(max_iters=1000, tol=TOL)
    g.solve(5, 4)
    lab = g.labels()
    assert len(set(lab[:40])) == 1 and len(set(lab[40:])) == 1 and lab[0] != lab[40]


@pytest.mark.parametrize("case", ["random3000", "moons2k"])
def test_unsupervised_run_parity(B, case):
    rp, col, w = CASES[case]()
    n = rp.shape[0] - 1
    lam_ref, v_ref = oracle.second_eigenpair(rp, col, w)
    u_ref = oracle.spectral_init(v_ref)
    g = unsup_problem(B, rp, col, w)
    _, u0, _ = g.spectral_init(max_iters=3000, tol=TOL)
    if np.abs(u0 + u_ref).max() < np.abs(u0 - u_ref).max():   # a sign tie (see assert_same_init)
        assert abs(u_ref.max() + u_ref.min()) <= 1e-3
        u_ref = -u_ref
    d0 = np.linalg.norm(u0 - u_ref) / np.linalg.norm(u_ref)
    ref = oracle.Problem(rp, col, w, 1, np.zeros(n, np.uint8), np.zeros(n, np.int32), 100.0, 100.0, 11.0,
                         precond=oracle.JACOBI_PERTURBED)
    g.solve(6, 4)
    u_end, e_ref, _ = ref.solve(6, 4, u_ref)
    d1 = np.linalg.norm(g.get_u() - u_end) / np.linalg.norm(u_end)
    print(f"{case}: init diff {d0:.2e}, after 6 x 4 sweeps {d1:.2e}")
    assert d1 <= 10 * d0 + 1e-5
    F, _ = g.energy()
    assert abs(F - e_ref[-1]) <= 1e-4 * abs(e_ref[-1])
    decided = np.abs(u_end) >= 1e-3
    assert np.all(g.labels()[decided] == (u_end[decided] >= 0))


def test_not_converged_still_sets_u0(B):
    rp, col, w = CASES["random500"]()
    g = unsup_problem(B, rp, col, w)
    with pytest.raises(B.PdcaError, match="NOT_CONVERGED"):
        g.spectral_init(max_iters=1, tol=1e-12)
    lam, u0, its = g.spectral_init(max_iters=1, tol=1e-12, strict=False)
    assert its == 1 and np.isfinite(lam) and np.abs(u0).max() == pytest.approx(1.0)
    np.testing.assert_array_equal(g.get_u(), u0)


def test_rejects_k_and_tiling(B):
    rp, col, w = CASES["random500"]()
    n = rp.shape[0] - 1
    prm = B.make_params(eps=1.0, eta=1.0, c=3.0)
    g = B.Problem(rp, col, w, 3, np.zeros(n, np.uint8), np.zeros(n, np.int32), prm)
    with pytest.raises(B.PdcaError, match="INVALID_ARG"):
        g.spectral_init()
    gt = B.Problem(rp, col, w, 1, np.zeros(n, np.uint8), np.zeros(n, np.int32), B.make_params(tiling=2))
    with pytest.raises(B.PdcaError, match="INVALID_ARG"):
        gt.spectral_init()


@pytest.mark.parametrize("precision", [1, 2])
def test_mixed_precision_operator(B, precision):
    """BF16 weights: the eigenpair of the BF16 operator, close to the FP32 one."""
    rp, col, w = CASES["random3000"]()
    lam_ref, v_ref = oracle.second_eigenpair(rp, col, w)
    g = unsup_problem(B, rp, col, w, precision=precision)
    lam, u0, _ = g.spectral_init(max_iters=3000, tol=TOL)
    assert abs(lam - lam_ref) <= 1e-2 * lam_ref
    assert_same_init(u0, oracle.spectral_init(v_ref), 0.05)


def test_ellipse_image_graph(B):
    """A 64 x 64 image graph (4 Ki nodes, window k-NN)."""
    wl = make_workload("ellipses256", size=64)
    lam_ref, v_ref = oracle.second_eigenpair(wl.row_ptr, wl.col, wl.w)
    g = unsup_problem(B, wl.row_ptr, wl.col, wl.w)
    lam, u0, its = g.spectral_init(max_iters=5000, tol=TOL, strict=False)
    print(f"ellipses64: lambda2 {lam:.6g} vs {lam_ref:.6g} after {its} iterations")
    assert abs(lam - lam_ref) <= 1e-5 + 1e-3 * lam_ref
