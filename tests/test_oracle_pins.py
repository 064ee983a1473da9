"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every check is a closed form, an
invariant, a brute-force computation on a tiny input or a direct dense solve
(numpy / scipy), chosen so that a dropped term, a wrong sign, a wrong index or
a transposed operand in the oracle fails at least one of them.
"""

import itertools
import math

import numpy as np
import pytest

import oracle
from gen import csr_from_pairs, random_graph


# ---------------------------------------------------------------------------
# small graphs with known spectra
# ---------------------------------------------------------------------------

def complete_graph(n, a=0.3):
    i, j = np.triu_indices(n, 1)
    return csr_from_pairs(n, i, j, np.full(i.size, a, np.float32))


def cycle_graph(n, a=0.7):
    i = np.arange(n)
    j = (i + 1) % n
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    return csr_from_pairs(n, lo, hi, np.full(n, a, np.float32))


def path_graph(n, seed=0):
    rng = np.random.default_rng(seed)
    i = np.arange(n - 1)
    return csr_from_pairs(n, i, i + 1, rng.uniform(0.2, 1.0, n - 1).astype(np.float32))


def dense_W(rp, col, w):
    n = rp.shape[0] - 1
    W = np.zeros((n, n))
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            W[i, col[e]] = float(w[e])
    return W


def dense_from_operator(apply, n, K=1):
    """Materialise a linear operator column by column (K = 1)."""
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = apply(e)
    return A


def mk(rp, col, w, K=1, mask=None, labels=None, **kw):
    n = rp.shape[0] - 1
    mask = np.zeros(n, np.uint8) if mask is None else mask
    labels = np.zeros(n, np.int32) if labels is None else labels
    args = dict(eps=1.0, eta=5.0, c=3.0)
    args.update(kw)
    return oracle.Problem(rp, col, w, K, mask, labels, **args)


# ---------------------------------------------------------------------------
# Laplacians (Sec. 2.2; Prop. diagonal:pre)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_complete_graph_spectrum(n):
    rp, col, w = complete_graph(n)
    d, bad = oracle.degrees(rp, col, w)
    assert bad == -1
    np.testing.assert_allclose(d, 0.3 * (n - 1), rtol=1e-7)
    Ls = dense_from_operator(lambda x: oracle.apply_Ls(rp, col, w, d, x), n)
    ev = np.sort(np.linalg.eigvalsh(0.5 * (Ls + Ls.T)))
    # normalized Laplacian of K_n: eigenvalues 0 and n/(n-1) (n-1 times)
    expect = np.array([0.0] + [n / (n - 1)] * (n - 1))
    np.testing.assert_allclose(ev, expect, atol=1e-12)


@pytest.mark.parametrize("n", [3, 4, 7, 10])
def test_cycle_spectrum(n):
    rp, col, w = cycle_graph(n)
    d, _ = oracle.degrees(rp, col, w)
    Ls = dense_from_operator(lambda x: oracle.apply_Ls(rp, col, w, d, x), n)
    ev = np.sort(np.linalg.eigvalsh(0.5 * (Ls + Ls.T)))
    expect = np.sort(1.0 - np.cos(2 * np.pi * np.arange(n) / n))
    np.testing.assert_allclose(ev, expect, atol=1e-12)
    # unnormalized: L = 2a I - a(P + P^T), eigenvalues 2a(1 - cos(2 pi j / n))
    L = dense_from_operator(lambda x: oracle.apply_L(rp, col, w, d, x), n)
    evL = np.sort(np.linalg.eigvalsh(0.5 * (L + L.T)))
    a = float(np.float32(0.7))
    np.testing.assert_allclose(evL, np.sort(2 * a * (1 - np.cos(2 * np.pi * np.arange(n) / n))), atol=1e-12)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_laplacian_invariants_random(seed):
    n = 23
    rp, col, w = random_graph(n, 4, seed)
    d, bad = oracle.degrees(rp, col, w)
    assert bad == -1
    W = dense_W(rp, col, w)
    np.testing.assert_allclose(d, W.sum(axis=1), rtol=1e-15)
    Ls = dense_from_operator(lambda x: oracle.apply_Ls(rp, col, w, d, x), n)
    L = dense_from_operator(lambda x: oracle.apply_L(rp, col, w, d, x), n)
    # symmetry
    np.testing.assert_allclose(Ls, Ls.T, atol=1e-15)
    np.testing.assert_allclose(L, L.T, atol=1e-15)
    # null vectors: L 1 = 0, L_s D^{1/2} 1 = 0
    np.testing.assert_allclose(L @ np.ones(n), 0.0, atol=1e-12)
    np.testing.assert_allclose(Ls @ np.sqrt(d), 0.0, atol=1e-12)
    # unit diagonal of L_s, diagonal d of L, off-diagonals -w and -w/sqrt(d_i d_j)
    np.testing.assert_allclose(np.diag(Ls), 1.0, atol=0)
    np.testing.assert_allclose(np.diag(L), d, atol=0)
    off = ~np.eye(n, dtype=bool)
    np.testing.assert_allclose(L[off], -W[off], atol=0)
    # spectra: 0 <= L_s <= 2I and 0 <= L <= 2D (Prop. diagonal:pre)
    ev = np.linalg.eigvalsh(Ls)
    assert ev.min() > -1e-12 and ev.max() < 2 + 1e-12
    assert np.linalg.eigvalsh(L).min() > -1e-12
    assert np.linalg.eigvalsh(2 * np.diag(d) - L).min() > -1e-12
    # <u, L u> = 1/2 sum_ij w_ij (u_i - u_j)^2 (Sec. 2.1), brute force
    u = np.random.default_rng(seed).normal(size=n)
    brute = 0.5 * sum(W[i, j] * (u[i] - u[j]) ** 2 for i in range(n) for j in range(n))
    assert abs(u @ oracle.apply_L(rp, col, w, d, u) - brute) < 1e-12 * max(1, brute)
    x = u / np.sqrt(d)
    brute_s = 0.5 * sum(W[i, j] * (x[i] - x[j]) ** 2 for i in range(n) for j in range(n))
    assert abs(u @ oracle.apply_Ls(rp, col, w, d, u) - brute_s) < 1e-12 * max(1, brute_s)


def test_isolated_node_detected():
    rp, col, w = csr_from_pairs(4, np.array([0, 1]), np.array([1, 2]), np.ones(2, np.float32))
    _, bad = oracle.degrees(rp, col, w)
    assert bad == 3


def test_multi_column_is_columnwise():
    n, K = 17, 3
    rp, col, w = random_graph(n, 4, 7)
    d, _ = oracle.degrees(rp, col, w)
    X = np.random.default_rng(0).normal(size=(n, K))
    Y = oracle.apply_Ls(rp, col, w, d, X)
    for k in range(K):
        np.testing.assert_array_equal(Y[:, k], oracle.apply_Ls(rp, col, w, d, X[:, k].copy()))


# ---------------------------------------------------------------------------
# Preconditioners: feasibility G > T (Sec. 3.1)
# ---------------------------------------------------------------------------

def dense_T(P):
    n = P.n
    return dense_from_operator(lambda x: P.apply_T(x), n)


@pytest.mark.parametrize("lap", [oracle.LAP_NORMALIZED, oracle.LAP_UNNORMALIZED])
def test_preconditioner_margins_bipartite(lap):
    """On a bipartite graph lambda_max(L_s) = 2 and D + W is singular, so the
    margins of Sec. 3.1 are attained exactly: G_Jp - T and G_R - T have
    smallest eigenvalue delta0, G_Jd(omega=1/2) - T has smallest eigenvalue c
    when no node is labelled."""
    n = 10
    rp, col, w = path_graph(n)
    d, _ = oracle.degrees(rp, col, w)
    delta0 = 1e-3
    W = dense_W(rp, col, w)
    L = np.diag(d) - W
    lam = 2.0 if lap == oracle.LAP_NORMALIZED else np.linalg.eigvalsh(L).max()
    for pc, margin in [(oracle.JACOBI_PERTURBED, delta0), (oracle.RICHARDSON, delta0),
                       (oracle.JACOBI_DAMPED, 3.0)]:
        P = mk(rp, col, w, eps=1.7, eta=5.0, c=3.0, precond=pc, damping=0.5, delta0=delta0,
               lambda_max=lam, laplacian=lap)
        G = np.diag(P.precond_diag())
        T = dense_T(P)
        np.testing.assert_allclose(T, T.T, atol=1e-13)
        emin = np.linalg.eigvalsh(G - T).min()
        assert abs(emin - margin) < 1e-9, (pc, emin, margin)


def test_preconditioner_values_with_labels():
    n = 9
    rp, col, w = random_graph(n, 3, 5)
    mask = np.zeros(n, np.uint8)
    mask[[1, 4]] = 1
    eps, eta, c, delta0, om, lam = 2.0, 7.0, 11.0, 1e-6, 0.8, 1.9
    for pc, expect in [
        (oracle.JACOBI_DAMPED, lambda lab: (eps + c + eta * lab) / om),
        (oracle.JACOBI_PERTURBED, lambda lab: 2 * eps + c + delta0 + eta * lab),
        (oracle.RICHARDSON, lambda lab: eps * lam + c + delta0 + eta * lab),
    ]:
        P = mk(rp, col, w, mask=mask, eps=eps, eta=eta, c=c, precond=pc, damping=om,
               delta0=delta0, lambda_max=lam)
        g = P.precond_diag()
        np.testing.assert_allclose(g, [expect(float(m)) for m in mask], rtol=1e-15)
        # the diagonal of T for L_s is eps + c + eta*Lambda_i
        np.testing.assert_allclose(np.diag(dense_T(P)), eps + c + eta * mask, rtol=1e-15)


@pytest.mark.parametrize("omega", [0.5, 0.6, 0.8])
def test_damped_jacobi_feasibility_rule(omega):
    """G = diag(T)/omega is feasible (G > T) for every graph iff
    c > eps (2 omega - 1)/(1 - omega); at the bound a bipartite graph makes
    G - T singular."""
    n = 8
    rp, col, w = path_graph(n, 3)
    eps = 1.0
    cb = eps * (2 * omega - 1) / (1 - omega)
    for c, ok in [(cb + 0.05, True), (max(cb - 0.05, 0.0) if cb > 0.05 else None, False)]:
        if c is None:
            continue
        P = mk(rp, col, w, eps=eps, eta=3.0, c=c, precond=oracle.JACOBI_DAMPED, damping=omega)
        emin = np.linalg.eigvalsh(np.diag(P.precond_diag()) - dense_T(P)).min()
        assert (emin > 0) == ok, (c, emin)


# ---------------------------------------------------------------------------
# The DCA step: fixed point of the sweeps = exact solve (eq. dca:linear:system:ori)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("pc", [oracle.JACOBI_DAMPED, oracle.JACOBI_PERTURBED, oracle.RICHARDSON])
@pytest.mark.parametrize("lap", [oracle.LAP_NORMALIZED, oracle.LAP_UNNORMALIZED])
def test_sweeps_converge_to_direct_solve(pc, lap):
    n = 30
    rp, col, w = random_graph(n, 5, 11)
    rng = np.random.default_rng(3)
    mask = (rng.uniform(size=n) < 0.3).astype(np.uint8)
    labels = rng.integers(0, 2, size=n).astype(np.int32)
    W = dense_W(rp, col, w)
    d = W.sum(1)
    if lap == oracle.LAP_NORMALIZED:
        Lap = np.eye(n) - W / np.sqrt(np.outer(d, d))
    else:
        Lap = np.diag(d) - W
    lam = np.linalg.eigvalsh(Lap).max()
    eps, eta, c = 1.3, 4.0, 5.0
    P = mk(rp, col, w, mask=mask, labels=labels, eps=eps, eta=eta, c=c, precond=pc,
           damping=0.8, delta0=1e-6, lambda_max=lam, laplacian=lap)
    y = np.where(mask == 1, 2.0 * labels - 1.0, 0.0)
    u = rng.uniform(-1, 1, size=n)
    b = P.rhs(u)
    # b^t = eta Lambda y + c u - (u^3 - u)/eps
    np.testing.assert_allclose(b, eta * mask * y + c * u - (u ** 3 - u) / eps, rtol=1e-14, atol=1e-14)
    T = eps * Lap + eta * np.diag(mask.astype(float)) + c * np.eye(n)
    exact = np.linalg.solve(T, b)
    g = P.precond_diag()
    v = u.copy()
    for _ in range(4000):
        v = P.sweep(g, b, v)
    np.testing.assert_allclose(v, exact, rtol=0, atol=1e-10)
    # one sweep is u + G^{-1}(b - T u)
    np.testing.assert_allclose(P.sweep(g, b, u), u + (b - T @ u) / g, atol=1e-13)
    # and the residual the oracle reports is ||b - T v|| / ||b||
    assert abs(P.residual(b, u) - np.linalg.norm(b - T @ u) / np.linalg.norm(b)) < 1e-13


def test_rhs_hand_values():
    """b for single nodes at hand-computed points (eps=1, c=2, eta=3)."""
    rp, col, w = csr_from_pairs(2, np.array([0]), np.array([1]), np.ones(1, np.float32))
    P = mk(rp, col, w, mask=np.array([1, 0], np.uint8), labels=np.array([1, 0], np.int32),
           eps=1.0, eta=3.0, c=2.0)
    # node 0 labelled +1, u = 0.5: 3*1 + 2*0.5 - (0.125 - 0.5) = 4.375
    # node 1 unlabelled, u = -1: 2*(-1) - (-1 + 1) = -2
    np.testing.assert_allclose(P.rhs(np.array([0.5, -1.0])), [4.375, -2.0], rtol=1e-15)


# ---------------------------------------------------------------------------
# Energy F(u) (eqs. gl:functional:graph and functional:GL, 1/2-reading)
# ---------------------------------------------------------------------------

def test_energy_special_values():
    n = 12
    rp, col, w = random_graph(n, 3, 2)
    mask = np.zeros(n, np.uint8)
    mask[:4] = 1
    labels = np.array([1, 0, 1, 0] + [0] * 8, np.int32)
    eps, eta = 0.7, 3.0
    P = mk(rp, col, w, mask=mask, labels=labels, eps=eps, eta=eta, c=1.0)
    d = dense_W(rp, col, w).sum(1)
    # u = 0: Laplacian and fidelity contribute (eta/2)*4, the double well n/(4 eps)
    assert abs(P.energy(np.zeros(n)) - (n / (4 * eps) + 0.5 * eta * 4)) < 1e-12
    # u = prior on labelled, constant-in-D^{1/2} +-1 impossible; use u in {+-1}
    u = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    u[:4] = [1, -1, 1, -1]
    W = dense_W(rp, col, w)
    x = u / np.sqrt(d)
    quad = 0.5 * sum(W[i, j] * (x[i] - x[j]) ** 2 for i in range(n) for j in range(n))
    assert abs(P.energy(u) - 0.5 * eps * quad) < 1e-12
    # u = D^{1/2} 1 / scale lies in the null space of L_s: only well + fidelity
    v = np.sqrt(d) / np.sqrt(d).max()
    well = np.sum((v ** 2 - 1) ** 2) / (4 * eps)
    y = np.array([1, -1, 1, -1], float)
    fid = 0.5 * eta * np.sum((v[:4] - y) ** 2)
    assert abs(P.energy(v) - (well + fid)) < 1e-12


def test_energy_monotone_binary():
    """Thm. decay:energy: F(u^{t+1}) <= F(u^t) for pDCA with feasible sweeps
    while P_2 is convex on the iterates (c >= (3 u^2 - 1)/eps)."""
    from gen import make_workload
    wl = make_workload("moons2k", n=400, cache=False)
    p = wl.params
    P = oracle.Problem(wl.row_ptr, wl.col, wl.w, 1, wl.fid_mask, wl.fid_labels,
                       p["eps"], p["eta"], p["c"], precond=p["precond"], damping=p["damping"])
    u0 = P.init_u()
    u, e, r = P.solve(15, 3, u0)
    f0 = P.energy(u0)
    seq = np.concatenate([[f0], e])
    assert np.all(np.diff(seq) <= 1e-12 * np.abs(seq[:-1])), seq
    # convexity of P_2 held along the run
    assert (3 * max(np.abs(u).max(), 1.0) ** 2 - 1) / p["eps"] <= p["c"]


@pytest.mark.parametrize("pc", [oracle.JACOBI_PERTURBED, oracle.RICHARDSON])
def test_energy_monotone_paper_setting(pc):
    """eps=100, c=11, eta=100 (the paper's image setting) with 4 sweeps."""
    n = 60
    rp, col, w = random_graph(n, 6, 4)
    rng = np.random.default_rng(9)
    mask = (rng.uniform(size=n) < 0.2).astype(np.uint8)
    labels = rng.integers(0, 2, size=n).astype(np.int32)
    P = mk(rp, col, w, mask=mask, labels=labels, eps=100.0, eta=100.0, c=11.0, precond=pc,
           lambda_max=2.0)
    u0 = P.init_u()
    u, e, _ = P.solve(30, 4, u0)
    seq = np.concatenate([[P.energy(u0)], e])
    assert np.all(np.diff(seq) <= 1e-12 * np.abs(seq[:-1]))
    assert (3 * max(np.abs(u).max(), 1.0) ** 2 - 1) / 100.0 <= 11.0


def test_stationarity_at_convergence():
    """After many exact-ish DCA steps, grad F(u) = eps L_s u + (u^3-u)/eps
    + eta Lambda (u - y) vanishes."""
    n = 40
    rp, col, w = random_graph(n, 5, 21)
    rng = np.random.default_rng(4)
    mask = (rng.uniform(size=n) < 0.25).astype(np.uint8)
    labels = rng.integers(0, 2, size=n).astype(np.int32)
    eps, eta, c = 0.5, 4.0, 8.0
    P = mk(rp, col, w, mask=mask, labels=labels, eps=eps, eta=eta, c=c,
           precond=oracle.JACOBI_PERTURBED)
    u, e, _ = P.solve(400, 20)
    W = dense_W(rp, col, w)
    d = W.sum(1)
    Ls = np.eye(n) - W / np.sqrt(np.outer(d, d))
    y = np.where(mask == 1, 2.0 * labels - 1.0, 0.0)
    grad = eps * Ls @ u + (u ** 3 - u) / eps + eta * mask * (u - y)
    assert np.abs(grad).max() < 1e-9


# ---------------------------------------------------------------------------
# Simplex projection (multi-class extension)
# ---------------------------------------------------------------------------

def brute_simplex(x):
    """Euclidean projection onto {v >= 0, sum v = 1} by enumerating supports."""
    K = x.size
    best, bestv = np.inf, None
    for r in range(1, K + 1):
        for S in itertools.combinations(range(K), r):
            S = list(S)
            theta = (x[S].sum() - 1.0) / len(S)
            v = np.zeros(K)
            v[S] = x[S] - theta
            if np.all(v[S] >= -1e-15):
                f = np.sum((v - x) ** 2)
                if f < best:
                    best, bestv = f, v
    return bestv


@pytest.mark.parametrize("K", [2, 3, 4, 5, 6])
def test_projection_brute_force(K):
    rng = np.random.default_rng(K)
    U = rng.normal(0, 1.2, size=(200, K))
    P = oracle.project_rows(U)
    for r in range(U.shape[0]):
        v = brute_simplex(0.5 * (U[r] + 1.0))
        np.testing.assert_allclose(0.5 * (P[r] + 1.0), v, atol=1e-13)


def test_projection_special_rows():
    K = 10
    # a constant row maps to the uniform point
    P = oracle.project_rows(np.full((3, K), 0.37))
    np.testing.assert_allclose(P, 2.0 / K - 1.0, atol=1e-15)
    # points already on the simplex are fixed (idempotence)
    rng = np.random.default_rng(0)
    V = rng.dirichlet(np.ones(K), size=50)
    U = 2 * V - 1
    np.testing.assert_allclose(oracle.project_rows(U), U, atol=1e-14)
    Q = oracle.project_rows(rng.normal(size=(50, K)))
    np.testing.assert_allclose(oracle.project_rows(Q), Q, atol=1e-14)
    np.testing.assert_allclose((0.5 * (Q + 1)).sum(1), 1.0, atol=1e-13)
    assert (0.5 * (Q + 1)).min() >= 0


def test_two_class_matches_binary_with_clipping():
    """K = 2 in the +-1 coding keeps u_0 = -u_1; projection then only clips to
    [-1, 1].  So the K = 2 run equals the binary run of column 1 with a clip
    after each outer step."""
    n = 50
    rp, col, w = random_graph(n, 5, 8)
    rng = np.random.default_rng(2)
    mask = (rng.uniform(size=n) < 0.3).astype(np.uint8)
    labels = rng.integers(0, 2, size=n).astype(np.int32)
    kw = dict(eps=1.0, eta=6.0, c=4.0, precond=oracle.JACOBI_PERTURBED)
    P2 = mk(rp, col, w, K=2, mask=mask, labels=labels, **kw)
    P1 = mk(rp, col, w, K=1, mask=mask, labels=labels, **kw)
    u2, _, _ = P2.solve(6, 3)
    u1 = P1.init_u()
    for _ in range(6):
        u1, _, _ = P1.solve(1, 3, u1)
        u1 = np.clip(u1, -1.0, 1.0)
    np.testing.assert_allclose(u2[:, 1], u1, atol=1e-12)
    np.testing.assert_allclose(u2[:, 0], -u1, atol=1e-12)


def test_labels_rule():
    rp, col, w = complete_graph(4)
    P = mk(rp, col, w, K=3)
    u = np.array([[0.1, 0.1, -1], [-1, 0.2, 0.2], [0.3, -0.2, 0.3], [-1, -1, 0]])
    np.testing.assert_array_equal(P.labels_of(u), [0, 1, 0, 2])
    P1 = mk(rp, col, w, K=1)
    np.testing.assert_array_equal(P1.labels_of(np.array([0.0, -1e-9, 2.0, -3.0])), [1, 0, 1, 0])


def test_init_u():
    rp, col, w = complete_graph(3)
    mask = np.array([1, 0, 1], np.uint8)
    labels = np.array([2, 0, 0], np.int32)
    P = mk(rp, col, w, K=4, mask=mask, labels=labels)
    np.testing.assert_allclose(P.init_u(), [[-1, -1, 1, -1], [-0.5] * 4, [1, -1, -1, -1]])
    P1 = mk(rp, col, w, K=1, mask=mask, labels=np.array([1, 0, 0], np.int32))
    np.testing.assert_allclose(P1.init_u(), [1, 0, -1])


# ---------------------------------------------------------------------------
# Power method for lambda_max (Sec. 3.1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("graph,expect", [
    (lambda: complete_graph(2), 2.0),
    (lambda: complete_graph(6), 6 / 5),
    (lambda: cycle_graph(7), 1 - math.cos(2 * math.pi * 3 / 7)),
    (lambda: cycle_graph(8), 2.0),
    (lambda: path_graph(9), 2.0),
])
def test_power_method_closed_forms(graph, expect):
    rp, col, w = graph()
    P = mk(rp, col, w)
    assert abs(P.power_max_eig(3000) - expect) < 1e-9


def test_power_method_random_vs_eigvalsh():
    n = 40
    rp, col, w = random_graph(n, 6, 13)
    W = dense_W(rp, col, w)
    d = W.sum(1)
    Ls = np.eye(n) - W / np.sqrt(np.outer(d, d))
    P = mk(rp, col, w)
    assert abs(P.power_max_eig(5000) - np.linalg.eigvalsh(Ls).max()) < 1e-8
    # unnormalized Laplacian, bound 2 max d
    P.s.laplacian = oracle.LAP_UNNORMALIZED
    lam = P.power_max_eig(5000)
    assert abs(lam - np.linalg.eigvalsh(np.diag(d) - W).max()) < 1e-8
    assert lam <= 2 * d.max()


def test_omp_build_is_bit_identical():
    from gen import make_workload
    wl = make_workload("moons2k", n=300, cache=False)
    p = wl.params
    args = (wl.row_ptr, wl.col, wl.w, 1, wl.fid_mask, wl.fid_labels, p["eps"], p["eta"], p["c"])
    a = oracle.Problem(*args, precond=p["precond"], damping=p["damping"]).solve(3, 5)
    b = oracle.Problem(*args, precond=p["precond"], damping=p["damping"], omp=True).solve(3, 5)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
