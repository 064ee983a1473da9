"""Pins of the oracle's finite step size k (Lemma preconditioned_DCA:stepsize,
eqs. btk:utk, pre:unnorm:jacob:richard:k, pre:norm:jacob:richard:k) and of the
unnormalized Laplacian's damped-Jacobi feasibility rule.

Every expected value is a closed form, a dense numpy solve, a finite
difference of the (separately pinned) energy or an eigenvalue bound.
"""

import numpy as np
import pytest

import oracle
from gen import csr_from_pairs, random_graph

PCS = [oracle.JACOBI_DAMPED, oracle.JACOBI_PERTURBED, oracle.RICHARDSON]
LAPS = [oracle.LAP_NORMALIZED, oracle.LAP_UNNORMALIZED]


def dense_W(rp, col, w):
    n = rp.shape[0] - 1
    W = np.zeros((n, n))
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            W[i, col[e]] = float(w[e])
    return W


def dense_lap(rp, col, w, lap):
    W = dense_W(rp, col, w)
    d = W.sum(1)
    if lap == oracle.LAP_NORMALIZED:
        return np.eye(len(d)) - W / np.sqrt(np.outer(d, d))
    return np.diag(d) - W


def path_graph(n, seed=0):
    rng = np.random.default_rng(seed)
    i = np.arange(n - 1)
    return csr_from_pairs(n, i, i + 1, rng.uniform(0.2, 1.0, n - 1).astype(np.float32))


def cycle_graph(n, a):
    i = np.arange(n)
    j = (i + 1) % n
    return csr_from_pairs(n, np.minimum(i, j), np.maximum(i, j), np.full(n, a, np.float32))


def materialise(apply, n):
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = apply(e)
    return A


def problem(rp, col, w, mask=None, labels=None, **kw):
    n = rp.shape[0] - 1
    mask = np.zeros(n, np.uint8) if mask is None else mask
    labels = np.zeros(n, np.int32) if labels is None else labels
    args = dict(eps=1.0, eta=5.0, c=3.0)
    args.update(kw)
    return oracle.Problem(rp, col, w, 1, mask, labels, **args)


@pytest.mark.parametrize("lap", LAPS)
@pytest.mark.parametrize("k", [0.01, 0.1, 1.0, 5.0])
def test_step_preconditioners_margins_bipartite(lap, k):
    """On a bipartite graph 2D - L = D + W (or 2I - L_s) is singular and
    lambda_max is attained, so the margins of G_k - T_k are exact:
    delta0 for G_Jp,k and G_R,k, and 1 + k c for G_Jd,k = 2 diag(T_k) with no
    labelled node.  T_k itself must be I + k T."""
    n = 10
    rp, col, w = path_graph(n, 2)
    Lap = dense_lap(rp, col, w, lap)
    lam = np.linalg.eigvalsh(Lap).max()
    eps, eta, c, delta0 = 1.7, 5.0, 3.0, 1e-3
    for pc, margin in [(oracle.JACOBI_PERTURBED, delta0), (oracle.RICHARDSON, delta0),
                       (oracle.JACOBI_DAMPED, 1.0 + k * c)]:
        P = problem(rp, col, w, eps=eps, eta=eta, c=c, precond=pc, damping=0.5, delta0=delta0,
                    lambda_max=lam, laplacian=lap, step_k=k)
        Tk = materialise(P.apply_system, n)
        np.testing.assert_allclose(Tk, np.eye(n) + k * (eps * Lap + c * np.eye(n)), rtol=0, atol=1e-12)
        G = np.diag(P.precond_diag())
        emin = np.linalg.eigvalsh(G - Tk).min()
        assert abs(emin - margin) < 1e-9 * max(1.0, k), (pc, emin, margin)


@pytest.mark.parametrize("lap", LAPS)
def test_step_preconditioner_values(lap):
    """G_k per row against the printed forms with hand-chosen numbers."""
    n = 7
    rp, col, w = random_graph(n, 3, 8)
    d = dense_W(rp, col, w).sum(1)
    a = np.ones(n) if lap == oracle.LAP_NORMALIZED else d
    mask = np.zeros(n, np.uint8)
    mask[[0, 5]] = 1
    eps, eta, c, delta0, om, lam, k = 2.0, 7.0, 11.0, 1e-6, 0.8, 1.9, 0.3
    lab = mask.astype(float)
    for pc, expect in [
        (oracle.JACOBI_DAMPED, (1 + k * (eps * a + c + eta * lab)) / om),
        (oracle.JACOBI_PERTURBED, 1 + k * (2 * eps * a + eta * lab + c) + delta0),
        (oracle.RICHARDSON, 1 + k * (eps * lam + eta * lab + c) + delta0),
    ]:
        P = problem(rp, col, w, mask=mask, eps=eps, eta=eta, c=c, precond=pc, damping=om,
                    delta0=delta0, lambda_max=lam, laplacian=lap, step_k=k)
        np.testing.assert_allclose(P.precond_diag(), expect, rtol=1e-15)


@pytest.mark.parametrize("pc", PCS)
@pytest.mark.parametrize("lap", LAPS)
def test_step_sweeps_converge_to_direct_solve(pc, lap):
    """The sweeps' fixed point is the solution of T_k u = b_k^t
    (eq. orig:equation:with:k), b_k^t = u^t + k b^t."""
    n = 30
    rp, col, w = random_graph(n, 5, 12)
    rng = np.random.default_rng(5)
    mask = (rng.uniform(size=n) < 0.3).astype(np.uint8)
    labels = rng.integers(0, 2, size=n).astype(np.int32)
    Lap = dense_lap(rp, col, w, lap)
    lam = np.linalg.eigvalsh(Lap).max()
    eps, eta, c, k = 1.3, 4.0, 5.0, 0.4
    P = problem(rp, col, w, mask=mask, labels=labels, eps=eps, eta=eta, c=c, precond=pc, damping=0.8,
                delta0=1e-6, lambda_max=lam, laplacian=lap, step_k=k)
    y = np.where(mask == 1, 2.0 * labels - 1.0, 0.0)
    u = rng.uniform(-1, 1, size=n)
    b = eta * mask * y + c * u - (u ** 3 - u) / eps
    bk = P.rhs(u)
    np.testing.assert_allclose(bk, u + k * b, rtol=1e-14, atol=1e-14)
    Tk = np.eye(n) + k * (eps * Lap + eta * np.diag(mask.astype(float)) + c * np.eye(n))
    exact = np.linalg.solve(Tk, bk)
    g = P.precond_diag()
    v = u.copy()
    for _ in range(3000):
        v = P.sweep(g, bk, v)
    np.testing.assert_allclose(v, exact, rtol=0, atol=1e-11)
    assert abs(P.residual(bk, u) - np.linalg.norm(bk - Tk @ u) / np.linalg.norm(bk)) < 1e-13


@pytest.mark.parametrize("pc", PCS)
@pytest.mark.parametrize("lap", LAPS)
def test_step_to_infinity(pc, lap):
    """Prop. k:infinity: with kappa = k -> infinity the preconditioned step
    with step size k tends to the infinite-step-size step."""
    n = 50
    rp, col, w = random_graph(n, 6, 13)
    rng = np.random.default_rng(6)
    mask = (rng.uniform(size=n) < 0.2).astype(np.uint8)
    labels = rng.integers(0, 2, size=n).astype(np.int32)
    lam = np.linalg.eigvalsh(dense_lap(rp, col, w, lap)).max()
    kw = dict(mask=mask, labels=labels, eps=1.0, eta=20.0, c=40.0, precond=pc, damping=0.7,
              delta0=1e-6, lambda_max=lam, laplacian=lap)
    u_inf, _, _ = problem(rp, col, w, **kw).solve(4, 5)
    errs = []
    for k in (1e2, 1e4, 1e6):
        u_k, _, _ = problem(rp, col, w, step_k=k, **kw).solve(4, 5)
        errs.append(np.linalg.norm(u_k - u_inf) / np.linalg.norm(u_inf))
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 1e-5, errs


@pytest.mark.parametrize("pc", PCS)
@pytest.mark.parametrize("lap", LAPS)
def test_small_step_is_gradient_flow(pc, lap):
    """k -> 0: one outer step moves u by k times the preconditioned steepest
    descent direction, (u^1 - u^0)/k -> -s grad F(u^0) with s = 1 for G_Jp,k and
    G_R,k (G_k -> (1 + delta0) I) and s = 1 - (1 - omega)^m for G_Jd,k after m
    sweeps (G_k -> I/omega).  grad F comes from central differences of the
    energy F."""
    n = 24
    rp, col, w = random_graph(n, 4, 14)
    rng = np.random.default_rng(7)
    mask = (rng.uniform(size=n) < 0.3).astype(np.uint8)
    labels = rng.integers(0, 2, size=n).astype(np.int32)
    om, m, k = 0.7, 3, 1e-7
    lam = np.linalg.eigvalsh(dense_lap(rp, col, w, lap)).max()
    P = problem(rp, col, w, mask=mask, labels=labels, eps=0.8, eta=3.0, c=4.0, precond=pc, damping=om,
                delta0=1e-9, lambda_max=lam, laplacian=lap, step_k=k)
    u0 = rng.uniform(-0.9, 0.9, size=n)
    u1, _, _ = P.solve(1, m, u0)
    h = 1e-4
    grad = np.array([(P.energy(u0 + h * e) - P.energy(u0 - h * e)) / (2 * h) for e in np.eye(n)])
    s = 1.0 - (1.0 - om) ** m if pc == oracle.JACOBI_DAMPED else 1.0
    np.testing.assert_allclose((u1 - u0) / k, -s * grad, rtol=0, atol=2e-5 * np.abs(grad).max())


@pytest.mark.parametrize("pc", PCS)
@pytest.mark.parametrize("k", [0.01, 0.1, 1.0, 5.0])
def test_energy_monotone_finite_step(pc, k):
    """Thm. decay:energy with a step size: the energy decreases for every
    k > 0 while P_2 stays convex on the iterates."""
    n = 80
    rp, col, w = random_graph(n, 6, 15)
    rng = np.random.default_rng(8)
    mask = (rng.uniform(size=n) < 0.2).astype(np.uint8)
    labels = rng.integers(0, 2, size=n).astype(np.int32)
    P = problem(rp, col, w, mask=mask, labels=labels, eps=1.0, eta=30.0, c=32.0, precond=pc, damping=0.8,
                lambda_max=2.0, step_k=k)
    u0 = P.init_u()
    u, e, _ = P.solve(20, 3, u0)
    seq = np.concatenate([[P.energy(u0)], e])
    assert np.all(np.diff(seq) <= 1e-12 * np.abs(seq[:-1])), seq
    assert seq[-1] < seq[0]
    assert 3 * max(np.abs(u).max(), 1.0) ** 2 - 1 <= 32.0


@pytest.mark.parametrize("pc", PCS)
@pytest.mark.parametrize("lap", LAPS)
def test_step_equals_shifted_infinite_step(pc, lap):
    """The algebra the CUDA path uses for a finite k: dividing T_k, b_k^t and
    G_k by k gives the infinite-step system with c + 1/k in place of c and
    delta0/k in place of delta0, so both iterations coincide."""
    n = 40
    rp, col, w = random_graph(n, 5, 16)
    rng = np.random.default_rng(9)
    mask = (rng.uniform(size=n) < 0.25).astype(np.uint8)
    labels = rng.integers(0, 2, size=n).astype(np.int32)
    k, c, delta0 = 0.05, 6.0, 1e-3
    kw = dict(mask=mask, labels=labels, eps=1.2, eta=8.0, precond=pc, damping=0.75, lambda_max=1.95,
              laplacian=lap)
    a, ea, _ = problem(rp, col, w, c=c, delta0=delta0, step_k=k, **kw).solve(5, 4)
    b, eb, _ = problem(rp, col, w, c=c + 1.0 / k, delta0=delta0 / k, **kw).solve(5, 4)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)
    np.testing.assert_allclose(ea, eb, rtol=1e-12)


@pytest.mark.parametrize("omega", [0.6, 0.8])
def test_unnormalized_damped_jacobi_feasibility_rule(omega):
    """For L = D - W, G = diag(T)/omega satisfies G - T >= eps (1/omega - 2) D
    + (1/omega - 1)(c + eta Lambda) (since W >= -D), so
    c > eps max_i d_i (2 omega - 1)/(1 - omega) is feasible on every graph; on
    a regular bipartite graph (even cycle) the bound is attained."""
    n, a, eps = 8, 0.6, 1.0
    rp, col, w = cycle_graph(n, a)
    cb = eps * 2 * a * (2 * omega - 1) / (1 - omega)
    for c, ok in [(cb + 0.05, True), (cb - 0.05, False)]:
        P = problem(rp, col, w, eps=eps, eta=3.0, c=c, precond=oracle.JACOBI_DAMPED, damping=omega,
                    laplacian=oracle.LAP_UNNORMALIZED)
        T = materialise(P.apply_T, n)
        emin = np.linalg.eigvalsh(np.diag(P.precond_diag()) - T).min()
        assert (emin > 0) == ok, (c, emin)
    rp, col, w = random_graph(40, 6, 17)
    dmax = dense_W(rp, col, w).sum(1).max()
    P = problem(rp, col, w, eps=eps, eta=3.0, c=eps * dmax * (2 * omega - 1) / (1 - omega) + 1e-3,
                precond=oracle.JACOBI_DAMPED, damping=omega, laplacian=oracle.LAP_UNNORMALIZED)
    T = materialise(P.apply_T, 40)
    assert np.linalg.eigvalsh(np.diag(P.precond_diag()) - T).min() > 0
