"""Pins of the oracle's second eigenpair of the graph Laplacian (the
initialisation of the unsupervised model): a closed form, a dense solve built
independently from the graph, the variational characterisation and the
cluster-splitting property."""

import numpy as np
import pytest

import oracle
from gen import csr_from_pairs, random_graph


def dense_W(rp, col, w):
    n = rp.shape[0] - 1
    W = np.zeros((n, n))
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            W[i, col[e]] = float(w[e])
    return W


@pytest.mark.parametrize("n", [5, 12, 40])
def test_path_closed_form_unnormalized(n):
    """Path with equal weights a: L = a (tridiagonal 1,2,...,2,1), whose
    eigenpairs are 2a (1 - cos(pi k / n)) and cos(pi k (i + 1/2) / n)."""
    a = 0.75
    i = np.arange(n - 1)
    rp, col, w = csr_from_pairs(n, i, i + 1, np.full(n - 1, a, np.float32))
    lam, v = oracle.second_eigenpair(rp, col, w, oracle.LAP_UNNORMALIZED)
    assert lam == pytest.approx(2 * a * (1 - np.cos(np.pi / n)), rel=1e-10)
    ref = np.cos(np.pi * (np.arange(n) + 0.5) / n)
    ref /= np.linalg.norm(ref)
    assert abs(abs(v @ ref) - 1.0) < 1e-10


@pytest.mark.parametrize("lap", [oracle.LAP_NORMALIZED, oracle.LAP_UNNORMALIZED])
def test_against_dense_eigh(lap):
    n = 60
    rp, col, w = random_graph(n, 5, seed=31)
    W = dense_W(rp, col, w)
    d = W.sum(1)
    M = np.eye(n) - W / np.sqrt(np.outer(d, d)) if lap == oracle.LAP_NORMALIZED else np.diag(d) - W
    ev, V = np.linalg.eigh(M)
    lam, v = oracle.second_eigenpair(rp, col, w, lap)
    assert lam == pytest.approx(ev[1], abs=1e-10)
    assert abs(abs(v @ V[:, 1]) - 1.0) < 1e-8
    # unit length, orthogonal to the null vector (D^1/2 1 or 1), eigen-residual
    q = np.sqrt(d) if lap == oracle.LAP_NORMALIZED else np.ones(n)
    assert abs(np.linalg.norm(v) - 1) < 1e-12
    assert abs(v @ q) / np.linalg.norm(q) < 1e-9
    assert np.linalg.norm(M @ v - lam * v) < 1e-9


def test_variational_bound():
    """lambda_2 = min of the Rayleigh quotient over vectors orthogonal to
    D^1/2 1: no random such vector goes below it."""
    n = 200
    rp, col, w = random_graph(n, 6, seed=32)
    d, _ = oracle.degrees(rp, col, w)
    lam, v = oracle.second_eigenpair(rp, col, w)
    q = np.sqrt(d) / np.linalg.norm(np.sqrt(d))
    rng = np.random.default_rng(0)
    for _ in range(100):
        x = rng.normal(size=n)
        x -= (x @ q) * q
        rq = x @ oracle.apply_Ls(rp, col, w, d, x) / (x @ x)
        assert rq >= lam - 1e-12
    assert v @ oracle.apply_Ls(rp, col, w, d, v) == pytest.approx(lam, abs=1e-12)


def test_two_cliques_split():
    """Two cliques joined by one weak edge: the sign of v_2 separates them,
    and the init u^0 lies in [-1, 1] with max |u| = 1 at a positive entry."""
    m = 15
    pairs = [(i, j) for c in (0, m) for i in range(c, c + m) for j in range(i + 1, c + m)] + [(m - 1, m)]
    i, j = np.array(pairs).T
    wt = np.ones(len(pairs), np.float32)
    wt[-1] = 0.01
    rp, col, w = csr_from_pairs(2 * m, i, j, wt)
    lam, v = oracle.second_eigenpair(rp, col, w)
    s = np.sign(v)
    assert np.all(s[:m] == s[0]) and np.all(s[m:] == -s[0])
    u0 = oracle.spectral_init(v)
    assert np.abs(u0).max() == 1.0 and u0[np.argmax(np.abs(u0))] == 1.0
    assert 0 < lam < 0.01


@pytest.mark.parametrize("lap", [oracle.LAP_NORMALIZED, oracle.LAP_UNNORMALIZED])
def test_disconnected_graph_closed_form(lap):
    """Two components A, B: 0 is a double eigenvalue; in the complement of
    the null vector the eigenvector is D^1/2 (vol_B 1_A - vol_A 1_B) for L_s
    (vol = sum of degrees) and |B| 1_A - |A| 1_B for L."""
    pairs = [(0, 1), (1, 2), (0, 2), (2, 3)] + [(4, 5), (5, 6), (6, 7), (7, 8), (4, 8)]
    i, j = np.array(pairs).T
    wt = np.array([1.0, 0.5, 2.0, 1.5, 1.0, 0.7, 1.2, 0.9, 1.1], np.float32)
    rp, col, w = csr_from_pairs(9, i, j, wt)
    d, _ = oracle.degrees(rp, col, w)
    A, Bm = np.arange(9) < 4, np.arange(9) >= 4
    if lap == oracle.LAP_NORMALIZED:
        ref = np.sqrt(d) * np.where(A, d[Bm].sum(), -d[A].sum())
    else:
        ref = np.where(A, Bm.sum(), -A.sum()).astype(float)
    ref /= np.linalg.norm(ref)
    lam, v = oracle.second_eigenpair(rp, col, w, lap)
    assert abs(lam) < 1e-10
    assert abs(abs(v @ ref) - 1.0) < 1e-10
