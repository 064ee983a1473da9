"""Pins of the oracle's point-cloud k-NN graph with local scaling: a 1-D
lattice worked by hand, pair-by-pair brute force, separated clusters, and the
structural invariants."""

import numpy as np
import pytest

from oracle import point_graph as PG


def test_lattice_by_hand():
    """Points 0, 1, 2, ..., 9 on a line, k = 2, m = 2: inner points keep both
    unit neighbours; the ends keep distance 1 and 2; ties (left and right at
    equal distance) go to the lower index."""
    X = np.arange(10, dtype=np.float32)[:, None]
    nbr, d2, _ = PG.knn(X, 2)
    assert list(nbr[0]) == [1, 2] and list(d2[0]) == [1.0, 4.0]
    assert list(nbr[5]) == [4, 6] and list(d2[5]) == [1.0, 1.0]
    rp, col, w, sigma = PG.point_graph(X, 3, 2)
    # k = 3 at point 5: 4 and 6 (d2 1), then 3 (d2 4, lower than 7); sigma_5 = 1
    assert sigma[5] == 1.0 and sigma[0] == 2.0
    row5 = dict(zip(col[rp[5]:rp[5 + 1]], w[rp[5]:rp[5 + 1]]))
    assert set(row5) >= {3, 4, 6}
    assert row5[4] == np.float32(np.exp(-1.0 / (sigma[5] * sigma[4])))


@pytest.mark.parametrize("n,d,k,m", [(40, 3, 5, 3), (60, 10, 7, 7), (25, 1, 4, 2)])
def test_against_pairwise(n, d, k, m):
    rng = np.random.default_rng(n + d)
    X = rng.normal(size=(n, d)).astype(np.float32)
    X[5] = X[3]           # an exact tie pair
    nbr, d2, _ = PG.knn(X, k)
    for i in range(n):
        cand = sorted((PG.pair_d2(X, i, j), j) for j in range(n) if j != i)[:k]
        assert list(nbr[i]) == [j for _, j in cand]
        np.testing.assert_allclose(d2[i], [v for v, _ in cand], rtol=1e-13)
    rp, col, w, sigma = PG.point_graph(X, k, m)
    edges = {(i, int(j)): float(v) for i in range(n) for j, v in zip(col[rp[i]:rp[i + 1]], w[rp[i]:rp[i + 1]])}
    for (i, j), v in edges.items():
        assert edges[(j, i)] == v and i != j
        assert (j in nbr[i]) or (i in nbr[j])
    for i in range(n):
        for j in nbr[i]:
            assert (i, int(j)) in edges
    assert np.all(np.diff(rp) >= k)


def test_separated_clusters():
    rng = np.random.default_rng(1)
    X = np.concatenate([rng.normal(size=(30, 4)), rng.normal(size=(30, 4)) + 100.0]).astype(np.float32)
    rp, col, w, _ = PG.point_graph(X, 6, 4)
    for i in range(60):
        assert np.all((col[rp[i]:rp[i + 1]] < 30) == (i < 30))
