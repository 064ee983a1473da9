"""Oracle of the k-NN graph of a point cloud (TEST INFRASTRUCTURE ONLY).

Sec. 2.3 for clustering: w_ij = K(i,j) N_c(i,j) with N_c the k-nearest-
neighbour indicator (Euclidean distance) and K the Gaussian kernel with the
local-scaling bandwidth of Zelnik-Manor and Perona, sigma_i = distance of i
to its m-th nearest neighbour (self excluded):
    w_ij = exp(-|x_i - x_j|^2 / (sigma_i sigma_j)),
symmetrised by union (an edge where either end keeps the other).

Definition written out: squared distances in float64 as sums of squared
coordinate differences, the k smallest (d2, j) kept (ties to the lower
index), weights in float64 rounded to float32.
"""

from __future__ import annotations

import numpy as np


def pair_d2(X: np.ndarray, i: int, j: int) -> float:
    """|x_i - x_j|^2 one coordinate at a time, in float64."""
    X = np.asarray(X)
    acc = 0.0
    for d in range(X.shape[1]):
        t = float(X[i, d]) - float(X[j, d])
        acc += t * t
    return acc


def all_d2(X: np.ndarray, chunk: int = 64) -> np.ndarray:
    """n x n squared distances in float64 (differences, then sums)."""
    Xd = np.asarray(X, np.float64)
    n = Xd.shape[0]
    out = np.empty((n, n), np.float64)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        diff = Xd[s:e, None, :] - Xd[None, :, :]
        out[s:e] = np.einsum("rcd,rcd->rc", diff, diff)
    return out


def knn(X: np.ndarray, k: int):
    """(nbr n x k, d2 n x k, next_d2 n): kept neighbours by (d2, index) and
    the distance of the first one not kept (to tell genuine near-ties)."""
    D = all_d2(X)
    n = D.shape[0]
    np.fill_diagonal(D, np.inf)
    idx = np.broadcast_to(np.arange(n), (n, n))
    order = np.lexsort((idx, D), axis=1)
    nbr = order[:, :k]
    d2 = np.take_along_axis(D, nbr, 1)
    nxt = np.take_along_axis(D, order[:, k:k + 1], 1)[:, 0] if k < n - 1 else np.full(n, np.inf)
    return nbr.astype(np.int64), d2, nxt


def point_graph(X: np.ndarray, k: int, m: int):
    """CSR (row_ptr int64, col int32 ascending, w float32) and sigma (n)."""
    nbr, d2, _ = knn(X, k)
    n = nbr.shape[0]
    sigma = np.sqrt(d2[:, m - 1])
    rows = np.repeat(np.arange(n), k)
    cols = nbr.ravel()
    vals = d2.ravel()
    R = np.concatenate([rows, cols])
    C = np.concatenate([cols, rows])
    V = np.concatenate([vals, vals])
    key = R * n + C
    order = np.argsort(key, kind="stable")
    key, R, C, V = key[order], R[order], C[order], V[order]
    first = np.ones(key.size, bool)
    first[1:] = key[1:] != key[:-1]
    R, C, V = R[first], C[first], V[first]
    row_ptr = np.zeros(n + 1, np.int64)
    np.add.at(row_ptr, R + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    w = np.exp(-V / (sigma[R] * sigma[C])).astype(np.float32)
    return row_ptr, C.astype(np.int32), w, sigma
