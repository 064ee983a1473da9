"""Oracle of the nonlocal image graph (TEST INFRASTRUCTURE ONLY).

Follows Sec. 2.3 of the paper (the weight of pixels i, j is the Gaussian
kernel K(i,j) of eq. kij times the window indicator N_s(i,j)), with the
window k-NN restriction the image workloads use: each pixel keeps the k
window pixels with the smallest patch distance, and the graph is the union of
those directed edges (symmetrised), weighted by K.

Definition, spelled out so that every floating-point decision is the same as
the CUDA builder's (the kept neighbours are decided by comparing distances,
so both sides take that decision in the same precision, FP32):
  * patch distance d2(i, j) = sum over patch offsets (oy, ox) in raster order
    (oy, then ox, from -p to p) and channels c of (A - B)^2, where A and B are
    the replicate-padded pixel values at i + (oy, ox) and j + (oy, ox); each
    square and each addition rounded to float32 in that order (no fused
    multiply-add);  alpha_n = 1;
  * candidates of i: the pixels j != i with max(|dy|, |dx|) <= r inside the
    image;  the k kept are the smallest (d2, j) in lexicographic order
    (ties of d2 go to the lower index j = y W + x);
  * w_ij = float32(exp(-float64(d2) / sigma^2)) for every edge of the union;
    d2(i, j) == d2(j, i) exactly, so w is symmetric bit for bit.
"""

from __future__ import annotations

import numpy as np


def _padded(img: np.ndarray, p: int) -> np.ndarray:
    img = np.ascontiguousarray(img, np.float32)
    return np.pad(img, ((p, p), (p, p), (0, 0)), mode="edge")


def patch_d2(img: np.ndarray, p: int, i: int, j: int) -> np.float32:
    """d2(i, j) for one pair, one term at a time (the definition above)."""
    H, W, C = img.shape
    P = _padded(img, p)
    yi, xi = divmod(i, W)
    yj, xj = divmod(j, W)
    acc = np.float32(0.0)
    for oy in range(-p, p + 1):
        for ox in range(-p, p + 1):
            for c in range(C):
                a = P[yi + p + oy, xi + p + ox, c]
                b = P[yj + p + oy, xj + p + ox, c]
                t = np.float32(a - b)
                acc = np.float32(acc + np.float32(t * t))
    return acc


def _d2_offset(P: np.ndarray, H: int, W: int, C: int, p: int, dy: int, dx: int) -> np.ndarray:
    """d2(i, i + (dy, dx)) for every pixel i (H x W, float32, same order of
    operations as patch_d2; +inf where the partner is outside the image)."""
    acc = np.zeros((H, W), np.float32)
    Hp, Wp = P.shape[:2]
    for oy in range(-p, p + 1):
        for ox in range(-p, p + 1):
            for c in range(C):
                ya, xa = p + oy, p + ox
                A = P[ya:ya + H, xa:xa + W, c]
                # partner rows / cols, clipped into the padded image (invalid ones masked below)
                yb = np.clip(np.arange(H) + p + oy + dy, 0, Hp - 1)
                xb = np.clip(np.arange(W) + p + ox + dx, 0, Wp - 1)
                Bv = P[yb[:, None], xb[None, :], c]
                t = (A - Bv).astype(np.float32)
                acc = (acc + (t * t).astype(np.float32)).astype(np.float32)
    ys, xs = np.arange(H)[:, None] + dy, np.arange(W)[None, :] + dx
    bad = (ys < 0) | (ys >= H) | (xs < 0) | (xs >= W)
    return np.where(bad, np.float32(np.inf), acc)


def knn_lists(img: np.ndarray, p: int, r: int, k: int):
    """(nbr, d2): for every pixel the k kept window neighbours (n x k, -1 and
    +inf where fewer than k candidates exist) ordered by (d2, index)."""
    img = np.ascontiguousarray(img, np.float32)
    H, W, C = img.shape
    n = H * W
    P = _padded(img, p)
    offs = [(dy, dx) for dy in range(-r, r + 1) for dx in range(-r, r + 1) if (dy, dx) != (0, 0)]
    D = np.stack([_d2_offset(P, H, W, C, p, dy, dx).ravel() for dy, dx in offs], axis=1)   # n x m
    idx = np.arange(n)[:, None] + np.array([dy * W + dx for dy, dx in offs])[None, :]
    idx = np.where(np.isinf(D), np.int64(1) << 40, idx)
    # lexicographic (d2, j): sort by j, then stable by d2
    o1 = np.argsort(idx, axis=1, kind="stable")
    D1 = np.take_along_axis(D, o1, 1)
    J1 = np.take_along_axis(idx, o1, 1)
    o2 = np.argsort(D1, axis=1, kind="stable")[:, :k]
    d2 = np.take_along_axis(D1, o2, 1)
    nbr = np.take_along_axis(J1, o2, 1)
    nbr = np.where(np.isinf(d2), -1, nbr).astype(np.int64)
    return nbr, d2


def image_graph(img: np.ndarray, p: int, r: int, k: int, sigma: float):
    """CSR (row_ptr int64, col int32 ascending, w float32) of the symmetrised
    window k-NN patch graph."""
    img = np.ascontiguousarray(img, np.float32)
    H, W, _ = img.shape
    n = H * W
    nbr, d2 = knn_lists(img, p, r, k)
    rows = np.repeat(np.arange(n), k)
    cols = nbr.ravel()
    vals = d2.ravel()
    ok = cols >= 0
    rows, cols, vals = rows[ok], cols[ok], vals[ok]
    # union of (i, j) and (j, i); d2 is symmetric, so duplicates carry equal values
    R = np.concatenate([rows, cols])
    Cc = np.concatenate([cols, rows])
    V = np.concatenate([vals, vals])
    key = R * n + Cc
    order = np.argsort(key, kind="stable")
    key, R, Cc, V = key[order], R[order], Cc[order], V[order]
    first = np.ones(key.size, bool)
    first[1:] = key[1:] != key[:-1]
    R, Cc, V = R[first], Cc[first], V[first]
    row_ptr = np.zeros(n + 1, np.int64)
    np.add.at(row_ptr, R + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    w = np.exp(-V.astype(np.float64) / (float(sigma) ** 2)).astype(np.float32)
    return row_ptr, Cc.astype(np.int32), w


def image_graph_rows(img: np.ndarray, p: int, r: int, k: int, sigma: float, rows):
    """The same graph restricted to the given pixels (for spot checks of large
    images): {i: (sorted columns int32, weights float32)}, computed from the
    k-NN lists of each pixel and of every pixel in its window, one pair at a
    time through patch_d2."""
    img = np.ascontiguousarray(img, np.float32)
    H, W, _ = img.shape

    def window(i):
        y, x = divmod(i, W)
        out = []
        for yy in range(max(0, y - r), min(H, y + r + 1)):
            for xx in range(max(0, x - r), min(W, x + r + 1)):
                j = yy * W + xx
                if j != i:
                    out.append(j)
        return out

    cache = {}

    def kept(i):
        if i not in cache:
            cand = sorted((patch_d2(img, p, i, j), j) for j in window(i))
            cache[i] = {j: d for d, j in cand[:k]}
        return cache[i]

    out = {}
    for i in rows:
        i = int(i)
        nb = {}
        for j in window(i):
            if j in kept(i):
                nb[j] = kept(i)[j]
            elif i in kept(j):
                nb[j] = kept(j)[i]
        cols = np.array(sorted(nb), np.int32)
        w = np.array([np.exp(-float(nb[j]) / float(sigma) ** 2) for j in sorted(nb)], np.float32)
        out[i] = (cols, w)
    return out


def image_graph_rows_crop(img: np.ndarray, p: int, r: int, k: int, sigma: float, rows):
    """image_graph restricted to the given pixels of a large image, through
    the full builder on a crop: the rows of pixel i depend only on the kept
    lists of the pixels within r of i, and those only on pixels within
    2r + p of i.  A crop of that radius (clipped to the image) keeps the
    row-major order of the indices, so ties break as in the whole image."""
    img = np.ascontiguousarray(img, np.float32)
    H, W, _ = img.shape
    R = 2 * r + p
    out = {}
    for i in rows:
        i = int(i)
        y, x = divmod(i, W)
        y0, y1 = max(0, y - R), min(H, y + R + 1)
        x0, x1 = max(0, x - R), min(W, x + R + 1)
        Wc = x1 - x0
        rp, col, w = image_graph(img[y0:y1, x0:x1], p, r, k, sigma)
        ic = (y - y0) * Wc + (x - x0)
        cc = col[rp[ic]:rp[ic + 1]].astype(np.int64)
        gy, gx = cc // Wc + y0, cc % Wc + x0
        out[i] = ((gy * W + gx).astype(np.int32), w[rp[ic]:rp[ic + 1]].copy())
    return out


# ---------------------------------------------------------------------------
# FP64 definition and the properties any FP32 builder must satisfy
# ---------------------------------------------------------------------------
def window_d2_f64(img: np.ndarray, p: int, r: int):
    """(D, offs): D[i, m] = the patch distance of pixel i to its window partner
    at offset offs[m], in FP64 (the FP32 pixel values are exact in FP64, the
    differences and squares nearly so); +inf where the partner is outside."""
    img = np.ascontiguousarray(img, np.float64)
    H, W, C = img.shape
    P = np.pad(img, ((p, p), (p, p), (0, 0)), mode="edge")
    offs = [(dy, dx) for dy in range(-r, r + 1) for dx in range(-r, r + 1) if (dy, dx) != (0, 0)]
    Hp, Wp = P.shape[:2]
    cols = []
    for dy, dx in offs:
        acc = np.zeros((H, W), np.float64)
        for oy in range(-p, p + 1):
            for ox in range(-p, p + 1):
                A = P[p + oy:p + oy + H, p + ox:p + ox + W, :]
                yb = np.clip(np.arange(H) + p + oy + dy, 0, Hp - 1)
                xb = np.clip(np.arange(W) + p + ox + dx, 0, Wp - 1)
                Bv = P[yb[:, None], xb[None, :], :]
                acc += ((A - Bv) ** 2).sum(axis=2)
        ys, xs = np.arange(H)[:, None] + dy, np.arange(W)[None, :] + dx
        bad = (ys < 0) | (ys >= H) | (xs < 0) | (xs >= W)
        cols.append(np.where(bad, np.inf, acc).ravel())
    return np.stack(cols, axis=1), offs


def check_against_f64(row_ptr, col, w, img: np.ndarray, p: int, r: int, k: int, sigma: float) -> dict:
    """Check a window k-NN patch graph built in FP32 against the FP64
    definition, where FP32 rounding cannot decide otherwise.

    An FP32 sum of m = (2p+1)^2 C non-negative rounded squares of rounded
    differences is within beta d2 of the exact sum, beta = (m + 4) 2^-24.  With
    d_k and d_{k+1} the k-th and (k+1)-th smallest exact distances of pixel i:
      * a partner closer than d_{k+1} (1 - 2 beta) is kept by i (fewer than
        k + 1 partners lie below d_{k+1}, and they all round below the rest);
      * a kept partner lies no farther than d_k + 2 beta d_{k+1}.
    The graph must hold every edge (i, j) that i or j must keep, and only
    edges that i or j may keep; weights exp(-d2 / sigma^2) within the FP32
    error of d2 plus a few ulps.  Returns the share of pixels whose kept set
    the FP64 distances decide alone (d_{k+1} - d_k > 4 beta d_{k+1})."""
    img = np.ascontiguousarray(img, np.float32)
    H, W, C = img.shape
    n = H * W
    D, offs = window_d2_f64(img, p, r)
    m_terms = (2 * p + 1) ** 2 * C
    beta = (m_terms + 4) * 2.0 ** -24
    Ds = np.sort(D, axis=1)
    dk = Ds[:, k - 1]
    dk1 = Ds[:, k] if Ds.shape[1] > k else np.full(n, np.inf)
    must_t = np.where(np.isfinite(dk1), dk1 * (1 - 2 * beta), np.inf)
    may_t = np.where(np.isfinite(dk1), dk + 2 * beta * dk1, np.inf)
    # partner index of every (pixel, offset)
    ii = np.arange(n)
    yy, xx = ii // W, ii % W
    J = np.stack([(yy + dy) * W + (xx + dx) for dy, dx in offs], axis=1)
    valid = np.isfinite(D)
    Jc = np.where(valid, J, 0)
    must = valid & ((D < must_t[:, None]) | (D < must_t[Jc]))
    may = valid & ((D <= may_t[:, None]) | (D <= may_t[Jc]))
    # the graph's edges as (pixel, offset) flags
    row_ptr = np.asarray(row_ptr, np.int64)
    col = np.asarray(col, np.int64)
    rows = np.repeat(ii, np.diff(row_ptr))
    dy = col // W - rows // W
    dx = col % W - rows % W
    if np.any((np.abs(dy) > r) | (np.abs(dx) > r) | (col == rows)):
        raise AssertionError("an edge outside the window")
    lut = {o: t for t, o in enumerate(offs)}
    side = 2 * r + 1
    table = np.full(side * side, -1, np.int64)
    for (a, b), t in lut.items():
        table[(a + r) * side + (b + r)] = t
    oi = table[(dy + r) * side + (dx + r)]
    have = np.zeros_like(valid)
    have[rows, oi] = True
    if np.any(must & ~have):
        bad = np.argwhere(must & ~have)[:5]
        raise AssertionError(f"edges that must be kept are missing: {[(int(a), int(J[a, b])) for a, b in bad]}")
    if np.any(have & ~may):
        bad = np.argwhere(have & ~may)[:5]
        raise AssertionError(f"edges that no FP32 rounding can keep: {[(int(a), int(J[a, b])) for a, b in bad]}")
    d = D[rows, oi]
    ref = np.exp(-d / float(sigma) ** 2)
    tol = ref * (beta * d / float(sigma) ** 2 + 4 * 2.0 ** -23)
    err = np.abs(np.asarray(w, np.float64) - ref)
    if np.any(err > tol):
        t = int(np.argmax(err - tol))
        raise AssertionError(f"weight {float(w[t])} against {float(ref[t])} at entry {t}")
    decided = np.isfinite(dk1) & (dk1 - dk > 4 * beta * dk1)
    return {"decided": float(np.mean(decided)), "edges": int(col.size)}
