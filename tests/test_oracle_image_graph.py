"""Pins of the oracle's nonlocal image graph (window k-NN of patch
distances, eq. kij with alpha_n = 1): hand-computed distances with replicate
padding, closed forms on constant and two-region images, the vectorised
builder against the pair-by-pair definition, and the structural invariants."""

import numpy as np
import pytest

from oracle import image_graph as IG


def test_patch_distance_by_hand():
    """3x3 single-channel image, 3x3 patches: the corner's patch repeats the
    border values (replicate padding)."""
    img = np.arange(9, dtype=np.float32).reshape(3, 3, 1)
    # patch of pixel 0 (0,0): rows [0,0,1] x cols [0,0,1] of the image
    # patch of pixel 1 (0,1): rows [0,0,1] x cols [0,1,2]
    a = np.array([[0, 0, 1], [0, 0, 1], [3, 3, 4]], np.float32)
    b = np.array([[0, 1, 2], [0, 1, 2], [3, 4, 5]], np.float32)
    assert IG.patch_d2(img, 1, 0, 1) == np.float32(((a - b) ** 2).sum())
    assert IG.patch_d2(img, 1, 0, 1) == IG.patch_d2(img, 1, 1, 0)


def test_constant_image_keeps_lowest_indices():
    H, W, r, k = 9, 11, 2, 5
    img = np.full((H, W, 3), 0.4, np.float32)
    nbr, d2 = IG.knn_lists(img, 1, r, k)
    assert np.all(d2 == 0)
    i = 5 * W + 6
    y, x = divmod(i, W)
    cand = [yy * W + xx for yy in range(y - r, y + r + 1) for xx in range(x - r, x + r + 1) if yy * W + xx != i]
    assert list(nbr[i]) == sorted(cand)[:k]
    rp, col, w = IG.image_graph(img, 1, r, k, 0.5)
    assert np.all(w == 1.0)


def test_two_regions_connect_within():
    """Left half colour a, right half b, single-pixel patches: distance 0
    inside a region and 3 (a-b)^2 across, so every kept neighbour of a pixel
    far from the boundary lies in its own region, with weight 1."""
    H, W = 12, 16
    img = np.zeros((H, W, 3), np.float32)
    img[:, W // 2:] = 0.5
    rp, col, w = IG.image_graph(img, 0, 2, 6, 0.5)
    for i in range(H * W):
        y, x = divmod(i, W)
        if 2 <= x < W // 2 - 2 or W // 2 + 2 <= x < W - 2:
            for j, wj in zip(col[rp[i]:rp[i + 1]], w[rp[i]:rp[i + 1]]):
                assert (j % W < W // 2) == (x < W // 2)
                assert wj == 1.0


@pytest.mark.parametrize("shape,p,r,k", [((7, 9, 3), 1, 2, 4), ((10, 6, 1), 0, 3, 7), ((8, 8, 2), 2, 1, 3)])
def test_vectorised_equals_pairwise(shape, p, r, k):
    rng = np.random.default_rng(sum(shape))
    img = rng.uniform(size=shape).astype(np.float32)
    img[2:4, 2:4] = img[0, 0]          # some exact ties
    rp, col, w = IG.image_graph(img, p, r, k, 0.7)
    n = shape[0] * shape[1]
    ref = IG.image_graph_rows(img, p, r, k, 0.7, range(n))
    for i in range(n):
        np.testing.assert_array_equal(col[rp[i]:rp[i + 1]], ref[i][0])
        np.testing.assert_array_equal(w[rp[i]:rp[i + 1]], ref[i][1])


def test_structure():
    rng = np.random.default_rng(3)
    img = rng.uniform(size=(20, 24, 3)).astype(np.float32)
    rp, col, w = IG.image_graph(img, 1, 3, 8, 0.5)
    n = 20 * 24
    deg = np.diff(rp)
    assert deg.min() >= 8 and deg.max() <= 48
    for i in range(n):
        c = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(c) > 0) and i not in c
    # symmetric, bit for bit
    pos = {(i, int(j)): float(w[e]) for i in range(n) for e, j in zip(range(rp[i], rp[i + 1]), col[rp[i]:rp[i + 1]])}
    for (i, j), v in pos.items():
        assert pos[(j, i)] == v


def test_crop_rows_equal_full():
    rng = np.random.default_rng(5)
    img = rng.uniform(size=(30, 34, 3)).astype(np.float32)
    img[10:14, 5:9] = 0.25
    rp, col, w = IG.image_graph(img, 1, 3, 6, 0.5)
    rows = [0, 33, 34 * 12 + 7, 34 * 15 + 20, 30 * 34 - 1]
    got = IG.image_graph_rows_crop(img, 1, 3, 6, 0.5, rows)
    for i in rows:
        np.testing.assert_array_equal(got[i][0], col[rp[i]:rp[i + 1]])
        np.testing.assert_array_equal(got[i][1], w[rp[i]:rp[i + 1]])


@pytest.mark.parametrize("shape,p,r,k", [((17, 23, 3), 1, 2, 6), ((30, 26, 3), 1, 4, 10), ((12, 40, 1), 2, 3, 8)])
def test_fp32_definition_within_fp64_bounds(shape, p, r, k):
    """The FP32 definition (patch sums in a fixed order) satisfies the FP64
    definition's bounds: an independent check of the builder's rounding, with
    most rows decided by the FP64 distances alone."""
    rng = np.random.default_rng(sum(shape) + k)
    img = rng.uniform(size=shape).astype(np.float32)
    rp, col, w = IG.image_graph(img, p, r, k, 0.5)
    st = IG.check_against_f64(rp, col, w, img, p, r, k, 0.5)
    assert st["decided"] > 0.9, st


def test_fp64_check_catches_planted_mistakes():
    """A dropped edge, an edge to a far partner and a wrong weight each fail."""
    rng = np.random.default_rng(5)
    img = rng.uniform(size=(20, 20, 3)).astype(np.float32)
    rp, col, w = IG.image_graph(img, 1, 3, 6, 0.5)
    IG.check_against_f64(rp, col, w, img, 1, 3, 6, 0.5)
    # drop the nearest partner of pixel 50
    D, offs = IG.window_d2_f64(img, 1, 3)
    y, x = divmod(50, 20)
    dy, dx = offs[int(np.argmin(D[50]))]
    j = (y + dy) * 20 + (x + dx)
    keep = np.ones(col.size, bool)
    keep[rp[50] + int(np.searchsorted(col[rp[50]:rp[51]], j))] = False
    keep[rp[j] + int(np.searchsorted(col[rp[j]:rp[j + 1]], 50))] = False
    rows = np.repeat(np.arange(400), np.diff(rp))[keep]
    rp2 = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=400))])
    with pytest.raises(AssertionError, match="must be kept"):
        IG.check_against_f64(rp2, col[keep], w[keep], img, 1, 3, 6, 0.5)
    # a wrong weight
    w2 = w.copy()
    w2[7] *= 1.001
    with pytest.raises(AssertionError, match="weight"):
        IG.check_against_f64(rp, col, w2, img, 1, 3, 6, 0.5)
    # the farthest partner of pixel 50 replacing its nearest (both directions)
    far = offs[int(np.argmax(np.where(np.isfinite(D[50]), D[50], -1)))]
    jf = (y + far[0]) * 20 + (x + far[1])
    col3 = col.copy()
    col3[rp[50] + int(np.searchsorted(col[rp[50]:rp[51]], j))] = jf
    with pytest.raises(AssertionError):
        IG.check_against_f64(rp, col3, w, img, 1, 3, 6, 0.5)
