"""Seeded synthetic graph workloads (inputs only; no solver arithmetic).

Every workload is a symmetric, non-negative weight matrix W in CSR form
(int64 row_ptr, int32 col with strictly increasing columns per row and no
self loops, float32 w), a fidelity mask Lambda (uint8 0/1), prior class ids y
on the labelled rows, the ground-truth classes and the solver settings of the
workload.  Graph construction follows Sec. 2.2 of the paper:

* weights w_ij = K(i,j) N(i,j) with the Gaussian similarity of eq. (K(i,j))
  on feature vectors D_i (3x3 RGB patches for images, coordinates for point
  clouds, alpha_n = 1);
* N_s: a square search window around each pixel (images), N_c: k nearest
  neighbours in feature space (point clouds); in both cases only the k
  nearest candidates are kept, then the edge set is symmetrised by union;
* point clouds use the local-scaling bandwidth of Zelnik-Manor and Perona,
  w = exp(-d^2 / (sigma_i sigma_j)) with sigma_i the distance to the 7th
  neighbour; images use a fixed bandwidth sigma.

Random numbers come from numpy's PCG64 seeded with 20230301 + workload id.
The paper's photographs, MNIST and its point sets are not available; these
generators stand in for them with the shapes, sizes and noise levels of the
paper's experiments (Sec. 5).
"""

from __future__ import annotations

import dataclasses
import hashlib
import json
import os
from typing import Callable, Dict, Optional, Tuple

import numpy as np

GEN_VERSION = 3
SEED_BASE = 20230301

# Preconditioner names, in the paper's terms (eq. for G_{Jd,s}, G_{Jp,s},
# G_{R,s}); the integer codes match the C interface.
JACOBI_DAMPED = 0
JACOBI_PERTURBED = 1
RICHARDSON = 2


@dataclasses.dataclass
class Workload:
    name: str
    n: int
    K: int                      # 1: binary +-1 model; >= 2: K label columns
    row_ptr: np.ndarray         # int64 [n+1]
    col: np.ndarray             # int32 [nnz]
    w: np.ndarray               # float32 [nnz]
    gt: np.ndarray              # int32 [n] ground-truth class ids
    fid_mask: np.ndarray        # uint8 [n] Lambda_i in {0,1}
    fid_labels: np.ndarray      # int32 [n] prior class id where fid_mask = 1, else 0
    params: Dict[str, float]    # eps, c, eta, precond, damping, delta0, outer, inner, power_iters
    meta: Dict[str, object]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


# ---------------------------------------------------------------------------
# CSR helpers
# ---------------------------------------------------------------------------

def csr_from_pairs(n: int, i: np.ndarray, j: np.ndarray, w: np.ndarray):
    """Build a symmetric CSR from undirected pairs (i < j) with one weight each.

    Both directions get the identical float32 weight, so w_ij = w_ji holds
    bit for bit.  Columns are strictly increasing within a row.
    """
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    w = np.asarray(w, dtype=np.float32)
    assert np.all(i != j)
    rows = np.concatenate([i, j])
    cols = np.concatenate([j, i])
    vals = np.concatenate([w, w])
    key = rows * n + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    assert key.size == 0 or np.all(np.diff(key) > 0), "duplicate pair"
    rows = rows[order]
    cols = cols[order].astype(np.int32)
    vals = vals[order]
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, cols, vals


def _union_pairs(n: int, src: np.ndarray, dst: np.ndarray, dist2: np.ndarray):
    """Union-symmetrise directed k-NN edges; keep one squared distance per pair.

    For a pair selected in both directions the distance of the direction with
    the smaller source index is kept (both are equal for the symmetric
    distances used here).
    """
    src = src.astype(np.int64)
    dst = dst.astype(np.int64)
    lo = np.minimum(src, dst)
    hi = np.maximum(src, dst)
    key = lo * n + hi
    # prefer the entry whose source is the lower index
    pref = (src != lo).astype(np.int64)
    order = np.lexsort((pref, key))
    key_s = key[order]
    first = np.ones(key_s.size, dtype=bool)
    first[1:] = key_s[1:] != key_s[:-1]
    sel = order[first]
    return lo[sel], hi[sel], dist2[sel]


def random_graph(n: int, avg_deg: int, seed: int, w_low: float = 0.05,
                 w_high: float = 1.0, connected: bool = True):
    """Random symmetric graph with positive weights (for tests of any size).

    A ring i -- i+1 guarantees d_i > 0 when ``connected``; extra edges are
    drawn uniformly.
    """
    rng = np.random.default_rng(seed)
    pairs = set()
    if connected and n >= 2:
        for a in range(n - 1):
            pairs.add((a, a + 1))
    m_extra = max(0, (avg_deg * n) // 2 - len(pairs))
    if n >= 2:
        a = rng.integers(0, n, size=2 * m_extra + 16)
        b = rng.integers(0, n, size=2 * m_extra + 16)
        for x, y in zip(a.tolist(), b.tolist()):
            if len(pairs) >= m_extra + (n - 1 if connected else 0):
                break
            if x == y:
                continue
            pairs.add((min(x, y), max(x, y)))
    if not pairs:
        return (np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))
    p = np.array(sorted(pairs), dtype=np.int64)
    w = rng.uniform(w_low, w_high, size=p.shape[0]).astype(np.float32)
    return csr_from_pairs(n, p[:, 0], p[:, 1], w)


def banded_graph(n: int, avg_deg: int, band: int, seed: int, far_frac: float = 0.0, hubs=(),
                 hub_deg: int = 100, w_low: float = 0.05, w_high: float = 1.0):
    """Random symmetric graph whose edges join nodes at most ``band`` apart in
    index (plus a ring i -- i+1), for tests of any size; ``far_frac`` of the
    extra edges join uniformly random nodes instead, and every node listed in
    ``hubs`` gets ``hub_deg`` extra neighbours between 1 and ``band``
    positions above it.
    """
    rng = np.random.default_rng(seed)
    a = [np.arange(n - 1, dtype=np.int64)]
    b = [np.arange(1, n, dtype=np.int64)]
    m = max(0, (avg_deg * n) // 2 - (n - 1))
    x = rng.integers(0, n, size=m)
    y = x + rng.integers(-band, band + 1, size=m)
    far = rng.uniform(size=m) < far_frac
    y[far] = rng.integers(0, n, size=int(far.sum()))
    a.append(x)
    b.append(y)
    for c in hubs:
        a.append(np.full(hub_deg, c, np.int64))
        b.append(c + rng.integers(1, band + 1, size=hub_deg))
    a = np.concatenate(a)
    b = np.concatenate(b)
    ok = (b >= 0) & (b < n) & (a != b)
    i = np.minimum(a[ok], b[ok])
    j = np.maximum(a[ok], b[ok])
    key = np.unique(i * n + j)
    i, j = key // n, key % n
    w = rng.uniform(w_low, w_high, size=i.shape[0]).astype(np.float32)
    return csr_from_pairs(n, i, j, w)


# ---------------------------------------------------------------------------
# Feature data
# ---------------------------------------------------------------------------

def two_moons(n: int, dim: int, noise: float, rng: np.random.Generator):
    """Two unit half circles in dims 0-1 (upper centred (0,0), lower centred
    (1, 0.5)), embedded in R^dim with N(0, noise^2) added to every coordinate."""
    n0 = n // 2
    n1 = n - n0
    t0 = rng.uniform(0.0, np.pi, size=n0)
    t1 = rng.uniform(0.0, np.pi, size=n1)
    X = np.zeros((n, dim), dtype=np.float64)
    X[:n0, 0] = np.cos(t0)
    X[:n0, 1] = np.sin(t0)
    X[n0:, 0] = 1.0 - np.cos(t1)
    X[n0:, 1] = 0.5 - np.sin(t1)
    X += rng.normal(0.0, noise, size=X.shape)
    gt = np.concatenate([np.zeros(n0, np.int32), np.ones(n1, np.int32)])
    return X, gt


def gmm_points(n_per: int, comps: int, dim: int, sigma: float, rng: np.random.Generator):
    """Isotropic Gaussian mixture with means uniform in [0,1]^dim, values
    clipped to [0,1]; equal class sizes."""
    means = rng.uniform(0.0, 1.0, size=(comps, dim))
    X = np.empty((n_per * comps, dim), dtype=np.float32)
    gt = np.empty(n_per * comps, dtype=np.int32)
    for c in range(comps):
        blk = means[c] + rng.normal(0.0, sigma, size=(n_per, dim))
        X[c * n_per:(c + 1) * n_per] = np.clip(blk, 0.0, 1.0)
        gt[c * n_per:(c + 1) * n_per] = c
    return X, gt


def ellipse_image(size: int, n_ellipses: int, noise: float, rng: np.random.Generator):
    """RGB image of random filled ellipses on a background; region colours are
    uniform in [0,1]^3; ground truth = inside any ellipse (1) or background (0)."""
    H = W = size
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    img = np.empty((H, W, 3), dtype=np.float64)
    img[:] = rng.uniform(0.0, 1.0, size=3)
    gt = np.zeros((H, W), dtype=np.int32)
    for _ in range(n_ellipses):
        cy, cx = rng.uniform(0.15 * H, 0.85 * H), rng.uniform(0.15 * W, 0.85 * W)
        a, b = rng.uniform(0.06 * size, 0.22 * size, size=2)
        th = rng.uniform(0.0, np.pi)
        col = rng.uniform(0.0, 1.0, size=3)
        dy, dx = yy - cy, xx - cx
        u = (dx * np.cos(th) + dy * np.sin(th)) / a
        v = (-dx * np.sin(th) + dy * np.cos(th)) / b
        inside = u * u + v * v <= 1.0
        img[inside] = col
        gt[inside] = 1
    img += rng.normal(0.0, noise, size=img.shape)
    return img.astype(np.float32), gt.reshape(-1)


def voronoi_image(size: int, n_seeds: int, n_classes: int, noise: float,
                  rng: np.random.Generator):
    """Piecewise-constant Voronoi image: seeds uniform in the square, each seed
    takes one of ``n_classes`` class colours (uniform in [0,1]^3; every class
    used at least once); Gaussian noise added."""
    H = W = size
    seeds = rng.uniform(0.0, size, size=(n_seeds, 2))
    seed_cls = rng.integers(0, n_classes, size=n_seeds)
    seed_cls[:n_classes] = np.arange(n_classes)
    rng.shuffle(seed_cls)
    colours = rng.uniform(0.0, 1.0, size=(n_classes, 3))
    owner = np.empty((H, W), dtype=np.int64)
    xs = np.arange(W, dtype=np.float64)
    for y in range(H):
        d = (seeds[:, 0:1] - y) ** 2 + (seeds[:, 1:2] - xs[None, :]) ** 2
        owner[y] = np.argmin(d, axis=0)
    gt = seed_cls[owner].astype(np.int32)
    img = colours[gt] + rng.normal(0.0, noise, size=(H, W, 3))
    return img.astype(np.float32), gt.reshape(-1)


# ---------------------------------------------------------------------------
# Graphs
# ---------------------------------------------------------------------------

def knn_graph_points(X: np.ndarray, k: int, scale_nn: int = 7, chunk: int = 2048,
                     device: str = "cpu"):
    """Symmetrised k-NN graph with local-scaling Gaussian weights.

    Candidates come from a float32 distance matrix (|x|^2 + |y|^2 - 2 x.y);
    the 3k best candidates of every point are re-ranked with exact float64
    distances, ties broken by the lower index.  sigma_i is the float64
    distance to the ``scale_nn``-th neighbour (self excluded).
    """
    import torch

    n = X.shape[0]
    Xd = np.ascontiguousarray(X, dtype=np.float64)
    Xt = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(device)
    sq = (Xt * Xt).sum(dim=1)
    n_cand = min(n - 1, 3 * k + 8)
    nbr = np.empty((n, k), dtype=np.int64)
    nd2 = np.empty((n, k), dtype=np.float64)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        blk = Xt[s:e]
        d = sq[s:e, None] + sq[None, :] - 2.0 * (blk @ Xt.T)
        idx = torch.arange(s, e, device=device)
        d[idx - s, idx] = float("inf")
        cand = torch.topk(d, n_cand, dim=1, largest=False, sorted=False).indices.cpu().numpy()
        cand.sort(axis=1)
        diff = Xd[cand] - Xd[s:e, None, :]
        exact = np.einsum("rcd,rcd->rc", diff, diff)
        # candidates ascending in index, so a stable sort by distance breaks
        # ties by the lower index
        order = np.argsort(exact, axis=1, kind="stable")[:, :k]
        nbr[s:e] = np.take_along_axis(cand, order, axis=1)
        nd2[s:e] = np.take_along_axis(exact, order, axis=1)
    sig = np.sqrt(nd2[:, scale_nn - 1])
    src = np.repeat(np.arange(n, dtype=np.int64), k)
    dst = nbr.reshape(-1)
    lo, hi, d2 = _union_pairs(n, src, dst, nd2.reshape(-1))
    w = np.exp(-d2 / (sig[lo] * sig[hi]))
    return csr_from_pairs(n, lo, hi, w.astype(np.float32))


def knn_graph_image(img: np.ndarray, k: int, window: int, sigma: float,
                    rows_per_chunk: int = 128, device: str = "cpu"):
    """Symmetrised window k-NN graph of an RGB image with 3x3 patch features.

    Patch distance between pixels p and q: sum over the 3x3 neighbourhood and
    the 3 channels of squared colour differences, patches replicate-padded at
    the border (alpha_n = 1).  Candidates are the pixels q != p of the
    ``window`` x ``window`` square centred on p, clipped to the image; the k
    with the smallest float64 patch distance are kept.  w = exp(-d^2/sigma^2).
    """
    import torch
    import torch.nn.functional as F

    H, W, _ = img.shape
    n = H * W
    r = window // 2
    I = torch.from_numpy(np.ascontiguousarray(img, dtype=np.float32)).to(device=device, dtype=torch.float64)
    I = I.permute(2, 0, 1).unsqueeze(0)                     # 1,3,H,W
    Ip1 = F.pad(I, (1, 1, 1, 1), mode="replicate")          # patch padding
    Ib = F.pad(Ip1, (r, r, r, r), mode="constant", value=0.0)[0]  # 3,H+2+2r,W+2+2r
    offs = [(dy, dx) for dy in range(-r, r + 1) for dx in range(-r, r + 1) if (dy, dx) != (0, 0)]
    nbr = np.empty((n, k), dtype=np.int64)
    nd2 = np.empty((n, k), dtype=np.float64)
    ys_all = torch.arange(H, device=device)
    xs_all = torch.arange(W, device=device)
    for y0 in range(0, H, rows_per_chunk):
        y1 = min(H, y0 + rows_per_chunk)
        R = y1 - y0
        D = torch.empty((len(offs), R, W), dtype=torch.float64, device=device)
        A = Ib[:, r + y0: r + y1 + 2, r: r + W + 2]
        for oi, (dy, dx) in enumerate(offs):
            B = Ib[:, r + y0 + dy: r + y1 + 2 + dy, r + dx: r + W + 2 + dx]
            t = A - B
            t = t * t
            delta = t[0] + t[1] + t[2]                           # (R+2, W+2)
            h = delta[:, 0:W] + delta[:, 1:W + 1] + delta[:, 2:W + 2]
            s = h[0:R] + h[1:R + 1] + h[2:R + 2]                # (R, W)
            ys = ys_all[y0:y1] + dy
            xs = xs_all + dx
            bad = ((ys < 0) | (ys >= H))[:, None] | ((xs < 0) | (xs >= W))[None, :]
            D[oi] = torch.where(bad, torch.full_like(s, float("inf")), s)
        Dt = D.permute(1, 2, 0).reshape(R * W, len(offs))
        vals, oidx = torch.topk(Dt, k, dim=1, largest=False, sorted=True)
        oidx = oidx.cpu().numpy()
        vals = vals.cpu().numpy()
        off_arr = np.array([dy * W + dx for dy, dx in offs], dtype=np.int64)
        p = np.arange(y0 * W, y1 * W, dtype=np.int64)
        nbr[y0 * W: y1 * W] = p[:, None] + off_arr[oidx]
        nd2[y0 * W: y1 * W] = vals
    assert np.all(np.isfinite(nd2)), "window too small for k"
    src = np.repeat(np.arange(n, dtype=np.int64), k)
    lo, hi, d2 = _union_pairs(n, src, nbr.reshape(-1), nd2.reshape(-1))
    w = np.exp(-d2 / (sigma * sigma))
    return csr_from_pairs(n, lo, hi, w.astype(np.float32))


def sample_labels(gt: np.ndarray, frac: float, n_classes: int, rng: np.random.Generator):
    """Uniform labelled set without replacement, resampled until every class
    has at least one labelled node."""
    n = gt.shape[0]
    m = max(n_classes, int(round(frac * n)))
    for _ in range(1000):
        sel = rng.choice(n, size=m, replace=False)
        if np.unique(gt[sel]).size == n_classes:
            break
    mask = np.zeros(n, dtype=np.uint8)
    mask[sel] = 1
    lab = np.where(mask == 1, gt, 0).astype(np.int32)
    return mask, lab


# ---------------------------------------------------------------------------
# The named workloads
# ---------------------------------------------------------------------------

def _params(eps, eta, c, precond, outer, inner, damping=0.0, delta0=1e-6, power_iters=150):
    return dict(eps=float(eps), eta=float(eta), c=float(c), precond=int(precond),
                outer=int(outer), inner=int(inner), damping=float(damping),
                delta0=float(delta0), power_iters=int(power_iters))


def _moons2k(device="cpu", **kw):
    rng = np.random.default_rng(SEED_BASE + 1)
    n = kw.get("n", 2000)
    X, gt = two_moons(n, 100, 0.02, rng)
    rp, col, w = knn_graph_points(X, 10, 7, device=device)
    mask, lab = sample_labels(gt, 0.05, 2, rng)
    eps, eta = 1.0, 500.0
    return Workload("moons2k", n, 1, rp, col, w, gt, mask, lab,
                    _params(eps, eta, 2.0 / eps + eta, JACOBI_DAMPED, 10, 5, damping=0.8),
                    dict(kind="points", dim=100))


def _ellipses256(device="cpu", **kw):
    rng = np.random.default_rng(SEED_BASE + 2)
    size = kw.get("size", 256)
    img, gt = ellipse_image(size, 6, 0.1, rng)
    rp, col, w = knn_graph_image(img, 10, 11, 0.5, device=device)
    mask, lab = sample_labels(gt, 0.02, 2, rng)
    eps, eta = 1.0, 500.0
    return Workload("ellipses256" if size == 256 else f"ellipses{size}", size * size, 1,
                    rp, col, w, gt, mask, lab,
                    _params(eps, eta, 2.0 / eps + eta, RICHARDSON, 4, 10),
                    dict(kind="image", shape=(size, size)))


def _gmm70k(device="cpu", **kw):
    rng = np.random.default_rng(SEED_BASE + 3)
    n_per = kw.get("n_per", 7000)
    dim = kw.get("dim", 784)
    X, gt = gmm_points(n_per, 10, dim, 0.15, rng)
    rp, col, w = knn_graph_points(X, 10, 7, device=device)
    mask, lab = sample_labels(gt, 0.035, 10, rng)
    eps, eta = 1.0, 500.0
    return Workload("gmm70k" if n_per == 7000 else f"gmm{10 * n_per}", 10 * n_per, 10,
                    rp, col, w, gt, mask, lab,
                    _params(eps, eta, 2.0 / eps + eta, JACOBI_DAMPED, 10, 5, damping=0.8),
                    dict(kind="points", dim=dim))


def _voronoi(device="cpu", **kw):
    size = kw.get("size", 2048)
    rng = np.random.default_rng(SEED_BASE + 4 + (0 if size == 2048 else 1000 + size))
    img, gt = voronoi_image(size, kw.get("seeds", 64), 4, 0.15, rng)
    rp, col, w = knn_graph_image(img, 10, 15, 0.5, device=device)
    mask, lab = sample_labels(gt, 0.01, 4, rng)
    eps, eta = 1.0, 500.0
    return Workload("voronoi2048" if size == 2048 else f"voronoi{size}", size * size, 4,
                    rp, col, w, gt, mask, lab,
                    _params(eps, eta, 2.0 / eps + eta, RICHARDSON, 4, 8),
                    dict(kind="image", shape=(size, size)))


WORKLOADS: Dict[str, Callable[..., Workload]] = {
    "moons2k": _moons2k,
    "ellipses256": _ellipses256,
    "gmm70k": _gmm70k,
    "voronoi2048": _voronoi,
}


def _cache_dir() -> str:
    d = os.environ.get("PDCA_GEN_CACHE") or os.path.join(
        os.environ.get("TMPDIR", "/tmp"), "pdca_gen_cache")
    os.makedirs(d, exist_ok=True)
    return d


def make_workload(name: str, device: str = "cpu", cache: bool = True, **kw) -> Workload:
    """Build (or load from the on-disk cache) a named workload.

    ``kw`` scales a workload down for tests (``size``, ``n_per``, ``dim``,
    ``n``, ``seeds``).  The cache key covers the name, the overrides and the
    generator version; cached arrays are exactly the generated ones.
    """
    key = hashlib.sha1(json.dumps([name, sorted(kw.items()), GEN_VERSION]).encode()).hexdigest()[:16]
    path = os.path.join(_cache_dir(), f"{name}_{key}.npz")
    if cache and os.path.exists(path):
        z = np.load(path, allow_pickle=False)
        meta = json.loads(str(z["meta"]))
        params = json.loads(str(z["params"]))
        return Workload(str(z["name"]), int(z["n"]), int(z["K"]), z["row_ptr"], z["col"], z["w"],
                        z["gt"], z["fid_mask"], z["fid_labels"], params, meta)
    wl = WORKLOADS[name](device=device, **kw)
    if cache:
        tmp = path + f".tmp{os.getpid()}.npz"
        np.savez(tmp, name=wl.name, n=wl.n, K=wl.K, row_ptr=wl.row_ptr, col=wl.col, w=wl.w,
                 gt=wl.gt, fid_mask=wl.fid_mask, fid_labels=wl.fid_labels,
                 params=json.dumps(wl.params), meta=json.dumps(wl.meta, default=list))
        os.replace(tmp, path)
    return wl
