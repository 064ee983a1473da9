"""Seeded request mix for the serving benchmark (inputs only).

Requests arrive as a Poisson process.  Half are image-segmentation problems
(window k-NN graphs of synthetic images, 3x3 patches), half are clustering
problems (k-NN graphs of Gaussian mixtures); node counts are log-uniform in
[n_min, n_max]; K is drawn from {2, 5, 10}.  Building a k-NN graph is far more
expensive than solving on it, so requests draw their graph from a pool of
templates spanning the size range (the nearest size of the request's kind)
and differ in K, labelled set and parameters.  Image requests use the
generalized Richardson preconditioner (4 outer x 10 sweeps), clustering
requests damped Jacobi (10 x 5), both with eps = 1, eta = 500, c = 2/eps + eta.
"""

from __future__ import annotations

import dataclasses
from typing import List

import numpy as np

from .workloads import (SEED_BASE, JACOBI_DAMPED, RICHARDSON, ellipse_image, gmm_points, knn_graph_image,
                        knn_graph_points, make_workload, _cache_dir)


@dataclasses.dataclass
class Template:
    kind: str
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    w: np.ndarray
    gt: np.ndarray


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start
    template: int
    K: int
    fid_mask: np.ndarray
    fid_labels: np.ndarray
    params: dict
    outer: int
    inner: int


IMAGE_SIDES = (64, 128, 256, 512, 1024)           # 4 Ki .. 1 Mi pixels
# point clouds from 4 Ki to 1 Mi points, dims from 784 (the small ones) down
# to 64 (the largest: an exact k-NN graph of 1 Mi points in 784 dims would
# cost minutes to build for every run)
POINT_SIZES = ((4096, 784), (16384, 784), (65536, 256), (262144, 128), (1048576, 64))


def _image_template(side: int, device: str) -> Template:
    rng = np.random.default_rng(SEED_BASE + 50 + side)
    img, gt = ellipse_image(side, 6, 0.1, rng)
    rp, col, w = knn_graph_image(img, 10, 11, 0.5, device=device)
    return Template("image", side * side, rp, col, w, gt)


def _point_template(n: int, dim: int, device: str) -> Template:
    rng = np.random.default_rng(SEED_BASE + 60 + n)
    X, gt = gmm_points(n // 10, 10, dim, 0.15, rng)
    rp, col, w = knn_graph_points(X, 10, 7, device=device, chunk=4096 if n <= 262144 else 2048)
    return Template("points", X.shape[0], rp, col, w, gt)


def templates(device: str = "cpu", max_n: int = 1 << 20, cache: bool = True) -> List[Template]:
    """The template pool (cached on disk like the named workloads)."""
    import os
    out = []
    specs = [("image", s, 0) for s in IMAGE_SIDES if s * s <= max_n] + \
            [("points", n, d) for n, d in POINT_SIZES if n <= max_n]
    for kind, a, b in specs:
        path = os.path.join(_cache_dir(), f"serving_{kind}_{a}_{b}_v3.npz")
        if cache and os.path.exists(path):
            z = np.load(path)
            out.append(Template(kind, int(z["n"]), z["row_ptr"], z["col"], z["w"], z["gt"]))
            continue
        t = _image_template(a, device) if kind == "image" else _point_template(a, b, device)
        if cache:
            tmp = path + f".tmp{os.getpid()}.npz"
            np.savez(tmp, n=t.n, row_ptr=t.row_ptr, col=t.col, w=t.w, gt=t.gt)
            os.replace(tmp, path)
        out.append(t)
    return out


def requests(pool: List[Template], n_requests: int = 512, rate: float = 200.0, n_min: int = 4096,
             n_max: int = 1 << 20, seed: int = SEED_BASE + 5) -> List[Request]:
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    by_kind = {k: [i for i, t in enumerate(pool) if t.kind == k] for k in ("image", "points")}
    out = []
    for r in range(n_requests):
        kind = "image" if r % 2 == 0 else "points"
        target = np.exp(rng.uniform(np.log(n_min), np.log(n_max)))
        cands = by_kind[kind]
        ti = min(cands, key=lambda i: abs(np.log(pool[i].n) - np.log(target)))
        t = pool[ti]
        K = int(rng.choice([2, 5, 10]))
        cls = (t.gt % K).astype(np.int32)
        frac = 0.02 if kind == "image" else 0.035
        m = max(K, int(round(frac * t.n)))
        sel = rng.choice(t.n, size=m, replace=False)
        sel[:K] = [int(np.flatnonzero(cls == k)[0]) if np.any(cls == k) else sel[k] for k in range(K)]
        mask = np.zeros(t.n, np.uint8)
        mask[sel] = 1
        lab = np.where(mask == 1, cls, 0).astype(np.int32)
        if kind == "image":
            params = dict(eps=1.0, eta=500.0, c=502.0, precond=RICHARDSON, damping=0.5, delta0=1e-6,
                          power_iters=150)
            outer, inner = 4, 10
        else:
            params = dict(eps=1.0, eta=500.0, c=502.0, precond=JACOBI_DAMPED, damping=0.8, delta0=1e-6,
                          power_iters=150)
            outer, inner = 10, 5
        out.append(Request(r, float(arrivals[r]), ti, K, mask, lab, params, outer, inner))
    return out
