"""GPU nonlocal image graph (pdca_image_graph) against the oracle's builder.

Bar: the CSR structure (row offsets and columns) is identical; weights agree
to 1e-6 relative (the oracle takes exp in FP64 of the same FP32 distance and
rounds to float32; the kernel evaluates it in FP32 with a correction for the
rounding of the exponent, a few float32 ulps from the oracle).  The kept
neighbours are decided by FP32 distances computed in the same order on both
sides, so ties (constant patches) must break identically.  Independently of
that shared order, the GPU graphs also meet the FP64 definition wherever
FP32 rounding cannot decide otherwise (check_against_f64: edges that must be
kept are present, only edges that may be kept appear, weights within the
FP32 error of the distance).
"""

import time

import numpy as np
import pytest

from gen.workloads import SEED_BASE, ellipse_image, voronoi_image
from oracle import image_graph as IG

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(cuda_lib):
    from paper_2303_14495_gb300 import binding
    return binding


def gpu_graph(B, img, p, r, k, sigma):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(img, np.float32)).cuda()
    rp, col, w = B.image_graph(t, p, r, k, sigma)
    torch.cuda.synchronize()
    return rp.cpu().numpy(), col.cpu().numpy(), w.cpu().numpy()


def assert_same_graph(got, ref):
    rp, col, w = got
    rp_r, col_r, w_r = ref
    np.testing.assert_array_equal(rp, rp_r)
    np.testing.assert_array_equal(col, col_r)
    np.testing.assert_allclose(w, w_r, rtol=1e-6, atol=0)


@pytest.mark.parametrize("shape,p,r,k", [((5, 7, 1), 0, 1, 3), ((17, 23, 3), 1, 2, 6), ((33, 31, 3), 1, 5, 10),
                                         ((40, 12, 2), 2, 3, 12), ((9, 64, 4), 1, 4, 32), ((64, 64, 3), 1, 7, 10)])
def test_random_images(B, shape, p, r, k):
    rng = np.random.default_rng(sum(shape) + p + r + k)
    img = rng.uniform(size=shape).astype(np.float32)
    img[2:5, 1:4] = img[0, 0]                  # exact ties
    assert_same_graph(gpu_graph(B, img, p, r, k, 0.5), IG.image_graph(img, p, r, k, 0.5))


def test_constant_image_ties(B):
    img = np.full((20, 25, 3), 0.3, np.float32)
    assert_same_graph(gpu_graph(B, img, 1, 3, 8, 0.5), IG.image_graph(img, 1, 3, 8, 0.5))


@pytest.mark.parametrize("kind", ["ellipses", "voronoi"])
def test_workload_images(B, kind):
    """The synthetic images of the workloads at 128 x 128, their settings
    (3x3 patches, k = 10 in an 11x11 / 15x15 window, sigma = 0.5)."""
    rng = np.random.default_rng(SEED_BASE + 99)
    if kind == "ellipses":
        img, _ = ellipse_image(128, 6, 0.1, rng)
        r = 5
    else:
        img, _ = voronoi_image(128, 16, 4, 0.15, rng)
        r = 7
    assert_same_graph(gpu_graph(B, img, 1, r, 10, 0.5), IG.image_graph(img, 1, r, 10, 0.5))


@pytest.mark.parametrize("kind,shape,p,r,k", [("random", (48, 40, 3), 1, 4, 10), ("random", (33, 31, 1), 2, 5, 12),
                                              ("ellipses", (96, 96, 3), 1, 5, 10), ("voronoi", (96, 96, 3), 1, 7, 10)])
def test_fp64_definition(B, kind, shape, p, r, k):
    rng = np.random.default_rng(SEED_BASE + 7 + shape[0])
    if kind == "random":
        img = rng.uniform(size=shape).astype(np.float32)
    elif kind == "ellipses":
        img, _ = ellipse_image(shape[0], 6, 0.1, rng)
    else:
        img, _ = voronoi_image(shape[0], 16, 4, 0.15, rng)
    st = IG.check_against_f64(*gpu_graph(B, img, p, r, k, 0.5), img, p, r, k, 0.5)
    print(f"{kind} {shape}: {st['decided']:.3f} of the rows decided by FP64 distances alone")
    assert st["decided"] > 0.5, st


def test_voronoi2048_spot_rows(B):
    """Full 2048 x 2048 image (4 Mi pixels, 15x15 window, k = 10): rows checked
    against the oracle on crops, the graph accepted by pdca_create."""
    import torch
    rng = np.random.default_rng(SEED_BASE + 4)
    img, gt = voronoi_image(2048, 64, 4, 0.15, rng)
    t = torch.from_numpy(img).cuda()
    B.image_graph(t, 1, 7, 10, 0.5)          # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rp, col, w = B.image_graph(t, 1, 7, 10, 0.5)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    print(f"voronoi2048 image graph: {col.numel()} entries in {ms:.1f} ms")
    rp_h = rp.cpu().numpy()
    n = 2048 * 2048
    pick = np.random.default_rng(0).choice(n, 12, replace=False).tolist() + [0, 2047, n - 1, n // 2 + 1024]
    ref = IG.image_graph_rows_crop(img, 1, 7, 10, 0.5, pick)
    col_h, w_h = col.cpu().numpy(), w.cpu().numpy()
    for i in pick:
        np.testing.assert_array_equal(col_h[rp_h[i]:rp_h[i + 1]], ref[i][0])
        np.testing.assert_allclose(w_h[rp_h[i]:rp_h[i + 1]], ref[i][1], rtol=1e-6)
    deg = np.diff(rp_h)
    assert deg.min() >= 10
    # the graph goes straight into a problem on the device
    mask = np.zeros(n, np.uint8)
    mask[::997] = 1
    lab = (gt.ravel() % 4).astype(np.int32)
    prm = B.make_params(eps=1.0, eta=500.0, c=502.0, precond=B.PDCA_RICHARDSON)
    g = B.Problem(rp, col, w, 4, torch.from_numpy(mask).cuda(), torch.from_numpy(lab).cuda(), prm)
    g.solve(1, 2)
    F, _ = g.energy()
    assert np.isfinite(F)


def test_argument_errors(B):
    import torch
    img = torch.zeros((8, 8, 3), dtype=torch.float32, device="cuda")
    for kw in [dict(k=0), dict(k=33), dict(window_radius=0), dict(k=9, window_radius=1), dict(patch_radius=5),
               dict(sigma=0.0)]:
        a = dict(patch_radius=1, window_radius=2, k=4, sigma=0.5)
        a.update(kw)
        with pytest.raises(B.PdcaError, match="INVALID_ARG"):
            B.image_graph(img, a["patch_radius"], a["window_radius"], a["k"], a["sigma"])
