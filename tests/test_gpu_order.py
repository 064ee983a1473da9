"""The BFS-block renumbering on the device (csrc/order_kernels.cu) against
the host implementation (csrc/reorder.cpp, pinned to the rule by
test_reorder_cpu.py): the same order, element for element, through
pdca_locality_order.  Graphs: an image graph over several 65536-node chunks,
random graphs whose levels explode, banded graphs with hubs, long paths (one
node per level), many tiny components, ragged and tiny sizes, repeated
columns, every sort window."""

import numpy as np
import pytest

from gen import make_workload, banded_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(cuda_lib):
    from paper_2303_14495_gb300 import binding
    return binding


def numpy_graph(n, avg, seed, local=0, dup=False):
    """Symmetric random CSR, increasing columns (repeated ones with dup)."""
    rng = np.random.default_rng(seed)
    m = max(1, n * avg // 2)
    a = rng.integers(0, n, m)
    b = (a + rng.integers(1, local + 1, m)) % n if local else rng.integers(0, n, m)
    keep = a != b
    e = np.concatenate([np.stack([a[keep], b[keep]], 1), np.stack([b[keep], a[keep]], 1)])
    e = np.unique(e, axis=0)
    if dup:   # every 5th entry twice
        e = np.concatenate([e, e[::5]])
        e = e[np.lexsort((e[:, 1], e[:, 0]))]
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, e[:, 0] + 1, 1)
    return np.cumsum(rp), e[:, 1].astype(np.int32)


def orders(B, rp, col, window):
    import torch
    n = rp.shape[0] - 1
    host = np.empty(n, np.int32)
    assert B.pdca_locality_order(rp, col, n, window, False, host) == 0
    d_rp = torch.from_numpy(rp).cuda()
    d_col = torch.from_numpy(col if col.size else np.zeros(1, np.int32)).cuda()
    d_out = torch.empty(n, dtype=torch.int32, device="cuda")
    st = B.pdca_locality_order(d_rp, d_col, n, window, True, d_out, torch.cuda.current_stream().cuda_stream)
    assert st == 0, B.STATUS_NAMES[st]
    return host, d_out.cpu().numpy()


def check(B, rp, col, window=0):
    host, dev = orders(B, rp, col, window)
    n = rp.shape[0] - 1
    assert np.array_equal(np.sort(host), np.arange(n))
    np.testing.assert_array_equal(dev, host)


@pytest.mark.parametrize("window", [0, 256, 32])
def test_image_graph(B, window):
    wl = make_workload("voronoi2048", size=512)       # 262144 nodes: four chunks
    check(B, wl.row_ptr, wl.col, window)


@pytest.mark.parametrize("n,avg,local", [(150000, 12, 0), (70001, 2, 1), (100000, 1, 0), (140000, 6, 40)])
def test_random_graphs(B, n, avg, local):
    """Exploding levels; a long path (one node per level); a random matching
    (tiny components); a long band."""
    rp, col = numpy_graph(n, avg, seed=n + avg, local=local)
    check(B, rp, col)


def test_banded_hubs(B):
    rp, col, _ = banded_graph(200000, 10, 3000, seed=3, far_frac=1e-3, hubs=(5, 70000, 150001), hub_deg=900)
    check(B, rp, col, 512)


@pytest.mark.parametrize("n", [1, 7, 33, 1025, 65537])
def test_small_and_ragged(B, n):
    if n == 1:
        rp, col = np.zeros(2, np.int64), np.zeros(0, np.int32)
    else:
        rp, col = numpy_graph(n, 5, seed=n)
    check(B, rp, col)


def test_repeated_columns(B):
    """A repeated column counts once, as on the host (pdca_create rejects
    such rows; the order itself does not need them excluded)."""
    rp, col = numpy_graph(20000, 6, seed=11, dup=True)
    rows = np.repeat(np.arange(20000), np.diff(rp))
    assert np.any((col[1:] == col[:-1]) & (rows[1:] == rows[:-1]))
    check(B, rp, col)


def test_bad_arguments(B):
    import torch
    rp, col = numpy_graph(100, 4, seed=1)
    out = np.empty(100, np.int32)
    assert B.pdca_locality_order(rp, col, 100, 48, False, out) == B.PDCA_ERR_INVALID_ARG     # not a power of two
    assert B.pdca_locality_order(rp, col, 100, 2048, False, out) == B.PDCA_ERR_INVALID_ARG   # above 1024
    bad = rp.copy()
    bad[50] = bad[51] + 1                                                                   # decreasing
    assert B.pdca_locality_order(bad, col, 100, 0, False, out) == B.PDCA_ERR_INVALID_ARG
    d_out = torch.empty(100, dtype=torch.int32, device="cuda")
    assert B.pdca_locality_order(rp, col, 100, 0, True, d_out) == B.PDCA_ERR_INVALID_ARG     # host graph
