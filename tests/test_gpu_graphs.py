"""pdca_solve replayed through cached CUDA graphs (pdca_graph_enable) runs
exactly the kernels of the direct path: iterates are bit-identical, in every
precision and for every starting buffer state, and the launch counter counts
the replayed kernels."""

import time

import numpy as np
import pytest

from gen import make_workload, random_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(cuda_lib):
    from paper_2303_14495_gb300 import binding
    return binding


def case(n, K, seed):
    rp, col, w = random_graph(n, 8, seed=seed)
    rng = np.random.default_rng(seed)
    mask = (rng.uniform(size=n) < 0.1).astype(np.uint8)
    lab = rng.integers(0, max(K, 2), size=n).astype(np.int32)
    return rp, col, w, mask, lab


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("K,precond", [(1, 0), (4, 2), (5, 1)])
def test_graph_replay_bitwise(B, precision, K, precond):
    import torch
    rp, col, w, mask, lab = case(1500, K, 40 + K + precision)
    prm = B.make_params(eps=1.0, eta=20.0, c=22.0, precond=precond, damping=0.8, precision=precision)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    direct = B.Problem(rp, col, w, K, mask, lab, prm, stream=s1)
    graphed = B.Problem(rp, col, w, K, mask, lab, prm, stream=s2)
    graphed.graphs(True)
    for rep in range(4):                  # set_u rotates the starting buffers
        n0 = B.pdca_kernel_launches()
        direct.set_u(None)
        direct.solve(3, 4)
        n1 = B.pdca_kernel_launches()
        graphed.set_u(None)
        graphed.solve(3, 4)
        n2 = B.pdca_kernel_launches()
        np.testing.assert_array_equal(graphed.get_u(), direct.get_u())
        assert n2 - n1 == n1 - n0   # the replayed kernels are counted like direct ones
    # continuing from the previous iterate (has_prev), and after a damping change
    direct.solve(2, 4, damping=0.7 if precond == 0 else 0.0)
    graphed.solve(2, 4, damping=0.7 if precond == 0 else 0.0)
    np.testing.assert_array_equal(graphed.get_u(), direct.get_u())
    assert direct.energy() == graphed.energy()
    graphed.graphs(False)
    graphed.solve(1, 2)
    direct.solve(1, 2)
    np.testing.assert_array_equal(graphed.get_u(), direct.get_u())


def test_graph_replay_small_problem_time(B):
    """The two-moons workload (2000 nodes): launch-bound, so the replay is faster."""
    import torch
    wl = make_workload("moons2k")
    p = wl.params
    prm = B.params_from_workload(p)
    st = torch.cuda.Stream()
    g = B.Problem(wl.row_ptr, wl.col, wl.w, wl.K, wl.fid_mask, wl.fid_labels, prm, stream=st)

    def run(reps=50):
        for _ in range(3):
            g.set_u(None)
            g.solve(p["outer"], p["inner"])
        st.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            g.set_u(None)
            g.solve(p["outer"], p["inner"])
        st.synchronize()
        return (time.perf_counter() - t0) / reps * 1e3

    direct = run()
    g.graphs(True)
    replay = run()
    print(f"moons2k solve ({p['outer']} x {p['inner']}): direct {direct:.3f} ms, graph replay {replay:.3f} ms")
    assert replay < direct
