"""pdca_energy_static: the energy entry point that allocates nothing.

It exists for callers that cannot allocate device memory and therefore cannot
hand the library a workspace: a framework that owns every device byte
through its own fixed pool and allows no other allocator (or a plug-in loaded
into such a process), or a loop that must not pay cudaMalloc's implicit
device-wide synchronisation.  Its scratch is a fixed array inside the
library.  These tests call it through the C interface and compare it, on two
calls in a row, with the FP64 oracle's F(u) of the same iterate and with
pdca_energy (which reduces the same F over the handle's own workspace).  They
pass alone in a fresh process and after the other tests.
"""

import ctypes as C

import numpy as np
import pytest

import oracle
from gen import make_workload, random_graph

pytestmark = pytest.mark.gpu

TOL_F = 1e-5


@pytest.fixture(scope="module")
def B(cuda_lib):
    from paper_2303_14495_gb300 import binding
    return binding


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _random_case(n, K, seed):
    rp, col, w = random_graph(n, 8, seed=seed)
    rng = np.random.default_rng(seed)
    mask = (rng.uniform(size=n) < 0.1).astype(np.uint8)
    lab = rng.integers(0, max(K, 2), size=n).astype(np.int32)
    return rp, col, w, K, mask, lab, dict(eps=1.0, eta=50.0, c=52.0, precond=1, inner=3, damping=0.5)


CASES = {
    "ellipses96_K1": lambda: make_workload("ellipses256", size=96),
    "voronoi128_K4": lambda: make_workload("voronoi2048", size=128),
    "gmm_K10": lambda: make_workload("gmm70k", n_per=300, dim=32),
    "random_K4": lambda: _random_case(3001, 4, 11),
}


def _unpack(case):
    if isinstance(case, tuple):
        return case
    return case.row_ptr, case.col, case.w, case.K, case.fid_mask, case.fid_labels, case.params


@pytest.mark.parametrize("name", list(CASES))
def test_static_energy_matches_oracle(B, name):
    import torch
    rp_h, col_h, w_h, K, mask_h, lab_h, p = _unpack(CASES[name]())
    n, nnz = len(rp_h) - 1, len(col_h)
    prob = B.Problem(rp_h, col_h, w_h, K, mask_h, lab_h,
                     B.make_params(eps=p["eps"], eta=p["eta"], c=p["c"], precond=p["precond"],
                                   damping=p.get("damping") or 0.5, lambda_max=2.0))
    ref = oracle.Problem(rp_h, col_h, w_h, K, mask_h, lab_h, p["eps"], p["eta"], p["c"])
    rp, col, w = _dev(rp_h), _dev(col_h), _dev(w_h)
    mask, lab = _dev(mask_h), _dev(lab_h)
    u = torch.empty(n * K, dtype=torch.float32, device="cuda")
    F_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    seen = []
    for call in range(2):          # two calls in a row, on different iterates
        prob.step(p["inner"])
        prob.get_u(u)
        u_h = u.cpu().numpy().astype(np.float64).reshape(n, K) if K > 1 else u.cpu().numpy().astype(np.float64)
        F_orc = ref.energy(u_h)
        F_lib, _ = prob.energy()
        st, F = B.pdca_energy_static(rp, col, w, n, nnz, K, u, mask, lab, p["eps"], p["eta"], stream)
        assert st == 0, B.STATUS_NAMES[st]
        assert abs(F - F_orc) <= TOL_F * abs(F_orc), (call, F, F_orc)
        assert abs(F - F_lib) <= TOL_F * abs(F_lib), (call, F, F_lib)
        # the same call with a device output pointer gives the same value
        st2 = B.lib().pdca_energy_static(rp.data_ptr(), col.data_ptr(), w.data_ptr(), n, nnz, K,
                                         u.data_ptr(), mask.data_ptr(), lab.data_ptr(),
                                         float(p["eps"]), float(p["eta"]), C.c_void_p(stream),
                                         C.cast(C.c_void_p(F_dev.data_ptr()), C.POINTER(C.c_double)))
        assert st2 == 0
        assert F_dev.item() == F
        seen.append(F)
    assert seen[0] != seen[1]


def test_static_energy_errors_then_recovers(B):
    """Bad input reports a clear status, a device output is left untouched on
    failure, and the shared scratch does not carry a failure into the next
    call."""
    import torch
    wl = make_workload("ellipses256", size=64)
    p = wl.params
    rp, col, w = _dev(wl.row_ptr), _dev(wl.col), _dev(wl.w)
    mask, lab = _dev(wl.fid_mask), _dev(wl.fid_labels)
    u = torch.zeros(wl.n, dtype=torch.float32, device="cuda")

    def call(rp_=rp, col_=col, w_=w, n=wl.n, K=1, mask_=mask, lab_=lab):
        return B.pdca_energy_static(rp_, col_, w_, n, wl.nnz, K, u, mask_, lab_, p["eps"], p["eta"])

    # too large for the fixed scratch
    assert B.STATUS_NAMES[call(n=B.PDCA_STATIC_MAX_N + 1)[0]] == "PDCA_ERR_TOO_LARGE"
    # host pointers are refused
    assert B.STATUS_NAMES[call(rp_=wl.row_ptr)[0]] == "PDCA_ERR_INVALID_ARG"
    # a column out of range is caught before it is used
    bad = col.clone()
    bad[5] = wl.n + 7
    assert B.STATUS_NAMES[call(col_=bad)[0]] == "PDCA_ERR_BAD_GRAPH"
    # a self loop
    bad = col.clone()
    bad[int(wl.row_ptr[3])] = 3
    assert B.STATUS_NAMES[call(col_=bad)[0]] == "PDCA_ERR_BAD_GRAPH"
    # a negative and a non-finite weight
    for v in (-0.5, float("nan")):
        bw = w.clone()
        bw[9] = v
        assert B.STATUS_NAMES[call(w_=bw)[0]] == "PDCA_ERR_BAD_GRAPH", v
    # a mask value other than 0/1
    bm = mask.clone()
    bm[2] = 2
    assert B.STATUS_NAMES[call(mask_=bm)[0]] == "PDCA_ERR_BAD_GRAPH"
    # a prior label out of range on a labelled row (K = 1 takes labels 0/1)
    i = int(np.nonzero(wl.fid_mask)[0][0])
    bl = lab.clone()
    bl[i] = 2
    assert B.STATUS_NAMES[call(lab_=bl)[0]] == "PDCA_ERR_BAD_GRAPH"
    # a device output stays untouched when the call fails
    F_dev = torch.full((1,), -7.0, dtype=torch.float64, device="cuda")
    st = B.lib().pdca_energy_static(rp.data_ptr(), bad.data_ptr(), w.data_ptr(), wl.n, wl.nnz, 1,
                                    u.data_ptr(), mask.data_ptr(), lab.data_ptr(), float(p["eps"]),
                                    float(p["eta"]), C.c_void_p(torch.cuda.current_stream().cuda_stream),
                                    C.cast(C.c_void_p(F_dev.data_ptr()), C.POINTER(C.c_double)))
    assert B.STATUS_NAMES[st] == "PDCA_ERR_BAD_GRAPH"
    assert F_dev.item() == -7.0
    # a valid call right after succeeds: u = 0 gives F = n/(4 eps) + (eta/2) * #labelled
    st, F = call()
    assert st == 0
    expect = wl.n / (4 * p["eps"]) + 0.5 * p["eta"] * int(wl.fid_mask.sum())
    assert abs(F - expect) <= 1e-12 * expect
