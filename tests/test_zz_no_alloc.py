"""pdca_energy_static: the energy entry point that allocates nothing.

It exists for callers that cannot allocate device memory and therefore cannot
hand the library a workspace (code inside a CUDA stream capture, frameworks
that own all device memory through a fixed pool, loops that must not pay
cudaMalloc's synchronisation).  Its scratch is a fixed array inside the
library.  These tests call it through the C interface and compare it with
pdca_energy, which reduces the same F(u) over the handle's own workspace, on
two calls in a row; they pass alone in a fresh process and after the other
tests.
"""

import numpy as np
import pytest

from gen import make_workload

pytestmark = pytest.mark.gpu

TOL_F = 1e-5


@pytest.fixture(scope="module")
def B(cuda_lib):
    from paper_2303_14495_gb300 import binding
    return binding


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("name,kw", [("ellipses256", {"size": 96}), ("voronoi2048", {"size": 128}),
                                     ("gmm70k", {"n_per": 300, "dim": 32})])
def test_static_energy_matches_pdca_energy(B, name, kw):
    import torch
    wl = make_workload(name, **kw)
    p = wl.params
    prob = B.Problem(wl.row_ptr, wl.col, wl.w, wl.K, wl.fid_mask, wl.fid_labels,
                     B.params_from_workload(p))
    rp, col, w = _dev(wl.row_ptr), _dev(wl.col), _dev(wl.w)
    mask, lab = _dev(wl.fid_mask), _dev(wl.fid_labels)
    u = torch.empty(wl.n * wl.K, dtype=torch.float32, device="cuda")
    F_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    seen = []
    for call in range(2):          # two calls in a row, on different iterates
        prob.step(p["inner"])
        F_ref, _ = prob.energy()
        prob.get_u(u)
        st, F = B.pdca_energy_static(rp, col, w, wl.n, wl.nnz, wl.K, u, mask, lab,
                                     p["eps"], p["eta"], stream)
        assert st == 0, B.STATUS_NAMES[st]
        assert abs(F - F_ref) <= TOL_F * abs(F_ref), (call, F, F_ref)
        # the same call with a device output pointer gives the same value
        import ctypes as C
        st2 = B.lib().pdca_energy_static(rp.data_ptr(), col.data_ptr(), w.data_ptr(), wl.n, wl.nnz,
                                         wl.K, u.data_ptr(), mask.data_ptr(), lab.data_ptr(),
                                         float(p["eps"]), float(p["eta"]), C.c_void_p(stream),
                                         C.cast(C.c_void_p(F_dev.data_ptr()), C.POINTER(C.c_double)))
        assert st2 == 0
        assert F_dev.item() == F
        seen.append(F)
    assert seen[0] != seen[1]


def test_static_energy_errors_then_recovers(B):
    """Bad input reports a clear status, and the shared scratch does not carry
    the failure into the next call."""
    import torch
    wl = make_workload("ellipses256", size=64)
    p = wl.params
    rp, col, w = _dev(wl.row_ptr), _dev(wl.col), _dev(wl.w)
    mask, lab = _dev(wl.fid_mask), _dev(wl.fid_labels)
    u = torch.zeros(wl.n, dtype=torch.float32, device="cuda")
    # too large for the fixed scratch
    st, _ = B.pdca_energy_static(rp, col, w, B.PDCA_STATIC_MAX_N + 1, wl.nnz, 1, u, mask, lab,
                                 p["eps"], p["eta"])
    assert B.STATUS_NAMES[st] == "PDCA_ERR_TOO_LARGE"
    # host pointers are refused
    st, _ = B.pdca_energy_static(wl.row_ptr, col, w, wl.n, wl.nnz, 1, u, mask, lab, p["eps"], p["eta"])
    assert B.STATUS_NAMES[st] == "PDCA_ERR_INVALID_ARG"
    # a column out of range is caught before it is used
    bad = col.clone()
    bad[5] = wl.n + 7
    st, _ = B.pdca_energy_static(rp, bad, w, wl.n, wl.nnz, 1, u, mask, lab, p["eps"], p["eta"])
    assert B.STATUS_NAMES[st] == "PDCA_ERR_BAD_GRAPH"
    # a valid call right after succeeds: u = 0 gives F = n/(4 eps) + (eta/2) * #labelled
    st, F = B.pdca_energy_static(rp, col, w, wl.n, wl.nnz, 1, u, mask, lab, p["eps"], p["eta"])
    assert st == 0
    expect = wl.n / (4 * p["eps"]) + 0.5 * p["eta"] * int(wl.fid_mask.sum())
    assert abs(F - expect) <= 1e-12 * expect
