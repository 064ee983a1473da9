"""Host-side checks of the C interface that need no GPU: the library builds,
loads, exports every symbol the header declares, and rejects bad arguments
before touching the device."""

import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_2303_14495_gb300 import build as bld
    bld.build()
    from paper_2303_14495_gb300 import binding
    binding.lib()
    return binding


def header_functions():
    src = open(os.path.join(ROOT, "include", "pdca.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pdca_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(B):
    names = header_functions()
    assert len(names) >= 15
    L = B.lib()
    for name in names:
        assert hasattr(L, name), name
    assert sorted(B.EXPORTS) == names


def test_status_strings_and_defaults(B):
    for st in range(10):
        assert B.pdca_status_string(st) not in ("", "unknown status")
    assert B.pdca_status_string(99) == "unknown status"
    p = B.pdca_default_params()
    assert (p.eps, p.c, p.eta, p.precond, p.delta0, p.power_iters) == (1.0, 3.0, 1.0, 1, 1e-6, 150)


def ring(n):
    from gen import csr_from_pairs
    i = np.arange(n - 1)
    return csr_from_pairs(n, i, i + 1, np.ones(n - 1, np.float32))


def test_workspace_size_host(B):
    rp, col, w = ring(1000)
    s1 = B.pdca_workspace_size(rp, 1000, 1)
    s4 = B.pdca_workspace_size(rp, 1000, 4)
    assert 0 < s1 < s4
    # the layout covers at least CSR staging + 3 iterates
    assert s4 >= 3 * 1000 * 4 * 4 + col.size * 8
    for n, k in [(0, 1), (1000, 0), (1000, 17)]:
        with pytest.raises(B.PdcaError, match="INVALID_ARG"):
            B.pdca_workspace_size(rp, n, k)
    bad = rp.copy()
    bad[5] = bad[6] + 1
    with pytest.raises(B.PdcaError, match="INVALID_ARG"):
        B.pdca_workspace_size(bad, 1000, 1)
    for sw in (16, 100, 16384):
        with pytest.raises(B.PdcaError, match="INVALID_ARG"):
            B.pdca_workspace_size(rp, 1000, 1, B.make_params(sort_window=sw))
    assert B.pdca_workspace_size(rp, 1000, 1, B.make_params(sort_window=32)) > 0


def test_create_rejects_before_device_work(B):
    rp, col, w = ring(64)
    mask = np.zeros(64, np.uint8)
    lab = np.zeros(64, np.int32)
    ws = C.create_string_buffer(1 << 16)
    addr = (C.addressof(ws) + 255) // 256 * 256

    def create(params, k=1, workspace=addr, n=64):
        st, h = B.pdca_create(rp, col, w, n, k, mask, lab, params, workspace, 1 << 16, 0)
        return st

    P = B.make_params
    assert create(P(), k=0) == 1
    assert create(P(), k=17) == 1
    assert create(P(), n=0) == 1
    # damped Jacobi with omega = 0.8 needs c > 3 eps (G > T, Sec. 3.1)
    st, h = B.pdca_create(rp, col, w, 64, 1, mask, lab,
                          P(eps=1.0, c=2.0, precond=B.PDCA_JACOBI_DAMPED, damping=0.8),
                          C.c_void_p(addr), 1 << 16, 0)
    assert st == 4
    st, h = B.pdca_create(rp, col, w, 64, 1, mask, lab,
                          P(precond=B.PDCA_JACOBI_PERTURBED, delta0=0.0), C.c_void_p(addr), 1 << 16, 0)
    assert st == 4
    # unknown Laplacian, tiled unnormalized Laplacian, bad step size / negative
    # eps / unaligned workspace
    for bad in (P(laplacian=2), P(laplacian=1, tiling=B.PDCA_TILING_ON), P(step_k=-1.0), P(entry_order=2),
                P(step_k=float("nan")), P(step_k=float("inf"))):
        st, _ = B.pdca_create(rp, col, w, 64, 1, mask, lab, bad, C.c_void_p(addr), 1 << 16, 0)
        assert st == 1
    st, _ = B.pdca_create(rp, col, w, 64, 1, mask, lab, P(eps=-1.0), C.c_void_p(addr), 1 << 16, 0)
    assert st == 1
    st, _ = B.pdca_create(rp, col, w, 64, 1, mask, lab, P(), C.c_void_p(addr + 8), 1 << 16, 0)
    assert st == 1
    # a workspace smaller than pdca_workspace_size is refused before any copy
    st, _ = B.pdca_create(rp, col, w, 64, 1, mask, lab, P(), C.c_void_p(addr), 1024, 0)
    assert st == 6


def test_no_oracle_in_product():
    """The library package never imports the oracle or falls back to the CPU."""
    pkg = os.path.join(ROOT, "paper_2303_14495_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "pdca_oracle" not in text, f


def test_async_entry_points_reject_before_device_work(B):
    """The asynchronous admission, labels and release calls check their
    arguments before any device work (NULL handles; NULL out pointer)."""
    lib = B.lib()
    h = C.c_void_p()
    mask = np.zeros(8, np.uint8)
    lab = np.zeros(8, np.int32)
    ws = C.create_string_buffer(1 << 12)
    p = B.make_params()
    assert lib.pdca_create_like_async(None, 2, mask.ctypes.data, lab.ctypes.data, C.byref(p), C.addressof(ws),
                                      1 << 12, C.byref(h)) == 1
    assert h.value is None
    assert lib.pdca_create_like_async(None, 2, mask.ctypes.data, lab.ctypes.data, C.byref(p), C.addressof(ws),
                                      1 << 12, None) == 1
    out = np.zeros(8, np.int32)
    st = np.zeros(1, np.uint32)
    assert lib.pdca_labels_async(None, out.ctypes.data, st.ctypes.data) == 1
    lib.pdca_release(None)          # ignored, like pdca_destroy(NULL)
