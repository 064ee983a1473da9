"""Thin Python binding of ``libpdca.so`` (argument marshalling only).

The functions ``pdca_*`` mirror the C interface of ``include/pdca.h`` one to
one.  ``Problem`` bundles them with a device workspace allocated by PyTorch
(PyTorch owns every byte of device memory; the library allocates none).
Every computation runs in the library's CUDA kernels; there is no CPU path.
If the library has not been built, ``lib()`` raises.
"""

from __future__ import annotations

import ctypes as C
import math
import os
import threading
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# PDCA_LIB may name another build of the same library (e.g. a tuning variant)
LIB_PATH = os.environ.get("PDCA_LIB") or os.path.join(HERE, "_build", "libpdca.so")

PDCA_MAX_K = 16

PDCA_OK = 0
STATUS_NAMES = {
    0: "PDCA_OK", 1: "PDCA_ERR_INVALID_ARG", 2: "PDCA_ERR_NOT_SYMMETRIC",
    3: "PDCA_ERR_ISOLATED_NODE", 4: "PDCA_ERR_INFEASIBLE", 5: "PDCA_ERR_NONFINITE",
    6: "PDCA_ERR_OOM", 7: "PDCA_ERR_CUDA", 8: "PDCA_ERR_TIMEOUT", 9: "PDCA_ERR_BAD_GRAPH",
    10: "PDCA_ERR_TOO_LARGE", 11: "PDCA_ERR_NOT_CONVERGED",
}
globals().update({name: code for code, name in STATUS_NAMES.items()})   # PDCA_ERR_* constants
PDCA_STATIC_MAX_N = 1 << 20
PDCA_LAP_NORMALIZED, PDCA_LAP_UNNORMALIZED = 0, 1
PDCA_JACOBI_DAMPED, PDCA_JACOBI_PERTURBED, PDCA_RICHARDSON = 0, 1, 2
PDCA_FP32, PDCA_MIXED_BF16W_FP16U, PDCA_MIXED_BF16W_BF16U = 0, 1, 2
PDCA_REORDER_NONE, PDCA_REORDER_BFS = 0, 1
PDCA_TILING_AUTO, PDCA_TILING_OFF, PDCA_TILING_ON = 0, 1, 2
PDCA_ENTRIES_SPREAD, PDCA_ENTRIES_CSR = 0, 1
PDCA_COLUMNS_AUTO, PDCA_COLUMNS_32 = 0, 1

# every symbol include/pdca.h declares
EXPORTS = [
    "pdca_default_params", "pdca_workspace_size", "pdca_create", "pdca_set_u", "pdca_step",
    "pdca_solve", "pdca_energy", "pdca_get_u", "pdca_labels", "pdca_lambda_max", "pdca_layout",
    "pdca_profile_enable", "pdca_profile_read", "pdca_kernel_launches", "pdca_destroy",
    "pdca_status_string", "pdca_energy_static",
    "pdca_batch_create", "pdca_batch_add", "pdca_batch_step", "pdca_batch_poll", "pdca_batch_remove",
    "pdca_batch_destroy", "pdca_workspace_size_like", "pdca_create_like",
    "pdca_spectral_workspace_size", "pdca_spectral_init",
    "pdca_image_graph_workspace_size", "pdca_image_graph",
    "pdca_point_graph_workspace_size", "pdca_point_graph", "pdca_graph_enable", "pdca_locality_order",
    "pdca_create_like_async", "pdca_labels_async", "pdca_release",
]


class PdcaError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)}")


class pdca_params(C.Structure):
    _fields_ = [
        ("eps", C.c_double), ("c", C.c_double), ("eta", C.c_double),
        ("laplacian", C.c_int32), ("precond", C.c_int32),
        ("damping", C.c_double), ("delta0", C.c_double), ("lambda_max", C.c_double),
        ("power_iters", C.c_int32), ("precision", C.c_int32),
        ("sort_window", C.c_int32), ("reorder", C.c_int32), ("tiling", C.c_int32),
        ("entry_order", C.c_int32), ("step_k", C.c_double), ("columns", C.c_int32),
        ("row_split", C.c_int32), ("block_slices", C.c_int32),
    ]


_lock = threading.Lock()
_lib = None


def lib():
    """Load the built CUDA library (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built ({LIB_PATH}); run __graft_entry__.build()")
            L = C.CDLL(LIB_PATH)
            vp, i32, i64, u64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
            P = C.POINTER(pdca_params)
            sig = {
                "pdca_default_params": (None, [P]),
                "pdca_workspace_size": (C.c_int, [vp, i32, i32, P, C.POINTER(C.c_size_t)]),
                "pdca_create": (C.c_int, [vp, vp, vp, i32, i32, vp, vp, P, vp, C.c_size_t, vp,
                                          C.POINTER(vp)]),
                "pdca_set_u": (C.c_int, [vp, vp]),
                "pdca_step": (C.c_int, [vp, i32]),
                "pdca_solve": (C.c_int, [vp, i32, i32, dbl, vp, vp]),
                "pdca_energy": (C.c_int, [vp, C.POINTER(dbl), C.POINTER(dbl)]),
                "pdca_get_u": (C.c_int, [vp, vp]),
                "pdca_labels": (C.c_int, [vp, vp]),
                "pdca_lambda_max": (C.c_int, [vp, C.POINTER(dbl), C.POINTER(dbl)]),
                "pdca_layout": (C.c_int, [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i32),
                                          C.POINTER(i32), C.POINTER(i64), C.POINTER(i32), C.POINTER(i64),
                                          C.POINTER(i32), C.POINTER(i64)]),
                "pdca_profile_enable": (C.c_int, [vp, i32]),
                "pdca_profile_read": (C.c_int, [vp, C.POINTER(dbl), C.POINTER(i64)]),
                "pdca_kernel_launches": (u64, []),
                "pdca_destroy": (None, [vp]),
                "pdca_status_string": (C.c_char_p, [C.c_int]),
                "pdca_energy_static": (C.c_int, [vp, vp, vp, i32, i64, i32, vp, vp, vp, dbl, dbl,
                                                 vp, C.POINTER(dbl)]),
                "pdca_batch_create": (C.c_int, [i32, vp, C.POINTER(vp)]),
                "pdca_batch_add": (C.c_int, [vp, vp, i32, i32]),
                "pdca_batch_step": (C.c_int, [vp, i32, C.POINTER(i32)]),
                "pdca_batch_poll": (C.c_int, [vp, C.POINTER(vp), i32, C.POINTER(i32)]),
                "pdca_batch_remove": (C.c_int, [vp, vp]),
                "pdca_batch_destroy": (None, [vp]),
                "pdca_workspace_size_like": (C.c_int, [vp, i32, P, C.POINTER(C.c_size_t)]),
                "pdca_create_like": (C.c_int, [vp, i32, vp, vp, P, vp, C.c_size_t, C.POINTER(vp)]),
                "pdca_create_like_async": (C.c_int, [vp, i32, vp, vp, P, vp, C.c_size_t, C.POINTER(vp)]),
                "pdca_labels_async": (C.c_int, [vp, vp, vp]),
                "pdca_release": (None, [vp]),
                "pdca_spectral_workspace_size": (C.c_int, [vp, C.POINTER(C.c_size_t)]),
                "pdca_spectral_init": (C.c_int, [vp, vp, C.c_size_t, i32, dbl, C.POINTER(dbl), vp,
                                                 C.POINTER(i32)]),
                "pdca_image_graph_workspace_size": (C.c_int, [i32, i32, i32, C.POINTER(C.c_size_t)]),
                "pdca_image_graph": (C.c_int, [vp, i32, i32, i32, i32, i32, i32, dbl, vp, C.c_size_t, vp, vp,
                                               vp, i64, C.POINTER(i64), vp]),
                "pdca_point_graph_workspace_size": (C.c_int, [i64, i32, i32, C.POINTER(C.c_size_t)]),
                "pdca_graph_enable": (C.c_int, [vp, i32]),
                "pdca_point_graph": (C.c_int, [vp, i64, i32, i32, i32, vp, C.c_size_t, vp, vp, vp, i64,
                                               C.POINTER(i64), vp]),
                "pdca_locality_order": (C.c_int, [vp, vp, i32, i32, i32, vp, vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
        return _lib


def _check(status: int, what: str):
    if status != PDCA_OK:
        raise PdcaError(status, what)


def _ptr(a) -> Optional[int]:
    """Address of a numpy array or torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, C.c_void_p):
        return a.value
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def make_params(eps=1.0, c=3.0, eta=1.0, precond=PDCA_JACOBI_PERTURBED, damping=0.5, delta0=1e-6,
                lambda_max=0.0, power_iters=150, laplacian=PDCA_LAP_NORMALIZED,
                precision=PDCA_FP32, sort_window=0, reorder=PDCA_REORDER_BFS,
                tiling=PDCA_TILING_AUTO, step_k=0.0, entry_order=PDCA_ENTRIES_SPREAD,
                columns=PDCA_COLUMNS_AUTO, row_split=0, block_slices=0) -> pdca_params:
    p = pdca_params()
    lib().pdca_default_params(C.byref(p))
    p.eps, p.c, p.eta = float(eps), float(c), float(eta)
    p.precond, p.damping, p.delta0 = int(precond), float(damping), float(delta0)
    p.lambda_max, p.power_iters = float(lambda_max), int(power_iters)
    p.laplacian, p.precision, p.sort_window = int(laplacian), int(precision), int(sort_window)
    p.reorder, p.tiling, p.step_k = int(reorder), int(tiling), float(step_k)
    p.entry_order = int(entry_order)
    p.columns = int(columns)
    p.row_split = int(row_split)
    p.block_slices = int(block_slices)
    return p


# ---- one-to-one wrappers of the C entry points ------------------------------

def pdca_default_params() -> pdca_params:
    p = pdca_params()
    lib().pdca_default_params(C.byref(p))
    return p


def pdca_workspace_size(row_ptr, n: int, k: int, params: Optional[pdca_params] = None) -> int:
    out = C.c_size_t(0)
    st = lib().pdca_workspace_size(_ptr(row_ptr), int(n), int(k),
                                   C.byref(params) if params is not None else None, C.byref(out))
    _check(st, "pdca_workspace_size")
    return int(out.value)


def workspace_size_like(base: "Problem", k: int, params: pdca_params) -> int:
    out = C.c_size_t(0)
    _check(lib().pdca_workspace_size_like(base.h, int(k), C.byref(params), C.byref(out)),
           "pdca_workspace_size_like")
    return int(out.value)


def pdca_create(row_ptr, col, w, n, k, fid_mask, labels, params, workspace, ws_bytes, stream=0):
    h = C.c_void_p()
    st = lib().pdca_create(_ptr(row_ptr), _ptr(col), _ptr(w), int(n), int(k), _ptr(fid_mask),
                           _ptr(labels), C.byref(params) if params is not None else None,
                           _ptr(workspace), int(ws_bytes), C.c_void_p(int(stream)), C.byref(h))
    return st, h


def pdca_set_u(h, u=None) -> int:
    return lib().pdca_set_u(h, _ptr(u))


def pdca_step(h, inner: int) -> int:
    return lib().pdca_step(h, int(inner))


def pdca_solve(h, outer: int, inner: int, damping: float = 0.0, energy_trace=None,
               residual_trace=None) -> int:
    return lib().pdca_solve(h, int(outer), int(inner), float(damping), _ptr(energy_trace),
                            _ptr(residual_trace))


def pdca_energy(h):
    F, r = C.c_double(0.0), C.c_double(0.0)
    st = lib().pdca_energy(h, C.byref(F), C.byref(r))
    return st, F.value, r.value


def pdca_get_u(h, out) -> int:
    return lib().pdca_get_u(h, _ptr(out))


def pdca_labels(h, out) -> int:
    return lib().pdca_labels(h, _ptr(out))


def pdca_lambda_max(h):
    a, b = C.c_double(0.0), C.c_double(0.0)
    st = lib().pdca_lambda_max(h, C.byref(a), C.byref(b))
    return st, a.value, b.value


def pdca_layout(h):
    e, s, w = C.c_int64(0), C.c_int64(0), C.c_int32(0)
    t, hr, mh, s16 = C.c_int32(0), C.c_int64(0), C.c_int32(0), C.c_int64(0)
    sl, sr = C.c_int32(0), C.c_int64(0)
    st = lib().pdca_layout(h, C.byref(e), C.byref(s), C.byref(w), C.byref(t), C.byref(hr), C.byref(mh),
                           C.byref(s16), C.byref(sl), C.byref(sr))
    return st, dict(sell_entries=e.value, n_slices=s.value, sort_window=w.value, tiled=bool(t.value),
                    halo_rows=hr.value, max_halo=mh.value, slices16=s16.value, split_len=sl.value,
                    split_rows=sr.value)


def pdca_locality_order(row_ptr, col, n: int, sort_window: int, device: bool, order, stream=0) -> int:
    """The BFS-block renumbering (order[p] = node at position p); device=True:
    the CUDA kernels (device arrays, ``stream`` a raw CUDA stream handle),
    else the host implementation (host arrays)."""
    return lib().pdca_locality_order(_ptr(row_ptr), _ptr(col), int(n), int(sort_window), 1 if device else 0,
                                     _ptr(order), C.c_void_p(int(stream)))


def pdca_profile_enable(h, on: bool) -> int:
    return lib().pdca_profile_enable(h, 1 if on else 0)


def pdca_profile_read(h):
    ms, cnt = C.c_double(0.0), C.c_int64(0)
    st = lib().pdca_profile_read(h, C.byref(ms), C.byref(cnt))
    return st, ms.value, cnt.value


def pdca_kernel_launches() -> int:
    return int(lib().pdca_kernel_launches())


def pdca_destroy(h) -> None:
    lib().pdca_destroy(h)


def pdca_energy_static(row_ptr, col, w, n, nnz, k, u, fid_mask, labels, eps, eta, stream=0):
    """F(u) from a device CSR without any allocation (fixed library scratch);
    returns (status, F).  F is the energy of the normalized Laplacian L_s
    only: for a problem created with PDCA_LAP_UNNORMALIZED it differs from
    pdca_energy's value.  Calls share the library's scratch, so calls that
    overlap on the GPU race; the call synchronises `stream`."""
    F = C.c_double(float("nan"))
    st = lib().pdca_energy_static(_ptr(row_ptr), _ptr(col), _ptr(w), int(n), int(nnz), int(k),
                                  _ptr(u), _ptr(fid_mask), _ptr(labels), float(eps), float(eta),
                                  C.c_void_p(int(stream)), C.byref(F))
    return st, F.value


def pdca_status_string(st: int) -> str:
    return lib().pdca_status_string(int(st)).decode()


# ---- convenience object -----------------------------------------------------

class Problem:
    """A created pDCA problem with a PyTorch-owned device workspace.

    Graph and fidelity arrays may be numpy arrays or torch tensors (host or
    CUDA).  ``stream``: a ``torch.cuda.Stream`` (default: the current one).
    """

    def __init__(self, row_ptr, col, w, K, fid_mask, fid_labels, params: pdca_params,
                 device="cuda", stream=None):
        import torch
        self.torch = torch
        self.n = int(row_ptr.shape[0] - 1)
        self.K = int(K)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._keep = (row_ptr, col, w, fid_mask, fid_labels)
        self.ws_bytes = pdca_workspace_size(row_ptr, self.n, self.K, params)
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        st, h = pdca_create(row_ptr, col, w, self.n, self.K, fid_mask, fid_labels, params,
                            self.workspace, self.ws_bytes, self.stream.cuda_stream)
        _check(st, "pdca_create")
        self.h = h

    @classmethod
    def like(cls, base: "Problem", K, fid_mask, fid_labels, params: pdca_params, wait: bool = True):
        """A problem on base's graph (shared, read-only operator); see pdca_create_like.

        wait=False calls pdca_create_like_async: nothing waits for the stream,
        the fidelity arrays must stay unchanged until the stream has copied
        them (pass device tensors or pinned host tensors), and a failed
        fidelity check shows in ``labels`` / ``labels_async``."""
        import torch
        self = cls.__new__(cls)
        self.torch = torch
        self.n, self.K = base.n, int(K)
        self.device, self.stream = base.device, base.stream
        self._base = base                      # keeps the shared operator alive
        self._keep = (fid_mask, fid_labels)
        out = C.c_size_t(0)
        _check(lib().pdca_workspace_size_like(base.h, self.K, C.byref(params), C.byref(out)),
               "pdca_workspace_size_like")
        self.ws_bytes = int(out.value)
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        h = C.c_void_p()
        name = "pdca_create_like" if wait else "pdca_create_like_async"
        _check(getattr(lib(), name)(base.h, self.K, _ptr(fid_mask), _ptr(fid_labels), C.byref(params),
                                    _ptr(self.workspace), self.ws_bytes, C.byref(h)), name)
        self.h = h
        return self

    def close(self):
        if getattr(self, "h", None):
            pdca_destroy(self.h)
            self.h = None

    def release(self):
        """pdca_release: drop the handle without waiting for the stream.  The
        workspace tensor goes back to PyTorch's caching allocator marked as
        used by the problem's stream (record_stream), so the allocator hands
        it out again only after the work enqueued there has finished."""
        if getattr(self, "h", None):
            lib().pdca_release(self.h)
            self.h = None
        ws = getattr(self, "workspace", None)
        if ws is not None:
            ws.record_stream(self.stream)
        self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_u(self, u=None):
        _check(pdca_set_u(self.h, u), "pdca_set_u")

    def step(self, inner: int):
        _check(pdca_step(self.h, inner), "pdca_step")

    def solve(self, outer: int, inner: int, damping: float = 0.0, trace: bool = False):
        if trace:
            e = np.zeros(max(outer, 1), np.float64)
            r = np.zeros(max(outer, 1), np.float64)
            _check(pdca_solve(self.h, outer, inner, damping, e, r), "pdca_solve")
            return e[:outer], r[:outer]
        _check(pdca_solve(self.h, outer, inner, damping), "pdca_solve")
        return None

    def energy(self):
        st, F, r = pdca_energy(self.h)
        _check(st, "pdca_energy")
        return F, r

    def get_u(self, out=None):
        if out is None:
            shape = (self.n,) if self.K == 1 else (self.n, self.K)
            out = np.empty(shape, np.float32)
        _check(pdca_get_u(self.h, out), "pdca_get_u")
        return out

    def labels(self, out=None):
        if out is None:
            out = np.empty(self.n, np.int32)
        _check(pdca_labels(self.h, out), "pdca_labels")
        return out

    def labels_async(self, out, status=None):
        """pdca_labels_async: enqueue the labels into ``out`` (a device or
        pinned host int32 tensor of n) and the fidelity-check word into
        ``status`` (one int32 or uint32 element, or None); both are valid once
        the stream has passed the call."""
        _check(lib().pdca_labels_async(self.h, _ptr(out), _ptr(status)), "pdca_labels_async")
        return out

    def spectral_init(self, max_iters: int = 500, tol: float = 1e-5, strict: bool = True):
        """u^0 from the second eigenvector of the Laplacian (pdca_spectral_init).

        Returns (lambda_2, u0 as a numpy array in node order, iterations).  The
        scratch is a PyTorch tensor freed on return.  strict=False accepts
        PDCA_ERR_NOT_CONVERGED (u^0 is then set from the last Ritz vector)."""
        out = C.c_size_t(0)
        _check(lib().pdca_spectral_workspace_size(self.h, C.byref(out)), "pdca_spectral_workspace_size")
        ws = self.torch.empty(int(out.value), dtype=self.torch.uint8, device=self.device)
        lam = C.c_double(0.0)
        its = C.c_int32(0)
        u0 = np.empty(self.n, np.float32)
        st = lib().pdca_spectral_init(self.h, _ptr(ws), int(out.value), int(max_iters), float(tol), C.byref(lam),
                                      _ptr(u0), C.byref(its))
        if not (st == PDCA_OK or (st == 11 and not strict)):
            _check(st, "pdca_spectral_init")
        return float(lam.value), u0, int(its.value)

    def lambda_max(self):
        st, used, est = pdca_lambda_max(self.h)
        _check(st, "pdca_lambda_max")
        return used, est

    def layout(self):
        st, d = pdca_layout(self.h)
        _check(st, "pdca_layout")
        return d

    def graphs(self, on: bool):
        """pdca_graph_enable: replay pdca_solve through cached CUDA graphs."""
        _check(lib().pdca_graph_enable(self.h, int(bool(on))), "pdca_graph_enable")

    def profile(self, on: bool):
        _check(pdca_profile_enable(self.h, on), "pdca_profile_enable")

    def profile_read(self):
        st, ms, cnt = pdca_profile_read(self.h)
        _check(st, "pdca_profile_read")
        return ms, cnt


class Batch:
    """Continuous batch of problems advanced together (pdca_batch_*).

    Problems must live on the batch's stream.  ``add`` a Problem with its
    outer / inner counts, ``step`` passes, ``poll`` the finished Problems."""

    def __init__(self, max_problems: int = 1024, stream=None):
        import torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        _check(lib().pdca_batch_create(int(max_problems), C.c_void_p(self.stream.cuda_stream), C.byref(h)),
               "pdca_batch_create")
        self.h = h
        self._by_handle = {}

    def add(self, prob: "Problem", outer: int, inner: int):
        _check(lib().pdca_batch_add(self.h, prob.h, int(outer), int(inner)), "pdca_batch_add")
        self._by_handle[prob.h.value] = prob

    def step(self, passes: int) -> int:
        active = C.c_int32(0)
        _check(lib().pdca_batch_step(self.h, int(passes), C.byref(active)), "pdca_batch_step")
        return int(active.value)

    def poll(self, capacity: int = 4096):
        arr = (C.c_void_p * max(capacity, 1))()
        cnt = C.c_int32(0)
        _check(lib().pdca_batch_poll(self.h, arr, int(capacity), C.byref(cnt)), "pdca_batch_poll")
        return [self._by_handle.pop(arr[i]) for i in range(cnt.value)]

    def remove(self, prob: "Problem"):
        _check(lib().pdca_batch_remove(self.h, prob.h), "pdca_batch_remove")
        self._by_handle.pop(prob.h.value, None)

    def close(self):
        if getattr(self, "h", None):
            lib().pdca_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def image_graph(image, patch_radius: int, window_radius: int, k: int, sigma: float, stream=None):
    """pdca_image_graph on a torch CUDA tensor image (H x W x C float32).

    Returns (row_ptr int64, col int32, w float32) as CUDA tensors trimmed to
    the graph's nnz; the scratch and the outputs are PyTorch allocations."""
    import torch
    img = image.contiguous()
    assert img.is_cuda and img.dtype == torch.float32 and img.dim() == 3
    H, W, Cc = (int(v) for v in img.shape)
    st = stream if stream is not None else torch.cuda.current_stream(img.device)
    out = C.c_size_t(0)
    _check(lib().pdca_image_graph_workspace_size(H, W, int(k), C.byref(out)), "pdca_image_graph_workspace_size")
    ws = torch.empty(int(out.value), dtype=torch.uint8, device=img.device)
    cap = 2 * int(k) * H * W
    rp = torch.empty(H * W + 1, dtype=torch.int64, device=img.device)
    col = torch.empty(cap, dtype=torch.int32, device=img.device)
    w = torch.empty(cap, dtype=torch.float32, device=img.device)
    nnz = C.c_int64(0)
    _check(lib().pdca_image_graph(_ptr(img), H, W, Cc, int(patch_radius), int(window_radius), int(k),
                                  float(sigma), _ptr(ws), int(out.value), _ptr(rp), _ptr(col), _ptr(w), cap,
                                  C.byref(nnz), C.c_void_p(st.cuda_stream)), "pdca_image_graph")
    m = int(nnz.value)
    return rp, col[:m], w[:m]


def point_graph(X, k: int, scale_nn: int = 7, stream=None):
    """pdca_point_graph on a torch CUDA tensor X (n x dim float32).

    Returns (row_ptr int64, col int32, w float32) CUDA tensors trimmed to nnz."""
    import torch
    Xc = X.contiguous()
    assert Xc.is_cuda and Xc.dtype == torch.float32 and Xc.dim() == 2
    n, dim = (int(v) for v in Xc.shape)
    st = stream if stream is not None else torch.cuda.current_stream(Xc.device)
    out = C.c_size_t(0)
    _check(lib().pdca_point_graph_workspace_size(n, dim, int(k), C.byref(out)), "pdca_point_graph_workspace_size")
    ws = torch.empty(int(out.value), dtype=torch.uint8, device=Xc.device)
    cap = 2 * int(k) * n
    rp = torch.empty(n + 1, dtype=torch.int64, device=Xc.device)
    col = torch.empty(cap, dtype=torch.int32, device=Xc.device)
    w = torch.empty(cap, dtype=torch.float32, device=Xc.device)
    nnz = C.c_int64(0)
    _check(lib().pdca_point_graph(_ptr(Xc), n, dim, int(k), int(scale_nn), _ptr(ws), int(out.value), _ptr(rp),
                                  _ptr(col), _ptr(w), cap, C.byref(nnz), C.c_void_p(st.cuda_stream)),
           "pdca_point_graph")
    m = int(nnz.value)
    return rp, col[:m], w[:m]


def params_from_workload(p: dict, **over) -> pdca_params:
    """pdca_params from a workload's parameter dict."""
    kw = dict(eps=p["eps"], c=p["c"], eta=p["eta"], precond=p["precond"],
              damping=p.get("damping", 0.5) or 0.5, delta0=p.get("delta0", 1e-6),
              power_iters=p.get("power_iters", 150))
    kw.update(over)
    return make_params(**kw)
