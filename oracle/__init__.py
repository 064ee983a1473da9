"""FP64 CPU oracle for pDCA on the graph Ginzburg-Landau model (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The
library under ``paper_2303_14495_gb300`` never imports it and never falls back
to it.

The arithmetic lives in ``pdca_oracle.c`` (plain C, double precision, one node
at a time, following the paper's equations); this module only compiles it
with gcc and marshals numpy arrays.  Building with ``omp=True`` compiles the
same file with OpenMP over independent rows (identical results).
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pdca_oracle.c")
HDR = os.path.join(HERE, "pdca_oracle.h")
BUILD = os.path.join(HERE, "_build")

LAP_NORMALIZED = 0
LAP_UNNORMALIZED = 1
JACOBI_DAMPED = 0
JACOBI_PERTURBED = 1
RICHARDSON = 2

_lock = threading.Lock()
_libs = {}


def build(omp: bool = False, force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FP contraction)."""
    os.makedirs(BUILD, exist_ok=True)
    out = os.path.join(BUILD, "liborc_omp.so" if omp else "liborc.so")
    newest = max(os.path.getmtime(SRC), os.path.getmtime(HDR))
    if force or not os.path.exists(out) or os.path.getmtime(out) < newest:
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, SRC, "-lm"]
        if omp:
            cmd.insert(1, "-fopenmp")
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


class _Problem(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("K", C.c_int32), ("laplacian", C.c_int32),
        ("precond", C.c_int32), ("pad_", C.c_int32),
        ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("w", C.c_void_p),
        ("d", C.c_void_p), ("mask", C.c_void_p), ("y", C.c_void_p),
        ("eps", C.c_double), ("eta", C.c_double), ("c", C.c_double),
        ("damping", C.c_double), ("delta0", C.c_double), ("lambda_max", C.c_double),
        ("step_k", C.c_double),
    ]


def _lib(omp: bool = False):
    with _lock:
        if omp not in _libs:
            lib = C.CDLL(build(omp))
            P = C.POINTER(_Problem)
            vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
            sig = {
                "orc_num_threads": (C.c_int, []),
                "orc_degrees": (i64, [i64, vp, vp, vp, vp]),
                "orc_apply_Ls": (None, [i64, i32, vp, vp, vp, vp, vp, vp]),
                "orc_apply_L": (None, [i64, i32, vp, vp, vp, vp, vp, vp]),
                "orc_apply_T": (None, [P, vp, vp]),
                "orc_apply_system": (None, [P, vp, vp]),
                "orc_prior": (None, [i64, i32, vp, vp, vp]),
                "orc_init_u": (None, [i64, i32, vp, vp, vp]),
                "orc_precond_diag": (None, [P, vp]),
                "orc_rhs": (None, [P, vp, vp]),
                "orc_sweep": (None, [P, vp, vp, vp, vp, vp]),
                "orc_project_row": (None, [i32, vp]),
                "orc_energy": (dbl, [P, vp, vp]),
                "orc_residual": (dbl, [P, vp, vp, vp]),
                "orc_labels": (None, [i64, i32, vp, vp]),
                "orc_power_max_eig": (dbl, [P, i32]),
                "orc_pdca_solve": (C.c_int, [P, i32, i32, vp, vp, vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _libs[omp] = lib
        return _libs[omp]


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def num_threads(omp: bool = False) -> int:
    return int(_lib(omp).orc_num_threads())


def degrees(row_ptr, col, w):
    n = row_ptr.shape[0] - 1
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    w = np.ascontiguousarray(w, np.float32)
    d = np.empty(n, np.float64)
    bad = _lib().orc_degrees(n, _p(row_ptr), _p(col), _p(w), _p(d))
    return d, int(bad)


def apply_Ls(row_ptr, col, w, d, x):
    x = np.ascontiguousarray(x, np.float64)
    n = row_ptr.shape[0] - 1
    K = 1 if x.ndim == 1 else x.shape[1]
    y = np.empty_like(x)
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    w = np.ascontiguousarray(w, np.float32)
    d = np.ascontiguousarray(d, np.float64)
    _lib().orc_apply_Ls(n, K, _p(row_ptr), _p(col), _p(w), _p(d), _p(x), _p(y))
    return y


def apply_L(row_ptr, col, w, d, x):
    x = np.ascontiguousarray(x, np.float64)
    n = row_ptr.shape[0] - 1
    K = 1 if x.ndim == 1 else x.shape[1]
    y = np.empty_like(x)
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    w = np.ascontiguousarray(w, np.float32)
    d = np.ascontiguousarray(d, np.float64)
    _lib().orc_apply_L(n, K, _p(row_ptr), _p(col), _p(w), _p(d), _p(x), _p(y))
    return y


def project_rows(u):
    """Simplex projection of every row (coding v = (u+1)/2)."""
    u = np.array(u, dtype=np.float64, copy=True, order="C")
    K = u.shape[-1]
    flat = u.reshape(-1, K)
    lib = _lib()
    for r in range(flat.shape[0]):
        row = np.ascontiguousarray(flat[r])
        lib.orc_project_row(K, _p(row))
        flat[r] = row
    return flat.reshape(u.shape)


class Problem:
    """One pDCA problem held by the oracle (arrays are kept alive here)."""

    def __init__(self, row_ptr, col, w, K, fid_mask, fid_labels, eps, eta, c,
                 precond=JACOBI_DAMPED, damping=0.5, delta0=1e-6, lambda_max=0.0,
                 laplacian=LAP_NORMALIZED, step_k=0.0, omp=False):
        self.omp = omp
        self.lib = _lib(omp)
        self.row_ptr = np.ascontiguousarray(row_ptr, np.int64)
        self.col = np.ascontiguousarray(col, np.int32)
        self.w = np.ascontiguousarray(w, np.float32)
        self.n = int(self.row_ptr.shape[0] - 1)
        self.K = int(K)
        self.mask = np.ascontiguousarray(fid_mask, np.uint8)
        self.labels = np.ascontiguousarray(fid_labels, np.int32)
        self.d = np.empty(self.n, np.float64)
        self.bad_node = int(self.lib.orc_degrees(self.n, _p(self.row_ptr), _p(self.col),
                                                 _p(self.w), _p(self.d)))
        self.y = np.empty(self.n * self.K, np.float64)
        self.lib.orc_prior(self.n, self.K, _p(self.mask), _p(self.labels), _p(self.y))
        self.s = _Problem()
        self.s.n, self.s.K = self.n, self.K
        self.s.laplacian, self.s.precond = int(laplacian), int(precond)
        self.s.row_ptr, self.s.col, self.s.w = _p(self.row_ptr), _p(self.col), _p(self.w)
        self.s.d, self.s.mask, self.s.y = _p(self.d), _p(self.mask), _p(self.y)
        self.s.eps, self.s.eta, self.s.c = float(eps), float(eta), float(c)
        self.s.damping, self.s.delta0 = float(damping), float(delta0)
        self.s.lambda_max = float(lambda_max)
        self.s.step_k = float(step_k)

    @property
    def ref(self):
        return C.byref(self.s)

    def _nk(self, x=None):
        shape = (self.n,) if self.K == 1 else (self.n, self.K)
        if x is None:
            return np.empty(shape, np.float64)
        return np.ascontiguousarray(np.asarray(x, np.float64).reshape(shape))

    def set_lambda_max(self, lam):
        self.s.lambda_max = float(lam)

    def init_u(self):
        u = self._nk()
        self.lib.orc_init_u(self.n, self.K, _p(self.mask), _p(self.labels), _p(u))
        return u

    def prior(self):
        return self.y.reshape((self.n,) if self.K == 1 else (self.n, self.K)).copy()

    def apply_lap(self, x):
        x = self._nk(x)
        y = self._nk()
        f = self.lib.orc_apply_Ls if self.s.laplacian == LAP_NORMALIZED else self.lib.orc_apply_L
        f(self.n, self.K, _p(self.row_ptr), _p(self.col), _p(self.w), _p(self.d), _p(x), _p(y))
        return y

    def apply_T(self, x):
        x = self._nk(x)
        y = self._nk()
        self.lib.orc_apply_T(self.ref, _p(x), _p(y))
        return y

    def apply_system(self, x):
        """T x (infinite step size) or T_k x = x + k T x (step size k)."""
        x = self._nk(x)
        y = self._nk()
        self.lib.orc_apply_system(self.ref, _p(x), _p(y))
        return y

    def precond_diag(self):
        g = np.empty(self.n, np.float64)
        self.lib.orc_precond_diag(self.ref, _p(g))
        return g

    def rhs(self, u):
        u = self._nk(u)
        b = self._nk()
        self.lib.orc_rhs(self.ref, _p(u), _p(b))
        return b

    def sweep(self, g, b, v):
        v = self._nk(v)
        b = self._nk(b)
        tv = self._nk()
        vn = self._nk()
        g = np.ascontiguousarray(g, np.float64)
        self.lib.orc_sweep(self.ref, _p(g), _p(b), _p(v), _p(tv), _p(vn))
        return vn

    def energy(self, u):
        u = self._nk(u)
        scratch = self._nk()
        return float(self.lib.orc_energy(self.ref, _p(u), _p(scratch)))

    def residual(self, b, u):
        b = self._nk(b)
        u = self._nk(u)
        scratch = self._nk()
        return float(self.lib.orc_residual(self.ref, _p(b), _p(u), _p(scratch)))

    def labels_of(self, u):
        u = self._nk(u)
        lab = np.empty(self.n, np.int32)
        self.lib.orc_labels(self.n, self.K, _p(u), _p(lab))
        return lab

    def power_max_eig(self, iters=150):
        return float(self.lib.orc_power_max_eig(self.ref, int(iters)))

    def solve(self, outer, inner, u0=None):
        """Run ``outer`` pDCA steps with ``inner`` sweeps; returns (u, energy[], residual[])."""
        u = self.init_u() if u0 is None else self._nk(np.array(u0, dtype=np.float64, copy=True))
        e = np.empty(max(outer, 1), np.float64)
        r = np.empty(max(outer, 1), np.float64)
        rc = self.lib.orc_pdca_solve(self.ref, int(outer), int(inner), _p(u), _p(e), _p(r))
        if rc != 0:
            raise FloatingPointError("oracle: non-finite iterate")
        return u, e[:outer], r[:outer]


def second_eigenpair(row_ptr, col, w, laplacian: int = LAP_NORMALIZED, tol: float = 1e-13):
    """(lambda_2, v_2): the smallest eigenvalue of L_s (or L) on the
    orthogonal complement of its null vector q = D^1/2 1 (or 1), and its unit
    eigenvector: the second eigenvector the paper initialises the unsupervised
    model with (Sec. 5.3, the unsupervised clustering experiments).  On a
    connected graph it is the second-smallest eigenpair; on a graph with
    several components (where 0 is a multiple eigenvalue) the restriction to
    the complement of q is what makes the vector unique.

    Definition written out: the largest eigenpair of Q (B I - L) Q with
    Q = I - q q^T / q^T q and B a bound of the spectrum (2 for L_s, 2 max d_i
    for L, Prop. diagonal:pre), by scipy's Lanczos (ARPACK) on the oracle's own
    C operator.  The eigenvector is normalised to unit length and its sign fixed
    so that its largest-magnitude component (lowest index among equal ones) is
    positive.
    """
    from scipy.sparse.linalg import LinearOperator, eigsh
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    w = np.ascontiguousarray(w, np.float32)
    n = row_ptr.shape[0] - 1
    d, bad = degrees(row_ptr, col, w)
    if bad >= 0:
        raise ValueError(f"isolated node {bad}")
    if laplacian == LAP_NORMALIZED:
        bound, apply, q = 2.0, (lambda x: apply_Ls(row_ptr, col, w, d, x)), np.sqrt(d)
    else:
        bound, apply, q = 2.0 * float(d.max()), (lambda x: apply_L(row_ptr, col, w, d, x)), np.ones(n)
    q = q / np.linalg.norm(q)

    def proj(x):
        return x - (q @ x) * q

    def mv(x):
        x = proj(np.asarray(x, np.float64).ravel())
        return proj(bound * x - apply(x))

    op = LinearOperator((n, n), matvec=mv, dtype=np.float64)
    v0 = proj(1.0 + 0.5 * np.sin(np.arange(1, n + 1, dtype=np.float64)))
    vals, vecs = eigsh(op, k=1, which="LA", tol=tol, v0=v0, maxiter=100000)
    lam2 = bound - float(vals[0])
    v = proj(vecs[:, 0].astype(np.float64))
    v /= np.linalg.norm(v)
    if v[int(np.argmax(np.abs(v)))] < 0:
        v = -v
    return lam2, v


def spectral_init(v2) -> np.ndarray:
    """u^0 of the unsupervised model from the second eigenvector: v_2 scaled
    to max |u_i| = 1 (values in [-1, 1], the sign pattern of v_2)."""
    v2 = np.asarray(v2, np.float64)
    return v2 / np.abs(v2).max()


def safe_lambda(lam_est: float, laplacian: int = LAP_NORMALIZED, dmax: float = 0.0) -> float:
    """lambda-hat used by the Richardson preconditioner: the power-method
    estimate raised by 0.1 % and capped by the Prop. (diagonal:pre) bound
    (2 for L_s, 2 max d_i for L)."""
    cap = 2.0 if laplacian == LAP_NORMALIZED else 2.0 * dmax
    return min(cap, 1.001 * lam_est)
