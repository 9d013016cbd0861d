"""CPU ORACLE -- test infrastructure, not part of the product.

A plain sequential FP64 implementation (``amg_oracle.c``) of the
matching-based aggregation AMG-PCG method of arXiv 2511.21268 (Sec. 3, 3.1,
3.2, 4), used to check the CUDA path.  It shares no code with the CUDA
library; the two meet only through the seeded inputs of
``paper_2511_21268_gb300.inputs``.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.

Every function follows the paper passage cited in ``amg_oracle.c``; the
readings taken where the paper is silent are listed at the top of that file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "amg_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

ERRORS = {0: "ok", -1: "bad argument", -2: "not SPD", -3: "breakdown", -4: "not converged", -7: "NaN",
          -8: "coarsest level too large", -9: "out of memory"}


def build(force: bool = False) -> str:
    """Compile the oracle (with OpenMP for the solve phase's row loops when
    the compiler supports it, sequential otherwise)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(SRC) > os.path.getmtime(LIB):
        tmp = LIB + ".tmp"
        base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"]
        r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
        if r.returncode != 0:
            r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
        os.replace(tmp, LIB)
    return LIB


class Opts(ctypes.Structure):
    _fields_ = [("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int), ("match_passes", ctypes.c_int),
                ("coarse_max", ctypes.c_int), ("max_levels", ctypes.c_int), ("testvec_sweeps", ctypes.c_int),
                ("testvec_kind", ctypes.c_int), ("seed", ctypes.c_uint64), ("stag", ctypes.c_double),
                ("dense_max", ctypes.c_int), ("smooth_levels", ctypes.c_int), ("smooth_omega", ctypes.c_double),
                ("cheb_degree", ctypes.c_int), ("coarse_solver", ctypes.c_int), ("coarse_tol", ctypes.c_double),
                ("coarse_maxit", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        L.orc_set_threads.argtypes = [i32]
        L.orc_opts_default.argtypes = [P]
        L.orc_setup.argtypes = [i64, P, P, P, P, P]
        L.orc_setup.restype = P
        L.orc_setup_ex.argtypes = [i64, P, P, P, P, P, P]
        L.orc_setup_ex.restype = P
        L.orc_level_sp_nnz.argtypes = [P, i32]
        L.orc_level_sp_nnz.restype = i64
        L.orc_level_sp.argtypes = [P, i32, P, P, P]
        L.orc_smooth_prolongator.argtypes = [i64, P, P, P, P, P, P, P, i64, P, P, P]
        L.orc_smooth_prolongator.restype = i32
        L.orc_galerkin_general.argtypes = [i64, P, P, P, P, P, P, i64, P, P, P]
        L.orc_galerkin_general.restype = i32
        L.orc_cheb4_smooth.argtypes = [i64, P, P, P, P, P, P, P, P, P, i32, i32]
        L.orc_coarse_cg.argtypes = [i64, P, P, P, P, dbl, i32, P]
        L.orc_free.argtypes = [P]
        L.orc_num_levels.argtypes = [P]
        L.orc_num_levels.restype = i32
        L.orc_level_n.argtypes = [P, i32]
        L.orc_level_n.restype = i64
        L.orc_level_nnz.argtypes = [P, i32]
        L.orc_level_nnz.restype = i64
        L.orc_level_npass.argtypes = [P, i32]
        L.orc_level_npass.restype = i32
        L.orc_level_pass_n.argtypes = [P, i32, i32]
        L.orc_level_pass_n.restype = i64
        L.orc_level_csr.argtypes = [P, i32, P, P, P]
        L.orc_level_vectors.argtypes = [P, i32, P, P]
        L.orc_level_map.argtypes = [P, i32, i32, P, P, P]
        L.orc_coarse_chol.argtypes = [P, P]
        L.orc_opc.argtypes = [P]
        L.orc_opc.restype = dbl
        L.orc_vcycle_apply.argtypes = [P, P, P]
        L.orc_pcg.argtypes = [P, P, P, dbl, i32, i32, P, P, P]
        L.orc_pcg.restype = i32
        L.orc_l1_diag.argtypes = [i64, P, P, P, P]
        L.orc_l1_diag.restype = i32
        L.orc_test_vector.argtypes = [i64, P, P, P, P, i32, ctypes.c_uint64, i32, P]
        L.orc_test_vector.restype = i32
        L.orc_edge_weight.argtypes = [dbl, dbl, dbl, dbl, dbl, P]
        L.orc_edge_weight.restype = i32
        L.orc_match_greedy.argtypes = [i64, P, P, P, P, P]
        L.orc_match_greedy.restype = i64
        L.orc_match_greedy_edges.argtypes = [i64, i64, P, P, P, P]
        L.orc_match_greedy_edges.restype = i64
        L.orc_aggregate.argtypes = [i64, P, P, P, P]
        L.orc_aggregate.restype = i64
        L.orc_restrict.argtypes = [i64, P, P, P, i64, P]
        L.orc_galerkin.argtypes = [i64, P, P, P, P, P, i64, P, P, P]
        L.orc_galerkin.restype = i32
        L.orc_cholesky.argtypes = [i64, P]
        L.orc_cholesky.restype = i32
        L.orc_chol_solve.argtypes = [i64, P, P, P]
        L.orc_spmv.argtypes = [i64, P, P, P, P, P]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(rowptr, col, val):
    return (np.ascontiguousarray(rowptr, np.int64), np.ascontiguousarray(col, np.int32),
            np.ascontiguousarray(val, np.float64))


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().orc_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


# ------------------------------------------------------------ building blocks
def l1_diag(rowptr, col, val):
    rp, ci, v = _csr(rowptr, col, val)
    d = np.empty(len(rp) - 1)
    rc = lib().orc_l1_diag(len(d), _p(rp), _p(ci), _p(v), _p(d))
    return d, rc


def test_vector(rowptr, col, val, seed=20251126, sweeps=4, kind=0):
    rp, ci, v = _csr(rowptr, col, val)
    d, _ = l1_diag(rp, ci, v)
    w = np.empty(len(d))
    lib().orc_test_vector(len(d), _p(rp), _p(ci), _p(v), _p(d), kind, seed, sweeps, _p(w))
    return w


def edge_weight(k, klo, khi, wlo, whi):
    c = ctypes.c_double()
    ok = lib().orc_edge_weight(k, klo, khi, wlo, whi, ctypes.byref(c))
    return c.value if ok else None


def match_greedy(rowptr, col, val, w):
    rp, ci, v = _csr(rowptr, col, val)
    w = np.ascontiguousarray(w, np.float64)
    mate = np.empty(len(rp) - 1, np.int32)
    lib().orc_match_greedy(len(mate), _p(rp), _p(ci), _p(v), _p(w), _p(mate))
    return mate


def match_greedy_edges(n, lo, hi, c):
    """Greedy matching on an explicit edge list with weights c (lo < hi)."""
    lo = np.ascontiguousarray(lo, np.int32)
    hi = np.ascontiguousarray(hi, np.int32)
    c = np.ascontiguousarray(c, np.float64)
    mate = np.empty(n, np.int32)
    lib().orc_match_greedy_edges(n, len(c), _p(lo), _p(hi), _p(c), _p(mate))
    return mate


def aggregate(mate, w):
    mate = np.ascontiguousarray(mate, np.int32)
    w = np.ascontiguousarray(w, np.float64)
    agg = np.empty(len(mate), np.int32)
    pval = np.empty(len(mate))
    nc = lib().orc_aggregate(len(mate), _p(mate), _p(w), _p(agg), _p(pval))
    return agg, pval, int(nc)


def restrict(agg, pval, x, nc):
    agg = np.ascontiguousarray(agg, np.int32)
    pval = np.ascontiguousarray(pval, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    out = np.empty(nc)
    lib().orc_restrict(len(agg), _p(agg), _p(pval), _p(x), nc, _p(out))
    return out


def galerkin(rowptr, col, val, agg, pval, nc):
    rp, ci, v = _csr(rowptr, col, val)
    agg = np.ascontiguousarray(agg, np.int32)
    pval = np.ascontiguousarray(pval, np.float64)
    orp, oci, ov = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    lib().orc_galerkin(len(rp) - 1, _p(rp), _p(ci), _p(v), _p(agg), _p(pval), nc, ctypes.byref(orp),
                       ctypes.byref(oci), ctypes.byref(ov))
    rpc = np.ctypeslib.as_array(ctypes.cast(orp, ctypes.POINTER(ctypes.c_int64)), (nc + 1,)).copy()
    z = int(rpc[-1])
    cic = np.ctypeslib.as_array(ctypes.cast(oci, ctypes.POINTER(ctypes.c_int32)), (max(z, 1),))[:z].copy()
    vc = np.ctypeslib.as_array(ctypes.cast(ov, ctypes.POINTER(ctypes.c_double)), (max(z, 1),))[:z].copy()
    libc = ctypes.CDLL(None)
    libc.free.argtypes = [ctypes.c_void_p]
    for ptr in (orp, oci, ov):
        libc.free(ptr)
    return rpc, cic, vc


def smooth_prolongator(rowptr, col, val, dl1, theta, agg, pval, nc):
    """P_bar = (I - diag(theta) D^-1 K) P as CSR (rowptr, col, val)."""
    rp, ci, v = _csr(rowptr, col, val)
    d = np.ascontiguousarray(dl1, np.float64)
    th = np.ascontiguousarray(theta, np.float64)
    a = np.ascontiguousarray(agg, np.int32)
    pv = np.ascontiguousarray(pval, np.float64)
    orp, oci, ov = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    rc = lib().orc_smooth_prolongator(len(rp) - 1, _p(rp), _p(ci), _p(v), _p(d), _p(th), _p(a), _p(pv), nc,
                                      ctypes.byref(orp), ctypes.byref(oci), ctypes.byref(ov))
    if rc != 0:
        raise RuntimeError(ERRORS.get(rc, rc))
    return _take_csr(len(rp) - 1, orp, oci, ov)


def galerkin_general(rowptr, col, val, prp, pci, pv, nc):
    """K_c = P^T (K P) for a general CSR prolongator P (n x nc)."""
    rp, ci, v = _csr(rowptr, col, val)
    a, b, c = _csr(prp, pci, pv)
    orp, oci, ov = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    rc = lib().orc_galerkin_general(len(rp) - 1, _p(rp), _p(ci), _p(v), _p(a), _p(b), _p(c), nc,
                                    ctypes.byref(orp), ctypes.byref(oci), ctypes.byref(ov))
    if rc != 0:
        raise RuntimeError(ERRORS.get(rc, rc))
    return _take_csr(nc, orp, oci, ov)


def cheb4_smooth(rowptr, col, val, dl1, f, x0=None, degree=4):
    """degree steps of the 4th-kind Chebyshev acceleration of l1-Jacobi on
    K x = f from x0 (None: from zero); returns (x, r), r the residual of the
    recurrence when starting from zero."""
    rp, ci, v = _csr(rowptr, col, val)
    n = len(rp) - 1
    d = np.ascontiguousarray(dl1, np.float64)
    f = np.ascontiguousarray(f, np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, np.float64)
    r, w1, w2 = np.empty(n), np.empty(n), np.empty(n)
    lib().orc_cheb4_smooth(n, _p(rp), _p(ci), _p(v), _p(d), _p(f), _p(x), _p(r), _p(w1), _p(w2), int(degree),
                           int(x0 is None))
    return x, r


def coarse_cg(rowptr, col, val, f, tol=1e-4, maxit=30):
    """Jacobi-preconditioned CG from zero (the coarse solver option)."""
    rp, ci, v = _csr(rowptr, col, val)
    f = np.ascontiguousarray(f, np.float64)
    x = np.empty(len(rp) - 1)
    lib().orc_coarse_cg(len(rp) - 1, _p(rp), _p(ci), _p(v), _p(f), float(tol), int(maxit), _p(x))
    return x


def _take_csr(n, orp, oci, ov):
    """Copy a CSR the C code allocated with malloc into numpy and free it."""
    libc = ctypes.CDLL(None)
    libc.free.argtypes = [ctypes.c_void_p]
    rp = np.ctypeslib.as_array(ctypes.cast(orp, ctypes.POINTER(ctypes.c_int64)), (n + 1,)).copy()
    z = int(rp[-1])
    ci = np.ctypeslib.as_array(ctypes.cast(oci, ctypes.POINTER(ctypes.c_int32)), (max(z, 1),))[:z].copy()
    v = np.ctypeslib.as_array(ctypes.cast(ov, ctypes.POINTER(ctypes.c_double)), (max(z, 1),))[:z].copy()
    for ptr in (orp, oci, ov):
        libc.free(ptr)
    return rp, ci, v


def cholesky(A):
    A = np.array(A, np.float64, order="C")
    rc = lib().orc_cholesky(A.shape[0], _p(A))
    return A, rc


def chol_solve(L, b):
    L = np.ascontiguousarray(L, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    x = np.empty_like(b)
    lib().orc_chol_solve(len(b), _p(L), _p(b), _p(x))
    return x


def spmv(rowptr, col, val, x):
    rp, ci, v = _csr(rowptr, col, val)
    x = np.ascontiguousarray(x, np.float64)
    y = np.empty(len(rp) - 1)
    lib().orc_spmv(len(y), _p(rp), _p(ci), _p(v), _p(x), _p(y))
    return y


def set_threads(t: int) -> int:
    """Threads of the solve phase's row loops (results do not depend on it);
    returns the count in effect (1 without OpenMP)."""
    L = lib()
    L.orc_set_threads(int(t) if L.orc_have_openmp() else 1)
    return L.orc_get_threads()


def have_openmp() -> bool:
    return bool(lib().orc_have_openmp())


# ------------------------------------------------------------- hierarchy ----
class Hierarchy:
    """Oracle AMG hierarchy built from a CSR matrix (host arrays)."""

    def __init__(self, rowptr, col, val, theta0=None, **opts):
        """opts: fields of Opts (smooth_levels, smooth_omega, ...); theta0:
        per-row smoothing weights of level 0 when its prolongator is
        smoothed (replacing smooth_omega there)."""
        self._keep = _csr(rowptr, col, val)
        rp, ci, v = self._keep
        self.opts = default_opts(**opts)
        st = ctypes.c_int()
        th = None if theta0 is None else np.ascontiguousarray(theta0, np.float64)
        self._theta = th
        self._h = lib().orc_setup_ex(len(rp) - 1, _p(rp), _p(ci), _p(v), ctypes.byref(self.opts),
                                     None if th is None else _p(th), ctypes.byref(st))
        self.status = st.value
        if not self._h:
            raise RuntimeError(f"oracle setup failed: {ERRORS.get(st.value, st.value)}")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_free(h)
            self._h = None

    @property
    def num_levels(self) -> int:
        return lib().orc_num_levels(self._h)

    @property
    def opc(self) -> float:
        return lib().orc_opc(self._h)

    def level_n(self, l):
        return int(lib().orc_level_n(self._h, l))

    def level_nnz(self, l):
        return int(lib().orc_level_nnz(self._h, l))

    def level_csr(self, l):
        n, z = self.level_n(l), self.level_nnz(l)
        rp = np.empty(n + 1, np.int64)
        ci = np.empty(z, np.int32)
        v = np.empty(z)
        lib().orc_level_csr(self._h, l, _p(rp), _p(ci), _p(v))
        return rp, ci, v

    def level_vectors(self, l):
        n = self.level_n(l)
        d = np.empty(n)
        w = np.empty(n)
        lib().orc_level_vectors(self._h, l, _p(d), _p(w))
        return d, w

    def level_npass(self, l):
        return lib().orc_level_npass(self._h, l)

    def level_map(self, l):
        """Composite map (agg, pval) from level l to level l+1."""
        n = self.level_n(l)
        agg = np.empty(n, np.int32)
        pv = np.empty(n)
        lib().orc_level_map(self._h, l, -1, _p(agg), _p(pv), None)
        return agg, pv

    def pass_map(self, l, s):
        """(mate, agg, pval) of matching pass s on level l."""
        n = int(lib().orc_level_pass_n(self._h, l, s))
        agg = np.empty(n, np.int32)
        pv = np.empty(n)
        mate = np.empty(n, np.int32)
        lib().orc_level_map(self._h, l, s, _p(agg), _p(pv), _p(mate))
        return mate, agg, pv

    def pass_sizes(self, l):
        return [int(lib().orc_level_pass_n(self._h, l, s)) for s in range(self.level_npass(l) + 1)]

    def prolongator(self, l):
        """Level l's prolongator as CSR (rowptr, col, val): the smoothed one
        where the level is smoothed, else the tentative one (one entry per
        row)."""
        n = self.level_n(l)
        z = int(lib().orc_level_sp_nnz(self._h, l))
        if z == 0:
            agg, pv = self.level_map(l)
            return np.arange(n + 1, dtype=np.int64), agg.astype(np.int32), pv
        rp = np.empty(n + 1, np.int64)
        ci = np.empty(z, np.int32)
        v = np.empty(z)
        lib().orc_level_sp(self._h, l, _p(rp), _p(ci), _p(v))
        return rp, ci, v

    def coarse_chol(self):
        n = self.level_n(self.num_levels - 1)
        L = np.empty((n, n))
        lib().orc_coarse_chol(self._h, _p(L))
        return L

    def vcycle(self, r):
        r = np.ascontiguousarray(r, np.float64)
        z = np.empty_like(r)
        lib().orc_vcycle_apply(self._h, _p(r), _p(z))
        return z

    def pcg(self, F, x0=None, rtol=1e-8, itmax=1000, flexible=False, history=False):
        F = np.ascontiguousarray(F, np.float64)
        u = np.zeros_like(F) if x0 is None else np.array(x0, np.float64)
        it = ctypes.c_int()
        rr = ctypes.c_double()
        hist = np.zeros(itmax + 1) if history else None
        rc = lib().orc_pcg(self._h, _p(F), _p(u), rtol, itmax, int(flexible), ctypes.byref(it), ctypes.byref(rr),
                           _p(hist) if history else None)
        out = dict(u=u, iters=it.value, relres=rr.value, status=rc)
        if history:
            out["history"] = hist[: it.value + 1]
        return out
