"""Thin Python binding of the C ABI in ``include/amg_gb300.h``.

Argument marshalling only: every step of setup and solve runs in the CUDA
library ``libamg_gb300.so``.  PyTorch is used for device buffers and
streams.  There is no fallback: if the library cannot be built or loaded,
or no CUDA device is present, the calls raise.

The module-level functions carry the C names (``amg_setup``,
``amg_pcg_solve``, ...); ``Hierarchy`` wraps them for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

AMG_OK = 0
AMG_ERR_ARG = -1
AMG_ERR_NOT_SPD = -2
AMG_ERR_BREAKDOWN = -3
AMG_ERR_NOT_CONVERGED = -4
AMG_ERR_TIMEOUT = -5
AMG_ERR_CUDA = -6
AMG_ERR_NAN = -7
AMG_ERR_COARSE_TOO_LARGE = -8
AMG_ERR_NOMEM = -9
AMG_ERR_ROW_TOO_LONG = -10

AMG_FP64, AMG_FP32, AMG_FP32_BF16FINE = 0, 1, 2
AMG_MEM_HOST, AMG_MEM_DEVICE = 0, 1
AMG_MAX_LEVELS = 32


class AmgCsr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p), ("mem", ctypes.c_int32)]


class AmgOpts(ctypes.Structure):
    _fields_ = [("nu_pre", ctypes.c_int32), ("nu_post", ctypes.c_int32), ("match_passes", ctypes.c_int32),
                ("coarse_max", ctypes.c_int32), ("max_levels", ctypes.c_int32), ("dense_max", ctypes.c_int32),
                ("testvec_sweeps", ctypes.c_int32), ("testvec_kind", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("stag", ctypes.c_double), ("max_match_rounds", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("flexible", ctypes.c_int32), ("resid_replace_every", ctypes.c_int32),
                ("matrix_format", ctypes.c_int32), ("mpnn_weights", ctypes.c_void_p), ("mpnn_bf16", ctypes.c_int32),
                ("smooth_levels", ctypes.c_int32), ("smooth_omega", ctypes.c_double),
                ("smooth_theta", ctypes.c_void_p), ("cheb_degree", ctypes.c_int32),
                ("coarse_solver", ctypes.c_int32), ("coarse_tol", ctypes.c_double), ("coarse_maxit", ctypes.c_int32),
                ("autotune", ctypes.c_int32)]


class AmgInfo(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("n", ctypes.c_int64 * AMG_MAX_LEVELS),
                ("nnz", ctypes.c_int64 * AMG_MAX_LEVELS), ("opc", ctypes.c_double), ("setup_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("iters", ctypes.c_int32), ("status", ctypes.c_int32),
                ("final_relres", ctypes.c_double), ("vcycle_bytes", ctypes.c_double),
                ("iter_bytes", ctypes.c_double), ("match_rounds", ctypes.c_int32 * AMG_MAX_LEVELS),
                ("setup_phase_ms", ctypes.c_double * 12), ("level_format", ctypes.c_int32 * AMG_MAX_LEVELS),
                ("staged_passes", ctypes.c_int32), ("staged_slots", ctypes.c_int64),
                ("staged_buffers", ctypes.c_int32 * 2), ("staged_window_bytes", ctypes.c_int32),
                ("staged_level1", ctypes.c_int32), ("graph_build_ms", ctypes.c_double),
                ("smoothed", ctypes.c_int32 * AMG_MAX_LEVELS), ("p_nnz", ctypes.c_int64 * AMG_MAX_LEVELS),
                ("sell64_warps", ctypes.c_int32), ("tune_ms", ctypes.c_double)]


AMG_GEOM_CUBE, AMG_GEOM_ANNULUS = 0, 1
AMG_SRC_ONE, AMG_SRC_SINE = 0, 1


class AmgIgaPatch(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("p", ctypes.c_int32), ("nq", ctypes.c_int32), ("geometry", ctypes.c_int32),
                ("with_boundary", ctypes.c_int32), ("source", ctypes.c_int32), ("kappa_m", ctypes.c_int32),
                ("kappa_sigma", ctypes.c_double), ("kappa_omega", ctypes.c_void_p), ("kappa_phi", ctypes.c_void_p)]


class AmgError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = amg_strerror(code)
        if code == AMG_ERR_CUDA:
            msg += ": " + lib().amg_last_cuda_error().decode()
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")


_lib = None

# exported entry points and their signatures
_SIGS = {
    "amg_opts_default": (ctypes.c_int, [ctypes.c_void_p]),
    "amg_setup": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "amg_pcg_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                     ctypes.c_double, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "amg_vcycle_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "amg_pcg_solve_multi": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                           ctypes.c_void_p, ctypes.c_void_p]),
    "amg_setup_batch": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "amg_pcg_solve_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                           ctypes.c_double, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "amg_level_spmv": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "amg_get_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "amg_export_level": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32] + [ctypes.c_void_p] * 7),
    "amg_export_pass": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32] + [ctypes.c_void_p] * 4),
    "amg_export_prolongator": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32] + [ctypes.c_void_p] * 4),
    "amg_export_coarse": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "amg_free": (ctypes.c_int, [ctypes.c_void_p]),
    "amg_kernel_launches": (ctypes.c_int64, []),
    "amg_relres_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "amg_profile_kernels": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "amg_kernel_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "amg_mpnn_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "amg_mpnn_omega": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "amg_mpnn_loss_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "amg_mpnn_theta_loss_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64,
                                                ctypes.c_void_p, ctypes.c_void_p]),
    "amg_mpnn_theta": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "amg_mpnn_adam": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 4 + [ctypes.c_int32] + [ctypes.c_float] * 4),
    "amg_mpnn_train": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_uint64, ctypes.c_float, ctypes.c_void_p]),
    "amg_mpnn_select": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                                       ctypes.c_double, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "amg_set_damping": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "amg_dfma_probe": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "amg_div_check": (ctypes.c_int, [ctypes.c_int64] + [ctypes.c_void_p] * 5),
    "amg_smoother_bound": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "amg_staged_wait_selftest": (ctypes.c_int, [ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]),
    "amg_iga_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "amg_iga_assemble": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 6),
    "amg_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "amg_last_cuda_error": (ctypes.c_char_p, []),
}


def library_path() -> str:
    return _build.AMG_LIB


def lib(build: bool = True):
    """Load (building first if needed) the CUDA library."""
    global _lib
    if _lib is None:
        path = _build.build_cuda() if build else _build.AMG_LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library missing: {path}")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != AMG_OK:
        raise AmgError(rc, what)


def amg_staged_wait_selftest(limit_ms: float = 2.0):
    """(timed_out, completed) of the bounded-wait self-test of the staged
    passes: a wait that nothing completes must give up after limit_ms, a
    completed one must return."""
    to, done = ctypes.c_int32(-1), ctypes.c_int32(-1)
    _check(lib().amg_staged_wait_selftest(limit_ms, ctypes.byref(to), ctypes.byref(done)), "amg_staged_wait_selftest")
    return to.value, done.value


def amg_strerror(code: int) -> str:
    return lib().amg_strerror(code).decode()


def amg_last_cuda_error() -> str:
    return lib().amg_last_cuda_error().decode()


def amg_opts_default(**overrides) -> AmgOpts:
    o = AmgOpts()
    _check(lib().amg_opts_default(ctypes.byref(o)), "amg_opts_default")
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        if k == "mpnn_weights" and v is not None and not isinstance(v, int):
            o._weights = _dev_weights(v)  # kept alive with the options
            v = o._weights.data_ptr()
        if k == "smooth_theta" and v is not None and not isinstance(v, int):
            torch = _torch()
            if isinstance(v, np.ndarray):
                v = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64))
            o._theta = v.to(device="cuda", dtype=torch.float64).contiguous()  # kept alive with the options
            v = o._theta.data_ptr()
        setattr(o, k, v)
    return o


def _torch():
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the AMG library runs on the GPU only")
    return torch


def _ptr(a):
    """(pointer, mem kind, keepalive) of a numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a)
        return a.ctypes.data, AMG_MEM_HOST, a
    if a.is_cuda:
        a = a.contiguous()
        return a.data_ptr(), AMG_MEM_DEVICE, a
    a = a.contiguous()
    return a.data_ptr(), AMG_MEM_HOST, a


def _stream_handle(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def amg_setup(rowptr, col, val, opts: AmgOpts | None = None, stream=None):
    """Build a hierarchy; arrays may be numpy (host) or torch (host/cuda)."""
    _torch()
    if isinstance(rowptr, np.ndarray):
        rowptr = np.ascontiguousarray(rowptr, np.int64)
        col = np.ascontiguousarray(col, np.int32)
        val = np.ascontiguousarray(val, np.float64)
    prp, m1, k1 = _ptr(rowptr)
    pci, m2, k2 = _ptr(col)
    pv, m3, k3 = _ptr(val)
    if not (m1 == m2 == m3):
        raise ValueError("rowptr, col and val must live in the same memory space")
    csr = AmgCsr(len(rowptr) - 1, len(val), prp, pci, pv, m1)
    h = ctypes.c_void_p()
    rc = lib().amg_setup(ctypes.byref(csr), ctypes.byref(opts) if opts is not None else None,
                         _stream_handle(stream), ctypes.byref(h))
    _check(rc, "amg_setup")
    del k1, k2, k3
    return h


def amg_pcg_solve(h, F, u, rtol: float, itmax: int):
    """Solve in place: u (numpy or torch, FP64) holds x0 and receives the
    solution.  Returns (status, iters, relres); status is AMG_OK or a
    convergence status (errors other than those raise)."""
    pF, mF, kF = _ptr(F)
    pu, mu, ku = _ptr(u)
    if mF != mu:
        raise ValueError("F and u must live in the same memory space")
    if ku is not u:
        raise ValueError("u must be contiguous (it is written in place)")
    it = ctypes.c_int32()
    rr = ctypes.c_double()
    rc = lib().amg_pcg_solve(h, pF, pu, mF, float(rtol), int(itmax), ctypes.byref(it), ctypes.byref(rr))
    if rc not in (AMG_OK, AMG_ERR_NOT_CONVERGED, AMG_ERR_BREAKDOWN, AMG_ERR_NAN):
        _check(rc, "amg_pcg_solve")
    return rc, it.value, rr.value


def amg_pcg_solve_multi(h, F, U, rtol: float, itmax: int):
    """F, U: (nrhs, n) C-contiguous arrays/tensors = column-major n x nrhs
    (ld = n); U holds the initial guesses and receives the solutions.
    Returns (status, iters[nrhs], relres[nrhs])."""
    pF, mF, kF = _ptr(F)
    pU, mU, kU = _ptr(U)
    if mF != mU or kU is not U:
        raise ValueError("F and U must share a memory space; U must be contiguous")
    nrhs, n = F.shape
    it = np.zeros(nrhs, np.int32)
    rr = np.zeros(nrhs)
    rc = lib().amg_pcg_solve_multi(h, nrhs, pF, pU, n, mF, float(rtol), int(itmax), it.ctypes.data, rr.ctypes.data)
    if rc not in (AMG_OK, AMG_ERR_NOT_CONVERGED, AMG_ERR_BREAKDOWN, AMG_ERR_NAN):
        _check(rc, "amg_pcg_solve_multi")
    return rc, it, rr


def amg_setup_batch(systems, opts: AmgOpts | None = None, stream=None):
    """systems: list of (rowptr, col, val) (numpy or torch, one memory space)."""
    _torch()
    keep = []
    arr = (AmgCsr * len(systems))()
    for k, (rp, ci, va) in enumerate(systems):
        if isinstance(rp, np.ndarray):
            rp = np.ascontiguousarray(rp, np.int64)
            ci = np.ascontiguousarray(ci, np.int32)
            va = np.ascontiguousarray(va, np.float64)
        prp, m1, k1 = _ptr(rp)
        pci, m2, k2 = _ptr(ci)
        pv, m3, k3 = _ptr(va)
        keep += [k1, k2, k3]
        arr[k] = AmgCsr(len(rp) - 1, len(va), prp, pci, pv, m1)
    h = ctypes.c_void_p()
    rc = lib().amg_setup_batch(len(systems), arr, ctypes.byref(opts) if opts is not None else None,
                               _stream_handle(stream), ctypes.byref(h))
    _check(rc, "amg_setup_batch")
    del keep
    return h


def amg_pcg_solve_batch(h, Fs, Us, rtol: float, itmax: int):
    """Fs, Us: per-system vectors (one memory space); Us solved in place.
    Returns (status, iters[count], relres[count])."""
    ptrF = [_ptr(F) for F in Fs]
    ptrU = [_ptr(U) for U in Us]
    mem = ptrF[0][1]
    if any(p[1] != mem for p in ptrF + ptrU) or any(p[2] is not U for p, U in zip(ptrU, Us)):
        raise ValueError("all vectors must share a memory space; U must be contiguous")
    cnt = len(Fs)
    aF = (ctypes.c_void_p * cnt)(*[p[0] for p in ptrF])
    aU = (ctypes.c_void_p * cnt)(*[p[0] for p in ptrU])
    it = np.zeros(cnt, np.int32)
    rr = np.zeros(cnt)
    rc = lib().amg_pcg_solve_batch(h, aF, aU, mem, float(rtol), int(itmax), it.ctypes.data, rr.ctypes.data)
    if rc not in (AMG_OK, AMG_ERR_NOT_CONVERGED, AMG_ERR_BREAKDOWN, AMG_ERR_NAN):
        _check(rc, "amg_pcg_solve_batch")
    return rc, it, rr


def amg_vcycle_apply(h, r, z):
    _check(lib().amg_vcycle_apply(h, r.data_ptr(), z.data_ptr()), "amg_vcycle_apply")


def amg_level_spmv(h, level: int, x, y):
    _check(lib().amg_level_spmv(h, level, x.data_ptr(), y.data_ptr()), "amg_level_spmv")


def amg_get_info(h) -> AmgInfo:
    info = AmgInfo()
    _check(lib().amg_get_info(h, ctypes.byref(info)), "amg_get_info")
    return info


def amg_export_level(h, level: int, n: int, nnz: int, with_map: bool, with_w: bool):
    rp = np.empty(n + 1, np.int64)
    ci = np.empty(nnz, np.int32)
    v = np.empty(nnz)
    d = np.empty(n)
    w = np.empty(n) if with_w else None
    agg = np.empty(n, np.int32) if with_map else None
    pv = np.empty(n) if with_map else None
    P = lambda a: a.ctypes.data if a is not None else None  # noqa: E731
    _check(lib().amg_export_level(h, level, P(rp), P(ci), P(v), P(d), P(w), P(agg), P(pv)), "amg_export_level")
    return dict(rowptr=rp, col=ci, val=v, dl1=d, w=w, agg=agg, pval=pv)


def amg_export_pass(h, level: int, pass_: int):
    ns = ctypes.c_int64()
    _check(lib().amg_export_pass(h, level, pass_, ctypes.byref(ns), None, None, None), "amg_export_pass")
    n = ns.value
    mate = np.empty(n, np.int32)
    agg = np.empty(n, np.int32)
    pv = np.empty(n)
    _check(lib().amg_export_pass(h, level, pass_, None, mate.ctypes.data, agg.ctypes.data, pv.ctypes.data),
           "amg_export_pass")
    return mate, agg, pv


def amg_kernel_launches() -> int:
    return int(lib().amg_kernel_launches())


def amg_profile_kernels(h, enable: bool):
    _check(lib().amg_profile_kernels(h, int(enable)), "amg_profile_kernels")


def amg_kernel_times(h):
    """(ms[3], count[3], bytes[3]) of the three fine-level matrix passes."""
    ms = np.zeros(3)
    cnt = np.zeros(3, np.int64)
    b = np.zeros(3)
    _check(lib().amg_kernel_times(h, ms.ctypes.data, cnt.ctypes.data, b.ctypes.data), "amg_kernel_times")
    return ms, cnt, b


def amg_relres_noalloc(rowptr, col, val, F, u, stream=None) -> float:
    """||F - K u|| / ||F|| for device tensors, through the entry point that
    allocates no device memory (see include/amg_gb300.h)."""
    csr = AmgCsr(len(rowptr) - 1, len(val), rowptr.data_ptr(), col.data_ptr(), val.data_ptr(), AMG_MEM_DEVICE)
    out = ctypes.c_double()
    _check(lib().amg_relres_noalloc(ctypes.byref(csr), F.data_ptr(), u.data_ptr(), ctypes.byref(out),
                                    _stream_handle(stream)), "amg_relres_noalloc")
    return out.value


def amg_free(h):
    _check(lib().amg_free(h), "amg_free")


# ------------------------------------------------------ learned damping
AMG_MPNN_HIDDEN = 32
AMG_MPNN_NPARAM = 4386


def _dev_weights(w):
    """FP32 device tensor of the flat weights (copy of a numpy/host array)."""
    torch = _torch()
    if isinstance(w, np.ndarray):
        w = torch.from_numpy(np.ascontiguousarray(w, dtype=np.float32))
    if w.dtype != torch.float32 or not w.is_cuda:
        w = w.to(device="cuda", dtype=torch.float32)
    w = w.contiguous()
    if w.numel() != AMG_MPNN_NPARAM:
        raise ValueError(f"expected {AMG_MPNN_NPARAM} weights, got {w.numel()}")
    return w


def amg_mpnn_apply(h, w, bf16_weights: bool = True):
    """Install the network's damping (w: weights) or, with w None, the plain
    smoother diagonal."""
    wd = None if w is None else _dev_weights(w)
    _check(lib().amg_mpnn_apply(h, None if wd is None else wd.data_ptr(), int(bf16_weights)), "amg_mpnn_apply")


def amg_mpnn_omega(h, level: int, n: int):
    torch = _torch()
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    _check(lib().amg_mpnn_omega(h, level, out.data_ptr()), "amg_mpnn_omega")
    return out


def amg_mpnn_loss_grad(h, w, nprobe: int, seed: int):
    """(loss, gradient as an FP64 device tensor)."""
    torch = _torch()
    wd = _dev_weights(w)
    g = torch.empty(AMG_MPNN_NPARAM, dtype=torch.float64, device="cuda")
    loss = ctypes.c_double()
    _check(lib().amg_mpnn_loss_grad(h, wd.data_ptr(), nprobe, seed & 0xFFFFFFFFFFFFFFFF, ctypes.byref(loss),
                                    g.data_ptr()), "amg_mpnn_loss_grad")
    return loss.value, g


def amg_mpnn_theta_loss_grad(h, w, nprobe: int, seed: int):
    """(loss, gradient) of the smoothing weights' two-grid loss."""
    torch = _torch()
    wd = _dev_weights(w)
    g = torch.empty(AMG_MPNN_NPARAM, dtype=torch.float64, device="cuda")
    loss = ctypes.c_double()
    _check(lib().amg_mpnn_theta_loss_grad(h, wd.data_ptr(), nprobe, seed & 0xFFFFFFFFFFFFFFFF, ctypes.byref(loss),
                                          g.data_ptr()), "amg_mpnn_theta_loss_grad")
    return loss.value, g


def amg_mpnn_theta(h, n: int):
    torch = _torch()
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    _check(lib().amg_mpnn_theta(h, out.data_ptr()), "amg_mpnn_theta")
    return out


def amg_mpnn_adam(h, w, grad, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam step on device tensors w, m, v (FP32) with FP64 grad."""
    _check(lib().amg_mpnn_adam(h, w.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), t, lr, beta1, beta2,
                               eps), "amg_mpnn_adam")


def amg_mpnn_train(hs, w, steps: int, nprobe: int, seed: int, lr: float):
    """Train the FP32 device tensor w in place on one hierarchy handle or a
    list of them (mean loss); returns the loss history."""
    hs = list(hs) if isinstance(hs, (list, tuple)) else [hs]
    arr = (ctypes.c_void_p * len(hs))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in hs])
    hist = np.zeros(max(steps, 1))
    _check(lib().amg_mpnn_train(arr, len(hs), w.data_ptr(), steps, nprobe, seed & 0xFFFFFFFFFFFFFFFF, lr,
                                hist.ctypes.data), "amg_mpnn_train")
    return hist[:steps]


def amg_mpnn_select(h, w, F, rtol: float, itmax: int, omega_ref: float = 1.0):
    """(used, iters_ref, iters_learned) of the fallback rule against the
    constant damping omega_ref (1: the plain smoother)."""
    wd = _dev_weights(w)
    used, ip, il = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().amg_mpnn_select(h, wd.data_ptr(), float(omega_ref), F.data_ptr(), rtol, itmax, ctypes.byref(used),
                                 ctypes.byref(ip), ctypes.byref(il)), "amg_mpnn_select")
    return bool(used.value), ip.value, il.value


def _iga_patch(n, p, nq=0, geometry=AMG_GEOM_CUBE, with_boundary=False, source=AMG_SRC_ONE, kappa=None):
    """The patch struct; kappa = (omega, phi, sigma) with omega (M, 3) and
    phi (M,) FP64 device tensors, or None (kappa = 1).  Returns the struct
    and the tensors it points to (keep them alive)."""
    P = AmgIgaPatch(int(n), int(p), int(nq), int(geometry), int(bool(with_boundary)), int(source), 0, 0.0, None, None)
    keep = ()
    if kappa is not None:
        om, ph, sigma = kappa
        if om.dtype != ph.dtype or str(om.dtype) != "torch.float64" or not (om.is_cuda and ph.is_cuda):
            raise ValueError("kappa's omega and phi must be FP64 device tensors")
        if om.numel() != 3 * ph.numel():
            raise ValueError("omega must hold 3 frequencies per phase")
        om = om.contiguous()
        ph = ph.contiguous()
        P.kappa_m = int(ph.numel())
        P.kappa_sigma = float(sigma)
        P.kappa_omega = om.data_ptr()
        P.kappa_phi = ph.data_ptr()
        keep = (om, ph)
    return P, keep


def amg_iga_size(patch) -> tuple[int, int]:
    """(unknowns, stored entries) of an AmgIgaPatch."""
    n, z = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().amg_iga_size(ctypes.byref(patch), ctypes.byref(n), ctypes.byref(z)), "amg_iga_size")
    return n.value, z.value


def amg_iga_assemble(patch, rowptr, col, val, F=None, stream=None) -> float:
    """Assemble into caller-allocated device tensors; returns the flop count
    of the quadrature sums."""
    fl = ctypes.c_double()
    _check(lib().amg_iga_assemble(ctypes.byref(patch), rowptr.data_ptr(), col.data_ptr(), val.data_ptr(),
                                  None if F is None else F.data_ptr(), _stream_handle(stream), ctypes.byref(fl)),
           "amg_iga_assemble")
    return fl.value


def iga_assemble(n, p, nq=0, geometry=AMG_GEOM_CUBE, with_boundary=False, source=AMG_SRC_ONE, kappa=None,
                 load=True, stream=None, device=None):
    """K (CSR) and F of a patch as new device tensors: dict with rowptr, col,
    val, F (or None), n, flops."""
    import torch

    P, keep = _iga_patch(n, p, nq, geometry, with_boundary, source, kappa)
    N, Z = amg_iga_size(P)
    dev = device or torch.device("cuda", torch.cuda.current_device())
    rowptr = torch.empty(N + 1, dtype=torch.int64, device=dev)
    col = torch.empty(max(Z, 1), dtype=torch.int32, device=dev)
    val = torch.empty(max(Z, 1), dtype=torch.float64, device=dev)
    F = torch.empty(max(N, 1), dtype=torch.float64, device=dev) if load else None
    fl = amg_iga_assemble(P, rowptr, col, val, F, stream)
    del keep
    return {"rowptr": rowptr, "col": col[:Z], "val": val[:Z], "F": None if F is None else F[:N], "n": N,
            "flops": fl}


def amg_dfma_probe_variants() -> int:
    """Number of FP64 probe variants."""
    n = ctypes.c_int32()
    _check(lib().amg_dfma_probe(-1, 0, 1, None, None, ctypes.byref(n), None), "amg_dfma_probe")
    return n.value


def amg_dfma_probe_threads(variant: int) -> int:
    """Block size of FP64 probe variant `variant`."""
    t = ctypes.c_int32()
    _check(lib().amg_dfma_probe(int(variant), 0, 1, None, None, ctypes.byref(t), None), "amg_dfma_probe")
    return t.value


def amg_dfma_probe(variant: int, blocks: int, trips: int, out, stream=None) -> float:
    """Enqueue FP64 probe variant `variant`; returns its flop count."""
    fl = ctypes.c_double()
    t = ctypes.c_int32()
    _check(lib().amg_dfma_probe(int(variant), int(blocks), int(trips), out.data_ptr(), _stream_handle(stream),
                                ctypes.byref(t), ctypes.byref(fl)), "amg_dfma_probe")
    return fl.value


def amg_div_check(a, b, stream=None):
    """(a / b rounded by the library's FP64 division, number of quotients its
    fast path accepted) for device float64 tensors a, b of equal length."""
    import torch
    a = a.contiguous()
    b = b.contiguous()
    q = torch.empty_like(a)
    cnt = torch.zeros(1, dtype=torch.int64, device=a.device)
    _check(lib().amg_div_check(a.numel(), a.data_ptr(), b.data_ptr(), q.data_ptr(), cnt.data_ptr(),
                               _stream_handle(stream)), "amg_div_check")
    return q, cnt


def amg_export_coarse(h):
    """(L, Ainv) of the coarsest level's dense factorisation, host arrays."""
    n = ctypes.c_int32()
    _check(lib().amg_export_coarse(h, ctypes.byref(n), None, None), "amg_export_coarse")
    L = np.zeros((n.value, n.value))
    Ai = np.zeros((n.value, n.value))
    _check(lib().amg_export_coarse(h, ctypes.byref(n), L.ctypes.data, Ai.ctypes.data), "amg_export_coarse")
    return L, Ai


def amg_export_prolongator(h, level: int, n: int):
    """(rowptr, col, val) of level `level`'s prolongator on the host."""
    nnz = ctypes.c_int64()
    _check(lib().amg_export_prolongator(h, level, ctypes.byref(nnz), None, None, None), "amg_export_prolongator")
    rp = np.empty(n + 1, np.int64)
    ci = np.empty(nnz.value, np.int32)
    v = np.empty(nnz.value)
    _check(lib().amg_export_prolongator(h, level, ctypes.byref(nnz), rp.ctypes.data, ci.ctypes.data, v.ctypes.data),
           "amg_export_prolongator")
    return rp, ci, v


def amg_set_damping(h, omega: float):
    """Install the constant damping omega / d on every smoothed level."""
    _check(lib().amg_set_damping(h, float(omega)), "amg_set_damping")


def amg_smoother_bound(h, level: int) -> float:
    """lam_hat, the Lanczos upper estimate of lambda_max(D^-1 K) on `level`."""
    out = ctypes.c_double()
    _check(lib().amg_smoother_bound(h, level, ctypes.byref(out)), "amg_smoother_bound")
    return out.value


class Hierarchy:
    """Owning wrapper of an ``amg_hierarchy*``."""

    def __init__(self, rowptr, col, val, stream=None, **opts):
        self.opts = amg_opts_default(**opts)
        self._h = amg_setup(rowptr, col, val, self.opts, stream)
        self.info = amg_get_info(self._h)

    def close(self):
        if getattr(self, "_h", None):
            amg_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def num_levels(self) -> int:
        return self.info.levels

    def level_n(self, l: int) -> int:
        return int(self.info.n[l])

    def level_nnz(self, l: int) -> int:
        return int(self.info.nnz[l])

    def solve(self, F, u=None, rtol: float = 1e-8, itmax: int = 10000):
        """u is created as zeros (same memory space as F) when not given."""
        if u is None:
            if isinstance(F, np.ndarray):
                u = np.zeros_like(F, dtype=np.float64)
            else:
                u = F.new_zeros(F.shape)
        status, iters, relres = amg_pcg_solve(self._h, F, u, rtol, itmax)
        self.info = amg_get_info(self._h)
        return dict(u=u, iters=iters, relres=relres, status=status)

    def solve_multi(self, F, U=None, rtol: float = 1e-8, itmax: int = 10000):
        """F: (nrhs, n) array/tensor; returns dict(u, iters[], relres[], status)."""
        if U is None:
            U = np.zeros_like(F, dtype=np.float64) if isinstance(F, np.ndarray) else F.new_zeros(F.shape)
        status, iters, relres = amg_pcg_solve_multi(self._h, F, U, rtol, itmax)
        self.info = amg_get_info(self._h)
        return dict(u=U, iters=iters, relres=relres, status=status)

    def vcycle(self, r):
        z = r.new_empty(r.shape)
        amg_vcycle_apply(self._h, r, z)
        return z

    def spmv(self, level: int, x):
        y = x.new_empty((self.level_n(level),))
        amg_level_spmv(self._h, level, x, y)
        return y

    def export_level(self, l: int):
        last = l == self.num_levels - 1
        return amg_export_level(self._h, l, self.level_n(l), self.level_nnz(l), not last, l == 0 and not last or l > 0)

    def export_pass(self, l: int, s: int):
        return amg_export_pass(self._h, l, s)

    def export_prolongator(self, l: int):
        return amg_export_prolongator(self._h, l, self.level_n(l))

    def export_coarse(self):
        return amg_export_coarse(self._h)

    # learned smoother damping
    def mpnn_apply(self, w=None, bf16_weights: bool = True):
        amg_mpnn_apply(self._h, w, bf16_weights)

    def mpnn_omega(self, level: int):
        return amg_mpnn_omega(self._h, level, self.level_n(level))

    def mpnn_loss_grad(self, w, nprobe: int = 4, seed: int = 99):
        return amg_mpnn_loss_grad(self._h, w, nprobe, seed)

    def mpnn_train(self, w, steps: int, nprobe: int = 4, seed: int = 1000, lr: float = 1e-2, others=()):
        """Train w on this hierarchy (and the hierarchies in `others`)."""
        return amg_mpnn_train([self._h] + [o._h for o in others], w, steps, nprobe, seed, lr)

    def mpnn_theta_loss_grad(self, w, nprobe: int = 4, seed: int = 99):
        return amg_mpnn_theta_loss_grad(self._h, w, nprobe, seed)

    def mpnn_theta(self):
        return amg_mpnn_theta(self._h, self.level_n(0))

    def mpnn_select(self, w, F, rtol: float = 1e-8, itmax: int = 10000, omega_ref: float = 1.0):
        return amg_mpnn_select(self._h, w, F, rtol, itmax, omega_ref)

    def set_damping(self, omega: float):
        amg_set_damping(self._h, omega)

    def smoother_bound(self, level: int) -> float:
        return amg_smoother_bound(self._h, level)


class BatchHierarchy(Hierarchy):
    """Owning wrapper of a batch hierarchy (amg_setup_batch)."""

    def __init__(self, systems, stream=None, **opts):
        self.opts = amg_opts_default(**opts)
        self._h = amg_setup_batch(systems, self.opts, stream)
        self.info = amg_get_info(self._h)
        self.sizes = [len(rp) - 1 for rp, _, _ in systems]

    def solve_batch(self, Fs, Us=None, rtol: float = 1e-8, itmax: int = 10000):
        if Us is None:
            Us = [np.zeros_like(F, dtype=np.float64) if isinstance(F, np.ndarray) else F.new_zeros(F.shape)
                  for F in Fs]
        status, iters, relres = amg_pcg_solve_batch(self._h, Fs, Us, rtol, itmax)
        self.info = amg_get_info(self._h)
        return dict(u=Us, iters=iters, relres=relres, status=status)
