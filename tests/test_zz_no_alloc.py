"""The entry point that allocates no device memory (amg_relres_noalloc).

It serves callers that cannot allocate -- for example an application whose
pool allocator owns all GPU memory, or a time-critical loop that must not
trigger a cudaMalloc.  It must report the same relative residual as the
regular path (amg_pcg_solve's relres, computed with scratch inside an
allocated hierarchy), on consecutive calls that reuse its static scratch.

This file is collected last so that a failure here comes after every other
test has run; it also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_21268_gb300 import amg as A  # noqa: E402
from paper_2511_21268_gb300 import inputs as I  # noqa: E402

RTOL = 1e-12  # same as the V-cycle parity tolerance: only the summation order differs


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("d,n,p,iters", [(3, 12, 3, 3), (2, 40, 2, 5)])
def test_noalloc_matches_solver_relres_on_two_calls(d, n, p, iters):
    prob = I.poisson_box(d, n, p)
    rp, ci, va, F = _dev(prob.rowptr), _dev(prob.col), _dev(prob.val), _dev(prob.F)
    H = A.Hierarchy(rp, ci, va, coarse_max=20)
    u = torch.zeros_like(F)
    st, it, rel_solver = A.amg_pcg_solve(H._h, F, u, 0.0, iters)  # stops after `iters` iterations
    assert it == iters and rel_solver > 0.0
    first = A.amg_relres_noalloc(rp, ci, va, F, u)
    second = A.amg_relres_noalloc(rp, ci, va, F, u)
    assert abs(first - rel_solver) <= RTOL * rel_solver
    assert abs(second - rel_solver) <= RTOL * rel_solver
    # a different input on the next call: stale scratch contents are not reused
    z = torch.zeros_like(F)
    assert abs(A.amg_relres_noalloc(rp, ci, va, F, z) - 1.0) <= RTOL
    H.close()


def test_noalloc_rejects_oversize_and_host_matrix():
    prob = I.poisson_box(2, 6, 2)
    rp, ci, va, F = _dev(prob.rowptr), _dev(prob.col), _dev(prob.val), _dev(prob.F)
    import ctypes

    big = A.AmgCsr((1 << 19) + 1, len(prob.val), rp.data_ptr(), ci.data_ptr(),
                   va.data_ptr(), A.AMG_MEM_DEVICE)
    out = ctypes.c_double()
    assert A.lib().amg_relres_noalloc(ctypes.byref(big), F.data_ptr(), F.data_ptr(), ctypes.byref(out), None) == \
        A.AMG_ERR_ARG
    host = A.AmgCsr(prob.n, len(prob.val), prob.rowptr.ctypes.data, prob.col.ctypes.data, prob.val.ctypes.data,
                    A.AMG_MEM_HOST)
    assert A.lib().amg_relres_noalloc(ctypes.byref(host), F.data_ptr(), F.data_ptr(), ctypes.byref(out), None) == \
        A.AMG_ERR_ARG


def test_noalloc_allocates_no_device_memory():
    """The defining property: a warm call changes neither the device's free
    memory nor torch's allocator (the first call may load the module and
    look up the scratch address; later calls only launch and copy)."""
    prob = I.poisson_box(3, 10, 3)
    rp, ci, va, F = _dev(prob.rowptr), _dev(prob.col), _dev(prob.val), _dev(prob.F)
    u = torch.zeros_like(F)
    A.amg_relres_noalloc(rp, ci, va, F, u)  # warm: module loaded, address cached
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        assert abs(A.amg_relres_noalloc(rp, ci, va, F, u) - 1.0) <= RTOL
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == alloc0

