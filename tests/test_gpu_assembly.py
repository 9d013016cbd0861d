"""GPU IgA assembly by sum factorization (Sec. 2.2) against the assembly
oracle's element loop, through the C ABI.

* Small patches (several elements, both geometries, with and without the
  boundary functions, kappa on and off, f = 1 and the sine source): the CSR
  pattern is exactly the band |i_k - j_k| <= p, every stored value and every
  load entry is within 1e-12 of the oracle's (relative to the largest entry:
  the sums run in another order).
* The learned-damping workload (quarter annulus, p = 3, n = 64, kappa with
  M = 256 features): sampled rows and load entries against the oracle's
  rows, and the whole matrix against the input generator's C element loop.
* Edge cases: one element, p = 1, an empty system (n = 1, p = 1 without the
  boundary), nq other than p + 1.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import iga  # noqa: E402
from paper_2511_21268_gb300 import amg as A  # noqa: E402
from paper_2511_21268_gb300 import inputs as I  # noqa: E402

GEOM = {"cube": A.AMG_GEOM_CUBE, "annulus": A.AMG_GEOM_ANNULUS}
SRC = {"one": A.AMG_SRC_ONE, "sine": A.AMG_SRC_SINE}


def band_pattern(m, p):
    rp = [0]
    cols = []
    for i3 in range(m):
        for i2 in range(m):
            for i1 in range(m):
                for j3 in range(max(0, i3 - p), min(m, i3 + p + 1)):
                    for j2 in range(max(0, i2 - p), min(m, i2 + p + 1)):
                        for j1 in range(max(0, i1 - p), min(m, i1 + p + 1)):
                            cols.append(j1 + m * (j2 + m * j3))
                rp.append(len(cols))
    return np.array(rp), np.array(cols)


def kappa_params(M, seed=5, ell=0.4):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(M, 3)) / ell, rng.uniform(0, 2 * math.pi, M)


def gpu(n, p, geom, wb, kap=None, src="one", nq=0):
    kappa = None
    if kap is not None:
        om, ph, sigma = kap
        kappa = (torch.tensor(om, dtype=torch.float64, device="cuda"),
                 torch.tensor(ph, dtype=torch.float64, device="cuda"), sigma)
    return A.iga_assemble(n, p, nq=nq, geometry=GEOM[geom], with_boundary=wb, source=SRC[src], kappa=kappa)


CASES = [(1, 1, "cube", True, 0, "one", 0), (3, 2, "cube", False, 0, "sine", 0), (4, 3, "cube", True, 0, "one", 0),
         (3, 2, "annulus", True, 0, "one", 0), (4, 2, "annulus", False, 6, "one", 0),
         (3, 3, "annulus", True, 4, "one", 0), (5, 1, "annulus", False, 3, "one", 0),
         (2, 2, "annulus", True, 3, "one", 5)]


@pytest.mark.parametrize("n,p,geom,wb,M,src,nq", CASES, ids=lambda c: str(c))
def test_small_patches_match_oracle(n, p, geom, wb, M, src, nq):
    kap = None
    kw = {}
    if M:
        om, ph = kappa_params(M)
        kap = (om, ph, 0.8)
        kw = dict(omega=om, phi=ph, sigma=0.8)
    g = gpu(n, p, geom, wb, kap, src, nq)
    P = iga.Patch(n, p, nq=nq or None, geom=geom, with_boundary=wb, src=src, **kw)
    K, F = P.assemble()
    m = P.m
    rp, ci = band_pattern(m, p)
    assert g["n"] == m ** 3
    assert np.array_equal(g["rowptr"].cpu().numpy(), rp)
    assert np.array_equal(g["col"].cpu().numpy(), ci)
    val = g["val"].cpu().numpy()
    dense = np.zeros_like(K)
    for i in range(m ** 3):
        dense[i, ci[rp[i]:rp[i + 1]]] = val[rp[i]:rp[i + 1]]
    scale = np.abs(K).max()
    assert np.abs(dense - K).max() <= 1e-12 * scale
    assert np.abs(g["F"].cpu().numpy() - F).max() <= 1e-12 * np.abs(F).max()
    assert g["flops"] > 0


def test_empty_system():
    g = gpu(1, 1, "cube", False)
    assert g["n"] == 0 and g["rowptr"].cpu().tolist() == [0] and len(g["val"]) == 0


def _learned_workload(n, p):
    """The annulus workload's kappa, drawn as the input generator draws it."""
    k = I.ANNULUS_KAPPA
    M, ell, sigma, seed = k["M"], k["ell"], k["sigma"], 7
    om = I.rng_normal(seed, 3 * M).reshape(M, 3) / ell
    ph = I.rng_u01(seed + 1, M) * 2 * math.pi
    return om, ph, sigma


def test_full_size_annulus_rows_match_oracle_and_generator():
    n, p = 64, 3
    om, ph, sigma = _learned_workload(n, p)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    g = gpu(n, p, "annulus", False, (om, ph, sigma))  # warm-up (pool, module load)
    t0.record()
    g = gpu(n, p, "annulus", False, (om, ph, sigma))
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    rp = g["rowptr"].cpu().numpy()
    ci = g["col"].cpu().numpy()
    val = g["val"].cpu().numpy()
    F = g["F"].cpu().numpy()
    P = iga.Patch(n, p, geom="annulus", omega=om, phi=ph, sigma=sigma)
    m = P.m
    rng = np.random.default_rng(1)
    rows = [0, m - 1, m * m * (m - 1), m ** 3 - 1, (m // 2) * (1 + m + m * m)] + list(rng.integers(0, m ** 3, 4))
    for Irow in rows:
        want, f = P.row(int(Irow))
        cols = ci[rp[Irow]:rp[Irow + 1]]
        got = val[rp[Irow]:rp[Irow + 1]]
        assert set(want) <= set(cols.tolist())
        w = np.array([want.get(int(c), 0.0) for c in cols])
        assert np.abs(got - w).max() <= 1e-12 * np.abs(w).max(), Irow
        assert abs(F[Irow] - f) <= 1e-12 * abs(f)
    # the input generator's C element loop, whole matrix
    prob = I.annulus_kappa(n, p)
    assert np.array_equal(prob.rowptr, rp) and np.array_equal(prob.col, ci)
    rel = np.abs(prob.val - val).max() / np.abs(prob.val).max()
    assert rel <= 1e-12, rel
    assert np.abs(prob.F - F).max() <= 1e-12 * np.abs(prob.F).max()
    print(f"\nassembly n={n} p={p}: {ms:.1f} ms on the GPU, {g['flops'] / ms / 1e9:.3f} TFLOP/s, max rel diff "
          f"vs the generator {rel:.2e}")
