"""Benchmark: time-to-solution of matching-based AMG-PCG on an IgA system.

Workload (one GPU): 3-D Poisson on the unit cube, B-splines of degree p=3
with C^2 continuity, n=64 elements per direction, homogeneous Dirichlet
data eliminated (N = 65^3 = 274,625 unknowns, 86,938,307 nonzeros, FP64
CSR 1.04 GB), f from the manufactured solution u = sin(pi x) sin(pi y)
sin(pi z); PCG with the matching-based aggregation AMG V-cycle (two matching
passes per level, one l1-Jacobi pre/post sweep, coarsest <= 200 rows solved
densely), x0 = 0, rtol 1e-8, all in FP64.

One step = amg_setup + amg_pcg_solve + amg_free on that system (the whole
hot path), inputs resident in HBM.  The matrix (1.04 GB) is larger than L2
(129 MB), so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own copy of the system (independent
replicas, no collective on the data path): weak scaling.  Rank 0 prints one
JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time-to-solution at rtol 1e-8 and V-cycle HBM GB/s: mixed/learned vs FP64 AMG"
WORKLOAD = "3-D Poisson unit cube, B-spline p=3 C^2, n=64 (N=274,625, nnz=86,938,307), FP64 AMG-PCG, rtol 1e-8"
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "fine_matrix_pass_fp64_3d_p3_n64.md")
STREAM_SUMMARY = os.path.join(ROOT, "profiles", "staged_mixed_passes_3d_p3_n64.md")
# FP64 finest-level passes by the layout the library chose (amg_info.staged_passes): 3 = sliced slabs
# with FP64 values (k_sell64), else the row-group kernels on run-encoded columns
FP64_KERNEL_NAMES = {
    3: ["k_sell64<7, Epi64PQ> (q = K p)", "k_sell64<7, Epi64Resid> (down-sweep residual)",
        "k_sell64<7, Epi64Up0> (up-sweep smoothing)"],
    0: ["k_spmv_pq<8> (q = K p)", "k_resid<8> (down-sweep residual)", "k_up0<8> (up-sweep smoothing)"],
}
FP64_SOURCES = {3: ("sell_kernels.cu",), 0: ("row_kernels.cuh",)}
# staged mixed-precision passes of the run-encoded finest matrix (matrix_format 2), by the
# layout the library chose (amg_info.staged_passes): 2 = sliced slabs with a lane per row
# (k_sell), 1 = slabs with a lane per run (k_stream)
MIXED_KERNEL_NAMES = {
    2: ["k_sell<7, f32, EpiPQ> (q = K p)", "k_sell<7, bf16, EpiResid> (down-sweep residual)",
        "k_sell<7, bf16, EpiUp0> (up-sweep smoothing)"],
    1: ["k_stream<EpiPQ, f32> (q = K p)", "k_stream<EpiResid, bf16> (down-sweep residual)",
        "k_stream<EpiUp0, bf16> (up-sweep smoothing)"],
    0: ["k_spmv_pq<8,f32> (q = K p)", "k_resid<8,bf16> (down-sweep residual)", "k_up0<8,bf16> (up-sweep smoothing)"],
}
STAGED_SOURCES = {2: ("sell_kernels.cu", "stream_common.cuh"), 1: ("stream_kernels.cu", "stream_common.cuh")}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--p", type=int, default=3)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-annulus", action="store_true")
    ap.add_argument("--no-smoothing", action="store_true")
    ap.add_argument("--no-paper-config", action="store_true")
    ap.add_argument("--no-paper-headline", action="store_true")
    ap.add_argument("--no-assembly", action="store_true")
    ap.add_argument("--train-steps", type=int, default=60)
    ap.add_argument("--matrix-format", type=int, choices=[0, 1, 2], default=2,
                    help="2 = run-encoded finest level + bulk-copy streamed mixed passes (default), 1 = run-encoded, 0 = CSR")
    ap.add_argument("--precision", choices=["fp64", "fp32", "bf16"], default="fp64",
                    help="precision of the main timed leg (profiling runs)")
    return ap.parse_args()


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def committed_traffic(summary=PROFILE_SUMMARY, sources=("row_kernels.cuh",)):
    """DRAM bytes per launch from a committed ncu summary, or None if the
    kernels' sources changed since the counters were taken (the summary
    records the SHA-256 of the concatenated source files)."""
    if not os.path.exists(summary):
        return None
    txt = open(summary).read()
    m = re.search(r"source_sha256:\s*([0-9a-f]{64})", txt)
    h = hashlib.sha256()
    for f in sources:
        h.update(open(os.path.join(ROOT, "paper_2511_21268_gb300", "csrc", f), "rb").read())
    if not m or m.group(1) != h.hexdigest():
        return None
    out = {}
    for k, v in re.findall(r"traffic_bytes_per_launch\[(\w+)\]:\s*([0-9.eE+]+)", txt):
        out[k] = float(v)
    return out or None


def fp64_peak_tflops():
    """FP64 rate from unit counts and clock: SMs x max SM clock x 2 DFMA/clk x 2 flop."""
    import torch

    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = 2070.0
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        mhz = float(json.load(open(path)).get("sm_max_mhz", mhz))
    return sms * mhz * 1e6 * 2 * 2 / 1e12


def measure_fp64_rate(A, torch, stream, uuid, seconds=2.0):
    """FP64 FMA rate of this GPU, measured: every variant of the library's
    FMA probe (independent chains per thread, shared or own operands, 2048 or
    512 threads per SM) timed with CUDA events on its stream, then the
    fastest for about `seconds` with the SM clocks sampled meanwhile.
    Returns (TFLOP/s, clocks, {variant: TFLOP/s})."""
    dev = torch.device("cuda", torch.cuda.current_device())
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def setup(v):
        th = A.amg_dfma_probe_threads(v)
        blocks = sms * (2048 // th if th >= 256 else 512 // th)
        return blocks, torch.empty(blocks * th, dtype=torch.float64, device=dev)

    def timed(v, blocks, out, trips, launches):
        e0.record(stream)
        fl = 0.0
        for _ in range(launches):
            fl += A.amg_dfma_probe(v, blocks, trips, out, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return fl, e0.elapsed_time(e1)

    rates, cal = {}, {}
    for v in range(A.amg_dfma_probe_variants()):
        blocks, out = setup(v)
        trips = 64
        for _ in range(4):  # calibrate one launch to about 0.2 s
            _, ms = timed(v, blocks, out, trips, 1)
            trips = max(64, int(trips * 200.0 / max(ms, 1e-3)))
        fl, ms = timed(v, blocks, out, trips, 2)
        rates[v] = fl / (ms * 1e-3) / 1e12
        cal[v] = (blocks, out, trips)
    best = max(rates, key=rates.get)
    blocks, out, trips = cal[best]
    clocks = ClockSampler(uuid)
    clocks.start()
    time.sleep(0.2)
    fl, ms = timed(best, blocks, out, trips, max(3, int(seconds / 0.2)))
    clk = clocks.stop()
    if not torch.isfinite(out).all():
        raise RuntimeError("FP64 probe produced non-finite values")
    return fl / (ms * 1e-3) / 1e12, clk, {str(k): round(v, 4) for k, v in rates.items()}


class ClockSampler:
    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            if self.uuid and parts[1] != self.uuid:
                continue
            rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def init_dist(world):
    import torch
    import torch.distributed as dist

    if world > 1 and not dist.is_initialized():
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return dist if world > 1 else None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x: float) -> float:
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------- oracle
def cpu_baseline(prob, iters_gpu: int, rtol: float) -> dict:
    """Time the CPU oracle on a bounded sample of the workload: the full setup
    (sequential: the greedy matching is defined by a sequential scan), CG
    with itmax = 0 (the start: median of three runs) and with itmax = 3
    (three iterations beyond the start), scaled to the iteration count of the
    GPU solve (the two agree within +-1).  The solve phase is timed on one
    core and with its row loops on all host cores (same results)."""
    import oracle as O

    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    H = O.Hierarchy(prob.rowptr, prob.col, prob.val)
    t_setup = time.perf_counter() - t0

    def solve_phase(threads):
        used = O.set_threads(threads)
        try:
            starts = []
            for _ in range(3):
                t0 = time.perf_counter()
                H.pcg(prob.F, rtol=rtol, itmax=0)
                starts.append(time.perf_counter() - t0)
            t_start = statistics.median(starts)
            t0 = time.perf_counter()
            H.pcg(prob.F, rtol=rtol, itmax=3)
            t_iter = max((time.perf_counter() - t0 - t_start) / 3, 0.0)
        finally:
            O.set_threads(1)
        return used, t_start, t_iter

    _, s1, i1 = solve_phase(1)
    used, sn, iN = solve_phase(cores)
    v1 = t_setup + s1 + iters_gpu * i1
    vn = t_setup + sn + iters_gpu * iN
    return {"value": vn, "unit": "s", "cores": used, "kind": "oracle",
            "sample": (f"full oracle setup ({t_setup:.2f} s, sequential) + CG start ({sn:.3f} s, median of 3) + "
                       f"{iN:.3f} s per CG iteration (three iterations timed) on the full system, scaled to "
                       f"{iters_gpu} iterations; plain C oracle, solve-phase row loops on {used} threads"),
            "setup_s": t_setup, "iter_s": iN,
            "one_core": {"value": v1, "cores": 1, "iter_s": i1, "start_s": s1}}


def run_reference(args):
    """--impl reference: the CPU oracle as the reference arm, rank 0 only."""
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    import oracle as O
    from paper_2511_21268_gb300 import inputs as I

    prob = I.poisson_box(3, args.n, args.p)
    t0 = time.perf_counter()
    H = O.Hierarchy(prob.rowptr, prob.col, prob.val)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    full = H.pcg(prob.F, rtol=args.rtol)
    t_full = time.perf_counter() - t0
    samples = []
    for k in range(args.warmup + args.steps):  # each step: one CG iteration of the oracle
        t0 = time.perf_counter()
        H.pcg(prob.F, rtol=args.rtol, itmax=0)
        a = time.perf_counter() - t0
        t0 = time.perf_counter()
        H.pcg(prob.F, rtol=args.rtol, itmax=1)
        b = time.perf_counter() - t0
        if k >= args.warmup:
            samples.append((a, b))
    t_start = statistics.median(a for a, _ in samples)
    t_iter = statistics.median(max(b - a, 0.0) for a, b in samples)
    value = t_setup + t_start + full["iters"] * t_iter
    sample = (f"oracle setup once ({t_setup:.2f} s), full oracle solve once ({full['iters']} iterations, "
              f"{t_full:.1f} s); each step = one oracle CG iteration on the full system; value = setup + start + "
              f"iterations x median step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_iter * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": args.n, "p": args.p, "N": prob.n, "nnz": prob.nnz,
                       "rtol": args.rtol},
            "cpu_baseline": {"value": value, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "iters": full["iters"], "measured_full_solve_s": t_full, "setup_s": t_setup}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------- ours
CONST_SWEEP = (1.0, 1.5, 1.8, 1.9, 1.95, 2.0, 2.2, 2.4, 2.6)


def omega_stats(A, h, torch):
    """min / max / mean / std of the installed network damping per smoothed
    level, with the level's cap omega_max = 2 / lam_hat."""
    info = A.amg_get_info(h)
    out = []
    for l in range(info.levels - 1):
        om = A.amg_mpnn_omega(h, l, int(info.n[l])).double()
        out.append({"level": l, "rows": int(info.n[l]), "min": float(om.min()), "max": float(om.max()),
                    "mean": float(om.mean()), "std": float(om.std()),
                    "omega_max": 2.0 / A.amg_smoother_bound(h, l)})
    return out


def constant_sweep(A, h, F, rtol, torch):
    """PCG iterations with the constant damping omega on every smoothed
    level, for each omega of CONST_SWEEP (None where the solve fails)."""
    its = {}
    for om in CONST_SWEEP:
        A.amg_set_damping(h, om)
        st, it, _ = A.amg_pcg_solve(h, F, torch.zeros_like(F), rtol, 3000)
        its[om] = it if st == A.AMG_OK else None
    A.amg_set_damping(h, 1.0)
    ok = {o: i for o, i in its.items() if i is not None}
    best = min(ok, key=lambda o: (ok[o], o))
    return its, best


def timed_steps(step, k, warm, stream, torch, dist):
    for _ in range(warm):
        step()
    torch.cuda.synchronize()
    barrier(dist)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(k):
        out = step()
    e1.record(stream)
    torch.cuda.synchronize()
    return max_over_ranks(dist, e0.elapsed_time(e1)) / k, out


def learned_leg(args, A, I, torch, np, stream, dist, rp, ci, va, F, ref_u, fp64_ms, mixed_ms):
    """Mixed precision + learned smoother damping on the bench workload,
    against mixed precision with the best constant damping of a sweep."""
    dev = F.device
    # training set: 3-D cube hierarchies, p in {2, 3, 4}, n = 16 (FP64)
    train = []
    for pp in (2, 3, 4):
        q = I.poisson_box(3, 16, pp)
        train.append(A.amg_setup(torch.from_numpy(q.rowptr).to(dev), torch.from_numpy(q.col).to(dev),
                                 torch.from_numpy(q.val).to(dev), A.amg_opts_default(), stream))
    w = torch.from_numpy(I.mpnn_init_weights(1).astype(np.float32)).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = A.amg_mpnn_train(train, w, args.train_steps, 4, 1000, 1e-2)
    train_s = time.perf_counter() - t0
    for h in train:
        A.amg_free(h)
    mopts = A.amg_opts_default(precision=A.AMG_FP32_BF16FINE, matrix_format=args.matrix_format)

    # constant damping sweep and the fallback rule against the best constant (untimed)
    h = A.amg_setup(rp, ci, va, mopts, stream)
    sweep, best = constant_sweep(A, h, F, args.rtol, torch)
    used, it_best, it_learned = A.amg_mpnn_select(h, w, F, args.rtol, 10000, omega_ref=best)
    # inference time alone (features and damping caps are computed on the first call)
    A.amg_mpnn_apply(h, w, True)
    stats = omega_stats(A, h, torch)
    i0 = torch.cuda.Event(enable_timing=True)
    i1 = torch.cuda.Event(enable_timing=True)
    i0.record(stream)
    for _ in range(5):
        A.amg_mpnn_apply(h, w, True)
    i1.record(stream)
    torch.cuda.synchronize()
    infer_ms = i0.elapsed_time(i1) / 5
    A.amg_free(h)
    h = A.amg_setup(rp, ci, va, A.amg_opts_default(matrix_format=args.matrix_format), stream)
    A.amg_mpnn_apply(h, w, True)
    u64 = torch.zeros_like(F)
    _, it64, _ = A.amg_pcg_solve(h, F, u64, args.rtol, 10000)
    A.amg_free(h)

    # the weights go to the setup: the finest level's network overlaps the
    # coarse-level setup on a second stream
    lopts = A.amg_opts_default(precision=A.AMG_FP32_BF16FINE, matrix_format=args.matrix_format,
                               mpnn_weights=w, mpnn_bf16=1)

    def lstep():
        h = A.amg_setup(rp, ci, va, lopts, stream)
        u = torch.zeros_like(F)
        st, it, rr = A.amg_pcg_solve(h, F, u, args.rtol, 10000)
        info = A.amg_get_info(h)
        A.amg_free(h)
        if st != A.AMG_OK:
            raise RuntimeError(f"learned solve failed: {A.amg_strerror(st)}")
        return u, it, rr, info

    def cstep():
        h = A.amg_setup(rp, ci, va, mopts, stream)
        A.amg_set_damping(h, best)
        u = torch.zeros_like(F)
        st, it, rr = A.amg_pcg_solve(h, F, u, args.rtol, 10000)
        info = A.amg_get_info(h)
        A.amg_free(h)
        if st != A.AMG_OK:
            raise RuntimeError(f"constant-damping solve failed: {A.amg_strerror(st)}")
        return u, it, rr, info

    torch.cuda.nvtx.range_push("learned")
    l_ms, (lu, lit, lrr, linfo) = timed_steps(lstep, args.steps, args.warmup, stream, torch, dist)
    torch.cuda.nvtx.range_pop()
    c_ms, (cu, cit, crr, cinfo) = timed_steps(cstep, args.steps, args.warmup, stream, torch, dist)
    # the fallback rule's choice is what a user gets
    chosen_ms = l_ms if used else c_ms
    err = float(torch.linalg.norm(lu - ref_u) / torch.linalg.norm(ref_u))
    cerr = float(torch.linalg.norm(cu - ref_u) / torch.linalg.norm(ref_u))
    return {"time_to_solution_s": chosen_ms / 1e3, "speedup_vs_fp64": fp64_ms / chosen_ms,
            "speedup_vs_mixed": mixed_ms / chosen_ms, "used": "learned" if used else f"constant omega {best}",
            "network": {"time_to_solution_s": l_ms / 1e3, "iters": lit, "speedup_vs_fp64": fp64_ms / l_ms,
                        "speedup_vs_best_constant": c_ms / l_ms, "final_relres_fp64": lrr,
                        "rel_error_vs_fp64_solution": err, "setup_ms": linfo.setup_ms,
                        "setup_damping_phase_ms": linfo.setup_phase_ms[9], "solve_ms": linfo.solve_ms,
                        "inference_ms_alone": infer_ms, "omega": stats, "iters_fp64_learned": it64},
            "best_constant": {"omega": best, "time_to_solution_s": c_ms / 1e3, "iters": cit,
                              "speedup_vs_fp64": fp64_ms / c_ms, "final_relres_fp64": crr,
                              "rel_error_vs_fp64_solution": cerr, "setup_ms": cinfo.setup_ms,
                              "solve_ms": cinfo.solve_ms},
            "constant_sweep_iters": {str(k): v for k, v in sweep.items()},
            "fallback_rule": {"reference": f"constant omega {best}", "iters_reference": it_best,
                              "iters_learned": it_learned, "learned_kept": bool(used)},
            "training": {"set": "3-D cube p in {2,3,4}, n=16, FP64 hierarchies", "steps": args.train_steps,
                         "probes": 4, "lr": 1e-2, "seconds": train_s,
                         "loss_first": float(hist[0]) if len(hist) else None,
                         "loss_last": float(hist[-1]) if len(hist) else None},
            "precision": "network BF16 weights / FP32 arithmetic; mixed-precision solve as in 'mixed'",
            "timed_step": "network: setup with the network weights (finest-level features, damping cap and network "
                          "on a second stream alongside the coarse-level setup; coarse levels and install at its "
                          "end) + solve + free; constant: setup + amg_set_damping + solve + free"}


def batched_leg(args, A, I, torch, np, stream, dist=None, rank=0, world=1):
    """Batched solves (FP32 V-cycle, FP64 outer FCG(1), rtol as the bench):
    48 uneven 2-D instances as one block-diagonal hierarchy, and one 3-D
    p=3 n=48 system with 16 right-hand sides (SpMM passes), each against the
    same systems solved one by one through amg_setup + amg_pcg_solve.
    Under torchrun the 48 instances are sharded across the ranks by stored
    entries (paper_2511_21268_gb300.dist; no collective on the data path):
    each rank times its share, the line reports the max over ranks."""
    from paper_2511_21268_gb300 import dist as D

    dev = torch.device("cuda", torch.cuda.current_device())
    fp32 = A.amg_opts_default(precision=A.AMG_FP32)
    reps = 3

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    all_probs = I.batch_instances(seed=20251126, count=48)
    share = D.assign_by_nnz([q.nnz for q in all_probs], world)[rank]
    probs = [all_probs[k] for k in share]
    systems = [tuple(torch.from_numpy(a).to(dev) for a in (q.rowptr, q.col, q.val)) for q in probs]
    Fs = [torch.from_numpy(q.F).to(dev) for q in probs]

    def batch_once():
        h = A.amg_setup_batch(systems, fp32, stream)
        Us = [torch.zeros_like(F) for F in Fs]
        st, it, rr = A.amg_pcg_solve_batch(h, Fs, Us, args.rtol, 10000)
        A.amg_free(h)
        assert st == A.AMG_OK
        return it

    def batch_seq():
        its = []
        for (rp, ci, va), F in zip(systems, Fs):
            h = A.amg_setup(rp, ci, va, fp32, stream)
            st, it, _ = A.amg_pcg_solve(h, F, torch.zeros_like(F), args.rtol, 10000)
            A.amg_free(h)
            assert st == A.AMG_OK
            its.append(it)
        return its

    tb, itb = timed(batch_once)
    ts, its = timed(batch_seq)
    tb, ts = max_over_ranks(dist, tb), max_over_ranks(dist, ts)
    q = I.poisson_box_random_rhs(3, 48, 3, seed=16, nrhs=16)
    rp, ci, va = (torch.from_numpy(a).to(dev) for a in (q.rowptr, q.col, q.val))
    Fm = torch.from_numpy(np.ascontiguousarray(q.F.reshape(16, q.n))).to(dev)

    def multi_once():
        h = A.amg_setup(rp, ci, va, fp32, stream)
        st, it, rr = A.amg_pcg_solve_multi(h, Fm, torch.zeros_like(Fm), args.rtol, 10000)
        A.amg_free(h)
        assert st == A.AMG_OK
        return it

    def multi_seq():
        h = A.amg_setup(rp, ci, va, fp32, stream)
        its = []
        for c in range(16):
            st, it, _ = A.amg_pcg_solve(h, Fm[c].contiguous(), torch.zeros(q.n, dtype=torch.float64, device=dev),
                                        args.rtol, 10000)
            assert st == A.AMG_OK
            its.append(it)
        A.amg_free(h)
        return its

    tm, itm = timed(multi_once)
    tq, itq = timed(multi_seq)
    return {"batch48": {"instances": "48 x 2-D, p in {2,3,4}, n in 32..256 (seeded), F = K u, u ~ N(0,1)",
                        "N_total": int(sum(p.n for p in all_probs)), "ms": tb, "ms_one_by_one": ts,
                        "ranks": world, "instances_on_rank0": len(D.assign_by_nnz([q.nnz for q in all_probs],
                                                                                 world)[0]),
                        "speedup": ts / tb, "iters_min_max": [int(min(itb)), int(max(itb))]},
            "rhs16": {"system": "3-D p=3 n=48 (N=117,649), 16 right-hand sides ~ N(0,1)", "ms": tm,
                      "ms_one_by_one": tq, "speedup": tq / tm, "iters_min_max": [int(min(itm)), int(max(itm))]},
            "timed": "setup + solve + free per batch (one-by-one: per system; the 16-RHS baseline shares one setup)"}


def annulus_leg(args, A, I, torch, np, stream, dist):
    """Learned-damping workload: quarter annulus (NURBS arc, radii 1 and 2)
    extruded over z in [0, 1], B-splines p=3, n=64, kappa = exp(g), g a
    seeded Gaussian random field (correlation length 0.2, sigma 1).  The
    network is trained (untimed) on annulus hierarchies with p in {2,3,4},
    n in {16,32}; timed: plain FP64 AMG-PCG vs mixed precision + learned
    damping, each step = setup (+ inference) + solve + free."""
    dev = torch.device("cuda", torch.cuda.current_device())
    t0 = time.perf_counter()
    prob = I.annulus_kappa(64, 3)
    asm_s = time.perf_counter() - t0
    rp, ci, va, F = (torch.from_numpy(a).to(dev) for a in (prob.rowptr, prob.col, prob.val, prob.F))
    train = []  # p in {2,3,4} x n in {16,32} x 4 coefficient fields (seeds 101-104; the workload uses 7)
    for n in (16, 32):
        for pp in (2, 3, 4):
            for ks in (101, 102, 103, 104):
                q = I.annulus_kappa(n, pp, kappa_seed=ks)
                train.append(A.amg_setup(torch.from_numpy(q.rowptr).to(dev), torch.from_numpy(q.col).to(dev),
                                         torch.from_numpy(q.val).to(dev), A.amg_opts_default(), stream))
    w = torch.from_numpy(I.mpnn_init_weights(1).astype(np.float32)).to(dev)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    hist = A.amg_mpnn_train(train, w, args.train_steps, 4, 2000, 1e-2)
    train_s = time.perf_counter() - t1
    for h in train:
        A.amg_free(h)
    o64 = A.amg_opts_default(matrix_format=args.matrix_format)
    omx = A.amg_opts_default(precision=A.AMG_FP32_BF16FINE, matrix_format=args.matrix_format)

    def step(opts, learned):
        if learned:
            opts = A.amg_opts_default(precision=opts.precision, matrix_format=opts.matrix_format, mpnn_weights=w,
                                      mpnn_bf16=1)
        h = A.amg_setup(rp, ci, va, opts, stream)
        u = torch.zeros_like(F)
        st, it, rr = A.amg_pcg_solve(h, F, u, args.rtol, 20000)
        A.amg_free(h)
        if st != A.AMG_OK:
            raise RuntimeError(f"annulus solve failed: {A.amg_strerror(st)}")
        return u, it, rr

    def timed(opts, learned, k):
        for _ in range(2):
            step(opts, learned)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            u, it, rr = step(opts, learned)
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(dist, e0.elapsed_time(e1)) / k, u, it, rr

    k = max(2, min(args.steps, 3))
    t64, u64, it64, rr64 = timed(o64, False, k)
    tml, uml, itml, rrml = timed(omx, True, k)
    h = A.amg_setup(rp, ci, va, omx, stream)
    sweep, best = constant_sweep(A, h, F, args.rtol, torch)
    used, ip, il = A.amg_mpnn_select(h, w, F, args.rtol, 20000, omega_ref=best)
    A.amg_mpnn_apply(h, w, True)
    stats = omega_stats(A, h, torch)
    A.amg_free(h)

    def cstep():
        h = A.amg_setup(rp, ci, va, omx, stream)
        A.amg_set_damping(h, best)
        u = torch.zeros_like(F)
        st, it, rr = A.amg_pcg_solve(h, F, u, args.rtol, 20000)
        A.amg_free(h)
        if st != A.AMG_OK:
            raise RuntimeError(f"annulus constant-damping solve failed: {A.amg_strerror(st)}")
        return it

    tc, itc = timed_steps(cstep, k, 2, stream, torch, dist)
    err = float(torch.linalg.norm(uml - u64) / torch.linalg.norm(u64))
    return {"workload": "quarter annulus x [0,1], NURBS geometry, B-spline p=3 C^2, n=64 (N=274,625, nnz=86,938,307), "
                        "kappa = exp(g), random Fourier features M=256, l=0.2, sigma=1",
            "assembly_s": asm_s, "fp64_time_to_solution_s": t64 / 1e3, "fp64_iters": it64,
            "mixed_learned_time_to_solution_s": tml / 1e3, "mixed_learned_iters": itml,
            "speedup_vs_fp64": t64 / tml, "rel_error_vs_fp64_solution": err, "final_relres_fp64": rrml,
            "best_constant": {"omega": best, "time_to_solution_s": tc / 1e3, "iters": itc,
                              "speedup_vs_fp64": t64 / tc},
            "network_vs_best_constant": tc / tml, "omega": stats,
            "constant_sweep_iters": {str(kk): v for kk, v in sweep.items()},
            "fallback_rule": {"reference": f"constant omega {best}", "learned_kept": bool(used),
                              "iters_reference": ip, "iters_learned": il},
            "training": {"set": "annulus hierarchies p in {2,3,4}, n in {16,32}, 4 coefficient seeds each (FP64)",
                         "steps": args.train_steps,
                         "probes": 4, "lr": 1e-2, "seconds": train_s,
                         "loss_first": float(hist[0]) if len(hist) else None,
                         "loss_last": float(hist[-1]) if len(hist) else None},
            "steps": k}


def smoothing_leg(args, A, I, torch, np, stream, dist, rp, ci, va, F, fp64_ms):
    """Prolongator smoothing on the bench workload (Sec. 3.1 "Variants"):
    level 0's prolongator smoothed with the constant theta = 4/3 and with the
    network's per-row theta (second head, trained on two-level 3-D cubes
    p in {2,3,4}, n = 8, jointly with the damping hierarchies of the learned
    leg), against the tentative prolongator; mixed precision, plain
    l1-Jacobi smoother in all three, each step = setup + solve + free."""
    dev = F.device
    dmp, sm = [], []
    for pp in (2, 3, 4):
        q = I.poisson_box(3, 8, pp)
        a = (torch.from_numpy(q.rowptr).to(dev), torch.from_numpy(q.col).to(dev), torch.from_numpy(q.val).to(dev))
        dmp.append(A.amg_setup(*a, A.amg_opts_default(), stream))
        sm.append(A.amg_setup(*a, A.amg_opts_default(smooth_levels=1, max_levels=2, coarse_max=20), stream))
    w = torch.from_numpy(I.mpnn_init_weights(1).astype(np.float32)).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = A.amg_mpnn_train(dmp + sm, w, 40, 4, 1000, 1e-2)
    train_s = time.perf_counter() - t0
    for h in dmp + sm:
        A.amg_free(h)
    base = dict(precision=A.AMG_FP32_BF16FINE, matrix_format=args.matrix_format)
    legs = {"tentative": A.amg_opts_default(**base),
            "theta_4/3": A.amg_opts_default(smooth_levels=1, **base),
            "theta_learned": A.amg_opts_default(smooth_levels=1, mpnn_weights=w, mpnn_bf16=1, **base)}
    out = {}
    k = max(2, min(args.steps, 3))
    for name, o in legs.items():
        def st(o=o, learned=name == "theta_learned"):
            h = A.amg_setup(rp, ci, va, o, stream)
            if learned:
                A.amg_set_damping(h, 1.0)  # compare the prolongators with the plain smoother
            u = torch.zeros_like(F)
            s_, it, rr = A.amg_pcg_solve(h, F, u, args.rtol, 10000)
            info = A.amg_get_info(h)
            A.amg_free(h)
            if s_ != A.AMG_OK:
                raise RuntimeError(f"smoothing leg {name}: {A.amg_strerror(s_)}")
            return it, info
        ms, (it, info) = timed_steps(st, k, 1, stream, torch, dist)
        out[name] = {"time_to_solution_s": ms / 1e3, "iters": it, "opc": info.opc, "setup_ms": info.setup_ms,
                     "solve_ms": info.solve_ms, "smoothing_phase_ms": info.setup_phase_ms[10],
                     "p0_nnz": int(info.p_nnz[0]), "speedup_vs_fp64": fp64_ms / ms}
    return {"legs": out, "steps": k, "training": {"steps": 40, "seconds": train_s,
                                                   "loss_first": float(hist[0]), "loss_last": float(hist[-1])},
            "note": "theta = 4/3 is the classical 4 / (3 rho(D^-1 K)) with rho <= 1 from the l1 diagonal"}


def paper_config_leg(args, A, I, torch, np, stream, dist, rp, ci, va, F, fp64_ms):
    """The paper's solver configuration of Sec. 5 on the bench workload:
    aggregates of up to 8 (three matching passes), smoothed prolongators on
    every level (theta = 4/3), 4th-kind Chebyshev l1-Jacobi of degree 8 (p =
    3), coarse CG to 1e-4 or 30 iterations, flexible CG; FP64 and mixed
    precision, rtol as the bench; each step = setup + solve + free."""
    out = {}
    k = max(2, min(args.steps, 3))
    for name, prec in (("fp64", A.AMG_FP64), ("mixed", A.AMG_FP32_BF16FINE)):
        o = A.amg_opts_default(match_passes=3, smooth_levels=-1, cheb_degree=8, coarse_solver=1, flexible=1,
                               precision=prec, matrix_format=args.matrix_format)

        def st(o=o):
            h = A.amg_setup(rp, ci, va, o, stream)
            u = torch.zeros_like(F)
            s_, it, rr = A.amg_pcg_solve(h, F, u, args.rtol, 10000)
            info = A.amg_get_info(h)
            A.amg_free(h)
            if s_ != A.AMG_OK:
                raise RuntimeError(f"paper configuration {name}: {A.amg_strerror(s_)}")
            return it, rr, info
        ms, (it, rr, info) = timed_steps(st, k, 1, stream, torch, dist)
        out[name] = {"time_to_solution_s": ms / 1e3, "iters": it, "final_relres_fp64": rr, "opc": info.opc,
                     "levels": [int(info.n[l]) for l in range(info.levels)], "setup_ms": info.setup_ms,
                     "smoothing_phase_ms": info.setup_phase_ms[10], "solve_ms": info.solve_ms,
                     "speedup_vs_plain_fp64": fp64_ms / ms}
    return {"legs": out, "steps": k, "settings": "m=3, smoothed P on every level (theta 4/3), Chebyshev degree 8, "
                                                 "coarse CG 1e-4 / 30 its, FCG; rtol as the bench (the paper: 1e-6)"}


PAPER_HEADLINE = {"k": 96, "p": 3, "unknowns": 941094, "solve_s": 1.566, "iters": 11,
                  "hardware": "1x NVIDIA A30 (24 GB HBM2), CUDA 12.9, FP64"}


def paper_headline_leg(args, A, I, torch, np, stream, dist):
    """The paper's headline system: the mixed Dirichlet/Neumann cube of
    Sec. 5 (F2) with k = 96 elements per direction, p = 3 (941,094
    unknowns), in the paper's solver configuration (as paper_config_leg) at
    its rtol 1e-6.  The paper reports the solve phase alone (1.566 s, FP64,
    one A30: another machine, context only); here the solve and the setup are
    reported separately, each step = setup + solve + free."""
    dev = torch.device("cuda", torch.cuda.current_device())
    t0 = time.perf_counter()
    prob = I.cube_mixed_bc(PAPER_HEADLINE["k"], PAPER_HEADLINE["p"])
    gen_s = time.perf_counter() - t0
    rp, ci, va, F = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (prob.rowptr, prob.col, prob.val,
                                                                                  prob.F))
    out = {}
    k = 2
    for name, prec in (("fp64", A.AMG_FP64), ("mixed", A.AMG_FP32_BF16FINE)):
        o = A.amg_opts_default(match_passes=3, smooth_levels=-1, cheb_degree=8, coarse_solver=1, flexible=1,
                               precision=prec, matrix_format=args.matrix_format)

        def st(o=o):
            h = A.amg_setup(rp, ci, va, o, stream)
            u = torch.zeros_like(F)
            s_, it, rr = A.amg_pcg_solve(h, F, u, 1e-6, 10000)
            info = A.amg_get_info(h)
            A.amg_free(h)
            if s_ != A.AMG_OK:
                raise RuntimeError(f"paper headline {name}: {A.amg_strerror(s_)}")
            return it, rr, info, u
        ms, (it, rr, info, u) = timed_steps(st, k, 1, stream, torch, dist)
        err = I.cube_mixed_bc_l2_error(prob, u.cpu().numpy())
        out[name] = {"time_to_solution_s": ms / 1e3, "solve_s": info.solve_ms / 1e3, "setup_s": info.setup_ms / 1e3,
                     "smoothing_phase_s": info.setup_phase_ms[10] / 1e3, "iters": it, "final_relres_fp64": rr,
                     "opc": info.opc, "levels": [int(info.n[l]) for l in range(info.levels)],
                     "l2_error_vs_exact": err,
                     "solve_vs_paper": PAPER_HEADLINE["solve_s"] / (info.solve_ms / 1e3)}
    return {"legs": out, "steps": k, "unknowns": prob.n, "nnz": prob.nnz, "generation_s": gen_s,
            "paper": PAPER_HEADLINE,
            "settings": "m=3, smoothed P on every level (theta 4/3), Chebyshev degree 8, coarse CG 1e-4 / 30 its, "
                        "FCG, rtol 1e-6 (the paper's)"}


def assembly_leg(args, A, I, torch, np, stream, dist, fp64_peak):
    """IgA assembly by sum factorization on the GPU (amg_iga_assemble) of the
    learned-damping workload's system: quarter annulus, p = 3, n = 64, kappa
    with 256 random Fourier features; against the input generator's element
    loop on the host cores (context).  Roofline: the FP64 multiply-adds of
    the quadrature sums (counted by the library) against the measured FP64
    FMA rate."""
    import math
    n, p = 64, 3
    kk = I.ANNULUS_KAPPA
    M, ell, sigma, seed = kk["M"], kk["ell"], kk["sigma"], 7
    dev = torch.device("cuda", torch.cuda.current_device())
    om = torch.from_numpy(I.rng_normal(seed, 3 * M).reshape(M, 3) / ell).to(dev)
    ph = torch.from_numpy(I.rng_u01(seed + 1, M) * 2 * math.pi).to(dev)
    P, keep = A._iga_patch(n, p, geometry=A.AMG_GEOM_ANNULUS, kappa=(om, ph, sigma))
    N, Z = A.amg_iga_size(P)
    rp = torch.empty(N + 1, dtype=torch.int64, device=dev)
    ci = torch.empty(Z, dtype=torch.int32, device=dev)
    va = torch.empty(Z, dtype=torch.float64, device=dev)
    F = torch.empty(N, dtype=torch.float64, device=dev)
    flops = [0.0]

    def st():
        flops[0] = A.amg_iga_assemble(P, rp, ci, va, F, stream)
    k = 3
    ms, _ = timed_steps(st, k, 2, stream, torch, dist)
    t0 = time.perf_counter()
    prob = I.annulus_kappa(n, p)
    host_s = time.perf_counter() - t0
    rel = float(np.abs(prob.val - va.cpu().numpy()).max() / np.abs(prob.val).max())
    tf = flops[0] / (ms * 1e-3) / 1e12
    del keep
    return {"ms": ms, "steps": k, "unknowns": N, "nnz": Z, "flops": flops[0],
            "roofline": {"bound": "alu", "achieved": tf, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": tf / fp64_peak if fp64_peak else None,
                         "peak_kind": "measured FP64 FMA rate (amg_dfma_probe)"},
            "host_element_loop_s": host_s, "host_threads": os.cpu_count(),
            "speedup_vs_host": host_s / (ms * 1e-3), "max_rel_diff_vs_host": rel}


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = env_rank()
    dist = init_dist(world)
    torch.cuda.set_device(local)
    from paper_2511_21268_gb300 import amg as A
    from paper_2511_21268_gb300 import inputs as I

    A.lib()  # build/load the CUDA library before anything is timed
    prob = I.poisson_box(3, args.n, args.p)
    dev = torch.device("cuda", local)
    rp = torch.from_numpy(prob.rowptr).to(dev)
    ci = torch.from_numpy(prob.col).to(dev)
    va = torch.from_numpy(prob.val).to(dev)
    F = torch.from_numpy(prob.F).to(dev)
    stream = torch.cuda.Stream(device=dev)
    prec = {"fp64": A.AMG_FP64, "fp32": A.AMG_FP32, "bf16": A.AMG_FP32_BF16FINE}[args.precision]
    opts = A.amg_opts_default(precision=prec, matrix_format=args.matrix_format)

    def step(profile=False):
        h = A.amg_setup(rp, ci, va, opts, stream)
        if profile:
            A.amg_profile_kernels(h, True)
        u = torch.zeros_like(F)
        st, it, rr = A.amg_pcg_solve(h, F, u, args.rtol, 10000)
        info = A.amg_get_info(h)
        kt = A.amg_kernel_times(h) if profile else None
        A.amg_free(h)
        if st != A.AMG_OK:
            raise RuntimeError(f"solve failed: {A.amg_strerror(st)}")
        return it, rr, info, kt

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        uuid = None
        try:
            uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
        except Exception:
            pass
        clocks = ClockSampler(uuid) if (rank == 0 and not args.no_clocks) else None
        barrier(dist)
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
            time.sleep(0.3)
        torch.cuda.nvtx.range_push("timed")
        l0 = A.amg_kernel_launches()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ms_sum = np.zeros(3)
        cnt_sum = np.zeros(3, np.int64)
        kbytes = None
        infos = []
        for _ in range(args.steps):
            it, rr, info, _ = step()
            infos.append((it, rr, info))
        e1.record(stream)
        torch.cuda.synchronize()
        launches = A.amg_kernel_launches() - l0
        torch.cuda.nvtx.range_pop()
        # per-kernel durations: event-record nodes around the finest-level
        # passes inside the iteration graph, in as many profiled steps run
        # right after the timed ones (their nodes stay out of the timed steps)
        for _ in range(args.steps):
            _, _, _, kt = step(profile=True)
            ms_sum += kt[0]
            cnt_sum += kt[1]
            kbytes = kt[2]
        torch.cuda.synchronize()
        clk = clocks.stop() if clocks else None
        barrier(dist)
        elapsed_ms = max_over_ranks(dist, e0.elapsed_time(e1))
        ms_per_step = elapsed_ms / args.steps
        it, rr, info = infos[-1]

        # the FP64 rate that bounds the FP64 passes, measured on this GPU
        fp64_meas, fp64_clk, fp64_variants = measure_fp64_rate(A, torch, stream, uuid)

        # V-cycle alone (standalone applications, events on the same stream)
        h = A.amg_setup(rp, ci, va, opts, stream)
        vinfo = A.amg_get_info(h)
        r = torch.randn(prob.n, dtype=torch.float64, device=dev)
        z = torch.empty_like(r)
        for _ in range(3):
            A.amg_vcycle_apply(h, r, z)
        v0 = torch.cuda.Event(enable_timing=True)
        v1 = torch.cuda.Event(enable_timing=True)
        v0.record(stream)
        nv = 20
        for _ in range(nv):
            A.amg_vcycle_apply(h, r, z)
        v1.record(stream)
        torch.cuda.synchronize()
        vcycle_ms = v0.elapsed_time(v1) / nv
        A.amg_free(h)

        # end to end through the public API with pinned host buffers
        e2e = None
        if not args.no_e2e:
            hrp = torch.from_numpy(prob.rowptr).pin_memory()
            hci = torch.from_numpy(prob.col).pin_memory()
            hva = torch.from_numpy(prob.val).pin_memory()
            hF = torch.from_numpy(prob.F).pin_memory()
            hu = torch.zeros(prob.n, dtype=torch.float64).pin_memory()
            e2e_steps = max(3, min(args.steps, 5))
            ts = []
            for k in range(e2e_steps + 1):
                hu.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                h = A.amg_setup(hrp, hci, hva, opts, stream)
                st, it2, rr2 = A.amg_pcg_solve(h, hF, hu, args.rtol, 10000)
                A.amg_free(h)
                torch.cuda.synchronize()
                if k > 0:
                    ts.append(time.perf_counter() - t0)
                assert st == A.AMG_OK
            e2e_s = max_over_ranks(dist, statistics.median(ts))
            h2d = prob.rowptr.nbytes + prob.col.nbytes + prob.val.nbytes + prob.F.nbytes + prob.n * 8
            e2e = {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(prob.n * 8),
                   "steps": e2e_steps, "host_buffers": "pinned"}

        # mixed precision on the same workload (FP32 V-cycle with BF16 finest values,
        # FP32 outer SpMV, FP64 flexible-CG recurrences and true-residual replacement)
        mixed = None
        if not args.no_mixed:
            mopts = A.amg_opts_default(precision=A.AMG_FP32_BF16FINE, matrix_format=args.matrix_format)
            ref_u = torch.zeros_like(F)
            h = A.amg_setup(rp, ci, va, opts, stream)
            A.amg_pcg_solve(h, F, ref_u, args.rtol, 10000)
            A.amg_free(h)

            def mstep(profile=False):
                h = A.amg_setup(rp, ci, va, mopts, stream)
                if profile:
                    A.amg_profile_kernels(h, True)
                u = torch.zeros_like(F)
                st, it, rr = A.amg_pcg_solve(h, F, u, args.rtol, 10000)
                info = A.amg_get_info(h)
                kt = A.amg_kernel_times(h) if profile else None
                A.amg_free(h)
                if st != A.AMG_OK:
                    raise RuntimeError(f"mixed solve failed: {A.amg_strerror(st)}")
                return u, it, rr, info, kt

            for _ in range(args.warmup):
                mstep()
            torch.cuda.synchronize()
            barrier(dist)
            m0 = torch.cuda.Event(enable_timing=True)
            m1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.nvtx.range_push("mixed")
            m0.record(stream)
            mms = np.zeros(3)
            mcnt = np.zeros(3, np.int64)
            for _ in range(args.steps):
                mu, mit, mrr, minfo, _ = mstep()
            m1.record(stream)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
            for _ in range(args.steps):  # per-kernel durations, as for the FP64 leg
                _, _, _, _, mkt = mstep(profile=True)
                mms += mkt[0]
                mcnt += mkt[1]
            torch.cuda.synchronize()
            m_ms = max_over_ranks(dist, m0.elapsed_time(m1)) / args.steps
            err = float(torch.linalg.norm(mu - ref_u) / torch.linalg.norm(ref_u))
            mavg = mms / np.maximum(mcnt, 1)
            mkind = int(minfo.staged_passes)
            mnames = MIXED_KERNEL_NAMES[mkind]
            mk = {name: {"bytes_per_launch": mkt[2][q], "avg_ms": mavg[q], "launches": int(mcnt[q]),
                         "achieved_gbs": mkt[2][q] / (mavg[q] * 1e-3) / 1e9 if mavg[q] > 0 else None}
                  for q, name in enumerate(mnames)}
            mdom = max(mk, key=lambda k: mk[k]["avg_ms"] * mk[k]["launches"])
            mixed = {"time_to_solution_s": m_ms / 1e3, "speedup_vs_fp64": ms_per_step / m_ms, "iters": mit,
                     "final_relres_fp64": mrr, "rel_error_vs_fp64_solution": err, "setup_ms": minfo.setup_ms,
                     "solve_ms": minfo.solve_ms, "precision": "fp32 V-cycle, bf16 finest values, fp32 outer SpMV, "
                     "fp64 FCG(1) recurrences, fp64 true-residual replacement every 20 iterations",
                     "iter_gbps": minfo.iter_bytes * mit / (minfo.solve_ms * 1e-3) / 1e9,
                     "roofline": {"bound": "hbm", "kernel": mdom, "achieved": mk[mdom]["achieved_gbs"],
                                  "unit": "GB/s", "traffic": None,
                                  "tkey": ["pq", "resid", "up0"][mnames.index(mdom)],
                                  "bytes_per_launch": mk[mdom]["bytes_per_launch"],
                                  "avg_launch_ms": mk[mdom]["avg_ms"], "all": mk},
                     "staged_passes": {"kind": ["row-group kernels", "slabs, lane per run",
                                                "sliced slabs, lane per row"][mkind],
                                       "value_slots": int(minfo.staged_slots),
                                       "ring_buffers_bf16_fp32": [int(x) for x in minfo.staged_buffers],
                                       "window_bytes": int(minfo.staged_window_bytes)}}

        # learned damping on top of mixed precision: the network is trained
        # (untimed) on small hierarchies of the same family, then each timed
        # step is setup + network inference (BF16 weights) + solve + free
        learned = None
        if not args.no_learned and not args.no_mixed:
            learned = learned_leg(args, A, I, torch, np, stream, dist, rp, ci, va, F, ref_u, ms_per_step, m_ms)

        smoothing = None
        if not args.no_smoothing:
            smoothing = smoothing_leg(args, A, I, torch, np, stream, dist, rp, ci, va, F, ms_per_step)
        paper_cfg = None
        if not args.no_paper_config:
            paper_cfg = paper_config_leg(args, A, I, torch, np, stream, dist, rp, ci, va, F, ms_per_step)

        headline = None
        if not args.no_paper_headline:
            headline = paper_headline_leg(args, A, I, torch, np, stream, dist)
        assembly = None
        if not args.no_assembly:
            assembly = assembly_leg(args, A, I, torch, np, stream, dist, fp64_meas)

        batched = None
        if not args.no_batched:
            batched = batched_leg(args, A, I, torch, np, stream, dist, rank, world)
        annulus = None
        if not args.no_annulus:
            annulus = annulus_leg(args, A, I, torch, np, stream, dist)

    peak, peak_kind = measured_peaks()
    avg_ms = ms_sum / np.maximum(cnt_sum, 1)
    per_kernel = {}
    fkind = 3 if int(info.staged_passes) == 3 else 0
    KERNEL_NAMES = FP64_KERNEL_NAMES[fkind]
    for q, name in enumerate(KERNEL_NAMES):
        gbs = kbytes[q] / (avg_ms[q] * 1e-3) / 1e9 if avg_ms[q] > 0 else None
        per_kernel[name] = {"bytes_per_launch": kbytes[q], "avg_ms": avg_ms[q], "launches": int(cnt_sum[q]),
                            "achieved_gbs": gbs}
    dom = int(np.argmax(ms_sum))
    traffic = committed_traffic(PROFILE_SUMMARY, FP64_SOURCES[fkind])
    tkey = ["spmv_pq", "resid", "up0"][dom]
    # The FP64 finest pass issues one DFMA per stored entry; on GB300 that is the binding limit (the FP64
    # pipe is far busier than DRAM), so its roofline is the FP64 rate derived from unit counts and clock.
    fpk = fp64_meas
    flops_tf = 2.0 * prob.nnz / (avg_ms[dom] * 1e-3) / 1e12 if avg_ms[dom] > 0 else 0.0
    roof = {"bound": "alu", "kernel": KERNEL_NAMES[dom], "achieved": flops_tf, "peak": fpk, "unit": "TFLOP/s",
            "frac": flops_tf / fpk, "traffic": (traffic or {}).get(tkey),
            "peak_kind": "measured on this GPU: amg_dfma_probe, the fastest of its variants (4 independent "
                         "FP64 FMA chains with their own operands per thread, 512 threads per SM, reaches "
                         "the unit-count rate; shared operands level off at 0.84 of it), ~2 s, CUDA events",
            "peak_variants_tflops": fp64_variants,
            "peak_clocks": fp64_clk, "peak_derived": fp64_peak_tflops(),
            "frac_of_derived": flops_tf / fp64_peak_tflops(),
            "flops_per_launch": 2.0 * prob.nnz, "bytes_per_launch": kbytes[dom], "avg_launch_ms": avg_ms[dom],
            "hbm": {"achieved_gbs": per_kernel[KERNEL_NAMES[dom]]["achieved_gbs"], "peak_gbs": peak,
                    "frac": (per_kernel[KERNEL_NAMES[dom]]["achieved_gbs"] or 0.0) / peak,
                    "peak_kind": f"{peak_kind} (hbm_gbs, STREAM-style copy)"},
            "all": per_kernel}

    line = {"metric": METRIC, "value": ms_per_step / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": args.n, "p": args.p, "N": prob.n, "nnz": prob.nnz,
                       "rtol": args.rtol, "precision": "fp64", "l2": "inputs larger than L2 (matrix 1.04 GB)",
                       "matrix_format": ["csr", "run-encoded finest level",
                                         "run-encoded + sliced finest-level passes"][args.matrix_format],
                       "fp64_passes": "sliced slabs, FP64 values, a warp per slab" if fkind == 3
                       else "row-group kernels",
                       "parallelism": f"replicas x{world}"},
            "iters": it, "final_relres": rr, "setup_ms": info.setup_ms, "solve_ms": info.solve_ms,
            "setup_phase_ms": dict(zip(["copy+checks", "l1+testvec+diag", "edge_weights", "matching",
                                        "aggregation", "galerkin", "composite+members", "coarse_inverse",
                                        "workspace"], [round(info.setup_phase_ms[k], 3) for k in range(9)])),
            "levels": [int(info.n[l]) for l in range(info.levels)], "opc": info.opc,
            "iter_gbps": info.iter_bytes * it / (info.solve_ms * 1e-3) / 1e9 if info.solve_ms > 0 else None,
            "vcycle_ms": vcycle_ms, "vcycle_gbps": vinfo.vcycle_bytes / (vcycle_ms * 1e-3) / 1e9,
            "throughput_systems_per_s": world * args.steps / (elapsed_ms * 1e-3),
            "roofline": roof, "e2e": e2e, "clocks": clk, "gpu_launches": int(launches), "mixed": mixed,
            "kernel_timing": "CUDA event-record nodes on the library's stream around each finest-level pass "
                             "inside the iteration graph, over as many profiled steps run right after the "
                             "timed (unprofiled) steps",
            "learned": learned, "batched": batched, "annulus_learned": annulus,
            "prolongator_smoothing": smoothing, "paper_configuration": paper_cfg,
            "paper_headline_cube_k96": headline, "assembly": assembly}
    if mixed is not None:
        mixed["roofline"]["peak"] = peak
        mixed["roofline"]["frac"] = (mixed["roofline"]["achieved"] or 0.0) / peak
        kind = next((k for k, v in MIXED_KERNEL_NAMES.items() if mixed["roofline"]["kernel"] in v), 0)
        st = committed_traffic(STREAM_SUMMARY, STAGED_SOURCES[kind]) if kind in STAGED_SOURCES else None
        if st:
            mixed["roofline"]["traffic"] = st.get(mixed["roofline"]["tkey"])
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(prob, it, args.rtol)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
