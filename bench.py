"""Benchmark: Hutch++ entropy estimates per second on a Barabasi-Albert graph.

Workload (one "step" = one full entropy estimate, every hot-path row):
  Barabasi-Albert n = 1,000,000, m = 4 (seed 3), rho = L / tr(L) as an implicit
  FP32 pattern Laplacian, nodes relabelled by descending degree; Hutch++ with
  N_r = 100 sketch columns and N_H = 100 Hutchinson vectors (300 Lanczos runs
  of 60 steps: 100 for f(A) Omega, 100 for Q, 100 for (I - QQ^T) G), FP32
  vectors with FP64 alpha/beta, tridiagonal eigensolve and quadrature.

Output: one JSON line (rank 0).  ``value`` is whole-job estimates/s with the
matrix resident on the device; ``e2e`` repeats the measurement through the C
ABI from host CSR buffers (matrix upload, relabelling and schedule included);
``roofline`` is the Lanczos step (SpMM) kernel's algorithmic HBM bandwidth
timed live with CUDA events on the library's stream; ``cpu_baseline`` times
the FP64 CPU oracle on a bounded sample of the same workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_NODES, BA_M, GRAPH_SEED = 1_000_000, 4, 3
N_SKETCH, N_HUTCH, M_STEPS = 100, 100, 60
METRIC = "entropy estimates/sec (Hutch++ N_r=100 N_H=100, 60 Lanczos steps, BA n=1e6 m=4, rel err vs FP64 <= 1e-4)"
UNIT = "estimates/s"
WORKLOAD = "BA n=1e6 m=4 (seed 3), rho=L/tr(L) FP32 implicit Laplacian, Hutch++ 300 matvec-equivalents, block 100, m=60"


def workload_name(n):
    """The headline workload's name, with the graph size when --n changes it."""
    return WORKLOAD if n == N_NODES else WORKLOAD.replace("BA n=1e6", f"BA n={n}")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-check", action="store_true")
    ap.add_argument("--n", type=int, default=N_NODES, help="graph size (default: the workload's 1e6)")
    ap.add_argument("--estimator", choices=["hutchpp", "hutchinson"], default="hutchpp",
                    help="hutchinson: one block of --vectors probes (small-memory case for profiling)")
    ap.add_argument("--vectors", type=int, default=112)
    ap.add_argument("--reorder", choices=["degree", "rcm", "none"], default="degree",
                    help="node relabelling of the headline matrix (default: descending degree)")
    ap.add_argument("--schedule", default="",
                    help="panel,item_nnz,step_variant[,interleave[,items_per_warp]] (skips the autotuner)")
    ap.add_argument("--reorth", choices=["none", "partial", "full"], default="none",
                    help="Lanczos reorthogonalisation of the FP32 estimate (partial: Simon's omega recurrence; "
                         "full: classical Gram-Schmidt twice at every step)")
    ap.add_argument("--workload", choices=["c2", "c1", "c3", "c4", "c5", "c6", "c7"], default="c2",
                    help="c2 = the headline workload; c1/c3/c4/c5/c6/c7 print measurement lines of the other configs")
    ap.add_argument("--requests", type=int, default=2000, help="c5: number of queries")
    ap.add_argument("--rate", type=float, default=200.0, help="c5: Poisson arrival rate (queries/s)")
    ap.add_argument("--at-once", action="store_true",
                    help="c5: every query arrives at the start (a saturated server, for profiling)")
    ap.add_argument("--fp64-limit-s", type=float, default=600.0,
                    help="c5: wall-time limit of the FP64 one-at-a-time arm (it serves a prefix of the queries)")
    ap.add_argument("--scaling-exponents", default="10,12,14,16,18,20", help="c7: n = 2^e for these e")
    ap.add_argument("--scaling-runs", type=int, default=10, help="c7: seeds averaged for the stochastic estimator")
    ap.add_argument("--serve-krylov-tol", type=float, default=-1.0,
                    help="c5: Krylov tolerance of the served blocks (< 0: half the query's accuracy, Section 5.2; "
                         "0: fixed 40 steps)")
    ap.add_argument("--serve-check", type=int, default=3, help="c5: Lanczos steps between Krylov-error checks")
    ap.add_argument("--serve-sketch", type=int, default=10,
                    help="c5/c7: Lanczos steps of each query's 4-column sketch f(A) Omega (0: 40)")
    ap.add_argument("--ba-max-colors", type=int, default=10000,
                    help="c7: BA probing is not run above a size whose colouring needed more colours")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.lines:
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_digest():
    """Digest of the step kernel's source: the k_step template and its
    launcher, the shared device header and the StepParams layout."""
    csrc = os.path.join(ROOT, "paper_2212_09642_gb300", "csrc")
    with open(os.path.join(csrc, "kernels_lanczos.cu")) as fh:
        src = fh.read()
    i = src.index("template <typename T, int KS, bool VALUED, int MINB, int UNR, bool STREAM, bool STAGE")
    j = src.index("// ------------", i)
    k = src.index("cudaError_t launch_step(")
    h = hashlib.sha256()
    h.update(src[i:j].encode())
    h.update(src[k:src.index("\n}\n", k)].encode())
    with open(os.path.join(csrc, "common.cuh"), "rb") as fh:
        h.update(fh.read())
    with open(os.path.join(csrc, "kernels.h")) as fh:
        hdr = fh.read()
    i = hdr.index("struct StepParams")
    h.update(hdr[i:hdr.index("};", i) + 2].encode())
    return h.hexdigest()[:16]


def recorded_traffic():
    """Per-launch DRAM bytes of the step kernel from the committed ncu summary,
    if it was taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    try:
        with open(p) as fh:
            rec = json.load(fh)
        if rec.get("source_digest") == kernel_digest():
            return float(rec["dram_bytes_per_launch_full_size"])
    except (OSError, KeyError, ValueError):
        pass
    return None


def make_graph(n):
    from paper_2212_09642_gb300 import graphs
    return graphs.barabasi_albert(n, BA_M, GRAPH_SEED)


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample of the same workload)

def oracle_sample(g, columns=1, seed=7):
    """Time the FP64 oracle on `columns` sketch matvecs and `columns`
    quadratic forms of the workload plus one orthonormalisation and projection
    of n x 100 blocks; return the extrapolated seconds per full estimate and
    the record of what was measured."""
    import numpy as np
    from oracle import density, estimators, krylov, rng

    A, _ = density.density_matrix(g)
    nA = density.gershgorin_norm(A)
    X = rng.rademacher(seed, g.n, 0, columns)
    t_all = time.perf_counter()
    t0 = time.perf_counter()
    for j in range(columns):
        krylov.lanczos_fmatvec(A, X[:, j], M_STEPS, reorth="none", norm_A=nA)
    t_f = (time.perf_counter() - t0) / columns
    t0 = time.perf_counter()
    for j in range(columns):
        krylov.lanczos_quadform(A, X[:, j], M_STEPS, reorth="none", norm_A=nA)
    t_q = (time.perf_counter() - t0) / columns
    Y = np.random.default_rng(0).standard_normal((g.n, N_SKETCH))
    t0 = time.perf_counter()
    Q = estimators.orthonormal_range(Y)
    G = rng.rademacher(seed, g.n, N_SKETCH, N_HUTCH)
    G - Q @ (Q.T @ G)
    t_o = time.perf_counter() - t0
    # context: one scipy sparse product with a 16-column block (one thread)
    X16 = rng.rademacher(seed, g.n, 0, 16)
    t0 = time.perf_counter()
    A @ X16
    t_s = time.perf_counter() - t0
    spmm_bytes = 4.0 * (g.n + 1) + 12.0 * A.nnz + 2.0 * g.n * 16 * 8
    measured = time.perf_counter() - t_all
    runs = N_SKETCH + N_SKETCH + N_HUTCH
    total = N_SKETCH * t_f + (N_SKETCH + N_HUTCH) * t_q + t_o
    rec = dict(extrapolated=True, sampled_krylov_runs=2 * columns, krylov_runs_per_estimate=runs,
               scale_factor=total / measured if measured > 0 else None, measured_seconds=measured,
               t_fmatvec_s=t_f, t_quadform_s=t_q, t_orth_s=t_o,
               threads={"krylov": 1, "orthonormalisation": blas_threads()},
               scipy_spmm_16_columns={"seconds": t_s, "algorithmic_gbs": spmm_bytes / t_s / 1e9 if t_s > 0 else None,
                                      "threads": 1, "counted_in_value": False})
    return total, rec


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def blas_threads():
    """Threads the oracle's dense BLAS calls may use (OpenBLAS / OpenMP
    environment, else the library default of one per core)."""
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        v = os.environ.get(var)
        if v and v.isdigit():
            return int(v)
    return cpu_cores()


def _krylov_worker(job):
    """One spawned process: build the workload's density matrix, wait for the
    other workers, time `runs` FP64 Lanczos quadratures (SciPy, one thread)."""
    n, runs, seed, barrier = job
    sys.path.insert(0, ROOT)
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    from oracle import density, krylov, rng
    g = make_graph(n)
    A, _ = density.density_matrix(g)
    nA = density.gershgorin_norm(A)
    X = rng.rademacher(seed, g.n, 0, runs)
    barrier.wait()
    t0 = time.perf_counter()
    for j in range(runs):
        krylov.lanczos_quadform(A, X[:, j], M_STEPS, reorth="none", norm_A=nA)
    return time.perf_counter() - t0


def oracle_all_cores(n, t_orth, runs_per_proc=1):
    """The same Krylov runs spread over the host cores, one spawned process
    per core; returns the extrapolated estimates/s and its record."""
    import multiprocessing as mp
    procs = cpu_cores()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    barrier = mgr.Barrier(procs)
    t0 = time.perf_counter()
    with ctx.Pool(procs) as pool:
        el = pool.map(_krylov_worker, [(n, runs_per_proc, 300 + i, barrier) for i in range(procs)])
    wall = time.perf_counter() - t0
    mgr.shutdown()
    runs = N_SKETCH + N_SKETCH + N_HUTCH
    per_run = max(el) / (procs * runs_per_proc)  # seconds per Krylov run at full occupancy
    t_est = runs * per_run + t_orth
    return 1.0 / t_est, dict(extrapolated=True, processes=procs, sampled_krylov_runs=procs * runs_per_proc,
                             krylov_seconds_max=max(el), wall_seconds=wall,
                             seconds_per_estimate=t_est, orthonormalisation_from_single_thread_sample=True)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    g = make_graph(args.n)
    t_run = time.perf_counter()
    for _ in range(args.warmup):
        oracle_sample(g, columns=1)
    times = []
    for k in range(args.steps):
        t, parts = oracle_sample(g, columns=1, seed=100 + k)
        times.append(t)
    per = sum(times) / len(times)
    value = 1.0 / per
    rec = dict(parts)
    rec["measured_seconds"] = time.perf_counter() - t_run
    rec["note"] = ("each step times 1 sketch matvec + 1 quadratic form + the n x 100 orthonormalisation and "
                   "scales them to one estimate (300 Krylov runs); measured_seconds is the whole run")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(g.n), "n": g.n, "nnz": g.nnz},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "per step: 1 sketch matvec + 1 quadratic form (FP64 scipy Lanczos, 60 steps, "
                                   "one thread) + one n x 100 orthonormalisation/projection (BLAS threads), "
                                   "scaled to 100 + 200 Krylov runs", **rec},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------

def oracle_c1_baseline(g):
    """The whole C1 estimate by the oracle on the host (no extrapolation):
    FP64 scipy Lanczos with full reorthogonalisation, 100 probes x 50 steps."""
    from oracle import density, estimators
    A, _ = density.density_matrix(g)
    estimators.hutchinson(A, 2, 50, 2, reorth="full")  # warm-up
    t0 = time.perf_counter()
    est, _ = estimators.hutchinson(A, 100, 50, 2, reorth="full")
    t = time.perf_counter() - t0
    return {"value": 1.0 / t, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
            "sample": "the whole estimate: 100 Rademacher probes x 50 FP64 Lanczos steps with full "
                      "reorthogonalisation (scipy sparse products on one thread, Gram-Schmidt by BLAS)",
            "extrapolated": False, "measured_seconds": t, "estimate": est,
            "threads": {"sparse_products": 1, "reorthogonalisation": blas_threads()}}


def oracle_c4_baseline(gs, sample=8, probes=16):
    """C4 by the oracle on a seeded sample of the 512 graphs (every 64th),
    `probes` of the 64 probes x 40 plain FP64 Lanczos steps each, scaled to
    the batch by the probes and by the work per graph, proportional to
    (n + nnz)."""
    from oracle import density, estimators
    pick = list(range(0, len(gs), max(1, len(gs) // sample)))[:sample]
    t = 0.0
    for i in pick:
        A, _ = density.density_matrix(gs[i])
        t0 = time.perf_counter()
        estimators.hutchinson(A, probes, 40, 1000 + i, reorth="none")
        t += time.perf_counter() - t0
    w_all = float(sum(gg.n + gg.nnz for gg in gs))
    w_s = float(sum(gs[i].n + gs[i].nnz for i in pick))
    scale = (w_all / w_s) * (64.0 / probes)
    return {"value": len(gs) / (t * scale), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{len(pick)} of the {len(gs)} graphs (every {max(1, len(gs) // sample)}th), {probes} of the "
                      "64 probes x 40 plain FP64 Lanczos steps each (scipy, one thread), scaled to the batch by "
                      "sum(n + nnz) and to 64 probes",
            "extrapolated": True, "scale_factor": scale, "measured_seconds": t, "sampled_graphs": len(pick),
            "sampled_probes_per_graph": probes}


def run_native(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_2212_09642_gb300 import _build, vne

    _build.build_all()
    dev = local
    torch.cuda.set_device(dev)
    g = make_graph(args.n)
    stream = torch.cuda.Stream(device=dev)
    ctx = vne.vne_ctx_create(dev)
    vne.vne_ctx_set_stream(ctx, stream)
    flags = vne.VNE_FP32 | {"degree": vne.VNE_REORDER, "rcm": vne.VNE_REORDER_RCM, "none": 0}[args.reorder]
    mat = vne.vne_create_density_matrix(ctx, g.n, g.rowptr, g.col, None, flags)
    reorth = {"none": 0, "partial": 2, "full": 1}[args.reorth]
    opt = vne.options(reorth=reorth)
    seed0 = 1000 * (rank + 1)
    if args.schedule:
        vals = [int(x) for x in args.schedule.split(",")] + [0, 0]
        pnl, itm, var, il, ipw = vals[:5]
        opt = vne.options(reorth=reorth, panel=pnl, item_nnz=itm, step_variant=var, interleave=il,
                          items_per_warp=ipw)
        tuned_cfg = {"panel": pnl, "item_nnz": itm, "step_variant": var, "interleave": il,
                     "items_per_warp": ipw, "source": "--schedule"}
    else:
        # schedule autotuner (once per matrix shape; cached in the context)
        tuned, tune_ms = vne.vne_autotune(ctx, mat, 112 if args.estimator == "hutchpp" else args.vectors, 8)
        tuned_cfg = {"panel": tuned.panel, "item_nnz": tuned.item_nnz, "step_variant": tuned.step_variant,
                     "interleave": tuned.interleave, "items_per_warp": tuned.items_per_warp,
                     "ms_per_lanczos_step_112_cols": tune_ms, "source": "vne_autotune"}

    def one(seed):
        if args.estimator == "hutchinson":
            return vne.vne_entropy_hutchinson(ctx, mat, args.vectors, M_STEPS, seed, opt=opt)
        return vne.vne_entropy_hutchpp(ctx, mat, N_SKETCH, N_HUTCH, M_STEPS, seed, opt=opt)

    for w in range(args.warmup):
        one(seed0 + w)
    torch.cuda.synchronize(dev)
    # ceiling of the step kernel's access pattern: random row gathers from a
    # table of one panel (n x panel FP32), untimed
    ks = int(tuned_cfg["panel"]) or 16
    probe_gbs = vne.vne_measure_gather(ctx, g.n * ks * 4, ks * 4, 32 << 20, 0, 3)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    ests = []
    sampler = ClockSampler(dev) if rank == 0 else None
    if sampler:
        sampler.__enter__()
    vne.vne_ctx_profile(ctx, True)
    barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nvtx_push("timed_steps")
    e0.record(stream)
    for k in range(args.steps):
        ests.append(one(seed0 + 100 + k)[0])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    nvtx_pop()
    barrier()
    if sampler:
        sampler.__exit__()
    elapsed_ms = e0.elapsed_time(e1)
    launches, kst = vne.vne_ctx_stats(ctx)
    vne.vne_ctx_profile(ctx, False)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([elapsed_ms], device=f"cuda:{dev}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    value = world * args.steps / (elapsed_ms / 1e3)

    # mixed-precision error against the FP64 GPU run on identical probes
    rel_err = None
    if not args.no_fp64_check and rank == 0 and args.estimator == "hutchpp":
        mat64 = vne.vne_create_density_matrix(ctx, g.n, g.rowptr, g.col, None, vne.VNE_FP64 | vne.VNE_REORDER)
        e64 = vne.vne_entropy_hutchpp(ctx, mat64, N_SKETCH, N_HUTCH, M_STEPS, seed0 + 100, opt=vne.options(reorth=0))[0]
        vne.vne_matrix_destroy(mat64)
        rel_err = abs(ests[0] - e64) / abs(e64)

    # end to end through the C ABI from host buffers
    e2e = None
    if not args.no_e2e and args.estimator == "hutchpp":
        k2 = max(1, min(args.steps, 3))
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for k in range(k2):
            m2 = vne.vne_create_density_matrix(ctx, g.n, g.rowptr, g.col, None, flags)
            vne.vne_entropy_hutchpp(ctx, m2, N_SKETCH, N_HUTCH, M_STEPS, seed0 + 200 + k, opt=opt)
            vne.vne_matrix_destroy(m2)
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([dt], device=f"cuda:{dev}", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        e2e = {"value": world * k2 / dt, "unit": UNIT, "h2d_bytes_per_step": int(8 * (g.n + 1) + 4 * g.nnz),
               "d2h_bytes_per_step": 8 + 3 * 8 + 2 * 4 + 8 * (N_SKETCH + N_HUTCH)}

    if rank != 0:
        vne.vne_matrix_destroy(mat)
        vne.vne_ctx_destroy(ctx)
        return

    n_, nnz_, tr_, nb_ = vne.vne_matrix_info(mat)
    peak, peak_kind = load_peaks()
    cnt, ms, byts = kst["step"]
    achieved = (byts / (ms / 1e3)) / 1e9 if ms > 0 else None
    per_launch_bytes = byts / cnt if cnt else None
    roof = {"kernel": "k_step (fused SpMM + Lanczos partial inner products)", "bound": "hbm",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak if achieved else None,
            "peak_kind": peak_kind, "nominal_peak": 7900.0,
            "frac_of_nominal": achieved / 7900.0 if achieved else None,
            "traffic": recorded_traffic(), "algorithmic_bytes_per_launch": per_launch_bytes,
            "avg_launch_ms": ms / cnt if cnt else None, "launches_timed": int(cnt),
            "share_of_step_time": (ms / elapsed_ms) if elapsed_ms else None}
    # the same launches counted by what they move through L2: every nonzero
    # gathers one row of KS columns per panel, besides the streams
    kp_s = -(-N_SKETCH // ks) * ks
    kp_avg = (kp_s + kp_s + -(-N_HUTCH // ks) * ks) / 2 if args.estimator == "hutchpp" else -(-args.vectors // ks) * ks
    gathered = float(nnz_) * kp_avg * 4
    csr_bytes = 4.0 * (g.n + 1) + 4.0 * float(nnz_)
    # gathers + the CSR once per panel + own rows of w_j, w_{j-1} and u
    l2_bytes = gathered + (kp_avg / ks) * csr_bytes + 3.0 * g.n * kp_avg * 4
    roof["l2_gather"] = {"gathered_bytes_per_launch": gathered, "l2_bytes_per_launch": l2_bytes,
                         "achieved_gbs": l2_bytes / (ms / cnt / 1e3) / 1e9 if cnt and ms > 0 else None,
                         "probe_gbs": probe_gbs,
                         "frac": (l2_bytes / (ms / cnt / 1e3) / 1e9) / probe_gbs if cnt and ms > 0 else None,
                         "probe": f"random {ks * 4}-byte row gathers from a {g.n * ks * 4 / 2**20:.0f} MiB table "
                                  f"(vne_measure_gather)"}
    ucnt, ums, ubytes = kst["update"]
    update = {"achieved_gbs": (ubytes / (ums / 1e3)) / 1e9 if ums > 0 else None,
              "avg_launch_ms": ums / ucnt if ucnt else None, "share_of_step_time": ums / elapsed_ms}

    cpu = None
    if not args.no_cpu_baseline and world == 1 and args.estimator == "hutchpp":
        t_est, parts = oracle_sample(g, columns=2)
        cpu = {"value": 1.0 / t_est, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "2 sketch matvecs + 2 quadratic forms (FP64 scipy Lanczos, 60 steps, one thread, same "
                         "graph) + one n x 100 orthonormalisation/projection (BLAS threads), extrapolated to "
                         "100 + 200 Krylov runs", **parts}
        try:
            v_all, rec_all = oracle_all_cores(g.n, parts["t_orth_s"])
            cpu["all_cores"] = {"value": v_all, "unit": UNIT, "cores": rec_all["processes"], **rec_all}
        except Exception as e:  # the single-thread figure stands on its own
            cpu["all_cores"] = {"unavailable": f"{type(e).__name__}: {e}"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload_name(g.n) if args.estimator == "hutchpp" else
                   f"Hutchinson {args.vectors} vectors x {M_STEPS} steps on BA n={args.n} m=4 (profiling case)",
                   "n": int(n_), "nnz": int(nnz_), "sketch_cols": N_SKETCH,
                   "hutch_vectors": N_HUTCH, "krylov_steps": M_STEPS, "scalars": "f64",
                   "l2": "inputs larger than L2 (each 100-column block is 400 MB; L2 129 MB)",
                   "parallelism": f"replicas x{world} (independent estimates)", "reorder": args.reorder,
                   "reorth": args.reorth},
        "roofline": roof, "update_kernel": update, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": int(launches), "clocks": sampler.summary() if sampler else None,
        "schedule": tuned_cfg,
        "rel_err_vs_fp64": rel_err, "estimates": ests,
    }
    print(json.dumps(line), flush=True)
    vne.vne_matrix_destroy(mat)
    vne.vne_ctx_destroy(ctx)


# ---------------------------------------------------------------------------
# measurement lines of the other configurations (not the headline)

def nvtx_push(name):
    """Mark a timed region (an ncu run can restrict its capture to it with
    --nvtx --nvtx-include name/)."""
    try:
        import torch
        torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def nvtx_pop():
    try:
        import torch
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def _timed(ctx, stream, fn, steps, warmup, label="timed_steps"):
    import torch
    from paper_2212_09642_gb300 import vne
    for w in range(warmup):
        fn(w)
    torch.cuda.synchronize()
    vne.vne_ctx_profile(ctx, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(0)
    sampler.__enter__()
    nvtx_push(label)
    e0.record(stream)
    outs = [fn(100 + k) for k in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    nvtx_pop()
    sampler.__exit__()
    ms = e0.elapsed_time(e1)
    launches, kst = vne.vne_ctx_stats(ctx)
    vne.vne_ctx_profile(ctx, False)
    return outs, ms, launches, kst, sampler.summary()


def _roof(kst, kind, ms_total, label):
    peak, kind_p = load_peaks()
    cnt, ms, byts = kst[kind]
    if not cnt or ms <= 0:
        return None
    ach = byts / (ms / 1e3) / 1e9
    return {"kernel": label, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "peak_kind": kind_p, "traffic": None, "algorithmic_bytes_per_launch": byts / cnt,
            "avg_launch_ms": ms / cnt, "launches_timed": int(cnt), "share_of_step_time": ms / ms_total}


def run_other(args):
    import numpy as np
    import torch
    from paper_2212_09642_gb300 import _build, graphs, vne
    _build.build_all()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    ctx = vne.vne_ctx_create(0)
    vne.vne_ctx_set_stream(ctx, stream)
    line = {"n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "data": "synthetic", "unit": UNIT}
    if args.workload == "c1":
        g = graphs.erdos_renyi(2000, 0.005, 1)
        mat = vne.matrix_from_graph(ctx, g, fp64=True)
        outs, ms, launches, kst, clk = _timed(ctx, stream, lambda s: vne.vne_entropy_hutchinson(
            ctx, mat, 100, 50, s), args.steps, args.warmup)
        line.update(metric="entropy estimates/sec (Hutchinson 100 x 50, ER n=2000 p=0.005, FP64)",
                    value=args.steps / (ms / 1e3), ms_per_step=ms / args.steps, dtype="f64",
                    config={"workload": "C1: ER G(2000,0.005) seed 1, FP64, Hutchinson 100 Rademacher x 50 Lanczos "
                                        "steps, full reorthogonalisation", "l2": "working set L2-resident (latency-bound)"},
                    roofline=_roof(kst, "step", ms, "k_step FP64"), gpu_launches=int(launches), clocks=clk,
                    estimate=outs[0][0], std_error=outs[0][1])
        # the same estimates with adaptive stopping by the Theorem 4.4
        # estimate (relative quadrature error 1e-8, checks every 5 steps)
        aopt = vne.options(quad_tol=1e-8, check_every=5)
        outs2, ms2, _, _, _ = _timed(ctx, stream, lambda s: vne.vne_entropy_hutchinson(
            ctx, mat, 100, 50, s, opt=aopt), args.steps, args.warmup)
        line["adaptive_quad_tol_1e-8"] = {"value": args.steps / (ms2 / 1e3), "unit": UNIT,
                                          "krylov_steps_taken": vne.vne_ctx_last_steps(ctx),
                                          "estimate": outs2[0][0],
                                          "rel_diff_vs_fixed_steps": abs(outs2[0][0] - outs[0][0]) / abs(outs[0][0])}
        vne.vne_matrix_destroy(mat)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = oracle_c1_baseline(g)
    elif args.workload == "c3":
        n = args.n if args.n != N_NODES else 4_000_000
        g = graphs.random_geometric(n, graphs.rgg_radius_for_degree(n, 6.0), 4)
        t0 = time.perf_counter()
        colors, s = vne.vne_greedy_coloring(g.n, g.rowptr, g.col, 2)
        t_col = time.perf_counter() - t0
        t1 = time.perf_counter()
        mat = vne.matrix_from_graph(ctx, g, fp64=False, reorder="rcm")
        t_asm = time.perf_counter() - t1
        # the device colouring alone (Algorithm 1 in rounds), checked against the host sweep
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        vne.vne_matrix_coloring(ctx, mat, g.n, 2)
        torch.cuda.synchronize()
        e0.record(stream)
        dcolors, ds, rounds = vne.vne_matrix_coloring(ctx, mat, g.n, 2)
        e1.record(stream)
        torch.cuda.synchronize()
        dev_col = {"ms": e0.elapsed_time(e1), "rounds": rounds, "colors": ds,
                   "equal_to_host_sweep": bool(np.array_equal(dcolors, colors)), "host_sweep_s": t_col}
        # SpMM schedule tuned on a block of one column per colour (cached in the context)
        tuned, _ = vne.vne_autotune(ctx, mat, s, 8)
        opt = vne.options(cg_tol=1e-8, n_inf_poles=2)
        # one step = Algorithm 1's colouring on the device + the probing estimate
        outs, ms, launches, kst, clk = _timed(ctx, stream, lambda sd: vne.vne_entropy_probing(
            ctx, mat, None, 2, 0, opt=opt, num_shifts=8), args.steps, args.warmup)
        line.update(metric="entropy estimates/sec (probing d=2, rational Krylov 8 poles + 2 at infinity, RGG n=4e6)",
                    value=args.steps / (ms / 1e3), ms_per_step=ms / args.steps, dtype="f32",
                    config={"workload": f"C3: RGG n={g.n} avg degree 6 (seed 4), generation order, greedy distance-2 "
                                        f"colouring on the device inside each step ({s} colours), matrix relabelled "
                                        f"by reverse Cuthill-McKee in vne_create_density_matrix ({t_asm:.1f} s, "
                                        "untimed), 8 log-spaced poles on [1e-4, 1] ||A||_G, multi-shift CG to "
                                        "recursive rel. residual 1e-8",
                            "nnz": g.nnz, "colors": s, "l2": "inputs larger than L2",
                            "schedule": {"panel": tuned.panel, "item_nnz": tuned.item_nnz,
                                         "step_variant": tuned.step_variant, "interleave": tuned.interleave}},
                    roofline=_roof(kst, "step", ms, "k_step (SpMM inside CG)"),
                    cg_update=_roof(kst, "cg_update", ms, "k_cg_update"),
                    cg_direction=_roof(kst, "cg_direction", ms, "k_cg_direction"),
                    gpu_launches=int(launches), clocks=clk, estimate=outs[0][0], device_coloring=dev_col)
        # the same estimate with the polynomial part chosen by the switching
        # rule of Section 5.3 (n_inf_poles = -1) instead of two poles at infinity
        mopt = vne.options(cg_tol=1e-8, n_inf_poles=-1)
        outs_m, ms_m, _, _, _ = _timed(ctx, stream, lambda sd: vne.vne_entropy_probing(
            ctx, mat, None, 2, 0, opt=mopt, num_shifts=8), max(1, args.steps // 2), 1, label="timed_sub")
        line["switching_rule"] = {"value": max(1, args.steps // 2) / (ms_m / 1e3), "unit": UNIT,
                                  "polynomial_dim": vne.vne_ctx_last_poly_dim(ctx), "estimate": outs_m[0][0],
                                  "diff_vs_two_poles_at_infinity": outs_m[0][0] - outs[0][0]}
        vne.vne_matrix_destroy(mat)
    elif args.workload == "c6":
        # Algorithm 2: T_1..T_3 (device colourings at d = 1, 2, 3), the fitted
        # error model for d, T_d with per-colour tolerances (Lanczos with the
        # Theorem 4.4 stop, checks every 2 steps)
        n = args.n if args.n != N_NODES else 4_000_000
        g = graphs.random_geometric(n, graphs.rgg_radius_for_degree(n, 6.0), 4)
        mat = vne.matrix_from_graph(ctx, g, fp64=False, reorder="rcm")
        tuned, _ = vne.vne_autotune(ctx, mat, 32, 8)
        eps = 1e-3
        aopt = vne.options(check_every=2)
        outs, ms, launches, kst, clk = _timed(ctx, stream, lambda sd: vne.vne_entropy_probing_auto(
            ctx, mat, eps, 128, 32, opt=aopt), args.steps, args.warmup)
        est, rep = outs[0]
        line.update(metric="entropy estimates/sec (probing with the heuristic choice of d, eps=1e-3, RGG n=4e6)",
                    value=args.steps / (ms / 1e3), ms_per_step=ms / args.steps, dtype="f32",
                    config={"workload": f"C6: RGG n={g.n} avg degree 6 (seed 4), relabelled by reverse Cuthill-McKee; "
                                        "probing with d from the fitted error model (T_1..T_3), device colourings "
                                        "inside each step, Lanczos stopped by the Theorem 4.4 estimate at "
                                        "eps/2 T_1 |V_l| / n (at most 128 steps, checks every 2)",
                            "nnz": g.nnz, "eps": eps, "l2": "inputs larger than L2"},
                    roofline=_roof(kst, "step", ms, "k_step"), update_kernel=_roof(kst, "update", ms, "k_update"),
                    gpu_launches=int(launches), clocks=clk, estimate=est, report=rep)
        vne.vne_matrix_destroy(mat)
    elif args.workload == "c7":
        line.update(run_scaling(args, ctx, stream))
    elif args.workload == "c4":
        gs = graphs.batched_uneven_family(512, 1000, 200000, 1000)
        mats = [vne.matrix_from_graph(ctx, gg, fp64=False) for gg in gs]
        outs, ms, launches, kst, clk = _timed(ctx, stream, lambda sd: vne.vne_batch_hutchinson(
            ctx, mats, 64, 40, sd, opt=vne.options(reorth=0)), args.steps, args.warmup)
        line.update(metric="entropy estimates/sec (512 uneven graphs batched, Hutchinson 64 x 40)",
                    value=512 * args.steps / (ms / 1e3), ms_per_step=ms / args.steps, dtype="f32",
                    config={"workload": "C4: 512 graphs, n log-uniform [1e3, 2e5], ER deg 8 / BA m=3 / WS k=6 b=0.1, "
                                        "64 Rademacher x 40 Lanczos steps each, one packed launch sequence (the packed layout of the "
                                        "batch is built by the first call and kept in the context)",
                            "sum_n": int(sum(gg.n for gg in gs)), "sum_nnz": int(sum(gg.nnz for gg in gs)),
                            "l2": "inputs larger than L2"},
                    roofline=_roof(kst, "step", ms, "k_step (packed segments)"),
                    update_kernel=_roof(kst, "update", ms, "k_update"), gpu_launches=int(launches), clocks=clk)
        for m in mats:
            vne.vne_matrix_destroy(m)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = oracle_c4_baseline(gs)
    else:
        line.update(run_serving(args, ctx, stream))
    vne.vne_ctx_destroy(ctx)
    print(json.dumps(line), flush=True)


def run_scaling(args, ctx, stream):
    """Scaling study of Section 6 (Figure 6): seconds per estimate against n =
    2^10 .. 2^20 for the 2D square grid and BA graphs, probing with the
    heuristic choice of d at eps = 1e-4 (grid: the optimal lattice colouring,
    BA: Algorithm 1 on the device) and the adaptive stochastic estimator at
    eps = 1e-2 (the served Hutch++ proxy: N_r = 4 sketch columns, then blocks
    of 64 deflated probes until 2.576 stderr <= eps/2 |S|, one query at a time
    on a server made for the graph), averaged over `--scaling-runs` seeds as
    the paper averages its adaptive Hutch++ over many runs.  Probing: one
    warm-up call, then the best of `steps` timed calls (CUDA events on the
    library stream).  BA probing stops growing n once the previous size took
    longer than 10 s or needed more than `--ba-max-colors` colours: the
    colour count of a distance-d colouring of a BA graph grows with n, and
    the probing cost with colours x n."""
    import numpy as np
    import torch
    from paper_2212_09642_gb300 import graphs, grid_coloring, vne

    def timed(fn, reps):
        fn()
        best, out = math.inf, None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            out = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        return best, out

    def stochastic(mat, n, seeds):
        """Seconds per served query (wall clock from submission to the
        result, device synchronised at both ends) for each seed, after one
        warm-up query; the server is created once per graph."""
        srv = vne.vne_server_create(ctx, (1 << 30) + 1200 * n, max_active=1, krylov_steps=40, block_vectors=64,
                                    opt=vne.options(reorth=0, quad_tol=args.serve_krylov_tol,
                                                    check_every=args.serve_check, sketch_steps=args.serve_sketch))
        try:
            def one(seed):
                t = vne.vne_server_submit(ctx, srv, mat, 1e-2, seed, 1 << 16)
                while vne.vne_server_result(srv, t)["state"] != 2:
                    vne.vne_server_step(ctx, srv)
                return vne.vne_server_result(srv, t)
            one(seeds[0] + 7919)
            times, res = [], []
            for sd in seeds:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = one(sd)
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t0)
                res.append(r)
        finally:
            vne.vne_server_destroy(srv)
        return times, res

    reps = max(1, min(args.steps, 3))
    exps = [int(e) for e in args.scaling_exponents.split(",")]
    curve = []
    sampler = ClockSampler(0)
    sampler.__enter__()
    ba_budget_s = 10.0  # BA probing stops growing n once one estimate takes longer
    ba_colors_ok = True  # ... or once it needs more than --ba-max-colors colours
    for kind in ("grid", "ba"):
        for e in exps:
            n = 1 << e
            if kind == "grid":
                side = 1 << (e // 2)
                g = graphs.grid2d(side, n // side)
                colfn = (lambda d, r=side, c=n // side: grid_coloring.lattice_coloring(r, c, d))
            else:
                g = graphs.barabasi_albert(n, 2, 100 + e)
                colfn = None
            mat = vne.matrix_from_graph(ctx, g, fp64=False, reorder=True)
            pt = {"graph": kind, "n": g.n, "nnz": g.nnz}
            if kind == "grid" or (ba_budget_s > 0 and ba_colors_ok):
                t_p, (est, rep) = timed(lambda: vne.vne_entropy_probing_auto(
                    ctx, mat, 1e-4, 128, 32, opt=vne.options(check_every=2), coloring=colfn), reps)
                pt["probing"] = {"s_per_estimate": t_p, "estimate": est, "d": rep["d"], "colors": rep["colors"],
                                 "colors_d123": rep["colors_d"], "rule": rep["rule"],
                                 "lanczos_steps": rep["steps_d"] + [rep["steps"]]}
                if kind == "ba" and t_p > ba_budget_s:
                    ba_budget_s = 0.0
                if kind == "ba" and rep["colors"] > args.ba_max_colors:
                    ba_colors_ok = False
            else:
                pt["probing"] = (f"not run: the previous BA size took longer than 10 s per estimate or needed "
                                 f"more than {args.ba_max_colors} colours")
            times, rs = stochastic(mat, g.n, [1000 * e + r for r in range(args.scaling_runs)])
            ests = np.array([r["estimate"] for r in rs])
            pt["stochastic"] = {"s_per_estimate_mean": float(np.mean(times)), "s_per_estimate_min": float(min(times)),
                                "s_per_estimate_max": float(max(times)), "runs": len(times),
                                "estimate_mean": float(np.mean(ests)),
                                "estimate_spread": float(np.std(ests) / abs(np.mean(ests))) if len(ests) > 1 else 0.0,
                                "vectors_mean": float(np.mean([r["vectors"] for r in rs])),
                                "vectors_min": int(min(r["vectors"] for r in rs)),
                                "vectors_max": int(max(r["vectors"] for r in rs))}
            curve.append(pt)
            vne.vne_matrix_destroy(mat)
            print(json.dumps(pt), file=sys.stderr, flush=True)
    sampler.__exit__()
    big = [p for p in curve if p["graph"] == "grid"][-1]
    return {"metric": f"entropy estimates/sec, probing eps=1e-4 on the 2D grid n={big['n']} (scaling study)",
            "value": 1.0 / big["probing"]["s_per_estimate"], "ms_per_step": 1e3 * big["probing"]["s_per_estimate"],
            "dtype": "f32",
            "config": {"workload": "scaling study: 2D square grids and BA m=2 graphs, n = 2^" + ",".join(map(str, exps))
                                   + "; probing with the heuristic choice of d at eps 1e-4 (grid: lattice "
                                   "colouring with ceil((d+1)^2/2) colours; BA: device greedy colouring), Lanczos "
                                   "stopped by Theorem 4.4 (checks every 2 steps, at most 128); adaptive Hutch++ "
                                   "proxy at eps 1e-2 (N_r = 4 sketch columns, blocks of 64 deflated probes, at "
                                   "most 40 Lanczos steps"
                                   + (", stopped by the Theorem 4.4 estimate" if args.serve_krylov_tol != 0 else "")
                                   + f"), mean over {args.scaling_runs} seeds",
                       "timing": f"probing: best of {reps} after one warm-up, CUDA events; stochastic: wall clock "
                                 "per served query, device synchronised, after one warm-up query",
                       "l2": "small sizes are L2-resident (the curve spans both regimes)"},
            "curve": curve, "clocks": sampler.summary()}


def run_serving(args, ctx, stream):
    """C5: Poisson arrivals of entropy queries (rel. accuracy 1e-3), continuous
    batching of the Hutch++ proxy (4 sketch columns, blocks of 64 deflated
    probes), one Lanczos step of every active query per tick; beside it the
    plain FP64 form one query at a time on the same queries and arrivals."""
    import numpy as np
    from paper_2212_09642_gb300 import graphs, vne
    rng = np.random.default_rng(5)
    pool_n = np.rint(np.exp(rng.uniform(math.log(1e3), math.log(1e6), size=24))).astype(int)
    pool = []
    for i, nn in enumerate(pool_n):
        kind = i % 3
        if kind == 0:
            pool.append(graphs.erdos_renyi(int(nn), 8.0 / (nn - 1), 500 + i))
        elif kind == 1:
            pool.append(graphs.barabasi_albert(int(nn), 3, 500 + i))
        else:
            pool.append(graphs.watts_strogatz(int(nn), 6, 0.1, 500 + i))
    R = args.requests
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, size=R))
    if args.at_once:
        arrivals[:] = 0.0  # every query arrives at the start: a saturated server (profiling)
    which = rng.integers(0, len(pool), size=R)
    eps, cap, m, block = 1e-3, 8192, 40, 64

    def serve(fp64, slots, budget, realtime, limit_s):
        """Run the queries through one server; with realtime, submissions follow
        the arrival clock, else each query runs alone (FIFO one at a time) and
        its latency is its FIFO queueing on the same arrivals plus its own
        service time.  Returns completion latencies, vectors, estimates."""
        mats = [vne.matrix_from_graph(ctx, g, fp64=fp64, reorder=True) for g in pool]
        srv = vne.vne_server_create(ctx, budget, max_active=slots, krylov_steps=m, block_vectors=block,
                                    opt=vne.options(reorth=0, quad_tol=args.serve_krylov_tol,
                                                    check_every=args.serve_check, sketch_steps=args.serve_sketch))
        lat, vecs, ests, served = {}, {}, {}, 0
        steps = {}  # Lanczos steps per block of each query (ticks from admission to completion / blocks)
        try:
            t0 = time.perf_counter()
            if realtime:
                nxt, tickets, live = 0, {}, set()
                while len(lat) < R:
                    now = time.perf_counter() - t0
                    while nxt < R and arrivals[nxt] <= now:
                        tickets[nxt] = vne.vne_server_submit(ctx, srv, mats[which[nxt]], eps, 9000 + nxt, cap)
                        live.add(nxt)
                        nxt += 1
                    q, a, _ = vne.vne_server_info(srv)
                    if q == 0 and a == 0:
                        if nxt < R:
                            time.sleep(max(0.0, arrivals[nxt] - now))
                        continue
                    done, _ = vne.vne_server_step(ctx, srv)
                    if done:
                        t_now = time.perf_counter() - t0
                        for i in list(live):
                            r = vne.vne_server_result(srv, tickets[i])
                            if r["state"] == 2:
                                lat[i] = t_now - arrivals[i]
                                vecs[i], ests[i] = r["vectors"], r["estimate"]
                                steps[i] = (r["done_tick"] - r["admit_tick"]) / (r["vectors"] / block)
                                live.discard(i)
                served = R
            else:
                free_at = 0.0
                for i in range(R):
                    if time.perf_counter() - t0 > limit_s:
                        break
                    ts = time.perf_counter()
                    t = vne.vne_server_submit(ctx, srv, mats[which[i]], eps, 9000 + i, cap)
                    while vne.vne_server_result(srv, t)["state"] != 2:
                        vne.vne_server_step(ctx, srv)
                    service = time.perf_counter() - ts
                    r = vne.vne_server_result(srv, t)
                    start = max(free_at, arrivals[i])
                    free_at = start + service
                    lat[i] = free_at - arrivals[i]
                    vecs[i], ests[i] = r["vectors"], r["estimate"]
                    steps[i] = (r["done_tick"] - r["admit_tick"]) / (r["vectors"] / block)
                    served = i + 1
            total = time.perf_counter() - t0
        finally:
            vne.vne_server_destroy(srv)
            for mt in mats:
                vne.vne_matrix_destroy(mt)
        return lat, vecs, ests, served, total, steps

    sampler = ClockSampler(0)
    sampler.__enter__()
    vne.vne_ctx_profile(ctx, True)
    lat, vecs, ests, _, total, steps = serve(False, 128, 120 << 30, True, None)
    launches, kst = vne.vne_ctx_stats(ctx)
    vne.vne_ctx_profile(ctx, False)
    sampler.__exit__()
    if args.fp64_limit_s > 0:
        lat64, vecs64, ests64, served64, total64, steps64 = serve(True, 1, 60 << 30, False, args.fp64_limit_s)
    else:  # the FP64 arm left out
        lat64, vecs64, ests64, served64, total64, steps64 = {}, {}, {}, 0, 1.0, {}
    idx = np.arange(R)
    L = np.array([lat[i] for i in idx])
    L64 = np.array([lat64[i] for i in range(served64)])
    Lsame = L[:served64]
    dev = [abs(ests[i] - ests64[i]) / abs(ests64[i]) for i in range(served64)]
    return {"metric": "served entropy estimates/sec at rel. accuracy 1e-3 (continuous batching), p50/p99 latency",
            "value": R / total, "ms_per_step": 1e3 * total / R, "dtype": "f32",
            "config": {"workload": f"C5: {R} queries, Poisson {args.rate}/s (seed 5), graphs from a pool of 24 "
                                   "(n log-uniform [1e3, 1e6], ER/BA/WS), eps 1e-3, Hutch++ proxy: 4 sketch columns "
                                   "+ blocks of 64 deflated probes until 2.576 se <= eps/2 |S|, cap 8192 probes, "
                                   + f"sketch of {args.serve_sketch or 40} Lanczos steps, "
                                   + ("Lanczos blocks of at most 40 steps stopped by the Theorem 4.4 estimate at "
                                      + ("eps/2" if args.serve_krylov_tol < 0 else f"{args.serve_krylov_tol}")
                                      + f" relative (checks every {args.serve_check} steps)"
                                      if args.serve_krylov_tol != 0 else "40 Lanczos steps per block")
                                   + ", 128 slots, one Lanczos step per tick",
                       "pool_n": [int(x) for x in pool_n]},
            "lanczos_steps_per_block": {"served_mean": float(np.mean(list(steps.values()))),
                                        "fp64_mean": float(np.mean(list(steps64.values()))) if steps64 else None},
            "latency_s": {"p50": float(np.percentile(L, 50)), "p99": float(np.percentile(L, 99)),
                          "mean": float(L.mean())},
            "fp64_one_at_a_time": {"queries": int(served64), "estimates_per_s": served64 / total64,
                                   "p50": float(np.percentile(L64, 50)), "p99": float(np.percentile(L64, 99)),
                                   "served_p50_same_queries": float(np.percentile(Lsame, 50)),
                                   "served_p99_same_queries": float(np.percentile(Lsame, 99)),
                                   "max_rel_dev_mixed_vs_fp64": float(max(dev)) if dev else None,
                                   "how": "the same server code with FP64 matrices and one slot; each query runs "
                                          "alone, latency = FIFO queueing on the same arrivals + its service time"}
            if served64 else None,
            "mean_vectors_per_query": float(np.mean([vecs[i] for i in idx])),
            "roofline": None, "roofline_note": "the served ticks launch step and update together per tick; the "
                                               "kernels' rooflines are those of the headline workload",
            "gpu_launches": int(launches), "clocks": sampler.summary()}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "c2":
        run_other(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
