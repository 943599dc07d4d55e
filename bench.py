#!/usr/bin/env python3
"""Benchmark of the SAP-multilevel solver on one GB300 (or N replicas).

One step = one call of mg_solve on the workload's right-hand sides, to a
relative residual of 1e-10 (verified in FP64 by the library), with the set-up
done once before the timed region and reported separately (as the paper's
tables do).  The default workload is the 32^3 x 64 lattice with the 12
spin-colour point sources, solved by the mixed-precision form (FP32
arithmetic, BF16-stored links and clover, FP16-stored test vectors, FP32
coarse operator; FP64 defect correction).  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

import os

# the CPU legs time the oracle on one core: keep numpy's BLAS single-threaded
for _v in ("OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12     # FP32 FMA lanes x 2 flop x max SM clock
FP64_PEAK_TFLOPS = 1.25                                # GB300 FP64 (nominal)
# DRAM bytes per (site of the colour, right-hand side) of one BF16 Schwarz colour pass,
# from ncu captures with 12 right-hand sides (traffic grows with the units), per
# launch shape of the paired kernels: shapes 0 (sap_colour_pair_kernel) and 3
# (sap_block_kernel) on the 16^3x32 lattice, shape 5 on 32^3x32; none for the others
SAP_DRAM_BYTES_PER_UNIT = {0: (266.179328e6 + 66.372352e6) / (65536 * 12),
                           3: (263.003904e6 + 52.152320e6) / (65536 * 12),
                           5: (2440.573e6 + 584.692736e6) / (524288 * 12)}
SAP_KERNEL = {-1: "sap_colour_kernel", 0: "sap_colour_pair_kernel", 1: "sap_colour_pair_kernel",
              2: "sap_colour_pair_kernel", 3: "sap_block_kernel", 4: "sap_block_kernel",
              5: "sap_block_kernel", 6: "sap_split_kernel"}


def flops_dirac_site():
    return 1848.0


def flops_sap_site(n_mr):
    # residual (D + subtraction) + n_MR x (block operator (6 hops on average) + dots + updates) + update
    return 1896.0 + 1854.0 * n_mr


def bytes_sap_spinor(prec):
    return 4 * 12 * (16 if prec == "fp64" else 8)             # b, z, halo z read; z written (per RHS)


def bytes_sap_fields(prec):
    store = {"fp64": 16, "fp32": 8, "fp16": 4, "bf16": 4}[prec]
    return 2 * 36 * store                                       # links (4 x 9 complex) + clover (36 slots)


def bytes_sap_site(prec):
    return bytes_sap_spinor(prec) + bytes_sap_fields(prec)


def bytes_dirac_site(prec):
    spinor = 2 * 12 * (16 if prec == "fp64" else 8)
    store = {"fp64": 16, "fp32": 8, "fp16": 4, "bf16": 4}[prec]
    return spinor + 2 * 36 * store


# the kernels behind each timed family (a family call may issue several launches)
FAMILY_KERNELS = {
    "dirac": "dirac_pair_kernel + dirac_kernel", "sap": "sap_colour_pair_kernel + sap_block_kernel + sap_split_kernel",
    "coarse": "coarse_apply_mma16_kernel",
    "restrict": "restrict0_mma_kernel", "prolong": "prolong0_mma_kernel",
    "blas": "dots2h_partial + dcgs2_coeff_kernel + axpy2h_kernel (outer Arnoldi, FP16 basis)",
    "coarse_blas": "multidot_h_partial + multiaxpy_h_kernel + normalize_h_kernel + hessenberg_solve_kernel",
    "sap1": "coarse_sap_mrhs_kernel (level-1 Schwarz of three levels)",
}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.lines = []
        self.proc = None
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def max_over_ranks(x, world, device):
    """The largest x over all ranks: the job's step time is its slowest rank's
    (replicas: each rank solves its own right-hand sides, no data exchange)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def make_rhs(wl, dims):
    if wl["rhs"] == "point12":
        return synth.point_sources(dims)
    if wl["rhs"] == "z2":
        return synth.z2_spinor(dims, wl["rhs_seed"])[None]
    return synth.random_spinor(dims, wl["rhs_seed"])[None]


def solver_kwargs(wl, precision, nrhs):
    """Solver parameters of the workload; the mixed form tunes its launch shapes at set-up."""
    kw = dict(n_levels=wl["n_levels"], n_vec=tuple(wl["n_vec"]), setup_iters=wl["setup_iters"],
              n_mr=wl["n_mr"], nu_post=wl["nu_post"], coarse_iters=wl["coarse_iters"],
              fgmres_m=wl["fgmres_m"], tol=wl["tol"], maxiter=wl.get("maxiter", 500),
              precision=precision, nrhs_max=min(nrhs, wl.get("nrhs_max", nrhs)), seed=wl.get("vec_seed", 1),
              autotune=int(precision != "fp64"))
    for k in ("inner_iters", "sap_block2", "agg2"):                # three levels: the level-1 parameters
        if k in wl:
            kw[k] = tuple(wl[k]) if isinstance(wl[k], (list, tuple)) else wl[k]
    return kw


# ----------------------------------------------------------------------------- CPU oracle sample
# The oracle (plain numpy FP64) cannot solve the full workload in minutes (one
# Schwarz sweep of 32^3 x 64 alone takes about 100 s on one core), so both CPU
# legs time a bounded sample and scale it: one outer flexible-GMRES iteration
# (the two-level cycle with the workload's parameters, one application of D
# and one Gram-Schmidt step) on a sub-lattice of 1/32 of the volume, run for
# independent right-hand sides in concurrent processes, one per core used.
SAMPLE_DIV = (2, 2, 2, 4)


def cpu_info():
    """Host CPU model and core counts (recorded beside every CPU figure)."""
    info = {"nproc": os.cpu_count(), "machine": platform.machine(), "model": None}
    try:
        info["usable_cores"] = len(os.sched_getaffinity(0))
    except AttributeError:
        info["usable_cores"] = os.cpu_count()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model"):
                info["model"] = ln.split(":", 1)[1].strip()
                if not info["model"].isdigit():
                    break
    except Exception:
        pass
    return info


def sample_dims(wl):
    return tuple(d // k for d, k in zip(wl["dims"], SAMPLE_DIV))


def _oracle_worker(wl, sub, n_iter, seed, barrier, q):
    """One process of the sample: build a two-level oracle hierarchy on the
    sub-lattice (initial random test vectors; the cost of a cycle does not
    depend on them), wait for the other processes, then time n_iter outer
    iterations on its own right-hand side."""
    sys.path.insert(0, ROOT)
    from oracle.dirac import WilsonClover
    from oracle.mg import Multigrid
    u = synth.random_gauge_field(sub, wl["eps"], wl["gauge_seed"])
    op = WilsonClover(u, wl["m0"], wl["c_sw"])
    n = wl["n_vec"][0]
    mg = Multigrid(op, dict(n_levels=2, n_vec=(n,), setup_iters=0, n_mr=wl["n_mr"], nu_post=wl["nu_post"],
                            coarse_iters=wl["coarse_iters"], sap_block=((4, 4, 4, 4),), agg=((4, 4, 4, 4),)),
                   synth.test_vector_draw(sub, n, 1))
    v = synth.random_spinor(sub, 7 + seed)
    v = v / np.linalg.norm(v)
    barrier.wait()
    times = []
    for _ in range(n_iter):
        t0 = time.perf_counter()
        z = mg.cycle(0, v)
        w = op.apply(z)
        h = np.vdot(v, w)                 # one orthogonalisation step of the Arnoldi process
        w = w - h * v
        times.append(time.perf_counter() - t0)
    q.put((seed, times))


def oracle_sample(wl, n_iter, procs):
    """Per-iteration wall times of the sample with `procs` concurrent processes
    (spawned: no CUDA state is inherited): iteration k's wall time is the
    slowest process's k-th iteration."""
    import multiprocessing as mp
    sub = sample_dims(wl)
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(procs)
    q = ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(wl, sub, n_iter, k, barrier, q)) for k in range(procs)]
    for p in ps:
        p.start()
    res = [q.get() for _ in ps]
    for p in ps:
        p.join()
    per = [max(t[i] for _, t in res) for i in range(n_iter)]
    return {"sub": sub, "procs": procs, "wall_per_iter": per}


def mem_available():
    """Host memory available to new processes (bytes), from /proc/meminfo."""
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) * 1024
    except Exception:
        pass
    return None


def oracle_bytes(dims, n_vec=0):
    """Rough host memory of one oracle process on `dims`: FP64 links (576 B
    per site), the 12 x 12 clover (2304 B), about ten spinors (192 B each) and
    n_vec test vectors with their aggregated copies."""
    return int(np.prod(dims)) * (576 + 2304 + 10 * 192 + 2 * n_vec * 192)


def cpu_procs(nrhs, per_proc_bytes=0):
    """Concurrent oracle processes: one per right-hand side, at most one per
    usable core, and no more than half the available host memory holds."""
    n = max(1, min(nrhs, cpu_info()["usable_cores"] or 1))
    avail = mem_available()
    if avail and per_proc_bytes:
        n = max(1, min(n, int(0.5 * avail // per_proc_bytes)))
    return n


def oracle_estimate(wl, smp, timed, iters_per_rhs, nrhs, iters_source):
    """Scale the sample to the workload: seconds for all right-hand sides =
    median wall time of a concurrent iteration x volume ratio x outer
    iterations per right-hand side x rounds of `procs` right-hand sides."""
    sub = smp["sub"]
    scale = int(np.prod(wl["dims"])) // int(np.prod(sub))
    t = statistics.median(timed)
    rounds = -(-nrhs // smp["procs"])
    value = t * scale * iters_per_rhs * rounds
    info = cpu_info()
    return value, {
        "value": value, "unit": "s", "cores": smp["procs"], "kind": "oracle", "estimate": True,
        "cpu": info,
        "sample": f"{len(timed)} timed outer FGMRES iterations of the oracle (two-level cycle with the workload's "
                  f"parameters + one D + one Gram-Schmidt step) on {sub[0]}x{sub[1]}x{sub[2]}x{sub[3]} "
                  f"(1/{scale} of the volume), {smp['procs']} right-hand sides at once in concurrent processes "
                  f"(one per core); median {t:.2f} s per iteration, scaled by the volume (x{scale}), by "
                  f"{iters_per_rhs:.1f} outer iterations per right-hand side ({iters_source}) and by "
                  f"{rounds} round(s) of {smp['procs']} of the {nrhs} right-hand sides: an estimate"}


def run_reference(a, wl):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    nrhs = 12 if wl["rhs"] == "point12" else 1
    if wl.get("fp64_iterations_per_rhs") is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no measured FP64 iteration count stored for "
                                                              f"workload {a.workload}"}), flush=True)
        return 0
    procs = cpu_procs(nrhs, oracle_bytes(sample_dims(wl), wl["n_vec"][0]))
    smp = oracle_sample(wl, a.warmup + a.steps, procs)
    timed = smp["wall_per_iter"][a.warmup:]
    value, cpu = oracle_estimate(wl, smp, timed, wl["fp64_iterations_per_rhs"], nrhs,
                                 "the FP64 method's count on this workload, stored with the workload")
    line = {
        "impl": "reference", "metric": wl["metric"], "value": value, "unit": "s", "n_gpus": 0,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": statistics.mean(timed) * 1e3,
        "step": "one concurrent sample iteration (see cpu_baseline.sample); value is the scaled estimate",
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": wl_config(wl, a.workload, "fp64"), "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _oracle_kernel_worker(dims, eps, seed, barrier, q):
    """One process of the per-kernel study: one oracle D application and one
    Schwarz sweep (n_MR = 4) of one right-hand side on `dims`."""
    sys.path.insert(0, ROOT)
    from oracle.dirac import WilsonClover
    from oracle.sap import BlockDecomposition, sap_sweep
    op = WilsonClover(synth.random_gauge_field(dims, eps, 1), -0.5, 1.0)
    x = synth.random_spinor(dims, 2 + seed)
    bl = BlockDecomposition(dims, (4, 4, 4, 4))
    barrier.wait()
    t0 = time.perf_counter()
    op.apply(x)
    t1 = time.perf_counter()
    sap_sweep(op, bl, x, np.zeros_like(x), 4)
    t2 = time.perf_counter()
    q.put((seed, t1 - t0, t2 - t1))


def oracle_study(a):
    """The CPU oracle on the host cores (one JSON line per measurement): one D
    application and one Schwarz sweep at every lattice size, on one core and
    with one right-hand side per core in concurrent processes; then the whole
    two-level FP64 solve of the 8^4 workload on one core."""
    import multiprocessing as mp
    info = cpu_info()
    print(json.dumps({"oracle_study": "cpu", "mem_available": mem_available(), **info}), flush=True)
    ctx = mp.get_context("spawn")
    sizes = [(8, 8, 8, 8), (16, 16, 16, 16), (16, 16, 16, 32), (32, 32, 32, 64)]
    for dims in sizes:
        for procs in sorted({1, cpu_procs(12, oracle_bytes(dims))}):
            barrier = ctx.Barrier(procs)
            q = ctx.Queue()
            ps = [ctx.Process(target=_oracle_kernel_worker, args=(dims, 0.5, k, barrier, q)) for k in range(procs)]
            for p in ps:
                p.start()
            res = [q.get() for _ in ps]
            for p in ps:
                p.join()
            d = max(r[1] for r in res)
            sw = max(r[2] for r in res)
            v = int(np.prod(dims))
            print(json.dumps({"oracle_study": "kernels", "dims": list(dims), "processes": procs,
                              "dirac_s": d, "sweep_s": sw, "dirac_sites_per_s": procs * v / d,
                              "sweep_sites_per_s": procs * v / sw}), flush=True)
    from oracle.dirac import WilsonClover
    from oracle.mg import Multigrid
    wl = synth.workload("8^4")
    dims = tuple(wl["dims"])
    op = WilsonClover(synth.random_gauge_field(dims, wl["eps"], wl["gauge_seed"]), wl["m0"], wl["c_sw"])
    b = synth.random_spinor(dims, wl["rhs_seed"])
    t0 = time.perf_counter()
    mg = Multigrid(op, dict(n_levels=2, n_vec=tuple(wl["n_vec"]), setup_iters=wl["setup_iters"], n_mr=wl["n_mr"],
                            nu_post=wl["nu_post"], coarse_iters=wl["coarse_iters"], fgmres_m=wl["fgmres_m"],
                            tol=wl["tol"], sap_block=((4, 4, 4, 4),), agg=((4, 4, 4, 4),)),
                   synth.test_vector_draw(dims, wl["n_vec"][0], 1))
    t1 = time.perf_counter()
    z, it, hist, ok = mg.solve(b)
    t2 = time.perf_counter()
    rel = float(np.linalg.norm(b - op.apply(z)) / np.linalg.norm(b))
    print(json.dumps({"oracle_study": "solve", "workload": "8^4", "cores": 1, "setup_s": t1 - t0,
                      "solve_s": t2 - t1, "iterations": it, "relres": rel, "converged": bool(ok)}), flush=True)
    return 0


def wl_config(wl, name, precision):
    d = wl["dims"]
    return {"workload": f"{d[0]}^3x{d[3]}" if d[0] == d[1] == d[2] else name,
            "lattice": list(d), "eps": wl["eps"], "c_sw": wl["c_sw"], "m0": wl["m0"],
            "rhs": wl["rhs"], "levels": wl["n_levels"], "n_vec": list(wl["n_vec"]), "n_mr": wl["n_mr"],
            **({"inner_iters": wl["inner_iters"]} if "inner_iters" in wl else {}),
            "nu_post": wl["nu_post"], "coarse_iters": wl["coarse_iters"], "fgmres_m": wl["fgmres_m"],
            "tol": wl["tol"], "storage": precision, "parallelism": "replicas",
            "l2": "inputs larger than L2 (fields of several GB)"}


# ----------------------------------------------------------------------------- our arm
def learned_init(wl, u):
    """Initial test vectors for workloads with init='learned': the gauge-
    covariant network trained on seeded 16^4 fields of the workload's eps at
    its bare mass (the library's training kernels), then BF16 inference on the
    workload's field from seeded device noise.  Returns (vectors as complex128
    on the device, a record of the training and inference)."""
    import torch
    from paper_1202_2462_gb300 import learned
    net, losses, t_train = learned.train(wl["c_sw"], wl["m0"], eps_train=wl["eps"])
    g = torch.Generator(device="cuda")
    g.manual_seed(wl.get("vec_seed", 1))
    noise = torch.randn((wl["n_vec"][0],) + tuple(u.shape[:4]) + (4, 3), dtype=torch.complex64, device="cuda",
                        generator=g)
    prop, t_infer = learned.infer(net, u, wl["c_sw"], wl["m0"], noise)
    del noise
    torch.cuda.empty_cache()
    return prop, {"train_s": t_train, "inference_s": t_infer, "inference": "bf16",
                  "train_fields": 20, "train_lattice": [16, 16, 16, 16], "train_eps": wl["eps"],
                  "train_loss_first": float(sum(losses[:8]) / 8), "train_loss_last": float(sum(losses[-8:]) / 8)}


def e2e_run(torch, s, b_pinned, z_pinned, stream, steps, pipelined):
    """Seconds per step of `steps` solves through the public API, each copying
    its right-hand sides in from pinned host memory and its solutions back
    out.  pipelined: the copies run on a second stream, the next step's
    sources while this step solves and this step's solutions while the next
    one solves (the first step's sources and the last step's solutions still
    inside the timed region); else each step copies, solves and copies back
    in line."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if not pipelined:
        for _ in range(steps):
            bd = b_pinned.to("cuda", non_blocking=True)
            zd, _, _ = s.solve(bd)
            z_pinned.copy_(zd, non_blocking=True)
            torch.cuda.synchronize()
        return (time.perf_counter() - t0) / steps
    side = torch.cuda.Stream()
    bufs = [torch.empty(b_pinned.shape, dtype=b_pinned.dtype, device="cuda") for _ in range(2)]
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    with torch.cuda.stream(side):
        bufs[0].copy_(b_pinned, non_blocking=True)
        ready[0].record(side)
    for k in range(steps):
        stream.wait_event(ready[k % 2])
        if k + 1 < steps:                          # the next step's sources, while this one solves
            with torch.cuda.stream(side):
                bufs[(k + 1) % 2].copy_(b_pinned, non_blocking=True)
                ready[(k + 1) % 2].record(side)
        zd, _, _ = s.solve(bufs[k % 2])            # returns when the solve is done
        done = torch.cuda.Event()
        done.record(stream)
        side.wait_event(done)
        zd.record_stream(side)
        with torch.cuda.stream(side):              # this step's solutions, while the next one solves
            z_pinned.copy_(zd, non_blocking=True)
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) / steps


def run_ours(a, wl):
    import torch
    import paper_1202_2462_gb300 as G
    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dims = tuple(wl["dims"])
    prec = a.precision or wl["precision"]
    t0 = time.perf_counter()
    u_h = synth.random_gauge_field(dims, wl["eps"], wl["gauge_seed"])
    rhs_h = make_rhs(wl, dims)
    gen_s = time.perf_counter() - t0
    nrhs = rhs_h.shape[0]
    u = torch.from_numpy(u_h).cuda()
    stream = torch.cuda.current_stream()
    init, learned = None, None
    if wl.get("init") == "learned":
        init, learned = learned_init(wl, u)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = G.Solver(u, wl["c_sw"], wl["m0"], init_vectors=init, **solver_kwargs(wl, prec, nrhs))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    tuning = G.mg_get_tuning(s.ctx)
    del u, init
    torch.cuda.empty_cache()
    free_b, total_b = torch.cuda.mem_get_info()
    # the right-hand sides reach the device after the set-up, whose peak they would raise
    b = torch.from_numpy(rhs_h).cuda()
    b_pinned = torch.from_numpy(rhs_h).pin_memory()
    z_pinned = torch.empty_like(b_pinned).pin_memory()

    # warm-up steps, profiled per kernel family to find the dominant one
    G.mg_set_profiling(s.ctx, 1)
    infos = []
    for _ in range(a.warmup):
        z, info, code = s.solve(b)
        infos.append((info.iterations, info.relres, code))
    fam = {}
    for f, i in G.PROFILE_FAMILIES.items():
        n_f, ms_f = G.mg_get_profile(s.ctx, i)
        b_f = G.mg_get_profile_bytes(s.ctx, i)
        fam[f] = {"ms_per_step": ms_f / max(a.warmup, 1), "calls_per_step": n_f / max(a.warmup, 1),
                  "alg_gbs": (b_f / (ms_f / 1e3) / 1e9) if ms_f > 0 and b_f > 0 else None}
    fam_ms = {f: v["ms_per_step"] for f, v in fam.items()}
    dominant = max(fam_ms, key=fam_ms.get)
    G.mg_reset_profile(s.ctx)
    G.mg_set_profiling(s.ctx, G.profile_mask(dominant))

    # timed region: K steps, barrier + synchronize on both sides, CUDA events on the stream
    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        gpu_id = None
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(gpu_id)
    l0 = G.mg_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    # the timed region is also the profiler range (ncu --profile-from-start off captures only it)
    torch.cuda.profiler.start()
    ev0.record(stream)
    codes = []
    for _ in range(a.steps):
        z, info, code = s.solve(b)
        codes.append((info.iterations, info.relres, code, info.restarts))
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    if world > 1:
        torch.distributed.barrier()
    launches = G.mg_launch_count() - l0
    clk = clocks.stop()
    if a.history and rank == 0:
        # the last timed solve's residual history as JSON lines (one per entry, then rho per RHS)
        with open(a.history, "w") as f:
            for q, d in sorted(s.history().items()):
                for kind in ("estimates", "fp64"):
                    for it, r in d[kind]:
                        f.write(json.dumps({"rhs": q, "iteration": it, "relres": r, "kind": kind}) + "\n")
                f.write(json.dumps({"rhs": q, "rho": d["rho"], "kind": "convergence_factor"}) + "\n")
    ms = ev0.elapsed_time(ev1) / a.steps
    n_prof, ms_prof = G.mg_get_profile(s.ctx, G.PROFILE_FAMILIES[dominant])
    bytes_prof = G.mg_get_profile_bytes(s.ctx, G.PROFILE_FAMILIES[dominant])
    G.mg_set_profiling(s.ctx, 0)
    ms = max_over_ranks(ms, world, "cuda")

    # end to end through the public API with host buffers
    del z, b
    torch.cuda.empty_cache()
    e2e_steps = max(2, min(a.steps, 3))
    e2e_serial = e2e_run(torch, s, b_pinned, z_pinned, stream, e2e_steps, False)
    free_now = torch.cuda.mem_get_info()[0]
    pipelined = free_now > 4 * b_pinned.numel() * 16                # two input buffers and two solutions
    e2e_s = e2e_run(torch, s, b_pinned, z_pinned, stream, e2e_steps, True) if pipelined else e2e_serial

    # Dirac-apply GB/s (storage precision of the smoother, blocked layout)
    v = dims[0] * dims[1] * dims[2] * dims[3]
    x = torch.randn((v * 12,), dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    pd = G.PRECISIONS[prec] | G.MG_BLOCKED
    for _ in range(3):
        G.dirac_apply(s.ctx, x, y, pd, 1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 20
    e0.record(stream)
    for _ in range(reps):
        G.dirac_apply(s.ctx, x, y, pd, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    dirac_s = e0.elapsed_time(e1) / reps / 1e3
    dirac_gbs = bytes_dirac_site(prec) * v / dirac_s / 1e9
    s.close()

    hbm, peak_kind = load_peaks()
    f32, f32x2, smem = G.mg_probe_peaks(stream)
    probe = {"fp32_tflops_scalar_fma": f32, "fp32_tflops_packed_fma": f32x2, "smem_gbs": smem,
             "how": "mg_probe_peaks: independent FMA chains and conflict-free 16-byte shared loads on every SM"}
    if dominant == "sap":
        # one launch = one colour pass over V/2 sites for every right-hand side
        units = (v // 2) * nrhs
        avg_s = ms_prof / max(n_prof, 1) / 1e3
        tflops = flops_sap_site(wl["n_mr"]) * units / avg_s / 1e12 if n_prof else None
        alg_bytes = (v // 2) * (nrhs * bytes_sap_spinor(prec) + bytes_sap_fields(prec))
        shape = tuning["sap_shape"] if nrhs % 2 == 0 else -1
        per_unit = SAP_DRAM_BYTES_PER_UNIT.get(shape) if prec == "bf16" else None
        roof = {"kernel": SAP_KERNEL[shape], "bound": "alu", "achieved": tflops, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": tflops / FP32_PEAK_TFLOPS if tflops else None,
                "traffic": per_unit * units if per_unit else None,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one colour pass of a "
                                  "12-RHS case with this launch shape (16^3x32, or 32^3x32 for shape 5), per site "
                                  "and RHS, scaled to this launch's units",
                "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                "peak_probe": probe,
                "hbm_gbs": alg_bytes / avg_s / 1e9 if n_prof else None,
                "hbm_frac": alg_bytes / avg_s / 1e9 / hbm if n_prof else None,
                "launches": n_prof, "avg_launch_ms": avg_s * 1e3, "sites_x_rhs_per_launch": units,
                "flop_per_site": flops_sap_site(wl["n_mr"]), "alg_bytes_per_launch": alg_bytes}
    else:
        avg_s = ms_prof / max(n_prof, 1) / 1e3
        gbs = bytes_prof / (ms_prof / 1e3) / 1e9 if ms_prof > 0 and bytes_prof > 0 else None
        roof = {"kernel": FAMILY_KERNELS.get(dominant, dominant), "bound": "hbm", "achieved": gbs, "peak": hbm,
                "unit": "GB/s", "frac": gbs / hbm if gbs else None, "traffic": None, "launches": n_prof,
                "avg_launch_ms": avg_s * 1e3, "alg_bytes_per_launch": bytes_prof / max(n_prof, 1)}

    iters = [c[0] for c in codes]
    line = {
        "metric": wl["metric"], "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": wl_config(wl, a.workload, prec),
        "iterations_per_step": iters, "restarts_per_step": [c[3] for c in codes],
        "relres": max(c[1] for c in codes), "status": [c[2] for c in codes], "rhs_per_step": nrhs * world,
        "setup_s": setup_s, "input_generation_s": gen_s, "tuning": tuning,
        "dirac_apply": {"storage": prec, "gbs": dirac_gbs, "frac_of_measured_hbm": dirac_gbs / hbm,
                        "frac_of_8tbs": dirac_gbs / 8000.0, "us": dirac_s * 1e6},
        "families_warmup": fam, "roofline": roof, "peak_hbm_gbs": hbm, "peak_kind": peak_kind,
        "clocks": clk, "gpu_launches": launches,
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(b_pinned.numel() * 16),
                "d2h_bytes_per_step": int(z_pinned.numel() * 16), "steps": e2e_steps,
                "copies": ("each step's sources in and solutions out on a second stream, overlapping the "
                           "neighbouring steps' solves" if pipelined else "in line with the solves"),
                "value_copies_in_line": e2e_serial},
    }
    line["device_memory_gb"] = {"in_use_after_setup": (total_b - free_b) / 1e9, "total": total_b / 1e9}
    if learned:
        line["learned_setup"] = learned
    if wl.get("nrhs_max", nrhs) < nrhs:
        line["config"]["rhs_batch"] = wl["nrhs_max"]
    if a.fp64_form and rank == 0:
        line["fp64_form"] = fp64_form(a, wl, u_h, rhs_h)
    if rank == 0 and world == 1 and not a.no_cpu:
        f64 = line.get("fp64_form")
        if f64:
            it_rhs, src = f64["iterations_per_rhs"], "this run's FP64 form"
        else:
            it_rhs, src = statistics.mean(iters) / nrhs, "this run's mixed form (the FP64 form was not run)"
        smp = oracle_sample(wl, 3, cpu_procs(nrhs, oracle_bytes(sample_dims(wl), wl["n_vec"][0])))
        line["cpu_baseline"] = oracle_estimate(wl, smp, smp["wall_per_iter"][1:], it_rhs, nrhs, src)[1]
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def fp64_form(a, wl, u_h, rhs_h):
    """Time-to-solution of the plain FP64 form (same method, FP64 everywhere,
    one right-hand side at a time): the first `--fp64-rhs` right-hand sides
    (default all) solved and timed one after the other; s_all_rhs is their sum
    scaled to all right-hand sides when fewer were measured."""
    import torch
    import paper_1202_2462_gb300 as G
    u = torch.from_numpy(u_h).cuda()
    kw = solver_kwargs(wl, "fp64", 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = G.Solver(u, wl["c_sw"], wl["m0"], **kw)
    torch.cuda.synchronize()
    setup = time.perf_counter() - t0
    del u
    n_all = rhs_h.shape[0]
    n = n_all if a.fp64_rhs is None else max(1, min(a.fp64_rhs, n_all))
    total, its, rel, codes = 0.0, [], 0.0, []
    for r in range(n):
        b = torch.from_numpy(rhs_h[r:r + 1]).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        z, info, code = s.solve(b)
        torch.cuda.synchronize()
        total += time.perf_counter() - t0
        its.append(info.iterations)
        rel = max(rel, info.relres)
        codes.append(code)
    s.close()
    return {"setup_s": setup, "s_measured": total, "s_all_rhs": total * n_all / n, "rhs_measured": n,
            "iterations": its, "iterations_per_rhs": statistics.mean(its), "relres": rel, "status": codes}


def run_cgn(a, wl):
    """The comparison of Sec. 4 (Tables 1-2) on this workload: the multilevel
    solve (set-up, one warm-up solve, one timed solve) against CG on the normal
    equations (CGN) for the same right-hand sides, FP32 iteration with FP64
    updates in the same context, and, with --cgn-fp64, CGN in FP64 on the
    first right-hand side (x nrhs for the whole set).  Prints one JSON line
    per part."""
    import torch
    import paper_1202_2462_gb300 as G
    torch.cuda.set_device(0)
    dims = tuple(wl["dims"])
    prec = a.precision or wl["precision"]
    u_h = synth.random_gauge_field(dims, wl["eps"], wl["gauge_seed"])
    rhs_h = make_rhs(wl, dims)
    nrhs = rhs_h.shape[0]
    u = torch.from_numpy(u_h).cuda()
    b = torch.from_numpy(rhs_h).cuda()
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) / 1e3

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = G.Solver(u, wl["c_sw"], wl["m0"], **solver_kwargs(wl, prec, nrhs))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    s.solve(b)
    (z, info, code), mg_s = timed(lambda: s.solve(b))
    mg = {"s": mg_s, "setup_s": setup_s, "iterations_per_rhs": info.iterations / nrhs, "relres": info.relres,
          "status": code}
    tol, cap = wl["tol"], 20000
    s.cgn_solve(b, tol=tol, maxiter=1, prec=G.MG_FP32)        # workspace allocation and first launches
    (z, info, code), cgn_s = timed(lambda: s.cgn_solve(b, tol=tol, maxiter=cap, prec=G.MG_FP32))
    cgn32 = {"s": cgn_s, "iterations_per_rhs": info.iterations / nrhs, "fp64_updates": info.restarts,
             "relres": info.relres, "status": code}
    sigma = None
    if a.sigma:
        from paper_1202_2462_gb300.tune import sigma_min
        sigma = sigma_min(s, s.lat + (4, 3), iters=8)[-1]
    s.close()
    out = {"metric": "time to solution, multilevel vs CGN (Sec. 4, Tables 1-2)", "workload": a.workload,
           "sigma_min": sigma,
           "nrhs": nrhs, "tol": tol, "m0": wl["m0"], "mg_mixed": mg, "cgn_fp32_fp64_updates": cgn32,
           "solve_speedup": cgn_s / mg_s, "speedup_with_setup": cgn_s / (mg_s + setup_s), "data": "synthetic"}
    print(json.dumps(out), flush=True)
    if a.cgn_fp64:
        p = G.Solver(u, wl["c_sw"], wl["m0"], n_levels=1, precision="fp64", nrhs_max=1, fgmres_m=2)
        b1 = b[:1].contiguous()
        p.cgn_solve(b1, tol=tol, maxiter=1)
        (z, info, code), t1 = timed(lambda: p.cgn_solve(b1, tol=tol, maxiter=cap))
        p.close()
        print(json.dumps({"cgn_fp64": {"s_per_rhs": t1, "s_all_rhs": t1 * nrhs, "iterations": info.iterations,
                                       "relres": info.relres, "status": code, "rhs_measured": 1}}), flush=True)
    return 0


def run_kernel(a, wl):
    """One kernel family of the path alone at the workload's lattice size
    (inputs resident on the device, blocked layout, 3 warm-up and --steps
    timed launches, CUDA events on the library's stream): 'dirac' applies D
    (storage precision of the workload) to --nrhs right-hand sides, 'sap' runs
    one Schwarz sweep (two colour passes) on them.  Prints one JSON line with
    the time per launch and the algorithmic bytes and flops behind it; the
    process launches nothing else in between, so it is the target of the
    profiles of these kernels."""
    import torch
    import paper_1202_2462_gb300 as G
    torch.cuda.set_device(0)
    dims = tuple(wl["dims"])
    prec = a.precision or wl["precision"]
    nrhs = a.nrhs
    u = torch.from_numpy(synth.random_gauge_field(dims, wl["eps"], wl["gauge_seed"])).cuda()
    s = G.Solver(u, wl["c_sw"], wl["m0"], n_levels=1, precision=prec, nrhs_max=nrhs, n_mr=wl["n_mr"], fgmres_m=1)
    del u
    v = int(np.prod(dims))
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    x = torch.randn((nrhs * v * 12, 2), device="cuda", generator=g).view(torch.complex64).reshape(-1)
    y = torch.zeros_like(x)
    pd = G.PRECISIONS[prec] | G.MG_BLOCKED
    stream = torch.cuda.current_stream()
    if a.kernel == "dirac":
        launch = lambda: G.dirac_apply(s.ctx, x, y, pd, nrhs)
        per_launch = 1
        alg = v * (nrhs * 2 * 12 * 8 + bytes_sap_fields(prec))
        flop = v * nrhs * flops_dirac_site()
    else:
        launch = lambda: G.sap_smooth(s.ctx, x, y, 1, pd, nrhs)
        per_launch = 2                                   # two colour passes per sweep
        alg = (v // 2) * (nrhs * bytes_sap_spinor(prec) + bytes_sap_fields(prec))
        flop = (v // 2) * nrhs * flops_sap_site(wl["n_mr"])
    for _ in range(3):
        launch()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(a.steps):
        launch()
    e1.record(stream)
    torch.cuda.synchronize()
    G.mg_sync(s.ctx)
    t = e0.elapsed_time(e1) / 1e3 / (a.steps * per_launch)
    hbm, kind = load_peaks()
    out = {"kernel": a.kernel, "workload": a.workload, "lattice": list(dims), "storage": prec, "nrhs": nrhs,
           "launches_timed": a.steps * per_launch, "ms_per_launch": t * 1e3,
           "alg_bytes_per_launch": alg, "alg_gbs": alg / t / 1e9, "hbm_frac": alg / t / 1e9 / hbm,
           "flop_per_launch": flop, "tflops": flop / t / 1e12, "peak_hbm_gbs": hbm, "peak_kind": kind,
           "sap_shape": os.environ.get("SAPMG_SAP_SHAPE", "default")}
    s.close()
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="32^3x64")
    ap.add_argument("--precision", default=None)
    ap.add_argument("--fp64-form", dest="fp64_form", action="store_true", default=True)
    ap.add_argument("--no-fp64-form", dest="fp64_form", action="store_false")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--kernel", choices=["dirac", "sap"], default=None,
                    help="instead of the bench line: time one kernel family alone (see run_kernel)")
    ap.add_argument("--nrhs", type=int, default=1, help="with --kernel: right-hand sides per launch")
    ap.add_argument("--history", default=None,
                    help="write the last timed solve's residual history to this file as JSON lines")
    ap.add_argument("--oracle-study", action="store_true",
                    help="instead of the bench line: oracle kernel timings at every size and the 8^4 oracle solve")
    ap.add_argument("--fp64-rhs", type=int, default=None,
                    help="right-hand sides the FP64 form solves and times (default: all)")
    ap.add_argument("--cgn", action="store_true",
                    help="instead of the bench line: the multilevel solve against CG on the normal equations")
    ap.add_argument("--cgn-fp64", action="store_true", help="with --cgn: also CGN in FP64 on one right-hand side")
    ap.add_argument("--m0", type=float, default=None, help="bare mass instead of the workload's")
    ap.add_argument("--sigma", action="store_true",
                    help="with --cgn: also sigma_min(D) by inverse iteration (16 solves of one right-hand side)")
    a = ap.parse_args()
    wl = synth.workload(a.workload)
    if a.m0 is not None:
        wl["m0"] = a.m0
    if a.oracle_study:
        return oracle_study(a)
    if a.kernel:
        return run_kernel(a, wl)
    if a.impl == "reference":
        return run_reference(a, wl)
    if a.cgn:
        return run_cgn(a, wl)
    return run_ours(a, wl)


if __name__ == "__main__":
    sys.exit(main())
