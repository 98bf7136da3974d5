#!/usr/bin/env python
"""Benchmark of the GMRES-GMG space-time solver (arXiv 2303.06742) on GB300.

Metric: slab solves per second (with p50/p99 latency per slab solve) of the
march of a 2D 64x64 Q3/Q2 dG(2) problem (5 GMG levels, tau = 1e-3, lognormal
per-cell permeability, log-uniform Lame parameters, c0 = 1e-2), solved to a
relative residual of 1e-8 with the FP32 V-cycle inside FP64 flexible GMRES;
the plain FP64 path is measured beside it.  One step = one slab of the march:
right-hand side assembly plus a full FGMRES-GMG solve (all hot-path steps).
The GMG hierarchy and patch inverses are built once before the timed region
and stay resident (setup time is reported separately).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Multi-GPU: independent replicas, one instance per rank, no collective on the
data path ("scaling": "weak").
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "c2_2d_q3_k2_64"
WORKLOAD_DESCS = {
    "c2_2d_q3_k2_64": ("2D unit square 64x64, 5 GMG levels, Q3^2/Q2 Taylor-Hood, dG(2) (3 Radau nodes), "
                       "tau=1e-3, lambda/mu log-uniform [0.5,50], kappa lognormal per cell (sigma=1), c0=1e-2, "
                       "alpha=1, manufactured sine solution, Dirichlet (Nitsche) on all faces; "
                       "N_slab=496,911; FGMRES(30) to 1e-8 relative"),
    "c3_3d_q2_k1_16": ("3D unit cube 16^3, 4 GMG levels, Q2^3/Q1 Taylor-Hood, dG(1), tau=1e-2, thermoelastic "
                       "set (alpha=0.5, c0=1, kappa=0.1, lambda=2, mu=1), manufactured sine solution, Dirichlet "
                       "on all faces; N_slab=441,070; one right-hand side; FGMRES(30) to 1e-8 relative"),
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--sweeps", type=int, default=1, help="pre- and post-smoothing sweeps per level")
    p.add_argument("--requests", type=int, default=64, help="requests of the serving workload")
    p.add_argument("--workers", type=int, default=8, help="concurrent requests of the serving workload")
    p.add_argument("--batched", action="store_true",
                   help="serving: lockstep groups with fused smoother launches (continuous batching)")
    p.add_argument("--members", type=int, default=16, help="serving, batched: most members of a group")
    p.add_argument("--rhs", type=int, default=1,
                   help="right-hand sides solved together (marches from t0 = 0, 0.1, ...): >1 times the "
                        "batched path with the tensor-core patch apply")
    p.add_argument("--form", default="3.1", choices=["3.1", "B.1"],
                   help="slab problem: Problem 3.1 (default) or Problem B.1 of Appendix B")
    p.add_argument("--pressure", default="continuous", choices=["continuous", "broken"],
                   help="pressure space: Taylor-Hood Q_{r-1} (default) or the broken pair's P_{r-1}^disc "
                        "with the interior penalty form")
    p.add_argument("--fine-operator", default="auto", choices=["auto", "assembled", "matrix-free"],
                   help="operator of the finest level inside the mixed-precision V-cycle")
    p.add_argument("--stream-shapes", default=None,
                   help="pin the streaming patch apply's shape per level, 'level:stages,ctas_per_sm,tile;...' "
                        "(default: the setup's autotuned shapes, printed in the roofline object)")
    p.add_argument("--tc-shapes", default=None,
                   help="with --rhs > 1: pin the tensor-core patch apply's shape per level, "
                        "'level:split,deep;...' (default: the setup's autotuned shapes, printed in the "
                        "roofline object)")
    p.add_argument("--cpu-leg", default=None, help=argparse.SUPPRESS)
    return p.parse_args()


# ------------------------------------------------------------------ oracle legs
def oracle_leg(workload, out_path, mode, steps=0, warmup=0, form="3.1", pressure="continuous"):
    """Runs the oracle (test infrastructure) in this process on the host cores.

    mode "solve": set up, time one full slab solve (slab 0), save the solution.
    mode "reference": set up, one full solve for the iteration count, then
    `warmup`+`steps` samples of two FGMRES iterations each.
    """
    import numpy as np
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import inputs
    from _cases import oracle_instance
    from oracle.slab import repeat_state
    c = inputs.case(workload)
    t0 = time.perf_counter()
    O = oracle_instance(c, form=form, pressure="disc" if pressure == "broken" else "cont")
    t_setup = time.perf_counter() - t0
    st0 = O.initial_state()
    b = O.rhs(0, st0)
    x0 = repeat_state(O.ops, O.tmp, st0)
    t0 = time.perf_counter()
    c0 = time.process_time()
    x, it, rel, _ = O.solve(b, x0, c["tol"])
    t_solve = time.perf_counter() - t0
    cpu_s = time.process_time() - c0
    res = dict(setup_s=t_setup, solve_s=t_solve, iters=it, rel=rel, cpu_s=cpu_s,
               threads_used=cpu_s / max(t_solve, 1e-9))
    if mode == "solve":
        np.save(out_path + ".npy", x)
    else:
        samples, steps_s = [], []
        for i in range(warmup + steps):
            t0 = time.perf_counter()
            O.solve(b, x0, 0.0, restart=30, max_it=2)
            if i >= warmup:
                steps_s.append(time.perf_counter() - t0)
                samples.append(steps_s[-1] / 2.0)
        res["per_iter_s"] = samples
        res["step_s"] = steps_s
    with open(out_path, "w") as f:
        json.dump(res, f)


def host_cpu():
    """(logical cores, CPU model) of the host the oracle runs on."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    return os.cpu_count() or 1, model


def run_oracle_subprocess(workload, mode, steps=0, warmup=0, form="3.1", threads=1, pressure="continuous"):
    """The oracle in a subprocess with `threads` BLAS/OpenMP threads (the
    oracle's library calls are the only parallel part of it)."""
    fd, path = tempfile.mkstemp(suffix=".json")
    os.close(fd)
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-leg", path, "--workload", workload,
           "--steps", str(steps), "--warmup", str(warmup), "--impl", "reference" if mode == "reference" else "ours",
           "--form", form, "--pressure", pressure]
    subprocess.run(cmd, check=True, env=env)
    with open(path) as f:
        res = json.load(f)
    os.unlink(path)
    sol = None
    if os.path.exists(path + ".npy"):
        import numpy as np
        sol = np.load(path + ".npy")
        os.unlink(path + ".npy")
    return res, sol


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, t0, t1):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, watts = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = [l for ts, l in self.lines if t0 - 0.25 <= ts <= t1 + 0.25] or [l for _, l in self.lines]
        for line in rows:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            try:
                watts.append(float(parts[2]))
            except ValueError:
                pass
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w": statistics.median(watts) if watts else None}


def energy_per_step(clk, ms_per_step):
    """Board energy per step: the median board power sampled during the timed
    region times the device time of a step (the GPU analogue of the paper's
    energy figures; coarse when the region holds few 200 ms samples)."""
    w = clk.get("power_w")
    if w is None:
        return None
    return {"j_per_step": w * ms_per_step / 1000.0, "power_w": w, "samples": clk.get("samples"),
            "method": "median nvidia-smi power.draw of this rank's GPU during the timed region x device time "
                      "per step"}


# ------------------------------------------------------------------ helpers
def peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the patch-apply kernels' source (the bulk-copy helpers and the
    streaming kernel, up to the next section of stfem.cu, and the wide kernel
    of vanka.cuh): the committed DRAM traffic is used only while this source is
    unchanged."""
    csrc = os.path.join(ROOT, "paper_2303_06742_gb300", "csrc")
    with open(os.path.join(csrc, "stfem.cu"), "rb") as f:
        src = f.read()
    a = src.index(b"// ---------------------------------------------------------------- bulk-copy streaming")
    b = src.index(b'#include "tc_patch.cuh"', a)
    with open(os.path.join(csrc, "vanka.cuh"), "rb") as f:
        van = f.read()
    c = van.index(b"// Time-diagonal patch apply for levels with few patches")
    d = van.index(b"// d = (zero ? 0 : d) + scale * sum of the patch results holding each dof.", c)
    return hashlib.sha256(src[a:b] + van[c:d]).hexdigest()[:16]


def dram_traffic(workload, precision, pressure="continuous"):
    """Per-launch DRAM bytes of the patch-apply kernel from the committed ncu
    summary of this workload and pressure space, if it was taken on the
    current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "traffic_k_patch_apply_stream_%s.json" % workload)
    try:
        with open(p) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    key = "%s/%s/patch_apply" % (workload, precision if pressure == "continuous" else precision + "-broken")
    r = rec.get(key)
    if not r or r.get("source_hash") != kernel_source_hash():
        return None
    return r.get("bytes_per_launch")


def tc_source_hash():
    """Hash of the tensor-core patch apply's source (tc_patch.cuh)."""
    with open(os.path.join(ROOT, "paper_2303_06742_gb300", "csrc", "tc_patch.cuh"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def dram_traffic_tc(workload, nb):
    """Per-launch DRAM bytes of the tensor-core patch apply with nb columns from
    the committed ncu summary, if it was taken on the current kernel source;
    else None."""
    p = os.path.join(ROOT, "profiles", "traffic_k_patch_apply_tc_%s.json" % workload)
    try:
        with open(p) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    r = rec.get("%s/tc%d/patch_apply" % (workload, nb))
    if not r or r.get("source_hash") != tc_source_hash():
        return None
    return r.get("bytes_per_launch")


def job_throughput(units_per_rank, total_ms, world, dist=None, device="cuda"):
    """Whole-job throughput of independent replicas: every rank processed
    units_per_rank units in its own total_ms; the job took the slowest rank's
    time, so value = units_per_rank * world / max over ranks of the time.
    Returns (value in units/s, the max time in ms).  The only collective is
    this one MAX reduction of a timing scalar; the solves exchange nothing."""
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return units_per_rank * world / (total_ms / 1000.0), total_ms


def pct(vals, q):
    v = sorted(vals)
    if not v:
        return None
    i = min(len(v) - 1, max(0, int(round(q / 100.0 * (len(v) - 1)))))
    return v[i]


# ------------------------------------------------------------------ GPU arm
FINE_OPERATORS = {"auto": 0, "assembled": 1, "matrix-free": 2}


def make_solver(c, precision, stream, sweeps=1, form="3.1", fine_operator="auto", pressure="continuous"):
    import paper_2303_06742_gb300 as st
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from _cases import gpu_problem
    f = st.FORM_PROBLEM_B_1 if form == "B.1" else st.FORM_PROBLEM_3_1
    pr = st.PRESSURE_BROKEN if pressure == "broken" else st.PRESSURE_CONTINUOUS
    return st.Solver(gpu_problem(c, form=f, pressure=pr), precision=precision, stream=stream, n_sweeps=sweeps,
                     fine_operator=FINE_OPERATORS[fine_operator])


def time_march(S, torch, stream, state, first, steps, tol, profile=False):
    """Marches `steps` slabs one by one; returns per-step device ms, iterations."""
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    iters = []
    if profile:
        S.profile(True)
    with torch.cuda.stream(stream):
        evs[0].record(stream)
        for i in range(steps):
            rc, it = S.march(first + i, 1, state, tol=tol)
            if rc != 0:
                raise RuntimeError("march returned %d at slab %d" % (rc, first + i))
            iters.append(it[0])
            evs[i + 1].record(stream)
    stream.synchronize()
    ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(steps)]
    return ms, iters


def gpu_arm(args):
    import numpy as np
    import torch
    import paper_2303_06742_gb300 as st
    import inputs
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    c = inputs.case(args.workload)
    tol = c["tol"]
    stream = torch.cuda.Stream()
    K, W = args.steps, args.warmup

    # ---- mixed precision (headline)
    t0 = time.perf_counter()
    S = make_solver(c, st.MIXED, stream, args.sweeps, args.form, args.fine_operator, args.pressure)
    setup_s = time.perf_counter() - t0
    if args.stream_shapes:
        for item in args.stream_shapes.split(";"):
            lev, shape = item.split(":")
            S.set_stream_shape(int(lev), *[int(v) for v in shape.split(",")])
    shapes = {str(l): list(S.stream_shape(l)) for l in range(1, S.n_levels)}
    state = torch.zeros(S.n_state, dtype=torch.float64, device="cuda")
    S.initial_state(state)
    # slab 0 solution for the error against the oracle
    x_slab0 = None
    with torch.cuda.stream(stream):
        rhs0 = torch.zeros(S.n_slab, dtype=torch.float64, device="cuda")
        S.slab_rhs(0, state, rhs0)
        x_slab0 = state.repeat(S.prob.q)
        rc0, it0, rel0 = S.slab_solve(rhs0, x_slab0, tol=tol)
    stream.synchronize()
    x_slab0_host = x_slab0.cpu().numpy()
    launches0 = S.launch_count()
    time_march(S, torch, stream, state, 0, W, tol)
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    tw0 = time.time()
    l0 = S.launch_count()
    ms, iters = time_march(S, torch, stream, state, W, K, tol)
    torch.cuda.synchronize()
    launches = S.launch_count() - l0
    tw1 = time.time()
    total_ms = sum(ms)
    clk = clocks.stop(tw0, tw1)
    # second pass of the march with per-launch events (eager launches) for
    # the per-kernel breakdown and the roofline of the patch apply
    KP = min(K, 5)
    _, _ = time_march(S, torch, stream, state, W + K, KP, tol, profile=True)
    prof = S.profile_read()
    S.profile(False)
    value, total_ms = job_throughput(K, total_ms, world, dist)

    # ---- end to end through the public call with host buffers
    E = min(K, 5)
    n = S.n_slab
    rhs_h = torch.empty(n, dtype=torch.float64, pin_memory=True)
    x0_h = torch.empty(n, dtype=torch.float64, pin_memory=True)
    x_h = torch.empty(n, dtype=torch.float64, pin_memory=True)
    with torch.cuda.stream(stream):
        rd = torch.zeros(n, dtype=torch.float64, device="cuda")
        S.slab_rhs(W + K + KP, state, rd)
        rhs_h.copy_(rd)
        x0_h.copy_(state.repeat(S.prob.q))
    stream.synchronize()
    rhs_d = torch.empty(n, dtype=torch.float64, device="cuda")
    x_d = torch.empty(n, dtype=torch.float64, device="cuda")
    e_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        e_ev[0].record(stream)
        for _ in range(E):
            rhs_d.copy_(rhs_h, non_blocking=True)
            x_d.copy_(x0_h, non_blocking=True)
            S.slab_solve(rhs_d, x_d, tol=tol)
            x_h.copy_(x_d, non_blocking=True)
        e_ev[1].record(stream)
    stream.synchronize()
    e2e_ms = e_ev[0].elapsed_time(e_ev[1])
    e2e_value = E * world / (e2e_ms / 1000.0)
    info = {l: S.level_info(l) for l in range(c["levels"])}
    S.close()

    # ---- plain FP64 path beside it
    fp64 = None
    if not args.no_fp64:
        t0 = time.perf_counter()
        S64 = make_solver(c, st.FP64, stream, args.sweeps, args.form, pressure=args.pressure)
        setup64 = time.perf_counter() - t0
        st64 = torch.zeros(S64.n_state, dtype=torch.float64, device="cuda")
        S64.initial_state(st64)
        K64 = min(K, 5)
        time_march(S64, torch, stream, st64, 0, min(W, 2), tol)
        ms64, it64 = time_march(S64, torch, stream, st64, min(W, 2), K64, tol)
        fp64 = {"value": K64 / (sum(ms64) / 1000.0), "unit": "slab solves/s", "steps": K64,
                "p50_ms": pct(ms64, 50), "p99_ms": pct(ms64, 99), "iters_per_slab": it64, "setup_s": setup64}
        S64.close()

    if rank != 0:
        return
    # ---- roofline of the dominant kernel (patch-inverse apply)
    pa = prof["patch_apply"]
    peak, peak_kind = peak_hbm()
    achieved = pa["bytes"] / (pa["ms"] / 1000.0) / 1e9 if pa["ms"] > 0 else None
    traffic = dram_traffic(args.workload, "mixed", args.pressure)
    roof = {"kernel": "patch apply: k_patch_apply_stream<float> (levels with more than one patch per SM), "
                      "k_patch_apply_wide<float> (the others)",
            "workload": args.workload, "bound": "hbm", "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak if achieved else None, "peak_source": peak_kind,
            "traffic": traffic,
            "algorithmic_bytes_per_launch": pa["bytes"] / max(pa["launches"], 1),
            "avg_launch_ms": pa["ms"] / max(pa["launches"], 1), "launches": pa["launches"],
            "measured": "per-launch CUDA events on the solver stream over %d profiled slabs after the timed "
                        "region (same kernels, eager launches)" % KP,
            "stream_shapes": shapes}
    breakdown = {k: {"ms": v["ms"], "share": v["ms"] / max(sum(x["ms"] for x in prof.values()), 1e-30),
                     "launches": v["launches"],
                     "gbs": (v["bytes"] / (v["ms"] / 1000.0) / 1e9) if v["ms"] > 0 else None}
                 for k, v in prof.items()}

    # ---- oracle on the host cores (bounded sample: one slab solve)
    cpu = None
    err_vs_oracle = None
    if not args.no_cpu_baseline:
        nproc, model = host_cpu()
        res, sol = run_oracle_subprocess(args.workload, "solve", form=args.form, pressure=args.pressure)
        cpu = {"value": 1.0 / res["solve_s"], "unit": "slab solves/s", "cores": 1, "kind": "oracle",
               "nproc": nproc, "cpu_model": model,
               "sample": "one full slab solve (slab 0, FGMRES-GMG to %g, %d iterations) of the same workload; "
                         "oracle setup (%.1f s) excluded as on the GPU; BLAS/OpenMP threads pinned to 1"
                         % (tol, res["iters"], res["setup_s"])}
        if sol is not None:
            err_vs_oracle = float(np.abs(x_slab0_host - sol).max() / np.abs(sol).max())
        # the same oracle with its library calls free to use every host core
        resa, _ = run_oracle_subprocess(args.workload, "solve", form=args.form, threads=nproc,
                                        pressure=args.pressure)
        cpu["all_cores"] = {
            "value": 1.0 / resa["solve_s"], "unit": "slab solves/s", "cores": round(resa["threads_used"], 2),
            "threads_allowed": nproc, "nproc": nproc, "cpu_model": model, "kind": "oracle",
            "sample": "the same slab solve with BLAS/OpenMP threads = nproc; cores = process CPU time / wall "
                      "time of the solve (the oracle's sparse products and patch loops are single-threaded, "
                      "only its dense library calls use more cores)"}

    out = {
        "metric": "slab solves/s",
        "value": value,
        "unit": "slab solves/s",
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": total_ms / K,
        "p50_ms": pct(ms, 50),
        "p99_ms": pct(ms, 99),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": bench_config(args, world),
        "precision": "FP32 V-cycle inside FP64 FGMRES",
        "levels": info,
        "inverse_bytes_per_sweep_set": sum(v["inv_bytes"] for v in info.values()),
        "iters_per_slab": iters,
        "first_slab": {"iters": it0, "rel_res": rel0, "err_vs_fp64_oracle": err_vs_oracle},
        "setup_s": setup_s,
        "roofline": roof,
        "breakdown": breakdown,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "slab solves/s", "steps": E,
                "h2d_bytes_per_step": 2 * n * 8, "d2h_bytes_per_step": n * 8},
        "fp64": fp64,
        "speedup_mixed_vs_fp64": (value / world) / fp64["value"] if fp64 else None,
        "gpu_launches": launches,
        "clocks": clk,
        "energy": energy_per_step(clk, total_ms / K),
    }
    print(json.dumps(out))


def bench_config(args, world):
    """The `config` of the JSON line: the workload, identical for both arms."""
    import inputs
    c = inputs.case(args.workload)
    cfg = {"workload": WORKLOAD_DESCS.get(args.workload, args.workload), "form": "Problem %s" % args.form,
           "tol": c["tol"], "restart": 30, "omega": 0.7, "sweeps": args.sweeps,
           "l2": "inputs larger than L2: the patch inverses streamed per sweep set exceed the 129 MB L2",
           "parallelism": "replicas" if world > 1 else "single"}
    if args.pressure == "broken":
        cfg["pressure_space"] = "broken P_{r-1}^disc with the interior penalty form (instead of Q_{r-1})"
    return cfg


# ------------------------------------------------------------------ reference arm
def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import inputs
    c = inputs.case(args.workload)
    res, _ = run_oracle_subprocess(args.workload, "reference", steps=args.steps, warmup=args.warmup,
                                   form=args.form, pressure=args.pressure)
    per_iter = res["per_iter_s"]
    iters = res["iters"]
    t_slab = statistics.mean(per_iter) * iters
    value = 1.0 / t_slab
    samples_ms = [p * iters * 1000.0 for p in per_iter]
    nproc, model = host_cpu()
    out = {
        "impl": "reference",
        "metric": "slab solves/s",
        "value": value,
        "unit": "slab solves/s",
        "n_gpus": 0,
        "steps": args.steps,
        "warmup": args.warmup,
        # the timed steps themselves: each is a bounded sample (two FGMRES-GMG
        # iterations); `value` scales the mean iteration time to a slab solve
        "ms_per_step": statistics.mean(res["step_s"]) * 1000.0,
        "ms_per_slab_solve": t_slab * 1000.0,
        "p50_ms": pct(samples_ms, 50),
        "p99_ms": pct(samples_ms, 99),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": bench_config(args, 1),
        "precision": "FP64 (oracle)",
        "cpu_baseline": {"value": value, "unit": "slab solves/s", "cores": 1, "kind": "oracle",
                         "nproc": nproc, "cpu_model": model,
                         "sample": "each step: 2 FGMRES-GMG iterations of slab 0 (ms_per_step); value = 1 / "
                                   "(mean iteration time x the %d iterations of a full slab solve, whose time is "
                                   "ms_per_slab_solve); oracle setup (%.1f s) excluded" % (iters, res["setup_s"])},
        "e2e": {"value": value, "unit": "slab solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


# ------------------------------------------------------------------ batched right-hand sides
def batch_arm(args):
    """n_rhs marches of the workload's operator (data phases t0 = 0.1 c) solved
    together: one step = one slab of every march (n_rhs slab solves), through
    march_batch with the tensor-core patch apply.  The same marches solved
    one after another on the single-column path are timed beside it."""
    import numpy as np
    import torch
    import paper_2303_06742_gb300 as st
    import inputs
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from _cases import gpu_problem
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    c = inputs.case(args.workload)
    nb, tol, K, W = args.rhs, c["tol"], args.steps, args.warmup
    t0s = [0.1 * k for k in range(nb)]
    stream = torch.cuda.Stream()
    ts = time.perf_counter()
    S = st.Solver(gpu_problem(c), precision=st.MIXED, stream=stream, n_sweeps=args.sweeps, n_rhs=nb)
    setup_s = time.perf_counter() - ts
    if args.tc_shapes:
        for item in args.tc_shapes.split(";"):
            lev, shape = item.split(":")
            S.set_tc_shape(int(lev), *[int(v) for v in shape.split(",")])
    tc_shapes = {str(l): list(S.tc_shape(l)) for l in range(1, S.n_levels)}
    states = torch.zeros((nb, S.n_state), dtype=torch.float64, device="cuda")
    for k, t0 in enumerate(t0s):
        S.initial_state_at(t0, states[k])

    def run(first, steps, profile=False):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        its = []
        if profile:
            S.profile(True)
        with torch.cuda.stream(stream):
            evs[0].record(stream)
            for i in range(steps):
                rc, it = S.march_batch(t0s, first + i, 1, states, tol=tol)
                if rc != 0:
                    raise RuntimeError("march_batch returned %d" % rc)
                its.append(it[0].tolist())
                evs[i + 1].record(stream)
        stream.synchronize()
        return [evs[i].elapsed_time(evs[i + 1]) for i in range(steps)], its

    run(0, W)
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    tw0 = time.time()
    l0 = S.launch_count()
    ms, its = run(W, K)
    torch.cuda.synchronize()
    launches = S.launch_count() - l0
    tw1 = time.time()
    clk = clocks.stop(tw0, tw1)
    total_ms = sum(ms)
    KP = min(K, 3)
    run(W + K, KP, profile=True)
    prof = S.profile_read()
    S.profile(False)
    value, total_ms = job_throughput(K * nb, total_ms, world, dist)

    # end to end: every step copies the nb right-hand sides and initial
    # guesses from pinned host memory and the solutions back
    E = min(K, 3)
    n = S.n_slab
    rhs_h = torch.empty((nb, n), dtype=torch.float64, pin_memory=True)
    x0_h = torch.empty((nb, n), dtype=torch.float64, pin_memory=True)
    x_h = torch.empty((nb, n), dtype=torch.float64, pin_memory=True)
    with torch.cuda.stream(stream):
        rd = torch.zeros(n, dtype=torch.float64, device="cuda")
        for k in range(nb):
            S.slab_rhs(0, states[k], rd)
            rhs_h[k].copy_(rd)
            x0_h[k].copy_(states[k].repeat(S.prob.q))
    stream.synchronize()
    rhs_d = torch.empty((nb, n), dtype=torch.float64, device="cuda")
    x_d = torch.empty((nb, n), dtype=torch.float64, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for _ in range(E):
            rhs_d.copy_(rhs_h, non_blocking=True)
            x_d.copy_(x0_h, non_blocking=True)
            S.slab_solve_batch(nb, rhs_d, x_d, tol=tol)
            x_h.copy_(x_d, non_blocking=True)
        ev[1].record(stream)
    stream.synchronize()
    e2e_value = E * nb * world / (ev[0].elapsed_time(ev[1]) / 1000.0)
    S.close()

    # the same marches one after another on the single-column FP32 path
    S1 = st.Solver(gpu_problem(c), precision=st.MIXED, stream=stream, n_sweeps=args.sweeps)
    one = []
    for k, t0 in enumerate(t0s[:min(nb, 2)]):
        st1 = torch.zeros(S1.n_state, dtype=torch.float64, device="cuda")
        S1.initial_state_at(t0, st1)
        time_march(S1, torch, stream, st1, 0, 2, tol)
        ms1, _ = time_march(S1, torch, stream, st1, 2, min(K, 4), tol)
        one += ms1
    S1.close()
    single = 1000.0 / (sum(one) / len(one))
    if rank != 0:
        return
    pa = prof["patch_apply"]
    peak, peak_kind = peak_hbm()
    achieved = pa["bytes"] / (pa["ms"] / 1000.0) / 1e9 if pa["ms"] > 0 else None
    breakdown = {k: {"ms": v["ms"], "share": v["ms"] / max(sum(x["ms"] for x in prof.values()), 1e-30),
                     "launches": v["launches"]} for k, v in prof.items()}
    print(json.dumps({
        "metric": "slab solves/s", "value": value, "unit": "slab solves/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": total_ms / K, "p50_ms": pct(ms, 50), "p99_ms": pct(ms, 99),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "tf32+f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESCS.get(args.workload, args.workload) + "; %d right-hand sides "
                   "(marches from t0 = 0, 0.1, ..) solved together, one step = one slab of each" % nb,
                   "precision": "TF32 tensor-core patch apply, FP32 V-cycle, FP64 FGMRES", "tol": tol,
                   "l2": "no flush: the patch inverses streamed per sweep exceed L2"},
        "iters_per_slab": its, "setup_s": setup_s,
        "e2e": {"value": e2e_value, "unit": "slab solves/s", "h2d_bytes_per_step": 2 * nb * n * 8,
                "d2h_bytes_per_step": nb * n * 8},
        "single_column_path": {"value": single, "unit": "slab solves/s",
                               "note": "same operator, one march at a time, FP32 CUDA-core patch apply"},
        "roofline": {"kernel": "k_patch_apply_tc", "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak if achieved else None, "peak_source": peak_kind,
                     "traffic": dram_traffic_tc(args.workload, nb),
                     "algorithmic_bytes_per_launch": pa["bytes"] / max(pa["launches"], 1),
                     "avg_launch_ms": pa["ms"] / max(pa["launches"], 1), "launches": pa["launches"],
                     "tc_shapes": tc_shapes},
        "breakdown": breakdown, "gpu_launches": launches, "clocks": clk,
        "energy": energy_per_step(clk, total_ms / K),
    }))


# ------------------------------------------------------------------ serving arm
def serving_arm(args):
    """Serving stream: requests arrive by a Poisson process and are admitted by
    HBM footprint; reports slab throughput, request and slab latencies."""
    import torch
    import paper_2303_06742_gb300 as st
    import inputs
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from _cases import gpu_problem
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    reqs = inputs.serving_stream(args.requests)
    probs = [gpu_problem(c) for c in reqs]
    free, total = torch.cuda.mem_get_info()
    budget = int(0.8 * free)
    S = st.Server(hbm_budget=budget, n_workers=args.workers, batched=args.batched, max_members=args.members)
    t0 = time.perf_counter()
    ids = []
    for p, c in zip(probs, reqs):
        wait = c["arrival"] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        ids.append(S.submit(p, c["slabs"], tol=c["tol"]))
    res = [S.result(i) for i in ids]
    makespan = max(r[0]["t_done"] for r in res) - min(r[0]["t_submit"] for r in res)
    S.close()
    if rank != 0:
        return
    slabs = sum(r[0]["n_slabs"] for r in res)
    lat = [r[0]["t_done"] - r[0]["t_submit"] for r in res]
    setup = [r[0]["t_ready"] - r[0]["t_admit"] for r in res]
    slab_ms = [x for r in res for x in r[2]]
    print(json.dumps({
        "metric": "slab solves/s", "value": slabs / makespan, "unit": "slab solves/s", "n_gpus": 1,
        "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "serving stream: %d 2D requests, Poisson arrivals (mean 2 ms), meshes "
                               "{16,32,64,128}^2, (Q2/Q1,k=1) or (Q3/Q2,k=2), 5-50 slabs, random materials; "
                               "%d workers, HBM budget %.0f GB" % (len(reqs), args.workers, budget / 1e9),
                   "mode": ("batched: lockstep groups of up to %d requests per class with fused smoother "
                            "launches" % args.members) if args.batched else "independent: one march per worker"},
        "requests": len(reqs), "slabs": slabs, "makespan_s": makespan,
        "request_latency_s": {"p50": pct(lat, 50), "p99": pct(lat, 99)},
        "slab_latency_ms": {"p50": pct(slab_ms, 50), "p99": pct(slab_ms, 99)},
        "setup_s": {"p50": pct(setup, 50), "p99": pct(setup, 99)},
        "status": sorted(set(r[0]["status"] for r in res)),
    }))


# ------------------------------------------------------------------ pulse march served with 3D requests
def served_pulse_arm(args):
    """The layered 3D 32^3 pulse march (40 slabs, 3.37 M unknowns per slab)
    served together with 16 concurrent 3D 16^3 marches (10 slabs each), all
    submitted at time 0 to the serving loop (one worker per request).  The
    big march is also run alone for its uncontended slab latency."""
    import torch
    import paper_2303_06742_gb300 as st
    import inputs
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from _cases import gpu_problem
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    reqs = inputs.served_with_pulse()
    probs = [gpu_problem(c) for c in reqs]
    free, _ = torch.cuda.mem_get_info()
    budget = int(0.8 * free)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    tw0 = time.time()
    S = st.Server(hbm_budget=budget, n_workers=len(reqs))
    ids = [S.submit(p, c["slabs"], tol=c["tol"]) for p, c in zip(probs, reqs)]
    res = [S.result(i) for i in ids]
    S.close()
    tw1 = time.time()
    clk = clocks.stop(tw0, tw1)
    A = st.Server(hbm_budget=budget, n_workers=1)
    alone = A.result(A.submit(probs[0], reqs[0]["slabs"], tol=reqs[0]["tol"]))
    A.close()
    big, small = res[0], res[1:]
    march_s = [r[0]["t_done"] - r[0]["t_ready"] for r in res]
    t_first = min(r[0]["t_ready"] for r in res)
    t_last = max(r[0]["t_done"] for r in res)
    slabs = sum(r[0]["n_slabs"] for r in res)
    print(json.dumps({
        "metric": "slab solves/s", "value": slabs / (t_last - t_first), "unit": "slab solves/s", "n_gpus": 1,
        "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "3D [0,2]^2x[0,1] 32^3 layered pulse (Q2^3/Q1, dG(1), 4 levels, tau 5e-3, "
                               "40 slabs, 3,367,374 unknowns per slab) served with 16 concurrent 3D 16^3 "
                               "thermoelastic marches (10 slabs each); FP32 V-cycle in FP64 FGMRES, tol 1e-8; "
                               "value = all slabs over the time from the first finished setup to the last "
                               "finished march"},
        "status": sorted(set(r[0]["status"] for r in res)),
        "pulse": {"slab_latency_ms": {"p50": pct(list(big[2]), 50), "p99": pct(list(big[2]), 99)},
                  "march_s": march_s[0], "setup_s": big[0]["t_ready"] - big[0]["t_admit"],
                  "iters_total": big[0]["iters_total"], "device_bytes": big[0]["device_bytes"],
                  "alone_slab_latency_ms": {"p50": pct(list(alone[2]), 50), "p99": pct(list(alone[2]), 99)},
                  "alone_march_s": alone[0]["t_done"] - alone[0]["t_ready"]},
        "small": {"march_s": {"p50": pct(march_s[1:], 50), "p99": pct(march_s[1:], 99)},
                  "slab_latency_ms": {"p50": pct([x for r in small for x in r[2]], 50),
                                      "p99": pct([x for r in small for x in r[2]], 99)},
                  "setup_s": {"p50": pct([r[0]["t_ready"] - r[0]["t_admit"] for r in small], 50)}},
        "clocks": clk,
    }))


def main():
    args = parse()
    if args.workload == "serving" and not args.cpu_leg:
        serving_arm(args)
        return
    if args.workload == "pulse_served" and not args.cpu_leg:
        served_pulse_arm(args)
        return
    if args.rhs > 1 and not args.cpu_leg and args.impl != "reference":
        batch_arm(args)
        return
    if args.cpu_leg:
        oracle_leg(args.workload, args.cpu_leg, "reference" if args.impl == "reference" else "solve",
                   args.steps, args.warmup, args.form, args.pressure)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
