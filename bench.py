"""Benchmark of the resolvent-sampling hot path on one GB300.

Workload: the rational 5-point-grid NEP T(z) = K - zM + (z/(z-300))E, n = 40000
(200 x 200 grid, natural ordering, half-bandwidth 200), ellipse centre 100,
semi-axes 80/20, N = 64 sampling points, L = 32 probe columns, mixed precision
(complex64 band LU, FP64 refinement to backward error <= 1e-10).

One step = one pass of the whole GPU hot path over the workload: rsrr_sample
(assembly, band LU, solves, FP64 refinement) + rsrr_project (normalisation,
Gram, truncated SVD basis, projections).  value = resolvent columns (N*L per
step) per second of device time; e2e = the same through the C ABI with the
probe U in pinned host memory copied in and the projected matrices copied
out every step.  The oracle (numpy/scipy, FP64) is timed on a bounded sample
of the same workload as the CPU baseline.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "grid5pt_rational_n40000_bw200_N64_L32"
METRIC = "resolvent columns/s at 1e-10 rel. residual (mixed vs FP64); RSRR p50/p99 latency"
UNIT = "resolvent columns/s"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e-3  # SMs x FP32 lanes x FMA x max SM clock (THz)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--g", type=int, default=200, help="grid side (n = g^2)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison step")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--workload", default="c1", choices=["c1", "c2", "c3"],
                    help="c1: banded grid (the benchmark line); c2: dense kernel, sampling only")
    ap.add_argument("--sample-points", type=int, default=2,
                    help="sampling points of the oracle's bounded sample")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving latency leg")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the dense-kernel and grouped-batch sub-measurements")
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--batch-full", action="store_true", help="c3 at its full sizes")
    ap.add_argument("--dense-n", type=int, default=4096, help="points of the dense kernel workload (c2)")
    ap.add_argument("--dense-flags", type=int, default=0, help="RSRR_FLAG_* bits of the dense run (c2)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- oracle leg
ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import oracle, workloads as W
p = W.rational_grid(g={g})
z = oracle.sample_points(p.region, p.N)[:{npts}]
oracle.resolvent_samples(p, z[:1])  # warm the code paths
t = time.perf_counter()
X = oracle.resolvent_samples(p, z)
dt = time.perf_counter() - t
print(json.dumps({{"seconds": dt, "columns": int(len(z) * p.L)}}))
"""


ORACLE_PAR_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import oracle, workloads as W
p = W.rational_grid(g={g})
z = oracle.sample_points(p.region, p.N)[{j}:{j} + 1]
oracle.resolvent_samples(p, z)  # warm the code paths
open(os.path.join({tmp!r}, "ready.{j}"), "w").close()
t_end = time.time() + 600
while len(os.listdir({tmp!r})) < {procs} and time.time() < t_end:  # every worker set up
    time.sleep(0.01)
t0 = time.time()
X = oracle.resolvent_samples(p, z)
t1 = time.time()
print(json.dumps({{"t0": t0, "t1": t1, "columns": int(len(z) * p.L)}}))
"""


def max_over_ranks(ms, dist=None, device="cpu"):
    """Step time of the whole job: the slowest rank's (all-reduce MAX; the
    identity on one rank)."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(cols_per_rank, world, ms):
    """Whole-job throughput of `world` replicas, each sampling `cols_per_rank`
    resolvent columns per step of `ms` milliseconds (the max over ranks)."""
    return cols_per_rank * world / (ms / 1e3)


def oracle_sample(g, npts):
    """Time the oracle's resolvent samples (LAPACK banded solves) on `npts`
    points of the workload in a 1-thread subprocess (BLAS pinned to 1 thread)."""
    env = dict(os.environ)
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    code = ORACLE_SNIPPET.format(root=ROOT, g=g, npts=npts)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["columns"] / d["seconds"], d


def oracle_parallel(g, procs):
    """The oracle on `procs` host processes at once, one sampling point each
    (1 BLAS thread each): every process sets up and warms up, they meet at a
    file barrier, then solve; wall time = last finish - first start."""
    import tempfile
    env = dict(os.environ)
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    with tempfile.TemporaryDirectory() as tmp:
        ps = [subprocess.Popen([sys.executable, "-c",
                                ORACLE_PAR_SNIPPET.format(root=ROOT, g=g, j=j, tmp=tmp, procs=procs)],
                               stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
              for j in range(procs)]
        outs = [q.communicate(timeout=1800) for q in ps]
    for q, (_, err) in zip(ps, outs):
        if q.returncode != 0:
            raise RuntimeError(err[-2000:])
    ds = [json.loads(o.strip().splitlines()[-1]) for o, _ in outs]
    wall = max(d["t1"] for d in ds) - min(d["t0"] for d in ds)
    cols = sum(d["columns"] for d in ds)
    return cols / wall, wall, cols


def cpu_model():
    """CPU model name of this host (lscpu), else the machine type."""
    import platform
    import shutil
    if shutil.which("lscpu"):
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=30).stdout
            for ln in out.splitlines():
                if ln.startswith("Model name:"):
                    return ln.split(":", 1)[1].strip() + f" ({platform.machine()})"
        except Exception:
            pass
    return platform.machine()


def cpu_baseline(g, npts, par=True):
    v, d = oracle_sample(g, npts)
    out = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{npts} of the 64 sampling points ({d['columns']} resolvent columns, "
                     f"scipy banded LU, FP64) in {d['seconds']:.1f} s, 1 BLAS thread",
           "cpu": cpu_model()}
    try:
        ncpu = len(os.sched_getaffinity(0))
    except AttributeError:
        ncpu = os.cpu_count() or 1
    out["host_cores"] = {"usable": ncpu, "total": os.cpu_count()}
    if par:
        # one process per core this process may run on, at most one per
        # sampling point (64; about 0.7 GB of host memory each)
        procs = max(1, min(64, ncpu))
        pv, wall, cols = oracle_parallel(g, procs)
        out["parallel"] = {"value": pv, "unit": UNIT, "cores": procs,
                            "sample": f"{procs} sampling points, one per process (1 BLAS thread "
                                      f"each), solved at once: {cols} columns in {wall:.1f} s"}
    return out


def measured_peaks():
    """Roofline denominators: the measured copy bandwidth and bf16 GEMM rates
    of this GPU model (MEASURED_PEAKS.json), else the fallback figures."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return {"hbm_gbs": d["hbm_gbs"], "bf16_burst": d["bf16_tflops"],
                "bf16_sustained": d["bf16_tflops_sustained"], "source": "of measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_burst": 1900.0, "bf16_sustained": 1700.0,
                "source": "of fallback"}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, val in zip(names, f[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_e2e(a, s, p, stats, stream, world, dist=None):
    """Same metric through the C ABI with host buffers: U copied from pinned
    host memory and the projected matrices copied back, every step."""
    import ctypes as C
    import numpy as np
    import torch
    from paper_1605_07951_gb300 import rsrr
    cols = p.N * p.L
    Uh = torch.from_numpy(np.ascontiguousarray(p.U.T)).pin_memory()  # column-major n x L
    k = stats["k"]
    Pout = torch.empty((p.m, k, k), dtype=torch.complex128).pin_memory()

    def e2e_step():
        st = rsrr.rsrr_set_probe(s.h, C.c_void_p(Uh.data_ptr()), 0, None)
        assert st == 0
        s.sample(stream)
        s.project(stream)
        sti = s.stats()
        assert sti["converged"] == 1 and sti["max_eta"] <= 1e-10, sti
        kk = sti["k"]
        st = rsrr.rsrr_get_projected(s.h, C.c_void_p(Pout.data_ptr()), 0,
                                     C.c_void_p(stream.cuda_stream))
        assert st == 0 and kk == k
    e2e_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) / a.steps * 1e3, dist, "cuda")
    e2e = {"value": replica_value(cols, world, e2e_ms), "unit": UNIT,
           "h2d_bytes_per_step": int(Uh.numel() * 16),
           "d2h_bytes_per_step": int(p.m * k * k * 16)}

    return e2e


# ---------------------------------------------------------------- serving leg
def serve_stream(rsrr, reqs, rate, precision, slots, seed):
    """Submit `reqs` to a request server with Poisson arrivals at `rate`
    requests/s (rate None: all at t = 0) and wait for every reply.  Latency is
    measured from the scheduled arrival to the result on the host."""
    import numpy as np
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, len(reqs)) if rate else np.zeros(len(reqs))
    sched = np.cumsum(gaps) - gaps[0]
    sv = rsrr.Server(slots=slots)
    ids, lag = [], []
    t0 = time.perf_counter()
    for (fam, p), ts in zip(reqs, sched):
        while time.perf_counter() - t0 < ts:
            time.sleep(min(1e-3, max(0.0, ts - (time.perf_counter() - t0))))
        lag.append(time.perf_counter() - t0 - ts)
        ids.append(sv.submit(p, rsrr.default_opts(precision=precision)))
    reps = [sv.wait(i, timeout=1800.0) for i in ids]
    t_end = time.perf_counter() - t0
    st = sv.stats()
    for i in ids:
        sv.release(i)
    sv.close()
    lat = np.array([(r["t_done"] - r["t_submit"]) + lg for r, lg in zip(reps, lag)])
    cols = sum(p.N * p.L for _, p in reqs)
    ok = sum(1 for r in reps if r["status"] >= 0)
    # where a request's time goes, per family (medians over the stream):
    # queueing, the three stages on the request's own stream, sweeps and rank
    stages = {}
    for fam in sorted({f for f, _ in reqs}):
        rr = [r for (f, _), r in zip(reqs, reps) if f == fam]
        med = lambda key, sc=1e3: float(np.median([r[key] for r in rr]) * sc)  # noqa: E731
        stages[fam] = {"count": len(rr), "queue_ms": float(np.median([r["t_admit"] - r["t_submit"] for r in rr]) * 1e3),
                       "sample_ms": med("t_sample"), "project_ms": med("t_project"), "solve_ms": med("t_solve"),
                       "refine_sweeps": med("refine_sweeps", 1), "k": med("k", 1)}
    return {"requests": len(reqs), "ok": ok, "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "makespan_s": t_end, "req_per_s": len(reqs) / t_end, "columns_per_s": cols / t_end,
            "peak_active": st["peak_active"], "peak_bytes": int(st["peak_bytes"]), "stages": stages}


def run_serving(a):
    """Serving of RSRR requests (rsrr_server_*): capacity from a closed burst,
    then Poisson arrivals at 0.7 x that capacity, mixed precision and the plain
    FP64 path, p50/p99 latency from arrival to eigenpairs on the host."""
    import workloads as W
    from paper_1605_07951_gb300 import rsrr
    reqs = W.serving_stream(a.serve_requests, seed=5000)
    mixed = rsrr.RSRR_PREC_MIXED
    serve_stream(rsrr, reqs[:4], None, mixed, a.serve_slots, 1)  # warm-up
    burst = serve_stream(rsrr, reqs, None, mixed, a.serve_slots, 5001)
    rate = 0.7 * burst["req_per_s"]
    poisson = serve_stream(rsrr, reqs, rate, mixed, a.serve_slots, 5002)
    poisson64 = serve_stream(rsrr, reqs, rate, rsrr.RSRR_PREC_FP64, a.serve_slots, 5002)
    return {"workload": f"{len(reqs)} requests, families c0/c1/c2 shapes (quadratic n=1000; "
                        "grid g=40..100; dense n=128..512), random regions, seed 5000",
            "slots": a.serve_slots, "budget_gb": 150, "burst": burst,
            "poisson_rate_req_per_s": rate, "poisson_mixed": poisson, "poisson_fp64_plain": poisson64}


# ---------------------------------------------------------------- our arm
def run_ours(a, rank, world, local):
    import numpy as np
    import torch
    import workloads as W
    from paper_1605_07951_gb300 import rsrr

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    p = W.rational_grid(g=a.g)
    opts = rsrr.default_opts(timing=1)
    s = rsrr.Solver(p, opts)
    stream = torch.cuda.current_stream()

    def step():
        s.sample(stream)
        s.project(stream)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    st = s.check_status()
    if st != rsrr.RSRR_OK:
        raise SystemExit(f"sampling did not converge: {rsrr.STATUS_NAMES.get(st, st)}")
    stats0 = s.stats()
    launches0 = stats0["launches"]

    clocks = ClockSampler(local)
    clocks.start()
    lu_ms, sample_ms, project_ms, gemm_ms, gemm_flops, tc_ms, tc_flops = [], [], [], [], [], [], []
    asm_ms, solve_ms = [], []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # the K timed steps back to back on the device (no host reads in between)
    e0.record(stream)
    for _ in range(a.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / a.steps, dist, "cuda")
    stats = s.stats()
    assert stats["converged"] == 1 and stats["max_eta"] <= 1e-10, stats
    launches = (stats["launches"] - launches0)
    # then K more steps, one at a time, for the stage times of the library's
    # own events (the rooflines) and the convergence of every step
    for _ in range(a.steps):
        step()
        torch.cuda.synchronize()
        sti = s.stats()
        assert sti["converged"] == 1 and sti["max_eta"] <= 1e-10, sti
        asm_ms.append(sti["stage_ms"][0])
        solve_ms.append(sti["stage_ms"][2])
        lu_ms.append(sti["stage_ms"][1])
        sample_ms.append(sum(sti["stage_ms"][:5]))
        project_ms.append(sti["stage_ms"][5])
        gemm_ms.append(sti["gemm_ms"])
        gemm_flops.append(sti["gemm_flops"])
        tc_ms.append(sti["tc_ms"])
        tc_flops.append(sti["tc_flops"])
    cols = p.N * p.L
    value = replica_value(cols, world, ms)

    # e2e: U from pinned host memory, projected matrices back to the host, per step
    e2e = None
    if not a.no_e2e:
        e2e = run_e2e(a, s, p, stats, stream, world, dist)
    fp64 = None
    # rooflines of the two kernels that dominate a step, from the library's
    # own CUDA events on the launching stream (opts.timing): the bf16 slice
    # products of the FP64-accurate GEMMs of rsrr_project (tensor pipe) and
    # the complex64 band LU of rsrr_sample (FP32 FMA pipe); "roofline" is the
    # one with more device time per step
    peaks = measured_peaks()
    # DRAM bytes of each roofline's kernel, dram__bytes_read.sum +
    # dram__bytes_write.sum from one ncu capture of this command at this size
    # (the DRAM traffic summary under profiles/); valid for the kernel
    # revisions captured there, and only at the default size
    full = a.g == 200
    traffic_tc = 101.9e9 if full else None      # all 37 slice GEMMs of one step
    traffic_lu = 39.66e9 if full else None      # one band LU launch
    traffic_asm = 13.32e9 if full else None     # one assembly launch
    traffic_solve = 16.78e9 if full else None   # the first solve (all 64 points)
    tc_avg = statistics.mean(tc_ms)
    tc_ach = statistics.mean(tc_flops) / (tc_avg / 1e3) / 1e12 if tc_avg > 0 else 0.0
    roof_tc = {"bound": "tensor", "kernel": "oz_gemm_tc_kernel (bf16 slice products on tcgen05, Ozaki GEMMs)",
               "achieved": tc_ach, "peak": peaks["bf16_sustained"], "unit": "TFLOP/s",
               "frac": tc_ach / peaks["bf16_sustained"], "traffic": traffic_tc,
               "tensor_flop_per_step": statistics.mean(tc_flops), "ms_per_step": tc_avg,
               "peak_note": f"bf16 dense, sustained, {peaks['source']}; flops = the 28 slice-pair "
                            "products per 128x64 tile the scheme needs (tcgen05.mma kind::f16); "
                            "achieved and traffic per step (all 37 slice-GEMM launches of a step)",
               "fp64_equivalent": {"flop_per_step": statistics.mean(gemm_flops),
                                   "gemm_ms_per_step": statistics.mean(gemm_ms),
                                   "tflops": statistics.mean(gemm_flops)
                                   / (statistics.mean(gemm_ms) / 1e3) / 1e12}}
    n, kl, ku = p.n, stats["kl"], stats["ku"]
    flop_per_point = 8.0 * sum(min(kl, n - 1 - j) * min(kl + ku, n - 1 - j) for j in range(n))
    lu_flops = flop_per_point * p.N
    lu_avg = statistics.mean(lu_ms)
    achieved = lu_flops / (lu_avg / 1e3) / 1e12
    ldab = 2 * kl + ku + 32
    roof_lu = {"bound": "alu", "kernel": "band_lu_cluster_kernel<float2> (complex64, two-CTA cluster per point)",
               "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
               "frac": achieved / FP32_PEAK_TFLOPS,
               "traffic": traffic_lu,
               "algorithmic_flop_per_launch": lu_flops, "avg_launch_ms": lu_avg,
               # the other roof: the band storage read and written once
               "algorithmic_bytes_per_launch": 2 * 8.0 * ldab * n * p.N,
               "hbm_frac": 2 * 8.0 * ldab * n * p.N / (lu_avg / 1e3) / 1e9 / peaks["hbm_gbs"],
               "peak_note": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz; traffic 1.53x the "
                            "algorithmic bytes: the trailing window written back every panel"}
    roof, roof_other = (roof_lu, roof_tc) if lu_avg >= tc_avg else (roof_tc, roof_lu)
    # band assembly: the complex64 band storage of every point written once
    asm_bytes = 8.0 * ldab * n * p.N
    asm_avg = statistics.mean(asm_ms)
    asm_gbs = asm_bytes / (asm_avg / 1e3) / 1e9
    roof_asm = {"bound": "hbm", "kernel": "assemble_band_kernel<float2> (one warp per band column)",
                "achieved": asm_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": asm_gbs / peaks["hbm_gbs"], "traffic": traffic_asm,
                "algorithmic_bytes_per_launch": asm_bytes, "avg_stage_ms": asm_avg,
                "pattern_only_bytes_per_launch": 8 * len(p.col_idx) * p.N,
                "peak_note": f"copy bandwidth, {peaks['source']}; time = the assembly stage "
                             "(the ||T(z_j)|| kernel + the assembly), so the fraction is a lower bound"}

    # first solve of all points: the complex64 factors streamed once per 16
    # right-hand sides (two CTAs per point), against the copy bandwidth
    solve_avg = statistics.mean(solve_ms)
    solve_bytes = 8.0 * ldab * n * p.N
    roof_solve = {"bound": "hbm", "kernel": "band_solve2_kernel<float2> (streaming banded solve, first solve)",
                  "achieved": solve_bytes / (solve_avg / 1e3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                  "frac": solve_bytes / (solve_avg / 1e3) / 1e9 / peaks["hbm_gbs"], "hbm_frac":
                  solve_bytes / (solve_avg / 1e3) / 1e9 / peaks["hbm_gbs"], "traffic": traffic_solve,
                  "algorithmic_bytes_per_launch": solve_bytes, "avg_stage_ms": solve_avg,
                  "peak_note": f"copy bandwidth, {peaks['source']}; the solve is a chain of 2n/32 dependent "
                               "block steps per point and is bound by its per-step latency, not by DRAM"}

    if not a.no_fp64:
        s64 = rsrr.Solver(p, rsrr.default_opts(precision=rsrr.RSRR_PREC_FP64, timing=1))
        s64.sample(stream)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        s64.sample(stream)
        f1.record(stream)
        torch.cuda.synchronize()
        st64 = s64.stats()
        fms = f0.elapsed_time(f1)
        fp64 = {"sample_value": cols / (fms / 1e3), "sample_ms": fms,
                "max_eta": float(np.max(s64.eta())), "lu_ms": st64["stage_ms"][1]}
        s64.close()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": p.n, "kl": kl, "ku": ku, "N": p.N, "L": p.L,
                   "precision": "mixed (complex64 band LU, FP64 refinement to eta<=1e-10)",
                   "step": "rsrr_sample + rsrr_project",
                   "l2": "inputs larger than L2: the 12.9 GB band workspace is rewritten every step",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "sample_only": {"value": cols / (statistics.mean(sample_ms) / 1e3),
                        "ms": statistics.mean(sample_ms), "stage_ms": stats["stage_ms"][:5],
                        "refine_sweeps": stats["refine_sweeps"], "max_eta": stats["max_eta"]},
        "project_ms": statistics.mean(project_ms), "rank_k": stats["k"],
        "pivoted_cholesky_kc": stats["kc"],
        "fp64_plain_path": fp64,
        "roofline": roof, "roofline_second": roof_other, "roofline_assembly": roof_asm,
        "roofline_solve": roof_solve,
        "e2e": e2e, "gpu_launches": int(launches),
        "clocks": clk,
    }
    s.close()
    if not a.no_extra and rank == 0:
        line["dense"] = dense_leg(a)
        line["batch_grouped"] = batch_leg(a)
    if not a.no_serving and rank == 0:
        line["serving"] = run_serving(a)
    if rank == 0 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(a.g, a.sample_points)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------- reference arm
def run_reference(a, rank, world):
    """The oracle (FP64 numpy/scipy) as the reference arm: each step is a
    bounded sample (a.sample_points sampling points) of the same workload."""
    if rank != 0:
        return
    times, cols = [], 0
    d = None
    for i in range(a.warmup + a.steps):
        v, d = oracle_sample(a.g, a.sample_points)
        if i >= a.warmup:
            times.append(d["seconds"])
    cols = d["columns"]
    sec = statistics.mean(times)
    value = cols / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": a.g * a.g, "N": 64, "L": 32,
                   "step": f"oracle resolvent samples at {a.sample_points} of the 64 points"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{a.sample_points} sampling points per step, 1 BLAS thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_dense(a):
    """Dense kernel workload (n = 4096 points on the unit sphere, N = 32,
    L = 64): rsrr_sample timed alone (the projection of this workload is
    dominated by FP64 Taylor products and is not part of the benchmark line)."""
    import torch
    import workloads as W
    from paper_1605_07951_gb300 import rsrr
    torch.cuda.set_device(0)
    p = W.helmholtz_sphere(n=a.dense_n, N=32, L=64)
    s = rsrr.Solver(p, rsrr.default_opts(timing=1, flags=a.dense_flags))
    stream = torch.cuda.current_stream()
    for _ in range(a.warmup):
        s.sample(stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        s.sample(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    st = s.stats()
    s.close()
    n = p.n
    lu_flops = 8.0 / 3.0 * n ** 3 * p.N
    print(json.dumps({"workload": f"helmholtz_sphere_n{n}_N32_L64", "metric": UNIT,
                      "dense_update": "fma" if a.dense_flags & rsrr.RSRR_FLAG_SIMT_DENSE_UPDATE else "tcgen05",
                      "sample_value": p.N * p.L / (ms / 1e3), "ms_per_sample": ms,
                      "stage_ms": st["stage_ms"][:5], "refine_sweeps": st["refine_sweeps"],
                      "max_eta": st["max_eta"],
                      "dense_lu_tflops": lu_flops / (st["stage_ms"][1] / 1e3) / 1e12}))


def dense_leg(a):
    """The dense kernel workload (n = 4096 points on the unit sphere, N = 32,
    L = 64) as a sub-measurement of the default line: rsrr_sample device time,
    the dense LU's roofline against the TF32 rate (the measured bf16 rate x the
    nominal TF32 / bf16 ratio 1.1 / 2.25; the update runs as 3xTF32 on
    tcgen05), and the oracle's dense LAPACK solve of one point on one core."""
    import numpy as np
    import torch
    import workloads as W
    from paper_1605_07951_gb300 import rsrr
    p = W.helmholtz_sphere(n=a.dense_n, N=32, L=64)
    s = rsrr.Solver(p, rsrr.default_opts(timing=1))
    stream = torch.cuda.current_stream()
    for _ in range(2):
        s.sample(stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.sample(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st = s.stats()
    ok = s.check_status() == rsrr.RSRR_OK
    s.close()
    n = p.n
    lu_flops = 8.0 / 3.0 * n ** 3 * p.N
    lu_tflops = lu_flops / (st["stage_ms"][1] / 1e3) / 1e12
    peaks = measured_peaks()
    tf32 = peaks["bf16_sustained"] * 1.1 / 2.25
    out = {"workload": f"helmholtz_sphere_n{n}_N32_L64", "value": p.N * p.L / (ms / 1e3), "unit": UNIT,
           "ms": ms, "converged": ok, "stage_ms": st["stage_ms"][:5], "max_eta": st["max_eta"],
           "roofline": {"bound": "tensor", "kernel": "dense LU (tcgen05 3xTF32 trailing update, panel kernels)",
                        "achieved": lu_tflops, "peak": tf32, "unit": "TFLOP/s", "frac": lu_tflops / tf32,
                        "traffic": None,
                        "peak_note": f"TF32 dense = bf16 sustained {peaks['source']} x 1.1/2.25 (nominal); "
                                     "achieved = 8/3 n^3 complex-LU flops per point; traffic null: the LU "
                                     "is many launches (a panel and an update per 32 columns)"}}
    if not a.no_cpu_baseline:
        import oracle
        zo = oracle.sample_points(p.region, p.N)
        t0 = time.perf_counter()
        oracle.resolvent_samples_dense(p, zo[:1])
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": p.L / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"1 of the 32 sampling points (64 columns, dense LAPACK solve, "
                                         f"FP64) in {dt:.1f} s"}
    return out


def batch_leg(a):
    """Grouped sampling of uneven band problems (the grid half of the batched
    workload at scaled sizes, g 40..100): rsrr_sample_batch (one persistent
    grouped band LU over all points of all handles) against the same handles
    sampled one after the other."""
    import torch
    import workloads as W
    from paper_1605_07951_gb300 import rsrr
    probs = [q for fam, q in W.batch_uneven(32, dense_n=(256, 1024), grid_g=(40, 100)) if fam == "grid"]
    solvers = [rsrr.Solver(q, rsrr.default_opts()) for q in probs]
    stream = torch.cuda.current_stream()
    cols = sum(sv.N * sv.L for sv in solvers)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    t_grouped = timed(lambda: rsrr.sample_batch(solvers, stream))
    t_single = timed(lambda: [sv.sample(stream) for sv in solvers])
    ok = all(sv.check_status() == rsrr.RSRR_OK for sv in solvers)
    for sv in solvers:
        sv.close()
    return {"workload": f"{len(probs)} uneven grid NEPs (g 40..100, N 16..64, L 8..32, seed 4000)",
            "value": cols / (t_grouped / 1e3), "unit": UNIT, "ms": t_grouped, "converged": ok,
            "one_by_one": {"value": cols / (t_single / 1e3), "ms": t_single}}


def run_batch(a):
    """Batched uneven workload through the request server: every problem
    submitted at t = 0, slots and memory budget admit them as room frees up.
    Scaled sizes by default (--batch-full for the full ranges)."""
    import torch
    import workloads as W
    from paper_1605_07951_gb300 import rsrr
    torch.cuda.set_device(0)
    if a.batch_full:
        probs = W.batch_uneven(256)
        desc = "256 problems: dense n 256..2048, grids g 100..316, N 16..64, L 8..32 (seed 4000)"
    else:
        probs = W.batch_uneven(32, dense_n=(256, 1024), grid_g=(40, 100))
        desc = "32 problems: dense n 256..1024, grids g 40..100, N 16..64, L 8..32 (seed 4000)"
    serve_stream(rsrr, probs[:2], None, rsrr.RSRR_PREC_MIXED, a.serve_slots, 1)  # warm-up
    r = serve_stream(rsrr, probs, None, rsrr.RSRR_PREC_MIXED, a.serve_slots, 4001)
    print(json.dumps({"workload": "batched uneven NEPs", "problems": desc, "metric": UNIT,
                      "value": r["columns_per_s"], "makespan_s": r["makespan_s"], "ok": r["ok"],
                      "requests": r["requests"], "slots": a.serve_slots, "peak_active": r["peak_active"],
                      "peak_bytes": r["peak_bytes"], "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"]}))


def main():
    a = parse()
    rank, world, local = dist_env()
    if a.workload == "c2":
        run_dense(a)
        return
    if a.workload == "c3":
        if rank == 0:
            run_batch(a)
        return
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    run_ours(a, rank, world, local)


if __name__ == "__main__":
    main()
