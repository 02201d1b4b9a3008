"""Benchmark of the parallel-CLS hot path on one B300 (or N replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--config mixed|3sat|red0|red10|red50|learned|partial]

A step is one full pass of the hot path over the batch: Walsh-Fourier FE and
literal partials of every constraint, gradient accumulation through the
variable-major transpose, projected step, rounding and exact scoring.  The
metric is constraint-literal FE+grad evaluations per second (R * nnz per
step).  Default workload: batched mixed symmetric PB, n = 5000, 20000 clauses
(len 2..8), 2000 XOR (len 3..20), 500 cardinality (len 10..300), planted,
4096 restarts, FP32.  Inputs are synthetic (seeded generators).

--impl reference times the FP64 CPU oracle (the only reference that exists:
the paper ships no code) on the same workload, a bounded sample of restarts
per step, on this machine's host cores.
"""
import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

SM_COUNT = 148
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2032.0
# algorithmic FP32 flops per (literal, root) of the DFT evaluation: factor
# (2 FMA), prefix complex product (2 MUL + 2 FMA), suffix complex product
# (2 MUL + 2 FMA), gradient accumulation (2 FMA); FMA = 2 flops.


# DRAM traffic of one launch (or one step of a kernel class) as ncu counted
# it, dram__bytes_read.sum + dram__bytes_write.sum, keyed by (kernel,
# workload), with the capture's restart count, the files and the SHA-256
# (first 16 hex digits) of the kernel sources it was taken on.  A figure is
# reported, scaled by R (every byte counted grows with the restarts), only
# while the sources still hash the same; otherwise traffic is null.  The
# captures and the command are in profiles/traffic_mixedpb_3sat.md.
_DFT_SOURCES = ("kernels.cu", "kernels_fr.cu", "kernels_series.cu", "kernels_corner.cu",
                "kernels_p2.cu", "kernels.cuh", "plan.h")
TRAFFIC = {
    # the DFT class over one step, mean of steps 0, 3, 6 and 9 of the run
    ("dft_class", "mixedpb_n5000_m22500"): dict(
        bytes=240030720, R=1024, sources=_DFT_SOURCES, sha="fee6c8bcc731e49d",
        profile="profiles/traffic_mixedpb_3sat.md"),
    ("k_accum_step", "mixedpb_n5000_m22500"): dict(
        bytes=868638656, R=1024, sources=("kernels.cu", "kernels.cuh"), sha="93757f47d435cb76",
        profile="profiles/traffic_mixedpb_3sat.md"),
    # few rows per variable and many restarts: four restart tiles per warp
    ("k_accum_step_nt<4>", "random3sat_n100_m426"): dict(
        bytes=380754176, R=65536, sources=("kernels.cu", "kernels.cuh"), sha="93757f47d435cb76",
        profile="profiles/traffic_mixedpb_3sat.md"),
    # the constraint statistics pass (adaptive weighting), one launch
    ("k_con_stats_tile", "mixedpb_n5000_m22500"): dict(
        bytes=848947712, R=1024, sources=("kernels.cu", "kernels.cuh"), sha="93757f47d435cb76",
        profile="profiles/traffic_mixedpb_3sat.md"),
}


def _sources_sha(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2606_06656_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, workload_name, R):
    rec = TRAFFIC.get((kernel, workload_name))
    if rec is None:
        return None, "no ncu capture of this kernel on this workload"
    if _sources_sha(rec["sources"]) != rec["sha"]:
        return None, "kernel sources changed since the ncu capture"
    return rec["bytes"] * R / rec["R"], (f"{rec['profile']}: ncu at R={rec['R']}"
                                         + (f", scaled to R={R}" if R != rec["R"] else ""))


def workload(name):
    if name == "mixed":
        return W.mixed_pb(), 4096, 0.1
    if name == "3sat":
        return W.random_ksat(), 64, 0.1
    if name.startswith("red"):
        red = {"red0": 0.0, "red10": 0.1, "red50": 0.5}[name]
        return W.redundant_5sat(redundancy=red), 2048, 0.1
    raise ValueError(name)


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples: CLS_BENCH_OUT if set (kept), else the temp directory
        out = os.environ.get("CLS_BENCH_OUT") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [l.strip().split(", ") for l in open(self.path) if l.strip()]
        except Exception:
            rows = []
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def cpu_oracle_step(inst, X, lr):
    """One oracle step: FP64 objective/gradient, FP32 projected step, score."""
    from oracle import cls as ocls
    _, g, _ = ocls.objective_grad(inst, X.astype(np.float64))
    Xn = ocls.pgd_step(X, g.astype(np.float32), lr, inst.fixed)
    ocls.score(inst, Xn)
    return Xn


def time_cpu_oracle(inst, R_sample, lr, steps, budget_s=25.0):
    X = W.uniform_points(inst.n, R_sample, seed=42)
    t_all, done = 0.0, 0
    for _ in range(max(1, steps)):
        t0 = time.perf_counter()
        X = cpu_oracle_step(inst, X, lr)
        t_all += time.perf_counter() - t0
        done += 1
        if t_all > budget_s:
            break
    return t_all / done, done


def threads_used():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        return 1


def _oracle_chunk(a):
    """One oracle step on a slice of restarts (run in a spawned worker);
    returns the new points and the seconds it took."""
    inst, X, lr = a
    t0 = time.perf_counter()
    Xn = cpu_oracle_step(inst, X, lr)
    return Xn, time.perf_counter() - t0


def _single_thread_env():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def time_cpu_oracle_all_cores(inst, lr, per_worker=8, steps=1, budget_s=25.0, seed=42):
    """The oracle, as it stands, on every host core: one spawned process per
    core, each stepping its own slice of per_worker restarts (restarts are
    independent, Sec. 3.3).  Wall time per parallel step, after the workers
    have started and imported the oracle; stops early once budget_s is
    spent.  Returns (record, steps done)."""
    import multiprocessing as mp
    cores = host_cores()
    X = W.uniform_points(inst.n, cores * per_worker, seed=seed)
    xs = [np.ascontiguousarray(X[:, i * per_worker:(i + 1) * per_worker]) for i in range(cores)]
    with mp.get_context("spawn").Pool(cores, initializer=_single_thread_env) as pool:
        pool.map(_oracle_chunk, [(inst, xs[0][:, :1].copy(), lr)] * cores, chunksize=1)  # warm
        wall, done = 0.0, 0
        for _ in range(max(1, steps)):
            t0 = time.perf_counter()
            out = pool.map(_oracle_chunk, [(inst, x, lr) for x in xs], chunksize=1)
            wall += time.perf_counter() - t0
            xs = [o[0] for o in out]
            done += 1
            if wall > budget_s:
                break
    per_step = wall / done
    return ({"value": cores * per_worker * inst.nnz / per_step, "unit": "literal-evals/s",
             "cores": cores, "restarts": cores * per_worker, "s_per_step": per_step,
             "cpu_model": cpu_model()}, done)


def run_reference(args, rank, world):
    """The oracle, as it stands, on all host cores (one spawned process per
    core over slices of restarts), a bounded sample of the workload per
    step; the single-core figure beside it."""
    inst, R, lr = workload(args.config)
    if rank != 0:
        return
    big = inst.nnz > 10000
    per_worker = 8 if big else max(1, min(R, 64) // host_cores())
    for _ in range(args.warmup if not big else 0):
        cpu_oracle_step(inst, W.uniform_points(inst.n, per_worker, 1), lr)
    allc, done = time_cpu_oracle_all_cores(inst, lr, per_worker, steps=args.steps)
    per_step = allc["s_per_step"]
    value = allc["value"]
    t1, d1 = time_cpu_oracle(inst, per_worker, lr, 1 if big else 3, budget_s=10.0)
    line = {
        "impl": "reference", "metric": "constraint-literal FE+grad evals/s",
        "value": value, "unit": "literal-evals/s", "n_gpus": args.gpus, "steps": done,
        "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": inst.name, "n": inst.n, "m": inst.m, "nnz": inst.nnz,
                   "R": R, "lr": lr},
        "cpu_baseline": {"value": value, "unit": "literal-evals/s", "cores": allc["cores"],
                         "kind": "oracle", "cpu_model": allc["cpu_model"],
                         "sample": f"{allc['restarts']} of {R} restarts per step "
                                   f"({per_worker} per core), {done} steps",
                         "single_core": {"value": per_worker * inst.nnz / t1,
                                         "unit": "literal-evals/s", "cores": 1,
                                         "sample": f"{per_worker} of {R} restarts, "
                                                   f"{d1} step(s)"}},
        "e2e": {"value": value, "unit": "literal-evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    from paper_2606_06656_b300 import Problem
    from paper_2606_06656_b300 import binding as B
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    inst, R, lr = workload(args.config)
    if args.R:
        R = args.R
    p = Problem(inst)
    info = p.info
    x0 = p.init_uniform(R, seed=42, r_offset=rank * R)   # restarts sharded by global id
    x = x0.clone()
    ws = p.workspace(R)
    tune_s = None
    if args.tuning:
        B.cls_tuning_set(p.handle, [int(v) for v in args.tuning.split(",")])
    elif not args.no_tune:
        # tune on the phases the timed run goes through: four blocks of
        # restarts taken from the same run at steps 0, 12, 25 and 60 (dense,
        # middle and corner-dominated points), so each configuration is
        # weighed on the mix of work a run sees, not on its first step only
        t0 = time.perf_counter()
        xt = x0.clone()
        if R >= 64 and args.steps >= 20:
            xs, done_steps = x0.clone(), 0
            q = R // 4
            for blk, at in enumerate(tune_points(args)):
                if at > done_steps:
                    B.cls_step(p.handle, R, xs, lr, at - done_steps, None, None, None, ws)
                    done_steps = at
                xt[:, blk * q:(blk + 1) * q if blk < 3 else R] = \
                    xs[:, blk * q:(blk + 1) * q if blk < 3 else R]
        B.cls_autotune(p.handle, R, xt, 2, ws)
        tune_s = time.perf_counter() - t0
    tuning = B.cls_tuning_get(p.handle)
    nsat = torch.empty(R, dtype=torch.int32, device="cuda")
    wsat = torch.empty(R, dtype=torch.float64, device="cuda")
    bits = torch.empty((inst.n, (R + 31) // 32), dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 126 MB L2
    stream = torch.cuda.current_stream()

    def step_eager():
        B.cls_step(p.handle, R, x, lr, 1, bits, nsat, wsat, ws)

    def step_persistent():
        B.cls_step_persistent(p.handle, R, x, lr, 1, bits, nsat, wsat, ws)

    if args.profile_step >= 0:
        # profiling window: S untimed steps of the run from x0, then one step
        # between cudaProfilerStart/Stop (ncu --profile-from-start off); no
        # bench line
        x.copy_(x0)
        if args.profile_step:
            B.cls_step(p.handle, R, x, lr, args.profile_step, bits, nsat, wsat, ws)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        step_eager()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profile_step": args.profile_step, "workload": inst.name, "R": R,
                          "tuning": tuning}), flush=True)
        return

    graph = None if (args.eager or args.persistent) else \
        B.cls_graph_create(p.handle, R, x, lr, 1, bits, nsat, wsat, ws)

    def step():
        if graph is not None:
            B.cls_graph_launch(graph)
        elif args.persistent:
            step_persistent()
        else:
            step_eager()

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    def timed(fn, k_steps):
        """k_steps of one run from the initial points x0 (reset untimed);
        per-step CUDA-event times on the launching stream, L2 flushed (an
        untimed 256 MB write) before every step."""
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(k_steps)]
        x.copy_(x0)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for k in range(k_steps):
            flush.fill_(k & 0xFF)
            evs[k][0].record(stream)
            fn()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    def class_stats(k_steps):
        out, n_launch = {}, 0
        for kc, name in enumerate(kc_names):
            n_l, t_ms = B.cls_profile_read(p.handle, kc)
            n_launch += n_l
            out[name] = {"launches_per_step": n_l / k_steps, "ms_per_step": t_ms / k_steps}
        return out, n_launch

    # timed region: the first K steps of one run from x0 (graph launches
    # unless --eager); then the same run eagerly with a CUDA event pair around
    # every launch on its stream, for the per-kernel durations -- once over
    # its first (dense-phase) steps for the roofline, once over all K steps
    kc_names = ["fe_thread", "fe_group_real", "fe_group_dft", "accum_step_round", "score",
                "reduce", "init"]
    K = args.steps
    n_dense = min(K, 10)
    with ClockSampler(local_rank) as clk:
        t0 = time.perf_counter()
        per_step = timed(step, K)
        wall = time.perf_counter() - t0
        B.cls_profile_reset(p.handle)
        B.cls_profile_enable(p.handle, True)
        B.cls_dft_flops_counter(p.handle, reset=True)
        timed(step_eager, n_dense)
        dft_flops_dense = B.cls_dft_flops_counter(p.handle) / n_dense
        kstats_dense, _ = class_stats(n_dense)
        B.cls_profile_reset(p.handle)
        per_eager = timed(step_eager, K)
        B.cls_profile_enable(p.handle, False)
    kstats, launches = class_stats(K)
    ms_step = sum(per_step) / K
    ms_eager = sum(per_eager) / K
    if args.persistent and B.cls_persistent_status(p.handle, R, ws) != 0:
        raise RuntimeError("persistent loop: a grid barrier timed out")
    if dist:
        t = torch.tensor([ms_step], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    graph_launches = B.cls_graph_kernel_count(graph) if graph is not None else None
    launches_timed = graph_launches * K if graph_launches is not None else launches
    if args.persistent:
        launches_timed = K                          # one cooperative kernel per step
    clocks = clk.summary()

    # end to end through host buffers: one cls_solve_host call per run --
    # H2D of x0 from pinned memory, the same K steps, D2H of the counts
    xh = x0.detach().cpu().pin_memory()
    nh = torch.empty(R, dtype=torch.int32).pin_memory()
    hws = p.workspace(R, host_solve=True)
    B.cls_solve_host(p.handle, R, xh, lr, 10, nh, None, hws)   # records its step graph
    t0 = time.perf_counter()
    B.cls_solve_host(p.handle, R, xh, lr, K, nh, None, hws)
    e2e_s = (time.perf_counter() - t0) / K

    units = R * inst.nnz * world
    value = units / (ms_step / 1e3)
    # roofline of the dominant kernel class
    dom = max(kstats, key=lambda k: kstats[k]["ms_per_step"])
    pk = peaks()
    if dom == "fe_group_dft":
        # flops the DFT path evaluated in the run's first steps (device
        # counter: the dense factored kernel's roots after the tail cutoff and
        # the power-sum pass's own arithmetic), before coordinates reach the
        # cube's faces (no tile on the corner passes)
        flops = dft_flops_dense
        t = kstats_dense[dom]["ms_per_step"] / 1e3
        peak = 2 * SM_COUNT * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
        # the dense count of the method's DFT work: 9 L^2 flops per
        # cardinality constraint and restart (J = L/2 roots, ~18 flops per
        # literal and root), with no tail cutoff, power sums or corner DPs
        Lc = inst.lengths()[np.isin(inst.ctype, (W.TYPE_CARD_GE, W.TYPE_CARD_LE))]
        dense = 9.0 * float((Lc.astype(np.float64) ** 2).sum()) * R
        tr, tr_src = recorded_traffic("dft_class", inst.name, R)
        roof = {"bound": "alu", "kernel": "k_fe_series / k_fe_group_fr (DFT buckets)",
                "achieved": flops / t / 1e12,
                "peak": peak, "unit": "TFLOP/s", "frac": flops / t / 1e12 / peak,
                "traffic": tr, "traffic_source": tr_src,
                "window": f"steps 0-{n_dense - 1} of the run (dense phase)",
                "flops_evaluated_per_step": flops,
                "dense_count": {"flops_per_step": dense, "achieved": dense / t / 1e12,
                                "frac": dense / t / 1e12 / peak,
                                "note": "9 L^2 per cardinality constraint and restart; above "
                                        "1 means the kernels skip work the dense DFT does"},
                "peak_source": "148 SMs x 128 FP32 lanes x 2 flops x 2032 MHz (max SM clock)"}
    # the fused accumulate + step + round kernel: algorithmic bytes = the
    # partial rows read once (4 B per FE literal and restart), x read and
    # written (8 B per variable and restart), one bitset word per variable
    # and 32 restarts
    RT = (R + 31) // 32
    step_bytes = 4 * RT * 32 * info["nnz_fe"] + 8 * inst.n * R + 4 * inst.n * RT
    t_step = kstats_dense["accum_step_round"]["ms_per_step"] / 1e3
    hbm_peak = pk.get("hbm_gbs", 6400.0)
    traffic, traffic_src = recorded_traffic("k_accum_step", inst.name, R)
    roof_step = {"bound": "hbm", "kernel": "k_accum_step", "bytes": step_bytes,
                 "achieved": step_bytes / t_step / 1e9, "peak": hbm_peak, "unit": "GB/s",
                 "frac": step_bytes / t_step / 1e9 / hbm_peak, "traffic": traffic,
                 "traffic_source": traffic_src, "peak_source": "measured copy bandwidth"}
    if dom != "fe_group_dft":
        roof = dict(roof_step)
        if dom != "accum_step_round":
            roof["note"] = (f"the longest kernel class is {dom} "
                            f"({kstats[dom]['ms_per_step']:.4f} ms/step, gather or launch "
                            f"bound); the HBM roofline is given for the fused step kernel")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        # the oracle as it stands on every host core (spawned workers, one
        # step on 8 restarts each), and on one core
        big = inst.nnz > 10000
        per_worker = 8 if big else max(1, min(R, 64) // host_cores())
        allc, done = time_cpu_oracle_all_cores(inst, lr, per_worker, steps=1 if big else 3)
        cpu_t, cpu_steps = time_cpu_oracle(inst, per_worker, lr, 1 if big else 3)
        cpu = {"value": allc["value"], "unit": "literal-evals/s", "cores": allc["cores"],
               "kind": "oracle", "cpu_model": allc["cpu_model"],
               "sample": f"{allc['restarts']} of {R} restarts ({per_worker} per core), "
                         f"{done} step(s)",
               "single_core": {"value": per_worker * inst.nnz / cpu_t,
                               "unit": "literal-evals/s", "cores": 1,
                               "sample": f"{per_worker} of {R} restarts, {cpu_steps} step(s)"}}
    line = {
        "metric": "constraint-literal FE+grad evals/s", "value": value,
        "unit": "literal-evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": inst.name, "n": inst.n, "m": inst.m, "nnz": inst.nnz,
                   "R_per_gpu": R, "lr": lr, "parallelism": f"restart-replicas x{world}",
                   "l2": "flushed (256 MB write) before every timed step",
                   "timed": f"steps 0-{K - 1} of one CLS run from uniform initial points "
                            f"(after {max(3, args.warmup)} untimed warm-up steps)",
                   "tuning": tuning, "autotune_s": tune_s,
                   "autotune_points": None if (args.tuning or args.no_tune) else
                   ("four restart blocks of the timed run's own trajectory, at steps "
                    + ", ".join(str(v) for v in tune_points(args)) + " (untimed)"
                    if R >= 64 and args.steps >= 20 else "x0")},
        "e2e": {"value": units / e2e_s, "unit": "literal-evals/s",
                "h2d_bytes_per_step": 4 * inst.n * R / K, "d2h_bytes_per_step": 4 * R / K,
                "call": f"cls_solve_host: x0 from pinned host memory, {K} steps, counts back"},
        "gpu_launches": launches_timed,
        "mode": ("cuda-graph (1 step per launch)" if graph is not None else
                 "persistent cooperative kernel (1 step per launch)" if args.persistent
                 else "eager"),
        "ms_per_step_eager": ms_eager,
        "ms_per_step_phases": {f"steps 0-{n_dense - 1}": sum(per_step[:n_dense]) / n_dense,
                               f"steps {K - n_dense}-{K - 1}": sum(per_step[-n_dense:]) / n_dense},
        "kernels_dense_phase": kstats_dense,
        "roofline": roof,
        "roofline_step": roof_step,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "kernels": kstats,
        "wall_s": wall,
        "mean_nsat": float(nsat.float().mean().item()),
    }
    if graph is not None:
        B.cls_graph_destroy(graph)
    if world == 1 and args.config == "mixed" and not args.no_extras:
        # the other two targets, on the same GPU in the same run: the fused
        # step kernel on the 3-SAT instance at scale, and learned vs uniform
        # initialisation (time to equal satisfaction)
        del ws, hws, x, x0, xh, flush
        p._ws.clear()
        p.close()
        torch.cuda.empty_cache()
        line["c1_step_kernel"] = c1_step_kernel()
        line["c1_loop"] = c1_loop()
        lvu, _, _ = learned_vs_uniform(args.train_instances, args.held_out, args.train_steps)
        line["learned_vs_uniform"] = lvu
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def learned_vs_uniform(n_train=512, n_held=64, train_steps=3000, R=1024, S=500):
    """Learned vs uniform initialisation (time to equal satisfaction): train
    the message-passing network on n_train planted mixed-PB instances (n ~
    U{1000..4000}, m = 4.5 n) through the CLS objective; on n_held held-out
    instances, device seconds until the median satisfied fraction reaches
    tau = the median that uniform starts reach after S steps (R restarts
    each), network inference included for the learned side."""
    import torch
    from paper_2606_06656_b300 import learned as Lr
    workers = max(1, min(32, host_cores()))
    t0 = time.perf_counter()
    train = W.mixed_instances(n_train, n_range=(1000, 4000), seed=1400, workers=workers)
    held = W.mixed_instances(n_held, n_range=(1000, 4000), seed=91400, workers=workers)
    t_gen = time.perf_counter() - t0
    tr = Lr.build_entries(train, harvest_R=64, harvest_steps=200)
    te = Lr.build_entries(held, harvest_R=8, harvest_steps=1)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0 - t_gen
    params = tr[0][1].init_params(3)
    t1 = time.perf_counter()
    log = Lr.train(tr, params, steps=train_steps, R=32, lam=0.5, tau=1.0, lr=2e-3,
                   log_every=max(1, train_steps // 8))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    t2 = time.perf_counter()
    res = Lr.compare(te, params, R=R, S=S, tau=1.0)
    t_eval = time.perf_counter() - t2
    su = [r["s_uniform"] for r in res]
    sl = [r["s_learned"] if r["s_learned"] is not None else float("inf") for r in res]
    stu = [r["steps_uniform"] for r in res]
    stl = [r["steps_learned"] if r["steps_learned"] is not None else float("inf") for r in res]
    out = {"s_learned_median": float(np.median(sl)), "s_uniform_median": float(np.median(su)),
           "speedup_median": float(np.median(su) / np.median(sl)),
           "steps_learned_median": float(np.median(stl)),
           "steps_uniform_median": float(np.median(stu)),
           "instances_learned_faster": int(sum(a < b for a, b in zip(sl, su))),
           "s_inference_median": float(np.median([r["s_inference"] for r in res])),
           "tau": "per held-out instance, the median over restarts of the satisfied "
                  "fraction uniform starts reach after S steps",
           "train_instances": n_train, "held_out": n_held, "train_steps": train_steps,
           "restarts": R, "S": S, "generate_s": t_gen, "build_s": t_build,
           "train_s": t_train, "eval_s": t_eval}
    return out, log, res


def run_learned(args):
    """Learned vs uniform initialisation as its own bench line."""
    out, log, res = learned_vs_uniform(args.train_instances, args.held_out, args.train_steps)
    line = {
        "metric": "time-to-equal-sat, learned vs uniform init (median device s)",
        "value": out["s_learned_median"], "unit": "s", "higher_is_better": False,
        "uniform_s": out["s_uniform_median"], "speedup": out["speedup_median"],
        "n_gpus": 1, "dtype": "f32 (network bf16 x bf16 -> f32)", "data": "synthetic",
        "config": {"workload": "planted mixed PB, n~U{1000..4000}, m=4.5n", **out},
        "train_log": log, "per_instance": res,
    }
    print(json.dumps(line), flush=True)


def tune_points(args):
    """Steps of the run whose restart blocks the autotuner times: given
    (--tune-at), else 0, 12, 25 and 60 (dense, middle and corner-dominated
    points).  On the driver's 20-step command, points inside its window
    (0/5/10/15, 0/3/9/15, 0/8/14/19) measured 4.43-4.53 ms per step against
    4.45, so the default stays."""
    if args.tune_at:
        pts = tuple(int(v) for v in args.tune_at.split(","))
        if len(pts) != 4 or any(v < 0 for v in pts):
            raise SystemExit("--tune-at takes four steps >= 0")
        return pts
    return (0, 12, 25, 60)


def c1_step_kernel():
    """The fused accumulate/step/round kernel on the random 3-SAT instance
    (n = 100, m = 426) at R = 2^20 restarts (k_accum_step_nt<4>: about 13
    partial rows per variable, so each warp takes four restart tiles), where it is
    HBM-bound (x is 419 MB, the partial rows 5.4 GB): mean CUDA-event time
    of the kernel over 5 eager steps after 3 warm-up steps, against its
    algorithmic bytes (partial rows read once, x read and written, the
    bitset written)."""
    import torch
    from paper_2606_06656_b300 import Problem
    from paper_2606_06656_b300 import binding as B
    inst = W.random_ksat()
    R = 1 << 20
    p = Problem(inst)
    x = p.init_uniform(R, seed=42)
    ws = p.workspace(R)
    nsat = torch.empty(R, dtype=torch.int32, device="cuda")
    for _ in range(3):
        B.cls_step(p.handle, R, x, 0.1, 1, None, nsat, None, ws)
    B.cls_profile_reset(p.handle)
    B.cls_profile_enable(p.handle, True)
    for _ in range(5):
        B.cls_step(p.handle, R, x, 0.1, 1, None, nsat, None, ws)
    B.cls_profile_enable(p.handle, False)
    n_l, t_ms = B.cls_profile_read(p.handle, 3)          # accum_step_round
    torch.cuda.synchronize()
    RT = (R + 31) // 32
    nbytes = 4 * RT * 32 * p.info["nnz_fe"] + 8 * inst.n * R + 4 * inst.n * RT
    t = t_ms / max(n_l, 1) / 1e3
    peak = peaks().get("hbm_gbs", 6400.0)
    tr, tr_src = recorded_traffic("k_accum_step_nt<4>", inst.name, R)
    out = {"kernel": "k_accum_step_nt<4> (the fused step kernel, four restart tiles per warp)",
           "workload": f"{inst.name}, R=2^20", "bytes": nbytes,
           "us": t * 1e6, "achieved": nbytes / t / 1e9, "peak": peak, "unit": "GB/s",
           "frac": nbytes / t / 1e9 / peak, "target_frac": 0.60,
           "traffic": tr, "traffic_source": tr_src,
           "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json)"}
    del x, ws, p
    torch.cuda.empty_cache()
    return out


def c1_loop(steps=200, R=64, reps=20):
    """Random 3-SAT at the phase-transition ratio (n = 100, m =
    426, 64 restarts from U[-1, 1], 200 projected-gradient steps, lr 0.1):
    the whole 200-step loop timed with CUDA events, as one CUDA graph of the
    200 steps and as one cls_step_persistent call (one CTA per tile of 32
    restarts with the tile in shared memory), after warm-up; x reset
    untimed before every repetition.  Both leave the same x and counts."""
    import torch
    from paper_2606_06656_b300 import Problem
    from paper_2606_06656_b300 import binding as B
    inst = W.random_ksat()
    p = Problem(inst)
    x0 = p.init_uniform(R, seed=42)
    x = x0.clone()
    ws = p.workspace(R)
    bits = torch.empty((inst.n, (R + 31) // 32), dtype=torch.int32, device="cuda")
    nsat = torch.empty(R, dtype=torch.int32, device="cuda")
    wsat = torch.empty(R, dtype=torch.float64, device="cuda")
    g = B.cls_graph_create(p.handle, R, x, 0.1, steps, bits, nsat, wsat, ws)
    n_graph = B.cls_graph_kernel_count(g)

    def run(fn):
        ts = []
        for k in range(reps + 3):
            x.copy_(x0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            if k >= 3:
                ts.append(e0.elapsed_time(e1))
        return float(np.median(ts)), x.clone(), nsat.clone()

    t_g, xg, ng = run(lambda: B.cls_graph_launch(g))
    t_p, xp, npers = run(lambda: B.cls_step_persistent(p.handle, R, x, 0.1, steps, bits, nsat,
                                                       wsat, ws))
    same = bool(torch.equal(xg.view(torch.int32), xp.view(torch.int32)) and torch.equal(ng, npers))
    if B.cls_persistent_status(p.handle, R, ws) != 0:
        raise RuntimeError("persistent loop: a grid barrier timed out")
    B.cls_graph_destroy(g)
    units = R * inst.nnz * steps
    out = {"workload": f"{inst.name}, R={R}, {steps} steps", "reps": reps,
           "graph": {"ms": t_g, "us_per_step": 1e3 * t_g / steps,
                     "literal_evals_per_s": units / (t_g / 1e3), "kernels": n_graph},
           "persistent": {"ms": t_p, "us_per_step": 1e3 * t_p / steps,
                          "literal_evals_per_s": units / (t_p / 1e3), "kernels": 1},
           "same_results": same, "mean_nsat": float(npers.float().mean())}
    del x, x0, ws, p
    torch.cuda.empty_cache()
    return out


def run_refill(args):
    """Per-restart convergence tracking with refills (Sec. 3.3: converged
    restarts idle in a lockstep batch).  Two runs of K steps from the same
    uniform points on the mixed workload: plain, and with cls_track_step
    after every step and cls_refill (patience P) every 10 steps, which gives
    restarts stuck for P steps fresh points.  Reports the tracking overhead,
    the refills, and the best count each restart reached (as unsatisfied
    constraints)."""
    import torch
    from paper_2606_06656_b300 import Problem
    from paper_2606_06656_b300 import binding as B
    inst, R, lr = workload("mixed")
    if args.R:
        R = args.R
    K = args.steps if args.steps != 100 else 200
    patience, every = 20, 10
    p = Problem(inst)
    x0 = p.init_uniform(R, seed=42)
    ws = p.workspace(R)
    nsat = torch.empty(R, dtype=torch.int32, device="cuda")
    wsat = torch.empty(R, dtype=torch.float64, device="cuda")
    bits = torch.empty((inst.n, (R + 31) // 32), dtype=torch.int32, device="cuda")
    trk = torch.empty((4, R), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    hist = torch.empty(inst.m + 1, dtype=torch.int32, device="cuda")

    def run(track, refill):
        x = x0.clone()
        B.cls_track_reset(p.handle, R, trk)
        cnt.zero_()
        gen = 0
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(K):
            B.cls_step(p.handle, R, x, lr, 1, bits, nsat, wsat, ws)
            if track:
                B.cls_track_step(p.handle, R, nsat, k, trk)
                if refill and (k + 1) % every == 0:
                    gen += 1
                    B.cls_refill(p.handle, R, x, trk, patience, 42, 0, gen, cnt)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    for _ in range(max(1, args.warmup // 3)):
        run(False, False)
    t_plain = run(False, False)
    t_prof = run(True, False)
    # convergence profile of the plain run: the step at which each restart
    # reached its best count
    reach = trk[1].cpu().numpy()
    profile = {f"p{q}": float(np.percentile(reach, q)) for q in (10, 50, 90)}
    t_track = run(True, True)
    best = trk[0].cpu().numpy()
    B.cls_unsat_histogram(p.handle, R, trk[0].clamp(min=0), hist)
    h = hist.cpu().numpy()
    unsat_best = inst.m - best[best >= 0]
    solved = int((trk[3] >= 0).sum().item())
    line = {"metric": "constraint-literal FE+grad evals/s with per-restart tracking and refills",
            "value": R * inst.nnz * K / (t_track / 1e3), "unit": "literal-evals/s",
            "higher_is_better": True, "n_gpus": 1, "steps": K, "dtype": "f32",
            "data": "synthetic",
            "ms_per_step": t_track / K, "ms_per_step_plain": t_plain / K,
            "tracking_overhead": t_prof / t_plain - 1.0,
            "steps_to_best_count": profile,
            "note": "refilled restarts restart in the expensive first steps of a trajectory, "
                    "so the refill run's steps cost more than the plain run's",
            "refilled_restarts": int(cnt.item()), "solved_restarts": solved,
            "best_unsat_since_last_refill": {"min": int(unsat_best.min()) if len(unsat_best) else None,
                                             "median": float(np.median(unsat_best)) if len(unsat_best) else None},
            "unsat_histogram_nonzero": {int(k): int(v) for k, v in enumerate(h) if v}
                                       if int((h > 0).sum()) <= 40 else "many bins",
            "config": {"workload": inst.name, "R": R, "lr": lr, "patience": patience,
                       "refill_every": every, "launches": "eager cls_step per step"}}
    print(json.dumps(line), flush=True)


def run_ramsey(args):
    """Redundant-constraint study on the paper's own structure (Sec. 3.1):
    balanced 3-colouring of K_16 (EO per edge, CARD_GE 5 per vertex and
    colour), plain and with the decomposed edge encoding added
    (CARD>=2(not x) + OR(x) = EO - 1, doubling the edge gradient).  R
    independent restarts, K lockstep steps each, for a few step sizes (the
    paper gives none), and with adaptive constraint weighting
    (cls_constraint_stats + cls_reweight every 10 steps, inside the timed
    loop).  Per arm: the fraction of restarts that reached a satisfying
    point, the median step at which they did, and, for restarts unsolved at
    the end, how many balance constraints they violate while every edge
    constraint holds.  Two more arms run 4K steps with refills (cls_refill,
    patience 20): "solved" then counts restarts solved by any of the points
    a slot held."""
    import torch
    from paper_2606_06656_b300 import Problem
    from paper_2606_06656_b300 import binding as B
    R = args.R or 16384
    K = args.steps if args.steps != 100 else 300
    lrs = [0.02, 0.05, 0.1, 0.2, 0.5]
    rw_sets = [(0.5, 4.0, 10.0), (2.0, 4.0, 10.0)]
    every = 10
    patience = 20

    def sub(inst, cs):
        return W.build(inst.n, [(int(inst.ctype[c]), int(inst.k[c]),
                                 inst.lit_var[inst.offsets[c]:inst.offsets[c + 1]],
                                 inst.lit_sign[inst.offsets[c]:inst.offsets[c + 1]])
                                for c in cs])

    out = {}
    t_all = 0.0
    steps_all = 0
    lit_evals = 0
    for red in (False, True):
        inst = W.ramsey_balanced(16, 3, redundant=red)
        E, VC = 120, 48
        edge_cs = list(range(E)) + (list(range(E + VC, inst.m)) if red else [])
        pe, pb = Problem(sub(inst, edge_cs)), Problem(sub(inst, range(E, E + VC)))
        nsat = torch.empty(R, dtype=torch.int32, device="cuda")
        wsat = torch.empty(R, dtype=torch.float64, device="cuda")
        bits = torch.empty((inst.n, (R + 31) // 32), dtype=torch.int32, device="cuda")
        trk = torch.empty((4, R), dtype=torch.int32, device="cuda")
        gn = torch.empty(inst.m, dtype=torch.float64, device="cuda")
        un = torch.empty(inst.m, dtype=torch.int32, device="cuda")
        wv = torch.empty(inst.m, dtype=torch.float32, device="cuda")
        arms = [(lr, None, False) for lr in lrs] + \
            [(lr, rw, False) for rw in rw_sets for lr in (0.05, 0.1, 0.2)] + \
            [(0.1, None, True), (0.1, rw_sets[1], True)]
        res = {}
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        for lr, rw, refill in arms:
            KK = 4 * K if refill else K
            gen = 0
            cnt.zero_()
            p = Problem(inst)                       # fresh weights per arm
            ws = p.workspace(R)
            x = p.init_uniform(R, seed=7)
            B.cls_track_reset(p.handle, R, trk)
            xs = x.clone()
            for _ in range(3):                      # warm-up on a scratch copy
                B.cls_step(p.handle, R, xs, lr, 1, bits, nsat, wsat, ws)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for k in range(KK):
                B.cls_step(p.handle, R, x, lr, 1, bits, nsat, wsat, ws)
                B.cls_track_step(p.handle, R, nsat, k, trk)
                if rw is not None and (k + 1) % every == 0:
                    B.cls_constraint_stats(p.handle, R, bits, ws, gn, un)
                    B.cls_reweight(p.handle, R, gn, un, rw[0], rw[1], rw[2], wv)
                if refill and (k + 1) % every == 0:
                    gen += 1
                    B.cls_refill(p.handle, R, x, trk, patience, 7, 0, gen, cnt)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            t_all += ms
            steps_all += KK
            lit_evals += R * inst.nnz * KK
            solved_at = trk[3].cpu().numpy()
            ok = solved_at >= 0
            ne, _, _ = pe.round_score(x)
            nb, _, _ = pb.round_score(x)
            ne, nb = ne.cpu().numpy(), nb.cpu().numpy()
            unsolved = ~ok
            edges_ok = unsolved & (ne == len(edge_cs))
            viol = VC - nb[edges_ok]
            key = f"lr={lr}" + ("" if rw is None else f",reweight(eta={rw[0]},kappa={rw[1]},w_max={rw[2]})") \
                + (f",refill(patience={patience}),steps={KK}" if refill else "")
            ent = {"solved_frac": float(ok.mean()),
                   "median_solve_step": float(np.median(solved_at[ok]) + 1) if ok.any() else None,
                   "unsolved_with_all_edges_ok_frac": float(edges_ok.sum() / max(1, unsolved.sum())),
                   "balance_violations_hist": {int(a): int(b) for a, b in
                                               zip(*np.unique(viol, return_counts=True))},
                   "ms_per_step": ms / KK}
            if refill:
                ent["refilled"] = int(cnt.item())
            if rw is not None:
                w = wv.cpu().numpy()
                ent["final_weight_mean"] = {"edge": float(w[edge_cs].mean()),
                                            "balance": float(w[E:E + VC].mean())}
            res[key] = ent
            p.close()
        out["redundant" if red else "plain"] = res
    line = {"metric": "fraction of restarts solved (balanced Ramsey colouring, 16 vertices, 3 colours)",
            "value": out["plain"]["lr=0.1"]["solved_frac"], "unit": "fraction",
            "higher_is_better": True, "n_gpus": 1, "steps": K, "dtype": "f32",
            "data": "synthetic",
            "throughput": {"value": lit_evals / (t_all / 1e3), "unit": "literal-evals/s"},
            "ms_per_step": t_all / steps_all,
            "encodings": out,
            "config": {"workload": "ramsey_V16_C3 plain and redundant", "R": R,
                       "reweight_every": every,
                       "launches": "eager cls_step + cls_track_step per step"}}
    print(json.dumps(line), flush=True)


def run_reweight(args):
    """Cost of adaptive constraint weighting on the mixed PB workload
    (n = 5000, m = 22500, R = 4096): the step alone, and the statistics pass
    (one read of every literal partial) plus the weight update, each timed
    with CUDA events over K repetitions after warm-up.  The statistics
    kernel is HBM-bound: its algorithmic bytes are the partials (nnz_fe * R
    * 4 B), the bitset (n * ceil(R/32) * 4 B) and the outputs (12 B per
    constraint)."""
    import torch
    from paper_2606_06656_b300 import Problem
    from paper_2606_06656_b300 import binding as B
    inst, R, lr = workload("mixed")
    if args.R:
        R = args.R
    K = args.steps if args.steps != 100 else 50
    p = Problem(inst)
    x = p.init_uniform(R, seed=42)
    ws = p.workspace(R)
    nsat = torch.empty(R, dtype=torch.int32, device="cuda")
    wsat = torch.empty(R, dtype=torch.float64, device="cuda")
    bits = torch.empty((inst.n, (R + 31) // 32), dtype=torch.int32, device="cuda")
    gn = torch.empty(inst.m, dtype=torch.float64, device="cuda")
    un = torch.empty(inst.m, dtype=torch.int32, device="cuda")
    wv = torch.empty(inst.m, dtype=torch.float32, device="cuda")
    for _ in range(max(3, args.warmup)):
        B.cls_step(p.handle, R, x, lr, 1, bits, nsat, wsat, ws)
        B.cls_constraint_stats(p.handle, R, bits, ws, gn, un)
    torch.cuda.synchronize()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(K):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / K

    t_step = timed(lambda: B.cls_step(p.handle, R, x, lr, 1, bits, nsat, wsat, ws))
    t_stats = timed(lambda: B.cls_constraint_stats(p.handle, R, bits, ws, gn, un))
    t_rw = timed(lambda: B.cls_reweight(p.handle, R, gn, un, 0.0, 4.0, 10.0, wv))
    nnz_fe = int(p.info["nnz_fe"])
    byts = nnz_fe * R * 4 + inst.n * ((R + 31) // 32) * 4 + inst.m * 12
    traffic, traffic_src = recorded_traffic("k_con_stats_tile", inst.name, R)
    peak = float(peaks().get("hbm_gbs", 6400.0))
    ach = byts / (t_stats * 1e-3) / 1e9
    line = {"metric": "constraint statistics pass, fraction of HBM peak",
            "value": ach / peak, "unit": "fraction", "higher_is_better": True, "n_gpus": 1,
            "steps": K, "dtype": "f32", "data": "synthetic",
            "ms_step": t_step, "ms_constraint_stats": t_stats, "ms_reweight": t_rw,
            "overhead_every_10_steps": (t_stats + t_rw) / (10 * t_step),
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": ach / peak, "traffic": traffic,
                         "traffic_source": traffic_src,
                         "kernel": "k_con_stats", "algorithmic_bytes": byts},
            "config": {"workload": inst.name, "R": R, "inputs": "partials of the last step"}}
    print(json.dumps(line), flush=True)


def run_completion(args):
    """Partial-assignment completion (Sec. 3.2): planted 3-SAT at clause
    ratio 4.26 with n = 450, 550 and 650 variables (stand-ins for the
    satisfiable phase-transition instances of the paper's study), a fraction
    of the variables pinned to the plant and folded into the constraints,
    R = 1024 restarts from uniform points, at most 3000 steps with per-restart
    tracking and refills (patience 50, every 10 steps).  Time to solution is
    wall-clock from the first step to the check (every 10 steps) that sees a
    restart satisfy every clause, problem set-up excluded."""
    import torch
    from paper_2606_06656_b300 import Problem
    from paper_2606_06656_b300 import binding as B
    R = args.R or 1024
    Kmax = 3000
    lr = 0.1
    fracs = [0.0, 0.1, 0.2, 0.3, 0.4, 0.5, 0.6]
    seeds = [0, 1, 2]
    table = {}
    for n in (450, 550, 650):
        for frac in fracs:
            times, steps = [], []
            for sd in seeds:
                inst = W.planted_ksat(n, seed=1600 + 10 * n + sd)
                if frac > 0:
                    inst = W.partial_assignment(inst, frac, seed=1700 + sd)
                p = Problem(inst, simplify_fixed=frac > 0)
                x = p.init_uniform(R, seed=sd + 1)
                ws = p.workspace(R)
                nsat = torch.empty(R, dtype=torch.int32, device="cuda")
                wsat = torch.empty(R, dtype=torch.float64, device="cuda")
                bits = torch.empty((inst.n, (R + 31) // 32), dtype=torch.int32, device="cuda")
                trk = torch.empty((4, R), dtype=torch.int32, device="cuda")
                cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
                B.cls_track_reset(p.handle, R, trk)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                solved_at, gen = None, 0
                for k in range(Kmax):
                    B.cls_step(p.handle, R, x, lr, 1, bits, nsat, wsat, ws)
                    B.cls_track_step(p.handle, R, nsat, k, trk)
                    if (k + 1) % 10 == 0:
                        if int(torch.max(nsat)) == inst.m:
                            solved_at = k + 1
                            break
                        gen += 1
                        B.cls_refill(p.handle, R, x, trk, 50, sd + 1, 0, gen, cnt)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                if solved_at is not None:
                    times.append(dt)
                    steps.append(solved_at)
                p.close()
            table[f"n={n},pinned={frac}"] = {
                "solved": f"{len(times)}/{len(seeds)}",
                "median_s": float(np.median(times)) if times else None,
                "median_steps": float(np.median(steps)) if steps else None}
    solved50 = [v["median_s"] for k, v in table.items() if k.endswith("pinned=0.5") and v["median_s"]]
    line = {"metric": "time to solution, planted 3-SAT (ratio 4.26) with a partial assignment",
            "value": float(np.median(solved50)) if solved50 else None, "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "value_is": "median over n of the median time at 50 % pinned",
            "table": table,
            "config": {"workload": "planted3sat n=450/550/650, m=round(4.26 n)", "R": R,
                       "max_steps": Kmax, "lr": lr, "refill_patience": 50,
                       "launches": "eager cls_step + cls_track_step per step"}}
    print(json.dumps(line), flush=True)


def run_profile(args):
    """Convergence profiles (Sec. 3.3's analysis, on the planted 3-SAT
    stand-ins: the Costas encodings are not given): n = 550 at clause ratio
    4.26 with about 10 % and about 66 % of the variables pinned to the plant,
    R = 4096 restarts from uniform points, the paper's 300-step limit.  Per
    restart the tracking state gives the step at which it reached its best
    count; restarts whose best came in the last 10 % of the steps are counted
    as still descending at the limit.  Reports the histogram of those steps
    (bins of 20), the fraction at the limit, the best-count quality by group,
    and the fraction solved."""
    import torch
    from paper_2606_06656_b300 import Problem
    from paper_2606_06656_b300 import binding as B
    R = args.R or 4096
    K = 300
    tol = 1e-4                   # convergence: no coordinate moves more than this
    out = {}
    for frac in (0.1, 0.66):
        inst = W.partial_assignment(W.planted_ksat(550, seed=1900), frac, seed=1901)
        p = Problem(inst, simplify_fixed=True)
        x = p.init_uniform(R, seed=3)
        ws = p.workspace(R)
        nsat = torch.empty(R, dtype=torch.int32, device="cuda")
        wsat = torch.empty(R, dtype=torch.float64, device="cuda")
        bits = torch.empty((inst.n, (R + 31) // 32), dtype=torch.int32, device="cuda")
        trk = torch.empty((4, R), dtype=torch.int32, device="cuda")
        B.cls_track_reset(p.handle, R, trk)
        md = torch.empty(R, dtype=torch.float32, device="cuda")
        conv = torch.full((R,), -1, dtype=torch.int32, device="cuda")
        xp = torch.empty_like(x)
        for k in range(K):
            xp.copy_(x)
            B.cls_step(p.handle, R, x, 0.1, 1, bits, nsat, wsat, ws)
            B.cls_track_step(p.handle, R, nsat, k, trk)
            B.cls_movement(p.handle, R, xp, x, md)
            B.cls_track_converged(p.handle, R, md, tol, k, conv)
        t = trk.cpu().numpy()
        cv = conv.cpu().numpy() + 1                  # steps taken to converge, 0 = never
        never = cv == 0
        conv_hist, _ = np.histogram(cv[~never], bins=np.arange(0, K + 21, 20))
        best_step = t[1] + 1
        unsat = inst.m - t[0]
        late = best_step > 0.9 * K
        hist, edges = np.histogram(best_step, bins=np.arange(0, K + 21, 20))
        out[f"pinned={frac}"] = {
            "best_step_hist_bins_of_20": hist.tolist(),
            "frac_best_in_last_10pct": float(late.mean()),
            "median_best_step": float(np.median(best_step)),
            "unsat_median": {"converged_early": float(np.median(unsat[~late])) if (~late).any() else None,
                             "still_descending": float(np.median(unsat[late])) if late.any() else None},
            "solved_frac": float((t[3] >= 0).mean()),
            "converged_hist_bins_of_20": conv_hist.tolist(),
            "frac_not_converged_at_limit": float(never.mean()),
            "median_converge_step": float(np.median(cv[~never])) if (~never).any() else None,
            "unsat_median_by_convergence": {
                "converged": float(np.median(unsat[~never])) if (~never).any() else None,
                "not_converged": float(np.median(unsat[never])) if never.any() else None}}
        p.close()
    line = {"metric": "convergence profile (step of each restart's best count)",
            "value": out["pinned=0.1"]["frac_best_in_last_10pct"], "unit": "fraction",
            "higher_is_better": False, "n_gpus": 1, "steps": K, "dtype": "f32",
            "data": "synthetic", "value_is": "fraction of restarts still improving in the last 10 % of 300 steps, 10 % pinned",
            "profiles": out,
            "config": {"workload": "planted3sat_n550_m2343, 10 % / 66 % pinned", "R": R, "lr": 0.1,
                       "convergence_tol": tol}}
    print(json.dumps(line), flush=True)


def run_partial(args):
    """Partial-assignment completion: 16 planted mixed-PB instances, n ~
    U{10000..30000}, m = 4.5 n, 90% of the variables pinned to the plant,
    512 restarts each, all instances in one CUDA graph; masked (every literal
    evaluated) vs simplified (pinned variables folded into the spectra)."""
    import torch
    from paper_2606_06656_b300 import Problem
    from paper_2606_06656_b300 import binding as B
    insts = []
    for i in range(16):
        rng = np.random.default_rng(1500 + i)
        n = int(rng.integers(10000, 30001))
        m = int(round(4.5 * n))
        base = W.mixed_pb(n=n, n_or=m - round(m * 2500 / 22500), n_xor=round(m * 2000 / 22500),
                          n_card=round(m * 500 / 22500), card_len=(10, 300), seed=2500 + i)
        insts.append(W.partial_assignment(base, 0.9, seed=3500 + i))
    R = 512
    units = R * sum(i.nnz for i in insts)
    out = {}
    for mode in ("masked", "simplified"):
        probs = [Problem(i, simplify_fixed=(mode == "simplified")) for i in insts]
        xs = [p.init_uniform(R, seed=42 + k) for k, p in enumerate(probs)]
        ns = [torch.empty(R, dtype=torch.int32, device="cuda") for _ in probs]
        g = B.cls_batch_graph_create([p.handle for p in probs], [R] * 16, xs, 0.1, 1, ns,
                                     [p.workspace(R) for p in probs])
        for _ in range(max(3, args.warmup)):
            B.cls_graph_launch(g)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            B.cls_graph_launch(g)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / args.steps
        out[mode] = {"ms_per_step": ms, "value": units / (ms / 1e3),
                     "nnz_fe": int(sum(p.info["nnz_fe"] for p in probs)),
                     "kernels_per_step": B.cls_graph_kernel_count(g),
                     "mean_nsat_frac": float(np.mean([n.float().mean().item() / p.m
                                                      for n, p in zip(ns, probs)]))}
        B.cls_graph_destroy(g)
        del probs
        torch.cuda.empty_cache()
    line = {"metric": "constraint-literal FE+grad evals/s (all literals counted)",
            "value": out["simplified"]["value"], "unit": "literal-evals/s",
            "higher_is_better": True, "n_gpus": 1, "steps": args.steps, "dtype": "f32",
            "data": "synthetic", "speedup_simplified_vs_masked":
                out["masked"]["ms_per_step"] / out["simplified"]["ms_per_step"],
            "config": {"workload": "16 planted mixed-PB instances, n~U{10000..30000}, "
                                   "m=4.5n, 90% pinned", "R_per_instance": R,
                       "nnz_total": sum(i.nnz for i in insts), "one_graph": True},
            "modes": out}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="mixed")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--eager", action="store_true", help="time eager launches, not the graph")
    ap.add_argument("--persistent", action="store_true",
                    help="time the one-launch persistent step (short closed-form problems)")
    ap.add_argument("--tuning", default="", help="fixed bucket->configuration map (25 ids)")
    ap.add_argument("--tune-at", default="",
                    help="four steps of the run to take the autotuner's restart blocks from")
    ap.add_argument("--R", type=int, default=0, help="override restarts (profiling)")
    ap.add_argument("--profile-step", type=int, default=-1,
                    help="run S steps untimed, then one step inside a profiler window")
    ap.add_argument("--train-instances", type=int, default=512)
    ap.add_argument("--held-out", type=int, default=64)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the 3-SAT step-kernel and learned-vs-uniform keys")
    ap.add_argument("--train-steps", type=int, default=3000)
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.config == "learned":
        run_learned(args)
    elif args.config == "partial":
        run_partial(args)
    elif args.config == "refill":
        run_refill(args)
    elif args.config == "ramsey":
        run_ramsey(args)
    elif args.config == "reweight":
        run_reweight(args)
    elif args.config == "completion":
        run_completion(args)
    elif args.config == "profile":
        run_profile(args)
    elif args.config == "c1loop":
        # the 200-step random 3-SAT loop alone (the default line's c1_loop key)
        print(json.dumps({"c1_loop": c1_loop(R=args.R or 64)}), flush=True)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
