"""Throughput of the tree-based column-density hot path on one GB300.

Workload (default): 256^3 uniform leaves (levels 0..8) in a 10 pc box, a
log-normal density n = exp(g) with g a seeded Gaussian random field of power
spectrum P(k) ~ k^-11/3 (mean 30 cm^-3, sigma_ln 2, seed 2), 48 HEALPix
directions.  One step = the per-simulation-step hot path: restriction of the
new leaf densities to every level (cd_tree_update) and the column densities
of every leaf and direction with the screening factor (cd_column_density,
N_H and shield written).  Geometry tables are built once beforehand, as the
precalculation module does (§3.3).

Metric: cell-directions/s = n_leaf * n_dir / step time (CUDA events on the
launching stream, L2 flushed between steps, max over ranks).  The headline
form is the BF16 tensor-core contraction; the same line reports the FP32
plain form ("compare"), the speed-up, and both forms' errors against the
FP64 oracle on a seeded leaf sample.  With --gpus N
every rank runs an independent replica of the workload (replicas only; the
value is the sum over ranks).

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores (the only other place this file runs the oracle).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-directions/s for N_H"
UNIT = "cell-dirs/s"
# algorithmic HBM bytes per cell-direction: the N_H store (4 B) plus, per leaf,
# the density read (4 B), the shield store (4 B) and the coarse-level reads
# (4/7 B: levels 0..L-1 hold 1/7 of the leaf count)
def algo_bytes_per_cell_dir(nd: int) -> float:
    return 4.0 + (4.0 + 4.0 + 4.0 / 7.0) / nd


def _rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def init_replicas(backend: str = "nccl"):
    """One process per GPU, launched by torch.distributed.run: (rank, world,
    local_rank, dist or None).  The process group exists only when WORLD_SIZE
    > 1; the replicas share nothing but the timing barrier and the max over
    ranks (the path has no exchange step).  With nccl the caller has set the
    CUDA device of local_rank."""
    rank, world, local = _rank()
    if world == 1:
        return rank, world, local, None
    import torch
    import torch.distributed as dist
    if backend == "nccl":
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist.init_process_group(backend)
    return rank, world, local, dist


def max_over_ranks(x: float, dist, device=None) -> float:
    """The largest x over the ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# nominal HBM3e bandwidth of the part, beside the measured copy peak
NOMINAL_HBM_GBS = 8000.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "samples": len(sm),
                "reasons": sorted(reasons)}


# source file of each kernel kind (the BF16 form.s leaf kernel lives in leaf_tc.cu)
KERNEL_SOURCES = {"leaf": "leaf.cu", "leaf_tc": "leaf_tc.cu", "shell": "colden_tc.cu", "restrict": "tree.cu"}


def _source_hash(name):
    import hashlib
    path = os.path.join(ROOT, "paper_1410_0624_gb300", "csrc", name)
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def measured_traffic(kind, L, nd, precision="bf16"):
    """DRAM bytes per step of a kernel kind (all its launches of one step) from
    the committed ncu summary (profiles/traffic.json), or None when the kernel
    source changed since."""
    if kind == "leaf" and precision == "bf16":
        kind = "leaf_tc"
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tr = json.load(f)
        e = tr.get("%s/L%d/nd%d" % (kind, L, nd))
        if e and e.get("source_sha256_16") == _source_hash(KERNEL_SOURCES[kind]):
            return e.get("dram_bytes_per_step", e.get("dram_bytes_per_launch"))
    except Exception:
        pass
    return None


def make_workload(args):
    from paper_1410_0624_gb300 import synth
    n = 1 << args.level
    t0 = time.time()
    rho = synth.lognormal_grf(n, 30.0, 2.0, seed=2)
    return rho, 10.0 * synth.PC_CM, time.time() - t0


def _sample_ijk(L, n, seed=11):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 1 << L, size=(n, 3)).astype(np.int64)


def _morton(ijk):
    m = np.zeros(len(ijk), dtype=np.int64)
    for b in range(21):
        for a in range(3):
            m |= ((ijk[:, a] >> b) & 1) << (3 * b + a)
    return m


def oracle_sample(rho, box, L, nside, target_s, min_leaves=16, max_leaves=400000, cone=False):
    """Times the FP64 oracle on a seeded leaf sample sized for ~target_s seconds.
    Returns (cell-dirs/s, n_leaves, seconds, ijk, N_ref); cone: the
    cone-averaged column (the mean over each direction's sub-rays)."""
    import oracle
    T = oracle.Tree.uniform(rho, box)
    dirs = oracle.dirs_healpix(nside)
    n = min_leaves
    while True:
        ijk = _sample_ijk(L, n)
        t0 = time.perf_counter()
        if cone:
            ref = T.column_density_cone(dirs, np.full(n, L), ijk)
        else:
            ref = T.column_density(dirs, np.full(n, L), ijk)
        dt = time.perf_counter() - t0
        if dt >= target_s or n >= max_leaves:
            return n * len(dirs) / dt, n, dt, ijk, ref
        n = int(min(max_leaves, max(2 * n, n * target_s / max(dt, 1e-3) * 1.1)))


def run_reference(args):
    rank, world, _ = _rank()
    if rank != 0:
        return 0
    rho, box, _ = make_workload(args)
    L, nd = args.level, 12 * args.nside ** 2
    # calibrate one step to ~2 s of CPU work, then time W + K such steps
    rate, n, dt, _, _ = oracle_sample(rho, box, L, args.nside, 2.0)
    import oracle
    T = oracle.Tree.uniform(rho, box)
    dirs = oracle.dirs_healpix(args.nside)
    times = []
    for s in range(args.warmup + args.steps):
        ijk = _sample_ijk(L, n, seed=100 + s)
        t0 = time.perf_counter()
        T.column_density(dirs, np.full(n, L), ijk)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    value = n * nd / (ms / 1e3)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "uniform %d^3 leaves, 10 pc, k^-11/3 log-normal (mean 30, sigma_ln 2, seed 2), "
                                   "%d HEALPix dirs" % (1 << L, nd), "sample_leaves_per_step": n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d seeded random leaves x %d dirs per step" % (n, nd)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _time_steps(step, flush, stream, steps):
    """Mean device time of `steps` calls of step(), L2 flushed before each."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in ev]))


def _kernel_breakdown(colden, step, flush, steps):
    """Per-kind launches, device ms and dense tensor-core flops per step
    (events on the launching stream)."""
    import torch
    colden.stats_reset(timing=True)
    for _ in range(steps):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    out = {}
    for k, name in enumerate(colden.KERNEL_KINDS):
        n, kms = colden.stats_get(k)
        if n:
            out[name] = {"launches_per_step": n / steps, "ms_per_step": kms / steps}
            fl = colden.stats_flops(k)
            if fl > 0:
                out[name]["tensor_flops_per_step"] = fl / steps
    colden.stats_reset(timing=False)
    return out


def _tensor_fraction(kern):
    """Dense BF16 tensor throughput of each kernel kind that issues tcgen05
    MMAs (its flops per step over its device time per step), against the
    measured sustained BF16 peak: these kernels run inside a longer step."""
    peak, kind = _tensor_peak(sustained=True)
    out = {}
    for name, k in kern.items():
        fl = k.get("tensor_flops_per_step", 0.0)
        if fl > 0 and k["ms_per_step"] > 0:
            tf = fl / (k["ms_per_step"] / 1e3) / 1e12
            out[name] = {"TFLOP/s": tf, "frac": tf / peak, "flops_per_step": fl}
    return {"peak": peak, "peak_kind": kind, "unit": "TFLOP/s", "kernels": out} if out else None


def _errors(got_nh, got_sh, ref):
    import oracle
    rel = np.abs(got_nh - ref) / ref
    return {"n_h_rel_max": float(rel.max()), "n_h_rel_p99": float(np.percentile(rel, 99)),
            "a_v_abs_max": float((np.abs(got_nh - ref) / 1.87e21).max()),
            "shield_abs_max": float(np.max(np.abs(got_sh - oracle.shield(ref)))), "leaves_checked": int(len(ref))}


def run_ours(args):
    import torch
    from paper_1410_0624_gb300 import colden

    torch.cuda.set_device(_rank()[2])
    rank, world, local, dist = init_replicas("nccl")
    colden.load()
    forms = {"fp32": colden.FP32, "bf16": colden.BF16}

    rho_np, box, gen_s = make_workload(args)
    L = args.level
    dev = torch.device("cuda", local)
    rho = torch.from_numpy(rho_np).to(dev).reshape(-1).contiguous()
    tree = colden.build_tree_uniform(rho.reshape(1 << L, 1 << L, 1 << L), box)
    cone = args.geometry == "cone"
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    geom = colden.precompute_geometry("healpix", args.nside, mode=colden.MODE_CONE if cone else colden.MODE_PREC)
    torch.cuda.synchronize()
    geom_ms = 1e3 * (time.perf_counter() - t0)
    nd = geom.n_dir
    n_leaf = tree.n_leaf
    n_h = torch.empty(n_leaf * nd, device=dev)
    sh = torch.empty(n_leaf, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, device=dev)
    stream = torch.cuda.current_stream()

    def make_step(prec):
        def step():
            colden.tree_update(tree, rho, stream=stream)
            colden.column_density(tree, geom, n_h=n_h, shield=sh, precision=forms[prec], stream=stream)
        return step

    def max_ranks(x):
        return max_over_ranks(x, dist, dev)

    # ---- the FP64 oracle on a seeded leaf sample: CPU baseline and reference values ----
    cpu = sample = None
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        rate, n, dt, ijk, ref = oracle_sample(rho_np, box, L, args.nside, args.cpu_seconds, cone=cone)
        cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d seeded random leaves x %d dirs%s (%.1f s)"
                         % (n, nd, " x 32 cone sub-rays" if cone else "", dt)}
        sample = (torch.from_numpy(_morton(ijk)).to(dev), ref)

    def score():
        if sample is None:
            return None
        rows, ref = sample
        return _errors(n_h.reshape(-1, nd)[rows].double().cpu().numpy(), sh[rows].double().cpu().numpy(), ref)

    # ---- the headline form: warm-up, timed steps with clocks sampled ----
    # A step is the density update + evaluation captured once as a CUDA graph
    # (cd_eval_graph) and replayed; --eager times the same calls one by one.
    step = make_step(args.precision)
    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    graph = None
    if not args.eager:
        graph = colden.EvalGraph(tree, geom, rho=rho, n_h=n_h, shield=sh, precision=forms[args.precision],
                                 stream=stream)
        for _ in range(args.warmup):
            flush.zero_()
            graph.launch(stream)
        torch.cuda.synchronize()
    timed = step if graph is None else (lambda: graph.launch(stream))
    clocks = ClockSampler(local)
    colden.stats_reset(timing=False)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ms = _time_steps(timed, flush, stream, args.steps)
    clk = clocks.stop()
    launches = sum(colden.stats_get(k)[0] for k in range(len(colden.KERNEL_KINDS)))
    if dist:
        dist.barrier()
    ms_eager = _time_steps(step, flush, stream, args.steps) if graph is not None else ms
    ms = max_ranks(ms)
    value = n_leaf * nd * world / (ms / 1e3)
    kern = _kernel_breakdown(colden, step, flush, args.steps)
    err = score()

    # ---- dominant kernel roofline (HBM: the algorithmic bytes of the path) ----
    # A kind may run as several launches a step (the BF16 oct level in Morton
    # ranges): bytes per launch / mean launch time = bytes per step / its time
    # per step, each launch timed alone (per-launch timing runs in order).
    dom = max(kern, key=lambda k: kern[k]["ms_per_step"])
    dom_launches = max(kern[dom]["launches_per_step"], 1)
    dom_ms = kern[dom]["ms_per_step"] / dom_launches
    peak, peak_kind = _peaks()
    bpu = algo_bytes_per_cell_dir(nd)
    achieved = bpu * n_leaf * nd / dom_launches / (dom_ms / 1e3) / 1e9
    traffic = measured_traffic(dom, L, nd, args.precision)
    if traffic is not None:
        traffic /= dom_launches

    # ---- the heating epilogue of §5 on the step's screening factor (HBM-bound, timed alone) ----
    heat = None
    if args.heating:
        g = torch.Generator(device=dev).manual_seed(5)
        T_k = 10.0 ** (1.0 + 3.2 * torch.rand(n_leaf, device=dev, generator=g))
        n_e = 10.0 ** (-4.0 + 4.5 * torch.rand(n_leaf, device=dev, generator=g))
        outs = [torch.empty(n_leaf, device=dev) for _ in range(3)]
        hstep = lambda: colden.heating(tree, sh, T_k, n_e, 1.7, *outs, stream=stream)
        for _ in range(args.warmup):
            hstep()
        hms = _time_steps(hstep, flush, stream, args.steps)
        hbytes = 28 * n_leaf
        heat = {"ms": hms, "algo_bytes": hbytes, "GB/s": hbytes / (hms / 1e3) / 1e9,
                "frac": hbytes / (hms / 1e3) / 1e9 / peak, "peak_kind": peak_kind,
                "note": "chi, T, n_e, leaf density in (16 B), G0_eff, Gamma_UV, Gamma_CR out (12 B) per leaf"}

    # ---- the other form (FP32 plain vs BF16 tensor cores), same workload ----
    other = None
    other_name = "fp32" if args.precision == "bf16" else "bf16"
    if not args.no_compare:
        ostep = make_step(other_name)
        for _ in range(args.warmup):
            flush.zero_()
            ostep()
        torch.cuda.synchronize()
        oms = max_ranks(_time_steps(ostep, flush, stream, args.steps))
        other = {"precision": other_name, "value": n_leaf * nd * world / (oms / 1e3), "ms_per_step": oms,
                 "kernels": _kernel_breakdown(colden, ostep, flush, args.steps), "error_vs_oracle": score()}

    # ---- e2e: host density in, host N_H + shield out, through the C-ABI's host entry point ----
    e2e = None
    if args.e2e_steps > 0:
        h_rho = torch.from_numpy(rho_np.reshape(-1)).pin_memory()
        h_nh = torch.empty(n_leaf * nd, dtype=torch.float32).pin_memory()
        h_sh = torch.empty(n_leaf, dtype=torch.float32).pin_memory()
        times = []
        for s in range(args.e2e_steps + 1):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            colden.column_density_host(tree, geom, rho=h_rho, n_h=h_nh, shield=h_sh,
                                       precision=forms[args.precision], stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            if s > 0:
                times.append(a.elapsed_time(b))
        e_ms = max_ranks(float(np.mean(times)))
        link = 4 * n_leaf * nd + 4 * n_leaf
        e2e = {"value": n_leaf * nd * world / (e_ms / 1e3), "unit": UNIT, "ms_per_step": e_ms,
               "h2d_bytes_per_step": 4 * n_leaf, "d2h_bytes_per_step": link,
               "d2h_GB/s": link / (e_ms / 1e3) / 1e9,
               "api": "cd_column_density_host (pinned host buffers; leaf stage in 8 chunks, copies overlapped)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "bf16",
                "data": "synthetic",
                "config": {"workload": "uniform %d^3 leaves (levels 0..%d), 10 pc box, k^-11/3 log-normal "
                                       "(mean 30, sigma_ln 2, seed 2), %d HEALPix dirs, N_H + shield out%s"
                                       % (1 << L, L, nd, ", cone-averaged factors" if cone else ""),
                           "precision": args.precision, "geometry": args.geometry,
                           "geometry_build_ms": geom_ms,
                           "l2": "512 MB buffer written between timed steps; N_H output (%.2f GB) > L2"
                                 % (4 * n_leaf * nd / 1e9),
                           "parallelism": "replicas" if world > 1 else "single",
                           "launch": "eager calls" if graph is None else
                                     "update + evaluation captured once as a CUDA graph (cd_eval_graph), "
                                     "one graph launch per step",
                           "eager_ms_per_step": ms_eager},
                "gpu_launches": int(launches),
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic, "kernel": dom, "kernel_ms": dom_ms,
                             "launches_per_step": dom_launches, "peak_kind": peak_kind,
                             "algo_bytes_per_cell_dir": bpu, "nominal_peak": NOMINAL_HBM_GBS,
                             "frac_of_nominal": achieved / NOMINAL_HBM_GBS},
                "step_roofline_frac": bpu * n_leaf * nd / (ms / 1e3) / 1e9 / peak,
                "kernels": kern, "clocks": clk, "e2e": e2e, "cpu_baseline": cpu, "error_vs_oracle": err}
        if heat is not None:
            line["heating"] = heat
        if other is not None:
            line["compare"] = other
            line["speedup_vs_" + other_name] = other["ms_per_step"] / ms
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_amr(args):
    """AMR mesh: base 128^3, three levels refined where the block mean exceeds
    10^(2+l) cm^-3 on a k^-11/3 log-normal field at 1024^3 (mean 30, sigma_ln 2,
    seed 2), 20 pc box, 48 HEALPix directions, N_H + screening factor out."""
    import torch
    import oracle
    from paper_1410_0624_gb300 import colden, synth
    rank, world, local = _rank()
    torch.cuda.set_device(local)
    colden.load()
    t0 = time.time()
    lf = args.amr_level          # finest level; the base is three levels coarser
    lb = lf - 3
    lv = synth.amr_leaves_grf_torch(lf, lb, [1e2, 1e3, 1e4], 30.0, 2.0, seed=2)
    torch.cuda.empty_cache()
    box = 20 * synth.PC_CM
    rho = torch.from_numpy(lv["rho"]).cuda()
    tree = colden.build_tree_amr(lb, lf, box, lv["level"], lv["ijk"], lv["rho"])
    build_s = time.time() - t0
    geom = colden.precompute_geometry("healpix", 2)
    nd = geom.n_dir
    n_h = torch.empty(tree.n_leaf * nd, device="cuda")
    sh = torch.empty(tree.n_leaf, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, device="cuda")
    stream = torch.cuda.current_stream()
    prec = {"fp32": colden.FP32, "bf16": colden.BF16}[args.precision]

    def step():
        colden.tree_update(tree, rho, stream=stream)
        colden.column_density(tree, geom, n_h=n_h, shield=sh, precision=prec, stream=stream)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    graph = None
    if not args.eager:
        graph = colden.EvalGraph(tree, geom, rho=rho, n_h=n_h, shield=sh, precision=prec, stream=stream)
        for _ in range(args.warmup):
            flush.zero_()
            graph.launch(stream)
        torch.cuda.synchronize()
    timed = step if graph is None else (lambda: graph.launch(stream))
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    colden.stats_reset(timing=False)
    ms = _time_steps(timed, flush, stream, args.steps)
    clk = clocks.stop()
    launches = sum(colden.stats_get(k)[0] for k in range(len(colden.KERNEL_KINDS)))
    ms_eager = _time_steps(step, flush, stream, args.steps) if graph is not None else ms
    kern = _kernel_breakdown(colden, step, flush, args.steps)
    units = tree.n_leaf * nd
    peak, peak_kind = _peaks()
    bpu = algo_bytes_per_cell_dir(nd)
    err = cpu = None
    if args.cpu_seconds > 0:
        # the FP64 oracle on a seeded sample of >= 1e5 leaves (uniform over the
        # output rows, plus 100 of every level), timed on the host cores and
        # extrapolated to the whole mesh; the same rows give the error
        olv, oijk = tree.leaves()
        rng = np.random.default_rng(3)
        n_s = int(min(tree.n_leaf, max(100_000, args.amr_sample)))
        sel = np.unique(np.concatenate([rng.choice(tree.n_leaf, n_s, replace=False)] +
                                       [rng.choice(np.nonzero(olv == l)[0], 100) for l in range(lb, lf + 1)]))
        T = oracle.Tree.amr(lb, lf, box, lv["level"], lv["ijk"], lv["rho"])
        t0 = time.perf_counter()
        ref = T.column_density(oracle.dirs_healpix(2), olv[sel], oijk[sel])
        dt = time.perf_counter() - t0
        rows = torch.from_numpy(sel).cuda()
        err = _errors(n_h.reshape(-1, nd)[rows].double().cpu().numpy(), sh[rows].double().cpu().numpy(), ref)
        rate = len(sel) * nd / dt
        cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d seeded leaves (uniform over the output rows + 100 per level) x %d dirs (%.1f s); "
                         "extrapolated to all %d leaves: %.1f s per step" % (len(sel), nd, dt, tree.n_leaf,
                                                                           units / rate)}
    dom = max(kern, key=lambda k: kern[k]["ms_per_step"])
    dom_ms = kern[dom]["ms_per_step"]
    # the other form (FP32 list kernels vs BF16 tensor-core lists), same mesh
    other = None
    if not args.no_compare:
        oprec = colden.FP32 if prec == colden.BF16 else colden.BF16

        def ostep():
            colden.tree_update(tree, rho, stream=stream)
            colden.column_density(tree, geom, n_h=n_h, shield=sh, precision=oprec, stream=stream)

        for _ in range(args.warmup):
            flush.zero_()
            ostep()
        torch.cuda.synchronize()
        oms = _time_steps(ostep, flush, stream, args.steps)
        other = {"precision": "fp32" if oprec == colden.FP32 else "bf16", "ms_per_step": oms,
                 "value": units / (oms / 1e3), "kernels": _kernel_breakdown(colden, ostep, flush, args.steps)}
    line = {"metric": METRIC, "value": units / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16" if prec == colden.BF16 else "f32", "data": "synthetic",
            "config": {"workload": ("AMR: base %d^3 + 3 levels (%d^3 effective), 20 pc, k^-11/3 log-normal "
                                    % (1 << lb, 1 << lf)) +
                                   "(mean 30, sigma_ln 2, seed 2), 48 HEALPix dirs, N_H + shield out",
                       "leaves": int(tree.n_leaf), "leaves_per_level": np.bincount(lv["level"])[lb:].tolist(),
                       "refined_octs": int(tree.n_oct), "precision": args.precision, "build_s": build_s,
                       "l2": "512 MB buffer written between timed steps",
                       "launch": "eager calls" if graph is None else
                                 "update + evaluation captured once as a CUDA graph (cd_eval_graph), "
                                 "one graph launch per step",
                       "eager_ms_per_step": ms_eager},
            "gpu_launches": int(launches), "kernels": kern,
            "roofline": {"bound": "hbm", "achieved": bpu * units / (dom_ms / 1e3) / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": bpu * units / (dom_ms / 1e3) / 1e9 / peak, "traffic": None,
                         "kernel": dom, "kernel_ms": dom_ms, "peak_kind": peak_kind,
                         "algo_bytes_per_cell_dir": bpu, "nominal_peak": NOMINAL_HBM_GBS,
                         "frac_of_nominal": bpu * units / (dom_ms / 1e3) / 1e9 / NOMINAL_HBM_GBS,
                         "note": "algorithmic bytes of the whole path over the dominant kernel kind's time"},
            "step_roofline_frac": bpu * units / (ms / 1e3) / 1e9 / peak, "dominant_kernel": dom,
            "tensor": _tensor_fraction(kern), "clocks": clk, "cpu_baseline": cpu, "error_vs_oracle": err}
    if other is not None:
        line["compare"] = other
        line["speedup_vs_" + other["precision"]] = other["ms_per_step"] / ms
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """64 independent boxes of uneven size and depth (screening factor out):
    the captured, autotuned graph vs per-box launches."""
    import torch
    from paper_1410_0624_gb300 import colden, synth
    rank, world, local = _rank()
    torch.cuda.set_device(local)
    colden.load()
    rng = np.random.default_rng(4)
    g12, g48 = colden.precompute_geometry("healpix", 1), colden.precompute_geometry("healpix", 2)
    trees, geoms, desc, srcs = [], [], [], []
    t0 = time.time()
    for i in range(args.boxes):
        base = int(rng.choice([5, 6, 7, 8]))
        ref = int(rng.integers(0, 3))
        sig = float(rng.uniform(1.0, 2.5))
        nd = int(rng.choice([12, 48]))
        lv = synth.amr_leaves_grf_torch(base + ref, base, [10.0 ** (2 + l) for l in range(ref)], 30.0, sig,
                                        seed=1000 + i)
        if ref == 0:
            n = 1 << base
            rho = np.zeros((n, n, n), np.float32)
            rho[lv["ijk"][:, 2], lv["ijk"][:, 1], lv["ijk"][:, 0]] = lv["rho"]
            trees.append(colden.build_tree_uniform(torch.from_numpy(rho).cuda(), 10 * synth.PC_CM))
            srcs.append(("u", rho))
        else:
            trees.append(colden.build_tree_amr(base, base + ref, 10 * synth.PC_CM, lv["level"], lv["ijk"], lv["rho"]))
            srcs.append(("a", lv))
        geoms.append(g12 if nd == 12 else g48)
        desc.append((1 << base, ref, nd, trees[-1].n_leaf))
        torch.cuda.empty_cache()
    gen_s = time.time() - t0
    units = sum(t.n_leaf * g.n_dir for t, g in zip(trees, geoms))
    prec = {"fp32": colden.FP32, "bf16": colden.BF16}[args.precision]
    sh = [torch.empty(t.n_leaf, device="cuda") for t in trees]
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / args.steps

    colden.stats_reset(timing=False)
    eager = lambda: colden.column_density_batch(trees, geoms, shield=sh, precision=prec, stream=stream)
    ms_eager = timed(eager)
    batch = colden.Batch(trees, geoms, shield=sh, precision=prec, stream=stream)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    colden.stats_reset(timing=False)
    ms_graph = timed(lambda: batch.run(stream=stream))
    clk = clocks.stop()
    info = batch.info()
    flush = torch.empty(512 * 1024 * 1024 // 4, device="cuda")
    # per-kind device time of the batch's own launches (with per-launch timing
    # on, cd_batch_run enqueues them directly instead of replaying the graph),
    # and of the per-box launches for comparison
    kern = _kernel_breakdown(colden, lambda: batch.run(stream=stream), flush, 1)
    kern_per_box = _kernel_breakdown(colden, eager, flush, 1)

    # ---- roofline: screening factor only, so the binding roof is the tensor
    # pipe of the shell contraction (the HBM bytes are ~9 B per leaf) ----
    tens = _tensor_fraction(kern)
    dom = "shell" if tens and "shell" in tens["kernels"] else max(kern, key=lambda k: kern[k]["ms_per_step"])
    roof = None
    if tens and dom in tens["kernels"]:
        t = tens["kernels"][dom]
        roof = {"bound": "tensor", "achieved": t["TFLOP/s"], "peak": tens["peak"], "unit": "TFLOP/s",
                "frac": t["frac"], "traffic": None, "kernel": dom, "kernel_ms": kern[dom]["ms_per_step"],
                "launches_per_step": kern[dom]["launches_per_step"], "peak_kind": tens["peak_kind"],
                "flops_per_step": t["flops_per_step"],
                "note": "dense BF16 MMA flops the shell kernels issue (2 M N K, padded tiles included) over their "
                        "summed device time, each launch of the batch timed alone"}

    # ---- FP64 oracle: every box on a seeded leaf sample (error of the replayed
    # screening factor), timed on the host cores ----
    cpu = err = None
    if args.cpu_seconds > 0:
        import oracle
        torch.cuda.synchronize()
        batch.run(stream=stream)
        torch.cuda.synchronize()
        srng = np.random.default_rng(17)
        per = max(200, int(args.batch_sample / len(trees)))
        t_or, n_or, worst, per_box = 0.0, 0, 0.0, []
        for (kind, data), t, g, out in zip(srcs, trees, geoms, sh):
            T = oracle.Tree.uniform(data, 10 * synth.PC_CM) if kind == "u" else \
                oracle.Tree.amr(data["base"], data["lmax"], 10 * synth.PC_CM, data["level"], data["ijk"], data["rho"])
            olv, oijk = t.leaves()
            rows = np.sort(srng.choice(t.n_leaf, size=min(per, t.n_leaf), replace=False))
            ta = time.perf_counter()
            ref = T.column_density(oracle.dirs_healpix(1 if g.n_dir == 12 else 2), olv[rows], oijk[rows])
            t_or += time.perf_counter() - ta
            n_or += len(rows) * g.n_dir
            e = float(np.max(np.abs(out.cpu().numpy()[rows] - oracle.shield(ref))))
            per_box.append(e)
            worst = max(worst, e)
            del T
        cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        cpu = {"value": n_or / t_or, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d seeded leaves per box x its directions, all %d boxes (%.1f s)"
                         % (per, len(trees), t_or)}
        err = {"shield_abs_max": worst, "shield_abs_max_per_box": per_box, "leaves_per_box": per,
               "tolerance": 5e-3 if prec == colden.BF16 else 1e-5}

    line = {"metric": METRIC, "value": units / (ms_graph / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_graph, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "bf16", "data": "synthetic",
            "config": {"workload": "%d boxes: base 32^3..256^3, 0-2 refined levels (thresholds 10^(2+l)), "
                                   "sigma_ln U[1,2.5], 12 or 48 HEALPix dirs, 10 pc, screening factor out"
                                   % args.boxes, "cell_dirs_per_step": units, "precision": args.precision,
                       "boxes": [{"base": b, "refined_levels": r, "n_dir": d, "leaves": n} for b, r, d, n in desc],
                       "generation_s": gen_s,
                       "l2": "inputs (%.1f GB of densities and levels) larger than L2" % (
                           sum(t.n_leaf for t in trees) * 4.6 / 1e9)},
            "gpu_launches": info["kernel_nodes"] * args.steps,
            "batch": {"graph_ms": ms_graph, "per_box_launches_ms": ms_eager, "speedup": ms_eager / ms_graph,
                      "autotune": info},
            "kernels": kern, "kernels_per_box_launches": kern_per_box, "roofline": roof, "tensor": tens,
            "cpu_baseline": cpu, "error_vs_oracle": err,
            "clocks": clk}
    print(json.dumps(line), flush=True)
    batch.free()
    return 0


def _learned_dataset(colden, synth, geom, L, seed, n_rows, x_out, y_out, nt_out=None, nr_out=None):
    """Rows of one seeded training field: network inputs and ray-marched
    targets of a random leaf subset, written into x_out / y_out (and the
    plain and ray-marched columns into nt_out / nr_out when given)."""
    import torch
    rho = synth.lognormal_grf_torch(1 << L, 30.0, 2.0, seed, device="cuda").contiguous()
    tree = colden.build_tree_uniform(rho, 10 * synth.PC_CM)
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    rows = torch.randperm(tree.n_leaf, generator=g)[:n_rows].cuda()
    nd = geom.n_dir
    nt = torch.empty((len(rows), nd), device="cuda") if nt_out is None else nt_out
    nr = torch.empty_like(nt) if nr_out is None else nr_out
    colden.learned_features(tree, geom, x_out, nt, leaves=rows)
    colden.raymarch(tree, geom, nr, leaves=rows)
    colden.learned_targets(nr, nt, y_out)
    tree.free()


def _ray_scores(n_h, sh, nd, rows, n_ray):
    """A_V and screening-factor errors of a form against the exact ray-marcher
    on sampled leaves."""
    import torch
    av = 1.0 / 1.87e21
    got = n_h.reshape(-1, nd)[rows].double()
    ray = n_ray.double()
    dav = (got - ray).abs() * av
    chi_ray = torch.exp(-2.5 * ray * av).mean(dim=1)
    return {"a_v_abs_mean": float(dav.mean()), "a_v_abs_p99": float(torch.quantile(dav.reshape(-1)[:10_000_000], 0.99)),
            "ln_err_mse": float(((got / ray).log() ** 2).mean()),
            "shield_abs_mean": float((sh[rows].double() - chi_ray).abs().mean()), "leaves": int(len(rows))}


def run_learned(args):
    """Learned correction: the network trained on 16 seeded 128^3 fields
    (1M leaves each, ray-marched targets) plus --matched-fields fields at the
    evaluation resolution (other seeds), its training stop chosen on a
    held-out field at that resolution, evaluated on a 512^3 field of the same
    recipe (seed 200).  A network trained on the 128^3 fields alone is
    scored beside it (its per-level inputs do not transfer across
    resolution).  One step = restriction + the BF16 learned form (per-level
    sums, per-oct layer 1, fused per-leaf network, N_H + shield)."""
    import torch
    from paper_1410_0624_gb300 import colden, synth
    rank, world, local = _rank()
    torch.cuda.set_device(local)
    colden.load()
    geom = colden.precompute_geometry("healpix", 2)
    nd = geom.n_dir
    H = 128
    # ---- training set and training (one-off, timed apart) ----
    # 16 seeded 128^3 fields, then resolution-matched fields at the evaluation
    # level (seeds 300+) and a held-out validation field there (seed 400)
    n_fields, rows_per, n_match = 16, args.train_rows, args.matched_fields
    t0 = time.time()
    n_rows = (n_fields + n_match) * rows_per
    # rows drawn in proportion to the squared mean ray-marched A_V: the fit follows the A_V error
    wrow = torch.empty(n_rows, dtype=torch.float64, device="cuda")
    x = torch.empty((n_rows, 8 * nd + 1), device="cuda")
    y = torch.empty((n_rows, nd), device="cuda")
    for i in range(n_fields + n_match):
        lev, seed = (7, 100 + i) if i < n_fields else (args.eval_level, 300 + i - n_fields)
        nr_i = torch.empty((rows_per, nd), device="cuda")
        _learned_dataset(colden, synth, geom, lev, seed, rows_per, x[i * rows_per:(i + 1) * rows_per],
                         y[i * rows_per:(i + 1) * rows_per], nr_out=nr_i)
        wrow[i * rows_per:(i + 1) * rows_per] = (nr_i.double() / 1.87e21).mean(1) ** 2
        del nr_i
    n_val = min(rows_per, 200_000)
    xv = torch.empty((n_val, 8 * nd + 1), device="cuda")
    yv = torch.empty((n_val, nd), device="cuda")
    ntv = torch.empty((n_val, nd), device="cuda")
    nrv = torch.empty((n_val, nd), device="cuda")
    _learned_dataset(colden, synth, geom, args.eval_level, 400, n_val, xv, yv, ntv, nrv)
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    # the 128^3-only network (scored on the evaluation field for comparison)
    net128 = colden.Net(nd, H, synth.mlp_init(nd, H, 12, out_scale=0.1))
    net128.fit_normaliser(x[:n_fields * rows_per])
    colden.train(net128, x[:n_fields * rows_per], y[:n_fields * rows_per], steps=args.train_steps, batch=8192,
                 lr=2e-3, lr_final=1e-4, seed=3)
    net = colden.Net(nd, H, synth.mlp_init(nd, H, 12, out_scale=0.1))
    t0 = time.time()
    net.fit_normaliser(x)
    dv = torch.empty_like(yv)

    def val_dav(nn):
        # training stop: mean |A_V| error on the held-out field at the evaluation resolution
        nn.forward(xv, dv)
        return float(((ntv.double() * torch.exp(dv.double()) - nrv.double()).abs() / 1.87e21).mean())

    losses = colden.train(net, x, y, steps=args.train_steps, batch=8192, lr=2e-3, lr_final=1e-4, seed=3,
                          val=val_dav, eval_every=args.eval_every, row_weights=wrow)
    torch.cuda.synchronize()
    train_s = time.time() - t0
    best_step, best_val = min(net.val_history, key=lambda h: h[1])
    # outside the targets' range (widened by the margin) the plain column is kept
    d_lo, d_hi = net.fit_delta_range(y, args.delta_margin)
    del x, y, xv, yv, ntv, nrv, dv
    torch.cuda.empty_cache()

    # ---- evaluation field ----
    L = args.eval_level
    rho = synth.lognormal_grf_torch(1 << L, 30.0, 2.0, 200, device="cuda").contiguous()
    box = 10 * synth.PC_CM
    tree = colden.build_tree_uniform(rho, box)
    torch.cuda.empty_cache()
    n_leaf = tree.n_leaf
    n_h = torch.empty(n_leaf * nd, device="cuda")
    sh = torch.empty(n_leaf, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, device="cuda")
    stream = torch.cuda.current_stream()
    P = {"fp32": colden.FP32, "bf16": colden.BF16}

    def make_step(prec, learned):
        def step():
            colden.tree_update(tree, rho, stream=stream)
            colden.column_density(tree, geom, n_h=n_h, shield=sh, precision=P[prec], net=net if learned else None,
                                  stream=stream)
        return step

    step = make_step("bf16", True)
    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    colden.device_status()
    clocks = ClockSampler(local)
    colden.stats_reset(timing=False)
    clocks.start()
    time.sleep(0.3)
    ms = _time_steps(step, flush, stream, args.steps)
    clk = clocks.stop()
    launches = sum(colden.stats_get(k)[0] for k in range(len(colden.KERNEL_KINDS)))
    kern = _kernel_breakdown(colden, step, flush, args.steps)
    units = n_leaf * nd

    # ---- accuracy against the exact ray-marcher on sampled leaves ----
    g = torch.Generator(device="cpu")
    g.manual_seed(7)
    rows = torch.randperm(n_leaf, generator=g)[:args.ray_leaves].cuda()
    n_ray = torch.empty((len(rows), nd), device="cuda")
    colden.raymarch(tree, geom, n_ray, leaves=rows)
    forms = {}
    step()
    torch.cuda.synchronize()
    forms["bf16_learned"] = {"ms_per_step": ms, "value": units / (ms / 1e3),
                             "vs_ray_marcher": _ray_scores(n_h, sh, nd, rows, n_ray)}
    # the 128^3-only network on the same leaves (FP32 forward on the sampled leaves' inputs)
    xs = torch.empty((len(rows), 8 * nd + 1), device="cuda")
    nts = torch.empty((len(rows), nd), device="cuda")
    colden.learned_features(tree, geom, xs, nts, leaves=rows)
    ds = torch.empty_like(nts)
    net128.forward(xs, ds)
    torch.cuda.synchronize()
    n128 = nts.double() * torch.exp(ds.double())
    forms["learned_128_only"] = {
        "vs_ray_marcher": {"a_v_abs_mean": float(((n128 - n_ray.double()).abs() / 1.87e21).mean()),
                           "ln_err_mse": float(((n128 / n_ray.double()).log() ** 2).mean()),
                           "leaves": int(len(rows))},
        "note": "network trained on the 16 128^3 fields alone (no resolution-matched rows), FP32 forward"}
    del xs, nts, ds, n128
    for name, prec, learned, k in (("bf16_plain", "bf16", False, args.steps), ("fp32_plain", "fp32", False, args.steps),
                                   ("fp32_learned", "fp32", True, 1)):
        if args.no_compare and name != "bf16_plain":
            continue
        st = make_step(prec, learned)
        flush.zero_()
        st()
        torch.cuda.synchronize()
        oms = _time_steps(st, flush, stream, k)
        st()
        torch.cuda.synchronize()
        forms[name] = {"ms_per_step": oms, "value": units / (oms / 1e3),
                       "vs_ray_marcher": _ray_scores(n_h, sh, nd, rows, n_ray)}

    # ---- parity with the FP64 oracle on sampled leaves (seeded weights) ----
    parity = cpu = None
    if args.cpu_seconds > 0:
        parity, cpu = _learned_oracle_checks(colden, synth, tree, geom, rho, box, L, args.cpu_seconds)

    # ---- dominant kernel: the fused per-leaf kernel ----
    dom = max(kern, key=lambda k: kern[k]["ms_per_step"])
    dom_ms = kern[dom]["ms_per_step"] / max(kern[dom]["launches_per_step"], 1)
    hbm_peak, peak_kind = _peaks()
    tflops_peak, tpk = _tensor_peak()
    # algorithmic work per leaf of learned_cell_tc: tensor FLOPs of the three
    # per-leaf products (unpadded) and the HBM bytes it must move
    flop_leaf = 2.0 * H * ((nd + 1) + H + nd)
    bytes_leaf = 4.0 * nd + 4 + 4 + (2.0 * H + 4.0 * nd) / 8
    t_achieved = flop_leaf * n_leaf / (kern["learned"]["ms_per_step"] / 1e3) / 1e12 if "learned" in kern else None
    h_achieved = bytes_leaf * n_leaf / (kern["learned"]["ms_per_step"] / 1e3) / 1e9 if "learned" in kern else None
    roof = {"bound": "tensor", "achieved": t_achieved, "peak": tflops_peak, "unit": "TFLOP/s",
            "frac": t_achieved / tflops_peak if t_achieved else None, "traffic": None, "kernel": "learned",
            "kernel_ms": kern.get("learned", {}).get("ms_per_step"), "peak_kind": tpk,
            "algo_flop_per_leaf": flop_leaf,
            "hbm": {"achieved": h_achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": h_achieved / hbm_peak if h_achieved else None, "algo_bytes_per_leaf": bytes_leaf}}
    if roof["hbm"]["frac"] and roof["frac"] and roof["hbm"]["frac"] > roof["frac"]:
        roof.update({"bound": "hbm", "achieved": h_achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": roof["hbm"]["frac"]})
    line = {"metric": METRIC, "value": units / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "learned correction (48 dirs x 8 slots + ln n -> 2 x 128 GELU -> 48) trained on "
                                   "16 seeded 128^3 fields + %d fields at %d^3 (other seeds), evaluated on a %d^3 "
                                   "uniform field (10 pc, k^-11/3 log-normal, mean 30, sigma_ln 2, seed 200), "
                                   "N_H + shield out" % (n_match, 1 << L, 1 << L),
                       "precision": "bf16", "l2": "512 MB buffer written between timed steps; N_H output %.1f GB"
                                                  % (4 * units / 1e9),
                       "training": {"fields": n_fields, "rows_per_field": rows_per, "steps": args.train_steps,
                                    "matched_fields": n_match, "matched_level": args.eval_level,
                                    "validation": "mean |A_V| error on a held-out field at level %d (seed 400), "
                                                  "%d leaves, every %d steps" % (args.eval_level, n_val, args.eval_every),
                                    "stop_step": int(best_step), "val_a_v_abs_mean": float(best_val),
                                    "delta_range": [d_lo, d_hi], "delta_margin": args.delta_margin,
                                    "row_sampling": "with replacement, probability proportional to the squared "
                                                    "mean ray-marched A_V of the leaf",
                                    "batch": 8192, "data_s": gen_s, "train_s": train_s,
                                    "loss_first": float(losses[:20].mean()), "loss_last": float(losses[-200:].mean())}},
            "gpu_launches": int(launches), "kernels": kern, "roofline": roof, "forms": forms,
            "speedup_vs_fp32_plain": forms["fp32_plain"]["ms_per_step"] / ms if "fp32_plain" in forms else None,
            "clocks": clk, "cpu_baseline": cpu, "error_vs_oracle": parity}
    print(json.dumps(line), flush=True)
    return 0


def _tensor_peak(sustained=False):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        if sustained:
            return float(p["bf16_tflops_sustained"]), "measured sustained"
        return float(p["bf16_tflops"]), "measured burst"
    except Exception:
        return (1700.0, "fallback sustained") if sustained else (1900.0, "fallback")


def _learned_oracle_checks(colden, synth, tree, geom, rho, box, L, cpu_seconds):
    """Learned form vs the FP64 oracle on sampled leaves of the evaluation
    field, with seeded weights and the oracle's own standardisation, and the
    oracle's learned inference timed on the host cores."""
    import torch
    import oracle
    from oracle import learned as ol
    nd = geom.n_dir
    T = oracle.Tree.uniform(rho.cpu().numpy(), box)
    rho_np = rho.reshape(-1).cpu().numpy().astype(np.float64)
    n_side = 1 << L
    dirs = oracle.dirs_healpix(2)          # the oracle's own direction set (48 HEALPix pixel centres)
    assert dirs.shape[0] == nd

    def oracle_rows(m):
        ijk = np.stack([_compact_np(m), _compact_np(m >> 1), _compact_np(m >> 2)], axis=1)
        _, pl = T.column_density(dirs, np.full(len(m), L), ijk, per_level=L)
        slots = ol.slots_from_levels(pl)
        nv = rho_np[(ijk[:, 2] * n_side + ijk[:, 1]) * n_side + ijk[:, 0]]
        return slots, nv

    rng = np.random.default_rng(5)
    ms = rng.choice(tree.n_leaf, 1000, replace=False)
    slots, nv = oracle_rows(ms)
    mu, sinv = ol.normaliser(ol.features(slots, nv))
    p = synth.mlp_init(nd, 128, 21, out_scale=0.5)
    net = colden.Net(nd, 128, p)
    st = net.state()
    st["mu"], st["sinv"] = mu.astype(np.float32), sinv.astype(np.float32)
    net.load_state(st)
    pd = ol.unpack(p.astype(np.float64), nd, 128)
    m = np.sort(rng.choice(tree.n_leaf, 200, replace=False))
    slots, nv = oracle_rows(m)
    delta, _ = ol.forward(pd, st["mu"].astype(np.float64), st["sinv"].astype(np.float64), ol.features(slots, nv))
    want = ol.apply(ol.tree_total(slots), delta)
    out = {}
    n_h = torch.empty(tree.n_leaf * nd, device="cuda")
    shd = torch.empty(tree.n_leaf, device="cuda")
    rows = torch.from_numpy(m).cuda()
    for name, prec in (("bf16_learned", colden.BF16), ("fp32_learned", colden.FP32)):
        colden.column_density(tree, geom, n_h=n_h, shield=shd, precision=prec, net=net)
        torch.cuda.synchronize()
        got = n_h.reshape(-1, nd)[rows].double().cpu().numpy()
        rel = np.abs(got - want) / want
        out[name] = {"n_h_rel_max": float(rel.max()), "n_h_rel_mean": float(rel.mean()),
                     "shield_abs_max": float(np.abs(shd[rows].double().cpu().numpy() - oracle.shield(want)).max()),
                     "delta_abs_max": float(np.abs(delta).max()), "leaves_checked": int(len(m))}
    del n_h
    net.free()
    # the oracle's learned inference (per-level walk, features, FP64 network), bounded sample
    n = 16
    while True:
        mm = rng.choice(tree.n_leaf, n, replace=False)
        t0 = time.perf_counter()
        slots, nv = oracle_rows(mm)
        d, _ = ol.forward(pd, mu, sinv, ol.features(slots, nv))
        ol.apply(ol.tree_total(slots), d)
        dt = time.perf_counter() - t0
        if dt >= cpu_seconds or n >= 2_000_000:
            break
        n = int(min(2_000_000, max(2 * n, n * cpu_seconds / max(dt, 1e-3) * 1.1)))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    cpu = {"value": n * nd / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "%d seeded random leaves of the %d^3 field x %d dirs: per-level walk, features, FP64 "
                     "network (%.1f s)" % (n, 1 << L, nd, dt)}
    return out, cpu


def _compact_np(v):
    v = np.asarray(v, dtype=np.uint64) & np.uint64(0x1249249249249249)
    for sh, mask in ((2, 0x10c30c30c30c30c3), (4, 0x100f00f00f00f00f), (8, 0x1f0000ff0000ff),
                     (16, 0x1f00000000ffff), (32, 0x1fffff)):
        v = (v ^ (v >> np.uint64(sh))) & np.uint64(mask)
    return v.astype(np.int64)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16"])
    ap.add_argument("--no-compare", action="store_true", help="skip the FP32-plain comparison run")
    ap.add_argument("--level", type=int, default=8)
    ap.add_argument("--nside", type=int, default=2)
    ap.add_argument("--heating", action="store_true", help="uniform workload: also time the heating epilogue")
    ap.add_argument("--geometry", default="ray", choices=["ray", "cone"],
                    help="uniform workload: one ray per direction, or factors averaged over each direction's cone")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--workload", default="uniform", choices=["uniform", "amr", "batch", "learned"])
    ap.add_argument("--train-rows", type=int, default=1_000_000, help="learned: training leaves per field")
    ap.add_argument("--train-steps", type=int, default=3000, help="learned: Adam steps")
    ap.add_argument("--ray-leaves", type=int, default=100_000, help="learned: leaves scored against the ray-marcher")
    ap.add_argument("--eval-level", type=int, default=9, help="learned: leaf level of the evaluation field")
    ap.add_argument("--eager", action="store_true",
                    help="uniform / amr: time the update and evaluation as eager calls instead of a captured graph")
    ap.add_argument("--eval-every", type=int, default=50,
                    help="learned: Adam steps between validation scores (the training stop)")
    ap.add_argument("--delta-margin", type=float, default=0.5,
                    help="learned: trusted delta range = training targets' range widened by this (ln units)")
    ap.add_argument("--matched-fields", type=int, default=4,
                    help="learned: training fields at the evaluation resolution (seeds 300+)")
    ap.add_argument("--boxes", type=int, default=64)
    ap.add_argument("--amr-level", type=int, default=10,
                    help="amr: finest level of the mesh (base three levels coarser); 9 is a small case for profiling")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--amr-sample", type=int, default=100_000, help="amr: leaves of the oracle sample (>= 1e5)")
    ap.add_argument("--batch-sample", type=int, default=64_000, help="batch: oracle leaves over all boxes")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "amr":
        return run_amr(args)
    if args.workload == "learned":
        return run_learned(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
