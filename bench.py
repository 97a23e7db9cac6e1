"""Benchmark: grid points per second of the vdW-DF nonlocal-correlation
evaluation (E_c^nl and its potential), FP32-mixed batched form against the
FP64 plain form, with latency, roofline and a CPU (oracle) baseline.

Workload (default): a batch of 8 dimer-like systems on 96^3 grids in an
18 x 18 x 24 bohr cell (seeds 0-3, vdW-DF1 and vdW-DF2), synthetic densities.
One step = the whole hot path (q0/theta, forward FFTs, kernel contraction and
energy, inverse FFTs, potential) over the batch: the library's batch graph,
one launch per stage for each of its parts (the batch runs as four parts
whose stage chains overlap).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload dimer96_batch8|cubic24|shell192|uneven64]

The other workloads (the small 24^3 case, one 192^3 ligand-shell-like system,
a batch of 64 uneven grids) measure the same quantities for the record; they
skip the serving stream, and the CPU baseline runs only on the default and
the 24^3 workload.

N > 1: run under torch.distributed.run; each rank evaluates its own batch
(independent systems, no data-path collective), weak scaling.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "dimer96_batch8"
SHAPE = (96, 96, 96)
CELL = (18.0, 18.0, 24.0)
METRIC = "grid pts/s for E_c^nl+potential, FP32 batched vs FP64 plain; p50/p99 latency"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD, "cubic24", "shell192", "uneven64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-stream measurement")
    ap.add_argument("--only-timed", action="store_true",
                    help="stop after the timed batched steps (for profiler launch lists)")
    return ap.parse_args()


def rank_seeds(rank, nb):
    """Seeds of the systems rank `rank` evaluates: independent systems per
    rank (weak scaling, no data exchange between ranks)."""
    return [rank * 1000 + i // 2 for i in range(nb)]


def reduce_max(x, device):
    """Max of a float over the ranks of the default process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
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
        os.unlink(self.f.name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


def stage_bytes(shape, prec_bytes):
    """Algorithmic DRAM bytes per launch of each stage for one system.
    c = complex element size; the half spectrum holds 20 * nx * ny * (nz/2+1)
    complex values; records are 16 B (FP32-mixed) or 32 B (FP64) per point;
    the contraction also reads one 4-byte k-point index per k-point."""
    nx, ny, nz = shape
    N = nx * ny * nz
    nk = nx * ny * (nz // 2 + 1)
    c = 2 * prec_bytes
    rec = 16 if prec_bytes == 4 else 32
    spec = 20 * nk * c
    return {
        "zfwd": 16 * N + rec * N + spec,          # n, sigma in; records, spectrum out
        "plane": 2 * spec,                         # cluster plane kernel (when enabled)
        "yfwd": 2 * spec,
        "xfwd": 2 * spec,
        "contract": 2 * spec + 4 * nk,
        "xinv": 2 * spec,
        "yinv": 2 * spec,
        "zinv": spec + rec * N + 16 * N,          # spectrum, records in; dedn, dedsigma out
        "efinish": 0,
    }


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of
# each stage kernel, per 96^3 dimer system: a single-pass ncu capture of the
# benchmarked 8-system launches themselves (one launch per stage,
# VDWGB_BATCH_SPLIT=0), divided by 8 (profiles/dram_traffic_dimer96_batch8_fp32.md).
# Clear an entry when its kernel changes.
MEASURED_TRAFFIC_PER_SYSTEM = {
    "zfwd": 755.6e6 / 8,
    "yfwd": 1097.2e6 / 8,
    "xfwd": 1093.0e6 / 8,
    "contract": 1116.7e6 / 8,
    "xinv": 1092.8e6 / 8,
    "yinv": 1097.6e6 / 8,
    "zinv": 794.6e6 / 8,
}


def run_reference(args, rank):
    """The oracle (FP64 CPU, test infrastructure) timed on the host cores on a
    bounded sample of the workload: one 48^3 grid of the same dimer density
    per step (the full 96^3 batch would take minutes per step)."""
    if rank != 0:
        return
    from paper_1703_06999_gb300 import inputs
    from oracle import vdw
    o = vdw.Oracle()
    s = inputs.dimer(0, shape=(48, 48, 48), cell_lengths=CELL, functional=1)
    n, sg = s.n.numpy(), s.sigma.numpy()
    for _ in range(args.warmup):
        o.energy_potential(n, sg, s.cell, 1)
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        o.energy_potential(n, sg, s.cell, 1)
        t.append(time.perf_counter() - t0)
    tot = sum(t)
    val = s.npts * args.steps / tot
    sample = "oracle on one 48^3 grid of the 96^3 dimer workload's density (18x18x24 bohr, seed 0, vdW-DF1) per step"
    out = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "grid pts/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD + " (oracle sample: 48^3)", "grid": [48, 48, 48]},
        "cpu_baseline": {"value": val, "unit": "grid pts/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "grid pts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(out), flush=True)


def serve_bench(B, inputs, torch, dev, local, seconds=3.0, rate=200.0, pool_entries=16):
    """Served form: Poisson arrivals (mean `rate` per second) of evaluations
    with grids from 48^3 to 160x192x224 (10-400 exponentials), FP32-mixed,
    admitted by footprint into an 8 GiB pool, continuous batching; against
    the same evaluations one at a time in FP64.  Inputs come from a pool of
    `pool_entries` distinct requests reused across arrivals (host arrays,
    page-locked)."""
    reqs = inputs.serving_requests(seed=0, count=pool_entries, rate=rate)
    pool = []
    for r in reqs:
        sy = inputs.realise(r, device=dev)
        hn = sy.n.cpu().pin_memory().numpy()
        hs = sy.sigma.cpu().pin_memory().numpy()
        dn = torch.empty(sy.shape, dtype=torch.float64).pin_memory().numpy()
        ds = torch.empty(sy.shape, dtype=torch.float64).pin_memory().numpy()
        pool.append((sy, hn, hs, dn, ds))
    # FP64 one at a time (plain form), device-resident inputs
    lat64, pts64 = [], 0
    for sy, *_ in pool:
        f = B.Functional(sy.shape, sy.cell, sy.functional, B.FP64, device=local)
        o1, o2 = torch.empty_like(sy.n), torch.empty_like(sy.n)
        en = torch.zeros(1, dtype=torch.float64, device=dev)
        f.calculate_device(sy.n, sy.sigma, o1, o2, en)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        f.calculate_device(sy.n, sy.sigma, o1, o2, en)
        b.record()
        b.synchronize()
        lat64.append(a.elapsed_time(b) / 1000.0)
        pts64 += sy.npts
        f.close()
    fp64_rate = pts64 / sum(lat64)
    sv = B.vdwgb_server_new(local, B.FP32_MIXED, pool_bytes=8 << 30, max_batch=16, max_inflight=3)
    try:
        # warm-up: every pool entry once
        for sy, hn, hs, dn, ds in pool:
            B.vdwgb_server_wait(sv, B.vdwgb_server_submit(sv, sy.functional, sy.shape, sy.cell, hn, hs, dn, ds), 120)
        B.vdwgb_server_free(sv)
        sv = B.vdwgb_server_new(local, B.FP32_MIXED, pool_bytes=8 << 30, max_batch=16, max_inflight=3)
        g = np.random.default_rng(1)
        arrivals = np.cumsum(g.exponential(1.0 / rate, int(rate * seconds * 1.5)))
        arrivals = arrivals[arrivals < seconds]
        ids = []
        t0 = time.perf_counter()
        for k, ta in enumerate(arrivals):
            while time.perf_counter() - t0 < ta:
                time.sleep(0.0002)
            sy, hn, hs, dn, ds = pool[k % len(pool)]
            ids.append(B.vdwgb_server_submit(sv, sy.functional, sy.shape, sy.cell, hn, hs, dn, ds))
        for rid in ids:
            B.vdwgb_server_wait(sv, rid, 300.0)
        wall = time.perf_counter() - t0
        st = B.vdwgb_server_stats(sv)
    finally:
        B.vdwgb_server_free(sv)
    return {"requests": len(ids), "rate_req_s": rate, "seconds": seconds, "value": st["pts_per_s"],
            "unit": "grid pts/s", "p50_ms": 1000 * st["p50_s"], "p99_ms": 1000 * st["p99_s"],
            "mean_batch": st["mean_batch"], "batches": st["batches"], "failed": st["failed"],
            "wall_s": wall, "pool_peak_GB": st["pool_used_peak"] / 1e9,
            "fp64_one_at_a_time": {"value": fp64_rate, "unit": "grid pts/s",
                                   "p50_ms": 1000 * float(np.median(lat64)),
                                   "p99_ms": 1000 * float(np.percentile(lat64, 99))},
            "grids": sorted({tuple(p[0].shape) for p in pool})}


def cpu_baseline():
    """Oracle (as it stands) on one 96^3 system of the workload, on the host."""
    from paper_1703_06999_gb300 import inputs
    from oracle import vdw
    o = vdw.Oracle()                      # table setup not timed
    s = inputs.dimer(0, shape=SHAPE, cell_lengths=CELL, functional=1)
    n, sg = s.n.numpy(), s.sigma.numpy()
    t0 = time.perf_counter()
    o.energy_potential(n, sg, s.cell, 1)
    dt = time.perf_counter() - t0
    return {"value": s.npts / dt, "unit": "grid pts/s", "cores": 1, "kind": "oracle",
            "sample": "one 96^3 dimer system (seed 0, vdW-DF1), %.1f s" % dt}


def cpu_baseline_small(s):
    """Oracle (as it stands) on the whole (small) workload system, on the host."""
    from oracle import vdw
    o = vdw.Oracle()
    n, sg = s.n.cpu().numpy(), s.sigma.cpu().numpy()
    t0 = time.perf_counter()
    o.energy_potential(n, sg, s.cell, s.functional)
    dt = time.perf_counter() - t0
    return {"value": s.npts / dt, "unit": "grid pts/s", "cores": 1, "kind": "oracle",
            "sample": "the whole %s system, %.2f s" % ("x".join(map(str, s.shape)), dt)}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank)
        return
    import torch
    from paper_1703_06999_gb300 import binding as B
    from paper_1703_06999_gb300 import inputs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    B.lib()   # fails loudly if the CUDA library is missing
    B.vdwgb_set_autotune(True)   # tile shapes measured once per grid at init (outside the timed region)

    default = args.workload == WORKLOAD
    if default:
        nb = args.batch
        seeds = rank_seeds(rank, nb)
        systems = [inputs.dimer(seeds[i], shape=SHAPE, cell_lengths=CELL, functional=1 + i % 2,
                                device=dev) for i in range(nb)]
    elif args.workload == "cubic24":
        systems = [inputs.small_cubic(rank, ngrid=24, device=dev)]
    elif args.workload == "shell192":
        systems = [inputs.ligand_shell(rank, device=dev)]
    else:
        systems = inputs.uneven_batch(rank, count=64, device=dev)
    if not default:
        nb = len(systems)
        args.no_serve = True
        if args.workload != "cubic24":
            args.no_cpu_baseline = True
    pts = sum(s.npts for s in systems)

    def make(prec):
        return [B.Functional(s.shape, s.cell, s.functional, prec, device=local) for s in systems]

    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    dn = [torch.empty_like(s.n) for s in systems]
    ds = [torch.empty_like(s.n) for s in systems]
    en = torch.zeros(nb, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 2x L2

    f32 = make(B.FP32_MIXED)
    plan_info = B.vdwgb_plan_info(f32[0].h)
    bt = B.vdwgb_batch_new([f.h for f in f32])
    ns = [s.n for s in systems]
    ss = [s.sigma for s in systems]
    for _ in range(args.warmup):
        B.vdwgb_batch_calculate_device(bt, ns, ss, dn, ds, en, sp)
    torch.cuda.synchronize()

    # ---- timed region: FP32-mixed batched (the captured graph) ----------------
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    torch.cuda.profiler.start()             # profilers started with capture off record the timed steps only
    for k in range(args.steps):
        flush.zero_()                       # L2 flushed between timed steps (outside the events)
        evs[k][0].record(stream)
        B.vdwgb_batch_calculate_device(bt, ns, ss, dn, ds, en, sp)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    clocks = clk.stop()
    if world > 1:
        torch.distributed.barrier()
    step_ms = np.array([a.elapsed_time(b) for a, b in evs])
    # per-stage breakdown, outside the timed region: the same steps with each
    # stage launched on its own between CUDA events (one stage at a time, so
    # each kernel's duration is its own)
    B.vdwgb_batch_set_timing(bt, True)
    for k in range(args.steps):
        flush.zero_()
        B.vdwgb_batch_calculate_device(bt, ns, ss, dn, ds, en, sp)
    torch.cuda.synchronize()
    stage_ms, ncalls = B.vdwgb_batch_stage_ms(bt)
    B.vdwgb_batch_set_timing(bt, False)
    tot_ms = float(step_ms.sum())
    if world > 1:
        tot_ms = reduce_max(tot_ms, dev)
    value = pts * world * args.steps / (tot_ms / 1000.0)
    if args.only_timed:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "grid pts/s", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
                              "partial": "only the timed batched steps were run",
                              "stage_ms_per_launch": (stage_ms / max(ncalls, 1)).tolist()}), flush=True)
        return
    e32 = en.cpu().numpy().copy()
    dn32 = [x.clone() for x in dn]
    ds32 = [x.clone() for x in ds]

    # ---- latency of single FP32 evaluations (one system at a time) -----------
    lat = []
    e1 = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    for i in range(220):
        f = f32[i % nb]
        e1[0].record(stream)
        f.calculate_device(ns[i % nb], ss[i % nb], dn[i % nb], ds[i % nb], en[i % nb:i % nb + 1], sp)
        e1[1].record(stream)
        e1[1].synchronize()
        if i >= 20:
            lat.append(e1[0].elapsed_time(e1[1]))
    lat = np.array(lat)

    # ---- FP64 plain, one system at a time, same inputs ------------------------
    f64 = make(B.FP64)
    k64 = max(2, args.steps // 4)
    for i, f in enumerate(f64):
        f.calculate_device(ns[i], ss[i], dn[i], ds[i], en[i:i + 1], sp)
    torch.cuda.synchronize()
    t64 = 0.0
    for _ in range(k64):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i, f in enumerate(f64):
            f.calculate_device(ns[i], ss[i], dn[i], ds[i], en[i:i + 1], sp)
        b.record(stream)
        b.synchronize()
        t64 += a.elapsed_time(b)
    fp64_value = pts * k64 / (t64 / 1000.0)
    e64 = en.cpu().numpy().copy()
    err_e = float(np.max(np.abs(e32 - e64)))
    err_n = max(float((dn32[i] - dn[i]).abs().max() / dn[i].abs().max()) for i in range(nb))
    err_s = max(float((ds32[i] - ds[i]).abs().max() / ds[i].abs().max()) for i in range(nb))
    for f in f64:
        f.close()

    # ---- end to end through the host-pointer batch API ------------------------
    hn = [s.n.cpu().pin_memory().numpy() for s in systems]
    hs = [s.sigma.cpu().pin_memory().numpy() for s in systems]
    hdn = [torch.empty(s.shape, dtype=torch.float64).pin_memory().numpy() for s in systems]
    hds = [torch.empty(s.shape, dtype=torch.float64).pin_memory().numpy() for s in systems]
    B.vdwgb_batch_calculate(bt, hn, hs, hdn, hds)
    ke = max(3, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(ke):
        B.vdwgb_batch_calculate(bt, hn, hs, hdn, hds)
    e2e_s = time.perf_counter() - t0
    e2e_val = pts * ke / e2e_s
    if world > 1:
        e2e_val = pts * world * ke / reduce_max(e2e_s, dev)
    h2d = sum(2 * s.npts * 8 for s in systems)
    d2h = sum(2 * s.npts * 8 for s in systems) + 8 * nb

    # ---- roofline of the dominant stage --------------------------------------
    names = [B.vdwgb_stage_name(i) for i in range(B.vdwgb_num_stages())]
    per_launch_ms = stage_ms / max(ncalls, 1)
    dom = int(np.argmax(per_launch_ms))
    sb = {k: 0 for k in names}
    for s in systems:
        for k, v in stage_bytes(s.shape, 4).items():
            sb[k] += v
    pk, pk_kind = peaks()
    achieved = sb[names[dom]] / (per_launch_ms[dom] / 1000.0) / 1e9
    tps = MEASURED_TRAFFIC_PER_SYSTEM.get(names[dom]) if default else None
    traffic = tps * nb if tps is not None else None
    roof = {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": pk["hbm_gbs"],
            "unit": "GB/s", "frac": achieved / pk["hbm_gbs"], "traffic": traffic,
            "peak_source": pk_kind,
            "traffic_source": "single-pass ncu capture of the 8-system launch (per system x systems)"
                              if traffic is not None else None,
            "stage_timing": "each stage launched on its own between CUDA events, outside the timed steps "
                            "(the timed steps replay the captured graph, where the two halves of the "
                            "batch overlap)",
            "stages": {n: {"ms_per_launch": float(m), "alg_bytes": int(sb[n]),
                           "GBps": (sb[n] / (m / 1000.0) / 1e9) if m > 0 else None}
                       for n, m in zip(names, per_launch_ms)}}

    launches_per_step = B.vdwgb_batch_launches(bt)
    for f in f32:
        f.close()
    B.vdwgb_batch_free(bt)
    serving = None if args.no_serve else serve_bench(B, inputs, torch, dev, local)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "grid pts/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32-mixed (f64 q0 and energy sum)",
            "data": "synthetic",
            "config": {"workload": args.workload,
                       "grid": list(SHAPE) if default else sorted({tuple(s.shape) for s in systems}),
                       "cell_bohr": list(CELL) if default else None, "systems": nb,
                       "functionals": sorted({int(s.functional) for s in systems}), "precision": "fp32_mixed",
                       "parallelism": "replicas", "plan": plan_info,
                       "l2": "flushed between timed steps (256 MB write); working set %.0f MB"
                             % (sum(s.shape[0] * s.shape[1] * (s.shape[2] // 2 + 1) * 160 + 48 * s.npts
                                    for s in systems) / 1e6)},
            "fp64_plain": {"value": fp64_value, "unit": "grid pts/s", "steps": k64,
                           "ms_per_step": t64 / k64, "form": "one system at a time"},
            "speedup_fp32_batched_vs_fp64_plain": value / (fp64_value * world),
            "latency_ms": {"single_system_fp32": {"p50": float(np.percentile(lat, 50)),
                                                  "p99": float(np.percentile(lat, 99)), "n": int(lat.size)},
                           "batch_step": {"p50": float(np.percentile(step_ms, 50)),
                                          "p99": float(np.percentile(step_ms, 99))}},
            "error_fp32_vs_fp64": {"max_abs_dE_Ha": err_e, "dedn_maxnorm_rel": err_n,
                                   "dedsigma_maxnorm_rel": err_s},
            "roofline": roof,
            "e2e": {"value": e2e_val, "unit": "grid pts/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "api": "vdwgb_batch_calculate (host arrays, pinned)"},
            "gpu_launches": int(args.steps * launches_per_step),
            "clocks": clocks,
            "table_build_s": B.vdwgb_table_build_seconds(local),
        }
        if serving is not None:
            out["serving"] = serving
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline() if default else cpu_baseline_small(systems[0])
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
