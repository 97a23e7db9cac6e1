"""Benchmark: grid points per second of the vdW-DF nonlocal-correlation
evaluation (E_c^nl and its potential), FP32-mixed batched form against the
FP64 plain form, with latency, rooflines, errors against the FP64 oracle and
the oracle timed on the host cores.

Workload (default, ``uneven64``): a batch of 64 independent systems whose
grid axes are drawn from {32, 48, 64, 80, 96, 128} (non-cubic mixes), grid
spacing 0.15-0.30 bohr, 4-60 exponentials each, vdW-DF1 and vdW-DF2 mixed
(25.8 M grid points), synthetic densities.  One step = the whole hot path
(q0/theta, forward FFTs, kernel contraction and energy, inverse FFTs,
potential) over the batch: the library's batch graph, one persistent launch
per stage for each of its parts, autotuned tile shapes.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload uneven64|dimer96_batch8|cubic24|shell192]

The default run also times the 8-system 96^3 dimer batch (``extra``), the
serving stream (Poisson arrivals, continuous batching) and the FP64 oracle
on every system of the batch on all host cores (errors of both GPU forms
against it, and the CPU baseline).  The other workloads measure the timed
quantities for the record.

N > 1: run under torch.distributed.run; each rank evaluates its own batch
(independent systems, no data-path collective), weak scaling.
"""
import argparse
import ctypes
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "uneven64"
DIMER_SHAPE = (96, 96, 96)
DIMER_CELL = (18.0, 18.0, 24.0)
METRIC = "grid pts/s for E_c^nl+potential, FP32 batched vs FP64 plain; p50/p99 latency"
PRECISION_NOTE = ("FP32 theta fields, FFTs and kernel contraction; q0 and saturation in double-float "
                  "(FP32 pairs, ~46 significant bits); per-warp energy sums in FP64, energy finish in "
                  "compensated FP32 pairs; outputs FP64")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "dimer96_batch8", "cubic24", "shell192", "shell640"])
    ap.add_argument("--no-oracle", action="store_true", help="skip the oracle errors and the CPU baseline")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-stream measurement")
    ap.add_argument("--no-extra", action="store_true", help="skip the extra 96^3 dimer batch")
    ap.add_argument("--only-timed", action="store_true",
                    help="stop after the timed batched steps (for profiler launch lists)")
    return ap.parse_args()


def rank_seeds(rank, nb):
    """Seeds of the dimer systems rank `rank` evaluates: independent systems
    per rank (weak scaling, no data exchange between ranks)."""
    return [rank * 1000 + i // 2 for i in range(nb)]


def job_points(pts, world, device):
    """Grid points of one step over all ranks (each rank its own systems)."""
    if world <= 1:
        return pts
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(pts)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def reduce_max(x, device):
    """Max of a float over the ranks of the default process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


_T0 = time.perf_counter()


def log(msg):
    """Progress of the run on stderr (the JSON line goes to stdout)."""
    sys.stderr.write("[bench %7.1f s] %s\n" % (time.perf_counter() - _T0, msg))
    sys.stderr.flush()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_workload(name, rank, device):
    """The systems of a workload (synthetic densities, built on `device`)."""
    from paper_1703_06999_gb300 import inputs
    if name == "dimer96_batch8":
        seeds = rank_seeds(rank, 8)
        return [inputs.dimer(seeds[i], shape=DIMER_SHAPE, cell_lengths=DIMER_CELL, functional=1 + i % 2,
                             device=device) for i in range(8)]
    if name == "cubic24":
        return [inputs.small_cubic(rank, ngrid=24, device=device)]
    if name == "shell192":
        return [inputs.ligand_shell(rank, device=device)]
    if name == "shell640":
        return [shell640(rank, device)]
    return inputs.uneven_batch(rank, count=64, device=device, shape_seed=0)


def shell160(seed, device):
    """A ligand-shell-like density on 160^3 points in a 27.4 bohr cell: a core
    of 12 exponentials and 8 radial chains of 4 (one quarter of the paper's
    (58 Angstrom)^3 box along each axis)."""
    from paper_1703_06999_gb300 import inputs
    g = np.random.default_rng(640 + seed)
    L = 109.6 / 4
    c0 = np.array([L / 2] * 3)
    atoms = []
    for _ in range(12):
        v = g.normal(size=3)
        v *= g.uniform(0, 3.0) / np.linalg.norm(v)
        atoms.append((float(g.uniform(6, 8)), float(g.uniform(2, 3)), tuple(c0 + v)))
    for _ in range(8):
        u = g.normal(size=3)
        u /= np.linalg.norm(u)
        for k in range(4):
            atoms.append((float(g.uniform(1, 6)), float(g.uniform(1, 2.5)), tuple(c0 + (4.0 + 1.2 * k) * u)))
    return inputs.make_system((160, 160, 160), np.diag([L, L, L]), atoms, 1, device=device, name="shell160")


def shell640(seed, device):
    """The paper's density-grid size: 640^3 points in a (58 Angstrom)^3 =
    109.6 bohr cubic box, the 4 x 4 x 4 supercell of shell160 (so that its
    energy is 64 times the 160^3 system's, a check at a size no oracle run
    reaches)."""
    from paper_1703_06999_gb300 import inputs
    b = shell160(seed, device)
    return inputs.System((640, 640, 640), 4 * b.cell, 1, b.n.repeat(4, 4, 4).contiguous(),
                         b.sigma.repeat(4, 4, 4).contiguous(), [], "shell640")


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    """SM clock and clock-event (throttle) reasons sampled during the timed
    region: NVML every 5 ms from a thread (read-only queries), else
    nvidia-smi every 50 ms."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, index):
        self.index = index
        self.sm, self.smax, self.reasons = [], [], set()
        self.stop_flag = False
        self.mode = None
        try:
            self.nv = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nv.nvmlInit_v2() != 0:
                raise OSError("nvmlInit")
            self.h = ctypes.c_void_p()
            if self.nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h)) != 0:
                raise OSError("handle")
            self.mode = "nvml"
            self.t = threading.Thread(target=self._loop, daemon=True)
            self.t.start()
        except (OSError, AttributeError):
            self._start_smi()

    def _loop(self):
        clk, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        get_r = getattr(self.nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.nv.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self.stop_flag:
            if self.nv.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(clk)) == 0:
                self.sm.append(float(clk.value))
            if self.nv.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0:
                self.smax.append(float(mx.value))
            if get_r(self.h, ctypes.byref(rs)) == 0:
                for bit, nm in self.REASONS.items():
                    if rs.value & bit:
                        self.reasons.add(nm)
            time.sleep(0.005)

    def _start_smi(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
            self.mode = "nvidia-smi"
        except OSError:
            self.p = None

    def stop(self):
        if self.mode == "nvml":
            self.stop_flag = True
            self.t.join(2)
        elif self.mode == "nvidia-smi" and self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(5)
            except subprocess.TimeoutExpired:
                self.p.kill()
            self.f.flush()
            self.f.seek(0)
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for line in self.f.read().splitlines():
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    self.sm.append(float(parts[1]))
                    self.smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        self.reasons.add(nm)
            os.unlink(self.f.name)
        else:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no clock source"], "samples": 0}
        return {"sm_mhz": float(np.median(self.sm)) if self.sm else None,
                "sm_max_mhz": float(max(self.smax)) if self.smax else None,
                "reasons": sorted(self.reasons), "samples": len(self.sm), "source": self.mode}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


# ---------------------------------------------------------------------------
# algorithmic work per stage
# ---------------------------------------------------------------------------
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


# Fused multiply-adds per half-spectrum k-point of the contraction: 210
# cubic evaluations (three per two pairs: 315), 400 complex multiply-adds by
# the real phi (one two-lane FMA each) and 20 for the energy, all two-lane
# FP32 FMAs (two FMAs, four flops each).
CONTRACT_FMA2_PER_KPOINT = 315 + 400 + 20
# FP64 form: 210 cubic evaluations (3 FMAs each), 400 complex multiply-adds
# (2 FMAs each) and 20 energy terms (2 each).
CONTRACT_FMA64_PER_KPOINT = 630 + 800 + 40

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of a stage over
# the whole batch, per workload: the six part launches of one timed step of
# a single-pass ncu capture of the benchmarked steps themselves (the launch
# list summarised in the profiles directory).  An entry is removed when its
# kernel changes.
MEASURED_TRAFFIC = {
    "uneven64": {"zfwd": 2616e6, "zinv": 2904e6, "contract": 3979e6},
}

# Instruction-issue utilisation of the z-forward kernel (the q0 step in
# double-float arithmetic makes it issue-bound): smsp__issue_active of a full
# ncu capture of one launch on two 96^3 systems (profiles directory).
ZFWD_ISSUE_ACTIVE = 0.718


# ---------------------------------------------------------------------------
# oracle legs (FP64 CPU, test infrastructure): process pool started with spawn
# ---------------------------------------------------------------------------
def _oracle_job(args):
    """One oracle evaluation in a worker process: (index, E, dedn, dedsigma, s)."""
    i, n, sg, cell, fn = args
    from oracle import vdw
    o = _oracle_job.o = getattr(_oracle_job, "o", None) or vdw.Oracle()
    t0 = time.perf_counter()
    r = o.energy_potential(n, sg, cell, fn)
    return i, r.energy, r.dedn, r.dedsigma, time.perf_counter() - t0


def oracle_workers(max_points):
    """Worker count for the oracle pool: every host core, bounded by the host
    memory the largest system needs (about 1.5 kB per grid point)."""
    cores = os.cpu_count() or 1
    try:
        with open("/proc/meminfo") as f:
            avail = next(int(l.split()[1]) * 1024 for l in f if l.startswith("MemAvailable"))
    except (OSError, StopIteration):
        avail = 16 << 30
    per = 1500 * max_points + (256 << 20)
    return max(1, min(cores, int(0.5 * avail // per)))


class OraclePool:
    """`workers` spawned processes evaluating the oracle, one system per job.
    The kernel table is built (or loaded from its cache) once in this
    process and then loaded by each worker in an untimed warm-up job."""

    def __init__(self, workers):
        import multiprocessing as mp
        from oracle import vdw
        vdw.Oracle()                       # build the table cache once, here
        self.workers = workers
        old = os.environ.get("OMP_NUM_THREADS")
        os.environ["OMP_NUM_THREADS"] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(workers)
        finally:
            if old is None:
                os.environ.pop("OMP_NUM_THREADS", None)
            else:
                os.environ["OMP_NUM_THREADS"] = old
        tiny = np.full((4, 4, 4), 0.01)
        self.pool.map(_oracle_job, [(-1, tiny, tiny * 0, np.eye(3) * 4, 1)] * workers, chunksize=1)

    def run(self, jobs):
        """Results by job index and the wall time of the whole set."""
        order = sorted(range(len(jobs)), key=lambda k: -jobs[k][1].size)   # largest first
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_job, [jobs[k] for k in order], chunksize=1)
        wall = time.perf_counter() - t0
        return {r[0]: r for r in res}, wall

    def close(self):
        self.pool.close()
        self.pool.join()


def errors_vs_oracle(gpu, ref):
    """Per system: |dE| (Ha) and max-norm relative errors of dedn, dedsigma."""
    out = []
    for i, (e, dn, ds) in enumerate(gpu):
        _, re, rdn, rds, _ = ref[i]
        out.append((abs(e - re), float(np.max(np.abs(dn - rdn)) / max(np.max(np.abs(rdn)), 1e-300)),
                    float(np.max(np.abs(ds - rds)) / max(np.max(np.abs(rds)), 1e-300))))
    a = np.array(out)
    return {"systems": len(out), "max_abs_dE_Ha": float(a[:, 0].max()), "dedn_maxnorm_rel": float(a[:, 1].max()),
            "dedsigma_maxnorm_rel": float(a[:, 2].max()), "median_abs_dE_Ha": float(np.median(a[:, 0]))}


def run_reference(args, rank):
    """The reference arm: the oracle (FP64 CPU, test infrastructure, as it
    stands) on the host cores.  Each step evaluates a bounded sample of the
    workload on a process pool: the 16 smallest systems of the 64-grid batch
    (about 1.7 M grid points), or one 48^3 grid of a dimer density for the
    dimer workload."""
    if rank != 0:
        return
    from paper_1703_06999_gb300 import inputs
    if args.workload == "dimer96_batch8":
        systems = [inputs.dimer(0, shape=(48, 48, 48), cell_lengths=DIMER_CELL, functional=1)]
        sample = "oracle on one 48^3 grid of the dimer density (18x18x24 bohr, seed 0) per step"
    elif args.workload == WORKLOAD:
        allsys = inputs.uneven_batch(0, count=64)
        systems = sorted(allsys, key=lambda s: s.npts)[:16]
        sample = ("oracle on the 16 smallest systems of the 64-grid batch (%d grid points) per step, one "
                  "system per worker process" % sum(s.npts for s in systems))
    else:
        systems = make_workload(args.workload, 0, "cpu")
        sample = "oracle on the whole workload per step"
    jobs = [(i, s.n.numpy(), s.sigma.numpy(), s.cell, s.functional) for i, s in enumerate(systems)]
    pts = sum(s.npts for s in systems)
    workers = min(len(jobs), oracle_workers(max(s.npts for s in systems)))
    pool = OraclePool(workers)
    try:
        for _ in range(args.warmup):
            pool.run(jobs)
        t = 0.0
        for _ in range(args.steps):
            _, w = pool.run(jobs)
            t += w
    finally:
        pool.close()
    val = pts * args.steps / t
    out = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "grid pts/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload + " (oracle sample)"},
        "cpu_baseline": {"value": val, "unit": "grid pts/s", "cores": workers, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "grid pts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# serving stream
# ---------------------------------------------------------------------------
def serve_bench(B, inputs, torch, dev, local, rate=200.0, count=2000, distinct=128,
                sweep=(400.0, 800.0, 1600.0, 3200.0), sweep_seconds=2.5):
    """Served form (the Poisson serving stream): arrivals with mean `rate`
    per second of evaluations with grids from 48^3 to 160x192x224 (sorted
    axes, 10-400 exponentials, spacing 0.15-0.30 bohr), FP32-mixed, admitted
    by footprint into a 160 GiB pool where plans stay resident, continuous
    batching (up to 16 requests per batch, 3 batches in flight).  `distinct`
    different requests (density, cell, grid) are drawn from the stream's
    distribution and the `count` arrivals cycle through them in a random
    order (host arrays, page-locked).  Reported against the same requests
    one at a time in FP64.  Then a sweep of higher rates (`sweep_seconds`
    each) up to saturation."""
    reqs = inputs.serving_requests(seed=0, count=distinct, rate=rate)
    log("serving: %d distinct requests" % distinct)
    pool = []
    for r in reqs:
        sy = inputs.realise(r, device=dev)
        hn = sy.n.cpu().pin_memory().numpy()
        hs = sy.sigma.cpu().pin_memory().numpy()
        dn = torch.empty(sy.shape, dtype=torch.float64).pin_memory().numpy()
        ds = torch.empty(sy.shape, dtype=torch.float64).pin_memory().numpy()
        pool.append((sy, hn, hs, dn, ds))
    # FP64 one at a time (plain form), device-resident inputs, on a sample of 32
    lat64, pts64 = [], 0
    for sy, *_ in pool[:32]:
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
    for sy, *_ in pool:
        sy.n = sy.sigma = None                      # device copies no longer needed
    torch.cuda.empty_cache()
    g = np.random.default_rng(1)

    def stream(rate_s, n_arrivals):
        log("serving: %g req/s, %d arrivals" % (rate_s, n_arrivals))
        sv = B.vdwgb_server_new(local, B.FP32_MIXED, pool_bytes=160 << 30, max_batch=16, max_inflight=3)
        try:
            for k in range(len(pool)):              # warm-up: every request once (plans built, resident)
                sy, hn, hs, dn, ds = pool[k]
                B.vdwgb_server_wait(sv, B.vdwgb_server_submit(sv, sy.functional, sy.shape, sy.cell, hn, hs, dn, ds),
                                    300.0)
            warm = B.vdwgb_server_stats(sv)
            arrivals = np.cumsum(g.exponential(1.0 / rate_s, n_arrivals))
            order = g.integers(0, len(pool), n_arrivals)
            ids, pts = [], 0
            t0 = time.perf_counter()
            for k, ta in enumerate(arrivals):
                while time.perf_counter() - t0 < ta:
                    time.sleep(0.0002)
                sy, hn, hs, dn, ds = pool[order[k]]
                ids.append(B.vdwgb_server_submit(sv, sy.functional, sy.shape, sy.cell, hn, hs, dn, ds))
                pts += sy.npts
            lat = [B.vdwgb_server_wait(sv, rid, 300.0)[1] for rid in ids]
            wall = time.perf_counter() - t0
            st = B.vdwgb_server_stats(sv)
        finally:
            B.vdwgb_server_free(sv)
        lat = np.array(lat)
        batches = st["batches"] - warm["batches"]
        return {"requests": len(ids), "rate_req_s": rate_s, "offered_s": float(arrivals[-1]),
                "value": pts / wall, "unit": "grid pts/s", "wall_s": wall,
                "p50_ms": 1000 * float(np.percentile(lat, 50)), "p99_ms": 1000 * float(np.percentile(lat, 99)),
                "mean_batch": (st["completed"] - warm["completed"]) / max(batches, 1), "batches": batches,
                "failed": st["failed"], "plans_reused": st["plans_reused"] - warm["plans_reused"],
                "plans_built": st["plans_built"] - warm["plans_built"], "pool_peak_GB": st["pool_used_peak"] / 1e9}

    # the GPU alone on one batch of the stream's requests (the batch graph,
    # device-resident inputs): what the served throughput is bounded by
    log("serving: one 16-request batch on the GPU alone")
    gsys = [inputs.realise(r, device=dev) for r in reqs[:16]]
    gf = [B.Functional(sy.shape, sy.cell, sy.functional, B.FP32_MIXED, device=local) for sy in gsys]
    gb = B.vdwgb_batch_new([f.h for f in gf])
    gdn = [torch.empty_like(sy.n) for sy in gsys]
    gds = [torch.empty_like(sy.n) for sy in gsys]
    gen = torch.zeros(len(gsys), dtype=torch.float64, device=dev)
    gsp = torch.cuda.current_stream(dev).cuda_stream
    run = lambda: B.vdwgb_batch_calculate_device(gb, [sy.n for sy in gsys], [sy.sigma for sy in gsys],  # noqa: E731
                                                 gdn, gds, gen, gsp)
    for _ in range(3):
        run()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(5):
        run()
    b.record()
    b.synchronize()
    gpu_batch = {"requests": len(gsys), "grid_points": sum(sy.npts for sy in gsys),
                 "value": 5 * sum(sy.npts for sy in gsys) / (a.elapsed_time(b) / 1000.0), "unit": "grid pts/s"}
    B.vdwgb_device_status(local)
    B.vdwgb_batch_free(gb)
    for f in gf:
        f.close()
    del gsys, gdn, gds
    torch.cuda.empty_cache()

    main = stream(rate, count)
    main["gpu_alone_one_batch"] = gpu_batch
    main["fp64_one_at_a_time"] = {"value": fp64_rate, "unit": "grid pts/s", "requests": len(lat64),
                                  "p50_ms": 1000 * float(np.median(lat64)),
                                  "p99_ms": 1000 * float(np.percentile(lat64, 99))}
    main["distinct_requests"] = len(pool)
    main["grids"] = len({tuple(p[0].shape) for p in pool})
    main["grid_points_mean"] = float(np.mean([p[0].npts for p in pool]))
    main["sweep"] = [stream(r, int(r * sweep_seconds)) for r in sweep]
    return main


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def timed_batch(B, torch, bt, ns, ss, dn, ds, en, sp, stream, steps, warmup, flush, world, dev, local):
    """Warm-up, then exactly `steps` timed replays of the batch graph
    (barrier + synchronize on both sides, L2 flushed between steps outside
    the events); returns per-step ms, total ms (max over ranks) and clocks."""
    for _ in range(warmup):
        B.vdwgb_batch_calculate_device(bt, ns, ss, dn, ds, en, sp)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    torch.cuda.profiler.start()             # profilers started with capture off record the timed steps only
    for k in range(steps):
        flush.zero_()
        evs[k][0].record(stream)
        B.vdwgb_batch_calculate_device(bt, ns, ss, dn, ds, en, sp)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    clocks = clk.stop()
    if world > 1:
        torch.distributed.barrier()
    step_ms = np.array([a.elapsed_time(b) for a, b in evs])
    tot = float(step_ms.sum())
    if world > 1:
        tot = reduce_max(tot, dev)
    return step_ms, tot, clocks


def stage_breakdown(B, torch, bt, ns, ss, dn, ds, en, sp, flush, steps):
    """The same evaluation with each stage launched on its own between CUDA
    events (one launch per stage over the whole batch), outside the timed
    steps: per-launch ms of every stage."""
    B.vdwgb_batch_set_timing(bt, True)
    for _ in range(steps):
        flush.zero_()
        B.vdwgb_batch_calculate_device(bt, ns, ss, dn, ds, en, sp)
    torch.cuda.synchronize()
    stage_ms, ncalls = B.vdwgb_batch_stage_ms(bt)
    B.vdwgb_batch_set_timing(bt, False)
    return stage_ms / max(ncalls, 1)


def _event_ms(torch, stream, fn, reps, flush):
    """Mean ms of fn() over reps calls, CUDA events on `stream`, L2 flushed
    before each call (outside the events)."""
    tot = 0.0
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        tot += a.elapsed_time(b)
    return tot / reps


def spin_bench(B, inputs, torch, dev, local, sp, stream, flush, reps=20):
    """The spin-polarised form on one 96^3 dimer (FP32-mixed and FP64, device
    form) against the plain form of the same handle; its error against the
    spin oracle on a 48^3 dimer."""
    s = inputs.dimer(0, shape=DIMER_SHAPE, cell_lengths=DIMER_CELL, functional=1, device=dev)
    nu, nd, su, sd = inputs.spin_split(s, 0.6, seed=1)
    out = {}
    for prec, name in ((B.FP32_MIXED, "fp32_mixed"), (B.FP64, "fp64")):
        f = B.Functional(s.shape, s.cell, s.functional, prec, device=local)
        o = [torch.empty_like(nu) for _ in range(4)]
        en = torch.zeros(1, dtype=torch.float64, device=dev)
        run_spin = lambda: B.vdwgb_calculate_spin_device(f.h, nu, nd, su, sd, *o, en, sp)   # noqa: E731
        run_plain = lambda: f.calculate_device(s.n, s.sigma, o[0], o[1], en, sp)            # noqa: E731
        for _ in range(3):
            run_spin()
            run_plain()
        torch.cuda.synchronize()
        t_spin = _event_ms(torch, stream, run_spin, reps, flush)
        t_plain = _event_ms(torch, stream, run_plain, reps, flush)
        B.vdwgb_device_status(local)
        f.close()
        out[name] = {"ms": t_spin, "value": s.npts / (t_spin / 1000.0), "unit": "grid pts/s",
                     "plain_ms_same_handle": t_plain}
    # results on a smaller dimer, for the comparison with the spin oracle
    # (made with the other oracle runs)
    sm = inputs.dimer(0, shape=(48, 48, 48), cell_lengths=DIMER_CELL, functional=1, device=dev)
    a = [x.cpu().numpy() for x in inputs.spin_split(sm, 0.6, seed=1)]
    gpu48 = {}
    for prec, name in ((B.FP32_MIXED, "fp32_mixed"), (B.FP64, "fp64")):
        f = B.Functional(sm.shape, sm.cell, sm.functional, prec, device=local)
        gpu48[name] = f.calculate_spin(*a)
        f.close()
    out["workload"] = "one 96^3 dimer (18 x 18 x 24 bohr), polarisation 0.6 sin cos texture"
    return out, (sm.cell, sm.functional, a, gpu48)


def spin_errors(case):
    """Errors of the spin-polarised GPU results against the spin oracle."""
    from oracle import spin as ospin
    from oracle import vdw as ovdw
    cell, functional, a, gpu48 = case
    ref = ospin.energy_potential_spin(ovdw.Oracle(ovdw.Params()), *a, cell, functional)
    errs = {}
    for name, (e, dn, ds) in gpu48.items():
        errs[name] = {"abs_dE_Ha": abs(e - ref[0]),
                      "dedn_rel_maxnorm": max(float(np.max(np.abs(x - y)) / np.max(np.abs(y)))
                                              for x, y in zip(dn, ref[1])),
                      "dedsigma_rel_maxnorm": max(float(np.max(np.abs(x - y)) / np.max(np.abs(y)))
                                                  for x, y in zip(ds, ref[2]))}
    return errs


def slab_bench(B, inputs, torch, dev, local, stream, flush, P=4, reps=10):
    """The slab decomposition with P virtual ranks on this GPU (each its own
    plans and buffers; the two all-to-alls as device copies between them, so
    the exchange runs at device-copy speed, not at a link's): per-phase
    times against one plan on the whole grid, 192^3 ligand shell."""
    from paper_1703_06999_gb300.slab import LibraryStages
    s = inputs.ligand_shell(0, device=dev)
    st = LibraryStages(local)
    prec = B.FP32_MIXED
    nbytes = st.slab_bytes(s.shape, P, prec)
    part = nbytes // P
    nxl = s.shape[0] // P
    R = []
    for r in range(P):
        a, b, x = st.buffer(nbytes), st.buffer(nbytes), st.buffer(nbytes)
        R.append(dict(h=st.new(s.functional, s.shape, s.cell, P, r, prec, a, b), a=a, b=b, x=x,
                      e=st.energy_buffer(), rho=s.n[r * nxl:(r + 1) * nxl].contiguous(),
                      sig=s.sigma[r * nxl:(r + 1) * nxl].contiguous(),
                      dn=torch.empty((nxl,) + s.shape[1:], dtype=torch.float64, device=dev),
                      ds=torch.empty((nxl,) + s.shape[1:], dtype=torch.float64, device=dev)))

    def exchange(src, dst):
        for r, Rr in enumerate(R):
            for q, Rq in enumerate(R):
                Rr[dst][q * part:(q + 1) * part].copy_(Rq[src][r * part:(r + 1) * part])

    phases = [("forward", lambda: [st.forward(x["h"], x["rho"], x["sig"]) for x in R]),
              ("pack", lambda: [st.pack(x["h"], x["x"]) for x in R]),
              ("exchange", lambda: exchange("x", "b")),
              ("contract", lambda: [st.contract(x["h"], x["e"]) for x in R]),
              ("exchange_back", lambda: exchange("b", "x")),
              ("unpack", lambda: [st.unpack(x["h"], x["x"]) for x in R]),
              ("inverse", lambda: [st.inverse(x["h"], x["dn"], x["ds"]) for x in R])]
    for _ in range(3):
        for _, fn in phases:
            fn()
    torch.cuda.synchronize()
    # whole evaluations, CUDA events between the phases (every phase runs once
    # per evaluation: the contraction works in place)
    per = {name: 0.0 for name, _ in phases}
    for _ in range(reps):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(phases) + 1)]
        ev[0].record(stream)
        for k, (_, fn) in enumerate(phases):
            fn()
            ev[k + 1].record(stream)
        ev[-1].synchronize()
        for k, (name, _) in enumerate(phases):
            per[name] += ev[k].elapsed_time(ev[k + 1]) / reps
    total = sum(per.values())
    st.status()
    f = B.Functional(s.shape, s.cell, s.functional, prec, device=local)
    dn1, ds1 = torch.empty_like(s.n), torch.empty_like(s.n)
    en1 = torch.zeros(1, dtype=torch.float64, device=dev)
    one = _event_ms(torch, stream, lambda: f.calculate_device(s.n, s.sigma, dn1, ds1, en1, stream.cuda_stream),
                    reps, flush)
    same = all(torch.equal(x["dn"], dn1[r * nxl:(r + 1) * nxl]) for r, x in enumerate(R))
    f.close()
    for x in R:
        st.free(x["h"])
    pack_bytes = 2 * nbytes * P                    # read and write of every rank's spectrum
    return {"workload": "192^3 ligand shell, FP32-mixed, %d virtual ranks on one GPU" % P,
            "phase_ms": per, "ms_all_ranks": total, "ms_one_plan_whole_grid": one,
            "pack_GBps": pack_bytes / (per["pack"] / 1000.0) / 1e9,
            "potentials_bitwise_equal_one_plan": bool(same),
            "exchange": "device copies between the ranks' buffers (an all-to-all's data movement "
                        "at device-copy speed; no link is measured)"}


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
    log("building the %s workload" % args.workload)
    systems = make_workload(args.workload, rank, dev)
    nb = len(systems)
    pts = sum(s.npts for s in systems)
    if not default:
        args.no_serve = True
        args.no_extra = True

    def make(prec, syss):
        return [B.Functional(s.shape, s.cell, s.functional, prec, device=local) for s in syss]

    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    dn = [torch.empty_like(s.n) for s in systems]
    ds = [torch.empty_like(s.n) for s in systems]
    en = torch.zeros(nb, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 2x L2
    ns = [s.n for s in systems]
    ss = [s.sigma for s in systems]

    log("planning %d FP32-mixed handles (autotuned tiles)" % nb)
    f32 = make(B.FP32_MIXED, systems)
    plan_info = B.vdwgb_plan_info(f32[0].h)
    fused = any(B.vdwgb_plan_info(f.h)["cluster"] for f in f32)   # plane kernel in use
    bt = B.vdwgb_batch_new([f.h for f in f32])

    # ---- timed region: FP32-mixed batched (the captured graph) ----------------
    log("timed batched steps")
    step_ms, tot_ms, clocks = timed_batch(B, torch, bt, ns, ss, dn, ds, en, sp, stream, args.steps, args.warmup,
                                          flush, world, dev, local)
    job_pts = job_points(pts, world, dev)
    value = job_pts * args.steps / (tot_ms / 1000.0)
    per_launch_ms = stage_breakdown(B, torch, bt, ns, ss, dn, ds, en, sp, flush, args.steps)
    if args.only_timed:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "grid pts/s", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
                              "partial": "only the timed batched steps were run",
                              "stage_ms_per_launch": per_launch_ms.tolist()}), flush=True)
        return
    # results of the FP32-mixed batch (the last timed call)
    B.vdwgb_batch_calculate_device(bt, ns, ss, dn, ds, en, sp)
    torch.cuda.synchronize()
    B.vdwgb_device_status(local)
    g32 = [(float(en[i]), dn[i].cpu().numpy(), ds[i].cpu().numpy()) for i in range(nb)]

    # ---- latency of single FP32 evaluations (one system at a time) -----------
    log("single-system latency")
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

    # ---- end to end through the host-pointer batch API ------------------------
    log("end to end through host arrays")
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
        e2e_val = job_pts * ke / reduce_max(e2e_s, dev)
    h2d = sum(2 * s.npts * 8 for s in systems)
    d2h = sum(2 * s.npts * 8 for s in systems) + 8 * nb
    launches_per_step = B.vdwgb_batch_launches(bt)
    for f in f32:
        f.close()
    B.vdwgb_batch_free(bt)

    # ---- FP64 plain, one system at a time, same inputs ------------------------
    log("FP64 plain form")
    try:
        f64 = make(B.FP64, systems)
    except B.VdwgbError:
        f64 = None                        # grids whose FP64 tiles do not fit shared memory (640 axes)
    supercell = None
    if f64 is None:
        fp64_value, k64, t64, g64, per_launch64, err_32_64 = None, 0, 0.0, None, None, None
        if args.workload == "shell640":
            # the 160^3 cell of the supercell in FP64: E(640^3) = 64 E(160^3), tiled potentials
            b = shell160(rank, dev)
            fb = B.Functional(b.shape, b.cell, 1, B.FP64, device=local)
            eb, dnb, dsb = fb.calculate(b.n.cpu().numpy(), b.sigma.cpu().numpy())
            fb.close()
            tile = lambda x: np.tile(x, (4, 4, 4))
            supercell = {"fp64_160cubed_energy_Ha": eb, "fp32_640cubed_energy_over_64_Ha": g32[0][0] / 64,
                         "abs_dE_per_160cubed_cell_Ha": abs(g32[0][0] / 64 - eb),
                         "rel_dE": abs(g32[0][0] / 64 - eb) / abs(eb),
                         "dedn_maxnorm_rel": float(np.max(np.abs(g32[0][1] - tile(dnb))) / np.max(np.abs(dnb))),
                         "dedsigma_maxnorm_rel": float(np.max(np.abs(g32[0][2] - tile(dsb))) / np.max(np.abs(dsb)))}
    else:
        k64 = max(2, args.steps // 4)
    if f64 is not None:
        for i, f in enumerate(f64):
            f.calculate_device(ns[i], ss[i], dn[i], ds[i], en[i:i + 1], sp)
        torch.cuda.synchronize()
        B.vdwgb_device_status(local)
        g64 = [(float(en[i]), dn[i].cpu().numpy(), ds[i].cpu().numpy()) for i in range(nb)]
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
        # FP64 stage breakdown (one launch per stage over the batch)
        bt64 = B.vdwgb_batch_new([f.h for f in f64])
        per_launch64 = stage_breakdown(B, torch, bt64, ns, ss, dn, ds, en, sp, flush, max(2, args.steps // 4))
        B.vdwgb_batch_free(bt64)
        for f in f64:
            f.close()
        err_32_64 = {"max_abs_dE_Ha": max(abs(a[0] - b[0]) for a, b in zip(g32, g64)),
                     "dedn_maxnorm_rel": max(float(np.max(np.abs(a[1] - b[1])) / np.max(np.abs(b[1])))
                                             for a, b in zip(g32, g64)),
                     "dedsigma_maxnorm_rel": max(float(np.max(np.abs(a[2] - b[2])) / np.max(np.abs(b[2])))
                                                 for a, b in zip(g32, g64))}

    # ---- rooflines of the stages ----------------------------------------------
    names = [B.vdwgb_stage_name(i) for i in range(B.vdwgb_num_stages())]
    dom = int(np.argmax(per_launch_ms))
    sb = {k: 0 for k in names}
    sb64 = {k: 0 for k in names}
    nk_total = sum(s.shape[0] * s.shape[1] * (s.shape[2] // 2 + 1) for s in systems)
    for s in systems:
        for k, v in stage_bytes(s.shape, 4).items():
            sb[k] += v
        for k, v in stage_bytes(s.shape, 8).items():
            sb64[k] += v
    if not fused:
        sb["plane"] = 0                   # not launched: separate y, x and contraction passes
    sb64["plane"] = 0
    pk, pk_kind = peaks()
    hbm = pk["hbm_gbs"]
    achieved = sb[names[dom]] / (per_launch_ms[dom] / 1000.0) / 1e9
    traffic = MEASURED_TRAFFIC.get(args.workload, {}).get(names[dom])
    fp32x2_peak = B.vdwgb_alu_peak(1, local)
    fp32_peak = B.vdwgb_alu_peak(0, local)
    fp64_peak = B.vdwgb_alu_peak(2, local)
    ic = names.index("contract")
    c_gflops = 4.0 * CONTRACT_FMA2_PER_KPOINT * nk_total / (per_launch_ms[ic] / 1000.0) / 1e9
    c64_gflops = (2.0 * CONTRACT_FMA64_PER_KPOINT * nk_total / (per_launch64[ic] / 1000.0) / 1e9
                  if per_launch64 is not None else None)
    roof = {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": hbm,
            "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
            "peak_source": pk_kind + " (copy bandwidth, MEASURED_PEAKS.json hbm_gbs)",
            "traffic_source": ("single-pass ncu capture of the timed steps (six part launches per step)"
                               if traffic is not None
                               else "no capture of the current kernel on this workload"),
            "stage_timing": "each stage launched on its own between CUDA events (one launch over the whole "
                            "batch), outside the timed steps; the timed steps replay the captured graph, where "
                            "the batch runs as overlapping parts",
            "stages": {n: {"ms_per_launch": float(m), "alg_bytes": int(sb[n]),
                           "GBps": (sb[n] / (m / 1000.0) / 1e9) if m > 0 else None,
                           "frac_hbm": (sb[n] / (m / 1000.0) / 1e9 / hbm) if m > 0 else None}
                       for n, m in zip(names, per_launch_ms)}}
    alu = {"peaks_gflops": {"fp32": fp32_peak, "fp32x2": fp32x2_peak, "fp64": fp64_peak,
                            "source": "vdwgb_alu_peak: FMA chains, CUDA events, timed alone"},
           "zfwd_issue": {"bound": "alu (instruction issue)", "frac": ZFWD_ISSUE_ACTIVE,
                          "source": "smsp__issue_active of an ncu capture (2 x 96^3 part launch)"},
           "contract_fp32": {"achieved_gflops": c_gflops, "peak_gflops": fp32x2_peak,
                             "frac": c_gflops / fp32x2_peak,
                             "flops_per_kpoint": 4 * CONTRACT_FMA2_PER_KPOINT},
           "contract_fp64": None if per_launch64 is None else
                            {"achieved_gflops": c64_gflops, "peak_gflops": fp64_peak,
                             "frac": c64_gflops / fp64_peak, "ms_per_launch": float(per_launch64[ic]),
                             "flops_per_kpoint": 2 * CONTRACT_FMA64_PER_KPOINT},
           "fp64_stages_ms_per_launch": None if per_launch64 is None else
                                        {n: float(m) for n, m in zip(names, per_launch64)}}

    # ---- extra workload: the 8-system 96^3 dimer batch ------------------------
    extra = None
    if not args.no_extra:
        log("extra workload: 8 x 96^3 dimers")
        dsys = make_workload("dimer96_batch8", rank, dev)
        fd = make(B.FP32_MIXED, dsys)
        btd = B.vdwgb_batch_new([f.h for f in fd])
        dnd = [torch.empty_like(s.n) for s in dsys]
        dsd = [torch.empty_like(s.n) for s in dsys]
        end = torch.zeros(len(dsys), dtype=torch.float64, device=dev)
        nsd, ssd = [s.n for s in dsys], [s.sigma for s in dsys]
        stepd, totd, clkd = timed_batch(B, torch, btd, nsd, ssd, dnd, dsd, end, sp, stream, args.steps,
                                        args.warmup, flush, world, dev, local)
        pld = stage_breakdown(B, torch, btd, nsd, ssd, dnd, dsd, end, sp, flush, args.steps)
        ptsd = sum(s.npts for s in dsys)
        sbd = {k: 0 for k in names}
        for s in dsys:
            for k, v in stage_bytes(s.shape, 4).items():
                sbd[k] += v
        if not any(B.vdwgb_plan_info(f.h)["cluster"] for f in fd):
            sbd["plane"] = 0
        extra = {"dimer96_batch8": {
            "value": job_points(ptsd, world, dev) * args.steps / (totd / 1000.0), "unit": "grid pts/s",
            "ms_per_step": totd / args.steps, "clocks": clkd,
            "stages": {n: {"ms_per_launch": float(m), "frac_hbm": (sbd[n] / (m / 1000.0) / 1e9 / hbm)
                           if m > 0 else None} for n, m in zip(names, pld)}}}
        B.vdwgb_batch_free(btd)
        for f in fd:
            f.close()

    spin_case = None
    if extra is not None:
        log("spin-polarised form")
        extra["spin_dimer96"], spin_case = spin_bench(B, inputs, torch, dev, local, sp, stream, flush)
        log("slab decomposition, virtual ranks")
        extra["slab_shell192_P4"] = slab_bench(B, inputs, torch, dev, local, stream, flush)

    if not args.no_serve:
        log("serving stream")
    serving = None if args.no_serve else serve_bench(B, inputs, torch, dev, local)

    # ---- oracle: errors of both forms and the CPU baseline (all host cores) ---
    err32 = err64 = cpu = None
    if not args.no_oracle and rank == 0 and world == 1 and args.workload != "shell640":
        jobs = [(i, s.n.cpu().numpy(), s.sigma.cpu().numpy(), s.cell, s.functional) for i, s in enumerate(systems)]
        workers = oracle_workers(max(s.npts for s in systems))
        log("oracle on %d host processes" % workers)
        pool = OraclePool(workers)
        try:
            ref, wall = pool.run(jobs)
        finally:
            pool.close()
        err32 = errors_vs_oracle(g32, ref)
        err64 = errors_vs_oracle(g64, ref) if g64 is not None else None
        if spin_case is not None:
            log("spin oracle on a 48^3 dimer")
            extra["spin_dimer96"]["error_vs_spin_oracle_48cubed"] = spin_errors(spin_case)
        one = float(np.mean([ref[i][4] / systems[i].npts for i in ref]))    # seconds per point, one core
        cpu = {"value": pts / wall, "unit": "grid pts/s", "cores": workers, "kind": "oracle",
               "sample": "the whole %s workload (%d systems, %d grid points), one system per worker process"
                         % (args.workload, nb, pts),
               "one_core_value": 1.0 / one, "host_cores": os.cpu_count(),
               "kernel_table": "built or loaded before timing"}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "grid pts/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload,
                       "grids": sorted({tuple(s.shape) for s in systems}), "systems": nb, "grid_points": pts,
                       "functionals": sorted({int(s.functional) for s in systems}), "precision": PRECISION_NOTE,
                       "parallelism": "replicas", "plan_first_system": plan_info,
                       "l2": "flushed between timed steps (256 MB write); working set %.0f MB"
                             % (sum(s.shape[0] * s.shape[1] * (s.shape[2] // 2 + 1) * 160 + 48 * s.npts
                                    for s in systems) / 1e6)},
            "fp64_plain": None if fp64_value is None else
                          {"value": fp64_value, "unit": "grid pts/s", "steps": k64,
                           "ms_per_step": t64 / k64, "form": "one system at a time"},
            "speedup_fp32_batched_vs_fp64_plain": None if fp64_value is None else value / (fp64_value * world),
            "latency_ms": {"single_system_fp32": {"p50": float(np.percentile(lat, 50)),
                                                  "p99": float(np.percentile(lat, 99)), "n": int(lat.size)},
                           "batch_step": {"p50": float(np.percentile(step_ms, 50)),
                                          "p99": float(np.percentile(step_ms, 99))}},
            "error_vs_oracle": {"fp32_mixed": err32, "fp64": err64},
            "error_fp32_vs_fp64": err_32_64,
            "roofline": roof,
            "alu": alu,
            "e2e": {"value": e2e_val, "unit": "grid pts/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "api": "vdwgb_batch_calculate (host arrays, pinned)"},
            "gpu_launches": int(args.steps * launches_per_step),
            "clocks": clocks,
            "table_build_s": B.vdwgb_table_build_seconds(local),
        }
        if cpu is not None:
            out["cpu_baseline"] = cpu
        if supercell is not None:
            out["supercell_check"] = supercell
        if extra is not None:
            out["extra"] = extra
        if serving is not None:
            out["serving"] = serving
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
