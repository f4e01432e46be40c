"""Benchmark: VR filtered-complex build throughput (simplices/s) on one cloud.

Workload (default): 1000 points on a torus (R=3, r=1) + N(0, 0.05^2) noise,
scaled by 30 to an int8 grid, radius cap at the 15th-percentile pairwise
squared distance, simplices up to dimension 2 (vertices, edges, triangles).

One step = one complete vr_build (distances, cap, ranking, enumeration,
(grade, lex) order, boundary CSC) from device-resident points; its result is
freed after the step's end event.  L2 is flushed (256 MB write) between timed
steps, outside the per-step events.  e2e repeats the step through the same
C-ABI call with the points in pinned host memory and copies every output
array back to pinned host memory inside the timed region.

--impl reference times the plain CPU oracle (the correctness reference) on
the host cores on the same workload; it is a deliberately slow program.
Multi-GPU (torchrun): the single-cloud build does not shard, so every rank
builds its own replica ("replicas only"); value = all ranks' simplices / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOADS = {
    "torus": ("torus n=1000 d=3 int8 (scale 30, noise 0.05), cap at 15th-pct d^2, maxdim 2",
              lambda: synth.config2(), "int64"),
    "plain64": ("uniform int32 n=64 d=3 in [-100,100], no cap, maxdim 2", lambda: synth.config1(), "int64"),
    "gauss32": ("8-Gaussian mixture n=4000 d=32 float32, cap at 5th-pct d^2, maxdim 2",
                lambda: synth.config3(), "f64"),
    "worldmap": ("WorldMap-shaped n=7322 d=3 float32 on the unit sphere (7 blobs + uniform), cap 0.15, maxdim 2",
                 lambda: synth.worldmap(), "f64"),
    "torus3": ("torus n=1000 d=3 int8 (scale 30, noise 0.05), cap at 15th-pct d^2, maxdim 3 (tetrahedra)",
               lambda: synth.Cloud(synth.config2().points, 3, synth.config2().maxrad), "int64"),
    "hiv": ("HIV-shaped 1088x1088 int32 Hamming distance matrix (9 subtypes), cap at its 10th percentile, maxdim 2",
            lambda: synth.hiv(), "int64"),
}


def oracle_build(cloud):
    import oracle
    if isinstance(cloud, synth.Matrix):
        return oracle.vr_build_dmat(cloud.points, cloud.maxdim, cloud.maxrad)
    return oracle.vr_build(cloud.points, cloud.maxdim, cloud.maxrad)


def gpu_build(cloud, src, **kw):
    import paper_1809_04424_b300 as vr
    if isinstance(cloud, synth.Matrix):
        if "d" in kw:
            kw.pop("d")
        return vr.vr_build_dmat(src, cloud.maxdim, cloud.maxrad, **kw)
    return vr.vr_build(src, cloud.maxdim, cloud.maxrad, **kw)
METRIC = "VR simplices/s"

# Algorithmic bytes per unit of each phase.
#   tri_emit:  36 B written per triangle (verts 12, grade 4, rowidx 12, colptr 8)
#   edge_sort: 8 B read + 8 B written per key per pass
#   edge_grades: keys 8 read, flags 4+4, outputs 8+4+8+8, CSR scatter 8 per edge


def roofline_bytes(cloud, E, T, T4=0, ngrades=0):
    """Algorithmic bytes of one launch of each single-kernel phase."""
    # Tetrahedron keys carry the packed vertices when the grades fit 12 bits;
    # otherwise the final write also reads an 8 B vertex record.
    tet_read = 8 if (ngrades - 1).bit_length() <= 12 else 16
    n = cloud.n
    Wd = (n + 31) // 32
    return {
        "tri_sort.pass": 16 * T,           # one digit pass: read + write one 8 B key
        "tri_sort.hist": 8 * T,            # all-digit histogram: read one 8 B key
        "tri_final": 44 * T,               # read key 8 B, write verts 12 + grade 4 + rowidx 12 + colptr 8
        "tri_lex_gen": 8 * T,              # write one 8 B key
        "tri_emit": 36 * T,                # write verts 12 + grade 4 + rowidx 12 + colptr 8
        "edge_sort.pass": 16 * E,
        "edge_sort.hist": 8 * E,
        "distance": cloud.points.nbytes + 4 * n * Wd,  # read points, write the bitmap
        "edge_keys": 8 * E,
        "tet_final": (tet_read + 36) * T4,  # read key (+ vertex record); write verts 16, grade 4, colptr 8, rowidx 16
    }


def sources_hash():
    """sha1 prefix over the CUDA sources and the C header (the key under which
    ncu traffic figures are recorded)."""
    import glob
    import hashlib
    h = hashlib.sha1()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_1809_04424_b300", "csrc", "*"))) + \
            [os.path.join(ROOT, "include", "vr.h")]:
        if f.endswith((".cu", ".cuh", ".h")):
            with open(f, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(region, workload):
    """DRAM bytes per launch (read + write) of `region` on `workload` from a
    profile summary's 'traffic:' line, if it was taken on the current
    sources; else None."""
    import glob
    cur = sources_hash()
    for f in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        with open(f) as fh:
            for line in fh:
                if not line.startswith("traffic:"):
                    continue
                kv = dict(x.split("=", 1) for x in line.split()[1:] if "=" in x)
                if kv.get("region") == region and kv.get("workload") == workload and kv.get("sources") == cur:
                    return int(kv["bytes_per_launch"])
    return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class NoGC:
    """The interpreter's cyclic garbage collector held off for a timed region
    (collected first), so that no collection pause lands inside a step."""

    def __enter__(self):
        gc.collect()
        gc.disable()
        return self

    def __exit__(self, *a):
        gc.enable()
        return False


class Clocks:
    """SM clock and throttle-reason samples taken DURING the timed region:
    NVML polled from a thread about every millisecond (reads only), else
    nvidia-smi at 20 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
            "hw_thermal_slowdown": 0x40, "hw_power_brake_slowdown": 0x80}

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.p = None
        self.nv = None
        self.samples = []
        self.max_mhz = None
        self.out = ""

    def _nvml_handle(self):
        """NVML through ctypes on the driver's libnvidia-ml (queries only)."""
        import ctypes
        import torch
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        want = ""
        try:
            want = str(torch.cuda.get_device_properties(self.gpu).uuid).replace("GPU-", "")
        except Exception:
            pass
        cnt = ctypes.c_uint()
        lib.nvmlDeviceGetCount_v2(ctypes.byref(cnt))
        pick = None
        for i in range(cnt.value):
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(i, ctypes.byref(h)) != 0:
                continue
            buf = ctypes.create_string_buffer(96)
            lib.nvmlDeviceGetUUID(h, buf, 96)
            if want and want in buf.value.decode():
                pick = h
                break
        if pick is None:
            pick = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(self.gpu, ctypes.byref(pick)) != 0:
                raise RuntimeError("no NVML handle")
        reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons

        def clock(kind_max=False):
            v = ctypes.c_uint()
            f = lib.nvmlDeviceGetMaxClockInfo if kind_max else lib.nvmlDeviceGetClockInfo
            if f(pick, 1, ctypes.byref(v)) != 0:  # 1 = NVML_CLOCK_SM
                raise RuntimeError("clock query failed")
            return float(v.value)

        def reasons():
            v = ctypes.c_ulonglong()
            reasons_fn(pick, ctypes.byref(v))
            return int(v.value)

        return clock, reasons

    def __enter__(self):
        try:
            clock, reasons = self._nvml_handle()
            self.nv = (clock, reasons)
            self.max_mhz = clock(True)
            self.stop = threading.Event()

            def poll():
                while not self.stop.is_set():
                    try:
                        self.samples.append((clock(), reasons()))
                    except Exception:
                        pass
                    time.sleep(0.001)

            self.th = threading.Thread(target=poll, daemon=True)
            self.th.start()
            t0 = time.time()
            while not self.samples and time.time() - t0 < 2:  # start with one sample in hand
                time.sleep(0.0005)
            return self
        except Exception:
            self.nv = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.nv is not None:
            try:
                self.samples.append((self.nv[0](), self.nv[1]()))
            except Exception:
                pass
            self.stop.set()
            self.th.join(timeout=2)
            return False
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
        return False

    def summary(self):
        if self.nv is not None and self.samples:
            reasons = set()
            for _, r in self.samples:
                for nm, bit in self.BITS.items():
                    if r & bit:
                        reasons.add(nm)
            return {"sm_mhz": statistics.median(c for c, _ in self.samples), "sm_max_mhz": self.max_mhz,
                    "reasons": sorted(reasons), "samples": len(self.samples), "source": "nvml"}
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "source": "nvidia-smi"}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Ranks:
    """One process per GPU (torchrun env).  The work shards by independent
    units (replicas of a cloud, clouds of a batch, requests of a stream) with
    no data-path collective: a barrier around the timed region and a max of
    the ranks' times are the only communication.  backend: "nccl" on GPUs,
    "gloo" for the host-only tests."""

    def __init__(self, backend="nccl"):
        self.world, self.rank, self.local = dist_env()
        self.dist = None
        self.backend = backend
        if self.world > 1:
            import torch.distributed as dist
            if not dist.is_initialized():
                dist.init_process_group(backend)
            self.dist = dist

    def shard(self, n_units):
        """This rank's contiguous share [lo, hi) of n_units (sizes differ by
        at most one)."""
        q, r = divmod(n_units, self.world)
        lo = self.rank * q + min(self.rank, r)
        return lo, lo + q + (1 if self.rank < r else 0)

    def barrier(self):
        if self.dist:
            self.dist.barrier()

    def max(self, x: float) -> float:
        """The largest x over the ranks (a rank's time: the job ends with the
        slowest)."""
        if not self.dist:
            return float(x)
        import torch
        dev = "cuda" if self.backend == "nccl" else "cpu"
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if not self.dist:
            return float(x)
        import torch
        dev = "cuda" if self.backend == "nccl" else "cpu"
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.dist:
            self.dist.destroy_process_group()
            self.dist = None


def whole_job_rate(units_all_ranks: float, slowest_seconds: float) -> float:
    """Units processed by every rank together over the slowest rank's time."""
    return units_all_ranks / slowest_seconds


def oracle_rate(cloud, seconds: float):
    """Time the oracle as it stands on full builds of the workload."""
    import oracle
    oracle.build()
    reps, t0 = 0, time.perf_counter()
    simp = 0
    while True:
        cx = oracle_build(cloud)
        simp += sum(d.count for d in cx.dims)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return simp / el, reps, el


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    WORKLOAD, make, dtype_name = WORKLOADS[args.config]
    cloud = make()
    for _ in range(args.warmup):
        oracle_build(cloud)
    t0 = time.perf_counter()
    simp = 0
    for _ in range(args.steps):
        cx = oracle_build(cloud)
        simp += sum(d.count for d in cx.dims)
    el = time.perf_counter() - t0
    v = simp / el
    line = {"metric": METRIC, "value": v, "unit": "simplices/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype_name, "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "n": cloud.n, "d": cloud.d, "maxdim": cloud.maxdim},
            "cpu_baseline": {"value": v, "unit": "simplices/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} full builds of the workload, single-threaded C oracle"},
            "e2e": {"value": v, "unit": "simplices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# Bytes of one cloud's descriptor in the batch path (struct CloudDesc of the
# batch source: 14 eight-byte fields and 8 four-byte ones); the library sends it
# to the device twice per batch and reads it back twice.
CLOUD_DESC_BYTES = 144


def run_batch_bench(args):
    """Batched clouds/s: all clouds of the uneven sphere workload in one
    vr_build_batch call per step, against the per-cloud path (one vr_build per
    cloud, plain launches, same GPU) timed on a sample of the same clouds."""
    import ctypes
    import torch
    import paper_1809_04424_b300 as vr
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    ranks = Ranks()
    lo, hi = ranks.shard(args.n_clouds)  # this rank's clouds of the batch
    clouds = synth.config4(args.n_clouds)[lo:hi]
    pts = np.concatenate([c.points for c in clouds], axis=0)
    off = np.concatenate([[0], np.cumsum([c.n for c in clouds])]).astype(np.int64)
    dev = torch.from_numpy(pts).cuda()
    L = vr.lib()
    W = max(args.warmup, 3)
    for _ in range(W):
        b = vr.vr_build_batch(dev, off, 2, 40.0)
        tot = b.info()["total_simplices"]
        del b
    torch.cuda.synchronize()
    L.vr_profile_reset()
    L.vr_profile_enable(1)
    launches0 = L.vr_launch_count()
    ranks.barrier()
    with NoGC(), Clocks(local) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            b = vr.vr_build_batch(dev, off, 2, 40.0)
            del b
        torch.cuda.synchronize()
        el = ranks.max(time.perf_counter() - t0)
    L.vr_profile_enable(0)
    launches = L.vr_launch_count() - launches0
    phases = {}
    for i in range(L.vr_profile_phases()):
        nm, ms, calls, nl = ctypes.c_char_p(), ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        L.vr_profile_phase(i, ctypes.byref(nm), ctypes.byref(ms), ctypes.byref(calls), ctypes.byref(nl))
        phases[nm.value.decode()] = round(ms.value / max(calls.value, 1), 4)
    batched = whole_job_rate(args.n_clouds * args.steps, el)
    tot = ranks.sum(tot)
    # per-cloud path on a sample
    sample = clouds[: min(len(clouds), 256)]
    devs = [torch.from_numpy(c.points).cuda() for c in sample]
    for c, dp in list(zip(sample, devs))[:8]:
        vr.vr_build(dp, 2, 40.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c, dp in zip(sample, devs):
        x = vr.vr_build(dp, 2, 40.0)
        del x
    torch.cuda.synchronize()
    per_cloud = len(sample) / (time.perf_counter() - t0)
    # e2e: host points in, each cloud's descriptor back, the complexes stay on the device
    host = torch.from_numpy(pts).pin_memory()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        b = vr.vr_build_batch(host.numpy(), off, 2, 40.0)
        if b.info()["n_failed"]:
            raise RuntimeError("batch build failed on some clouds")
        del b
    torch.cuda.synchronize()
    e2e = args.n_clouds * args.steps / (time.perf_counter() - t0)
    line = {"metric": "batched clouds/s", "value": batched, "unit": "clouds/s", "n_gpus": world,
            "scaling_note": "clouds sharded across ranks, no collective on the data path",
            "steps": args.steps, "warmup": W, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": f"{args.n_clouds} sphere clouds n~U[32,512] d=3 int8 (scale 100, noise 0.02), "
                                   "cap 40, maxdim 2", "simplices_per_step": tot,
                       "l2": "inputs and outputs larger than L2 per step"},
            "simplices_per_s": tot * args.steps / el,
            "per_cloud_path": {"value": per_cloud, "unit": "clouds/s", "sample_clouds": len(sample),
                               "speedup_batched": batched / per_cloud},
            "e2e": {"value": e2e, "unit": "clouds/s",
                    "h2d_bytes_per_step": int(pts.nbytes) + len(clouds) * (2 * CLOUD_DESC_BYTES + 4),
                    "d2h_bytes_per_step": len(clouds) * 2 * CLOUD_DESC_BYTES,
                    "read_back": "each cloud's descriptor (sizes, status, grade count) after the sizing pass "
                                 "and after the build; the complexes stay on the device"},
            "gpu_launches": launches, "phases_ms": phases, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ranks.close()
    return 0


def _open_loop(submit_fn, poll_fn, reqs, arrivals, n_pollers=16):
    """Submit request i at arrivals[i] (seconds from start) and record when
    its result is back.  Returns (latencies in s, wall time of the run)."""
    import threading
    N = len(reqs)
    tickets = [None] * N
    ready = [threading.Event() for _ in range(N)]
    done = [0.0] * N
    t_start = time.perf_counter() + 0.05

    def submitter():
        for i, r in enumerate(reqs):
            dt = t_start + arrivals[i] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets[i] = submit_fn(r)
            ready[i].set()

    def poller(k):
        for i in range(k, N, n_pollers):
            ready[i].wait()
            poll_fn(tickets[i])
            done[i] = time.perf_counter()

    th = [threading.Thread(target=submitter)] + [threading.Thread(target=poller, args=(k,)) for k in range(n_pollers)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    lat = np.array([done[i] - (t_start + arrivals[i]) for i in range(N)])
    return lat, max(done) - t_start


def run_serve_bench(args):
    """Serving: a Poisson stream of mixed requests (n log-uniform in
    [50, 5000]; half int8 d=3 torus/sphere, half float32 d=16 mixtures;
    maxdim in {1, 2}; per-request cap) through the continuous-batching server
    at 0.8x its measured capacity: p50/p99 latency and clouds/s, against the
    per-cloud path (one vr_build per request, FIFO) on the same arrivals."""
    import torch
    import paper_1809_04424_b300 as vr
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    ranks = Ranks()
    _, reqs_all = synth.config5(args.n_requests)
    lo, hi = ranks.shard(args.n_requests)  # this rank's share of the stream
    reqs = reqs_all[lo:hi]
    N = len(reqs)
    srv = vr.Server(n_streams=3, max_batch_clouds=256, n_large_workers=4)
    submit = lambda r: srv.submit(r.points, r.maxdim, r.maxrad)
    poll = lambda t: srv.poll(t, 120_000_000)
    for r in reqs[:64]:  # warm-up
        poll(submit(r))
    # capacity, closed loop
    C = min(N, 4000)
    t0 = time.perf_counter()
    ts = [submit(r) for r in reqs[:C]]
    for t in ts:
        poll(t)
    cap = C / (time.perf_counter() - t0)
    lam = 0.8 * cap
    g = synth.rng(1809 + 50)
    arrivals = np.cumsum(g.exponential(1.0 / lam, size=N))
    ranks.barrier()
    with Clocks(local) as clk:
        lat, wall = _open_loop(submit, poll, reqs, arrivals)
    wall_all = ranks.max(wall)
    sweep = {}
    for f in (0.5, 1.0):
        M = min(N, 4000)
        a = np.cumsum(synth.rng(1809 + 51).exponential(1.0 / (f * cap), size=M))
        l2, w2 = _open_loop(submit, poll, reqs[:M], a)
        sweep[str(f)] = {"p50_ms": 1e3 * float(np.percentile(l2, 50)), "p99_ms": 1e3 * float(np.percentile(l2, 99)),
                         "clouds_per_s": M / w2}
    srv.close()
    # per-cloud path: one vr_build per request in arrival order, one worker
    M = min(N, 2000)
    devq = []
    import threading
    lock = threading.Lock()

    def per_submit(r):
        return r

    results = {}

    def per_poll(r):
        with lock:  # a single FIFO worker: plain launches, one cloud at a time
            x = vr.vr_build(r.points, r.maxdim, r.maxrad)
            del x
    t0 = time.perf_counter()
    for r in reqs[:200]:
        per_poll(r)
    per_cap = 200 / (time.perf_counter() - t0)
    a = np.cumsum(synth.rng(1809 + 52).exponential(1.0 / lam, size=M))
    lp, wp = _open_loop(per_submit, per_poll, reqs[:M], a, n_pollers=1)
    line = {"metric": "served clouds/s", "value": whole_job_rate(args.n_requests, wall_all), "unit": "clouds/s",
            "n_gpus": world, "steps": N,
            "warmup": 64, "ms_per_step": 1e3 * wall / N, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "mixed int64/f64", "data": "synthetic",
            "config": {"workload": f"Poisson stream of {N} requests, n log-uniform [50,5000], half int8 d=3 "
                                   "torus/sphere, half f32 d=16 Gaussian mixtures, maxdim {1,2}, per-request cap",
                       "arrival_rate_per_s": lam, "capacity_closed_loop": cap},
            "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)), "p99": 1e3 * float(np.percentile(lat, 99)),
                           "mean": 1e3 * float(lat.mean())},
            "rate_sweep": sweep,
            "per_cloud_path": {"capacity_clouds_per_s": per_cap, "requests": M,
                               "p50_ms": 1e3 * float(np.percentile(lp, 50)),
                               "p99_ms": 1e3 * float(np.percentile(lp, 99)), "clouds_per_s": M / wp},
            "e2e": {"value": N / wall, "unit": "clouds/s", "h2d_bytes_per_step": int(np.mean([r.points.nbytes for r in reqs])),
                    "d2h_bytes_per_step": 2 * CLOUD_DESC_BYTES,
                    "read_back": "per request its descriptor (batched requests, twice) or the status word the "
                                 "device writes to mapped host memory (large ones); the complexes stay on the device"},
            "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ranks.close()
    return 0


def run_bars_bench(args):
    """One step = build the complex and compute its barcodes in every
    dimension on the device (GPU reduction of the boundary matrix)."""
    import ctypes
    import torch
    import paper_1809_04424_b300 as vr
    WORKLOAD, make, dtype_name = WORKLOADS[args.config]
    cloud = make()
    L = vr.lib()
    src = torch.from_numpy(cloud.points).cuda()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    W = max(args.warmup, 3)

    def step():
        c = gpu_build(cloud, src)
        nb = [len(c.barcode(k)) for k in range(cloud.maxdim + 1)]
        return c, nb

    for _ in range(W):
        c, nbars = step()
        counts = c.counts()[0]
        del c
    torch.cuda.synchronize()
    L.vr_profile_select(None)
    L.vr_profile_reset()
    L.vr_profile_enable(1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with Clocks(0) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record()
            c, _ = step()
            ev[k][1].record()
            del c
        torch.cuda.synchronize()
    L.vr_profile_enable(0)
    ms = sum(a.elapsed_time(b) for a, b in ev)
    phases = {}
    for i in range(L.vr_profile_phases()):
        nm, t, calls, nl = ctypes.c_char_p(), ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        L.vr_profile_phase(i, ctypes.byref(nm), ctypes.byref(t), ctypes.byref(calls), ctypes.byref(nl))
        if nm.value.decode().startswith("bars."):
            phases[nm.value.decode()] = round(t.value / max(calls.value, 1), 3)
    simplices = sum(counts)
    cpu = None
    if args.cpu_seconds > 0:
        t0 = time.perf_counter()
        reps = 0
        while True:
            cx = oracle_build_keep(cloud)
            for k in range(cloud.maxdim + 1):
                cx.barcode(k)
            reps += 1
            if time.perf_counter() - t0 >= args.cpu_seconds:
                break
        el = time.perf_counter() - t0
        cpu = {"value": simplices * reps / el, "unit": "simplices/s", "cores": 1, "kind": "oracle",
               "sample": f"{reps} build(s) + barcodes of the workload in {el:.1f} s, single-threaded "
                         "(column algorithm in homology)"}
    line = {"metric": "VR simplices/s, build + barcodes of every dimension", "value": simplices * args.steps / (ms / 1e3),
            "unit": "simplices/s", "n_gpus": 1, "steps": args.steps, "warmup": W,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_name, "data": "synthetic",
            "config": {"workload": WORKLOAD, "counts": counts, "bars_per_dim": nbars,
                       "l2": "flushed between steps (256 MB write)"},
            "e2e": None, "gpu_launches": None, "roofline": None,
            "roofline_note": "the reduction is latency-bound on chains of column additions; see bars phases",
            "bars_phases_ms": phases, "clocks": clk.summary(), "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    return 0


def oracle_build_keep(cloud):
    import oracle
    if isinstance(cloud, synth.Matrix):
        return oracle.vr_build_dmat(cloud.points, cloud.maxdim, cloud.maxrad, keep_handle=True)
    return oracle.vr_build(cloud.points, cloud.maxdim, cloud.maxrad, keep_handle=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="length of the CPU-oracle baseline sample (0 skips it)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--config", default="torus", choices=sorted(WORKLOADS) + ["batch", "serve"],
                    help="workload (default: the headline torus cloud)")
    ap.add_argument("--n-clouds", type=int, default=4096, help="clouds of the batch workload")
    ap.add_argument("--n-requests", type=int, default=20000, help="requests of the serving workload")
    ap.add_argument("--bars", action="store_true",
                    help="time build + persistence barcodes of every dimension (the reduction step)")
    args = ap.parse_args()
    if args.bars and args.impl != "reference":
        return run_bars_bench(args)
    if args.config == "batch" and args.impl != "reference":
        return run_batch_bench(args)
    if args.config == "serve" and args.impl != "reference":
        return run_serve_bench(args)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_1809_04424_b300 as vr

    world, rank, local = dist_env()
    assert torch.cuda.is_available(), "bench needs a CUDA device"
    torch.cuda.set_device(local)
    ranks = Ranks()
    W = max(args.warmup, 3)
    L = vr.lib()

    WORKLOAD, make, dtype_name = WORKLOADS[args.config]
    cloud = make()
    pts_dev = torch.from_numpy(cloud.points).cuda()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        return gpu_build(cloud, pts_dev)

    for _ in range(W):
        c = step()
        counts = c.counts()[0]
        ngrades = c.stats()["ngrades"]
        del c
    torch.cuda.synchronize()
    simplices = sum(counts)

    import ctypes
    L.vr_profile_select.argtypes = [ctypes.c_char_p]

    def read_phases():
        out = {}
        for i in range(L.vr_profile_phases()):
            nm, ms, calls, nl = ctypes.c_char_p(), ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
            L.vr_profile_phase(i, ctypes.byref(nm), ctypes.byref(ms), ctypes.byref(calls), ctypes.byref(nl))
            out[nm.value.decode()] = {"ms_per_call": ms.value / max(calls.value, 1), "calls": calls.value,
                                      "launches_per_call": nl.value / max(calls.value, 1)}
        return out

    # ---- calibration (untimed): every phase timed by the library's events.
    L.vr_profile_select(None)
    L.vr_profile_reset()
    L.vr_profile_enable(1)
    for _ in range(min(args.steps, 20)):
        flush.zero_()
        c = step()
        del c
    torch.cuda.synchronize()
    L.vr_profile_enable(0)
    phases = read_phases()
    per_launch_bytes = roofline_bytes(cloud, counts[1], counts[2], counts[3] if len(counts) > 3 else 0, ngrades)
    # Regions of one kernel (a sort's digit passes: several launches of the
    # same kernel, each timed).
    single = {k: v for k, v in phases.items() if k in per_launch_bytes
              and (v["launches_per_call"] == 1 or k.endswith(".pass"))}
    dom = max(single, key=lambda k: single[k]["ms_per_call"]) if single else None

    # ---- timed region: K steps, per-step CUDA events, L2 flushed between;
    # inside it the library times only the dominant kernel's region.
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    L.vr_profile_select(dom.encode() if dom else b"-")
    L.vr_profile_reset()
    L.vr_profile_enable(1)
    ranks.barrier()
    torch.cuda.synchronize()
    launches0 = L.vr_launch_count()
    with NoGC(), Clocks(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            c = step()
            ev[k][1].record(stream)
            del c
        torch.cuda.synchronize()
    launches = L.vr_launch_count() - launches0
    L.vr_profile_enable(0)
    ranks.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = ranks.max(sum(step_ms))
    value = whole_job_rate(simplices * args.steps * world, total_ms / 1e3)

    timed_phases = read_phases()
    L.vr_profile_select(None)

    # ---- e2e: host (pinned) points in, every output array back to pinned host.
    host_pts = torch.from_numpy(cloud.points).pin_memory()
    c0 = gpu_build(cloud, pts_dev)
    cnt, _ = c0.counts()
    del c0
    bufs = []
    for k in range(3):
        m = cnt[k]
        bufs.append([torch.empty(m * (k + 1), dtype=torch.int32).pin_memory(),
                     torch.empty(m, dtype=torch.int32).pin_memory(),
                     torch.empty(m + 1, dtype=torch.int64).pin_memory() if k else None,
                     torch.empty(m * (k + 1), dtype=torch.int32).pin_memory() if k else None])
    d2h = sum(b.numel() * b.element_size() for bb in bufs for b in bb if b is not None)
    gv = None

    def e2e_step():
        nonlocal gv
        c = gpu_build(cloud, host_pts.data_ptr(), n=cloud.n, d=cloud.d,
                        dtype=cloud.dtype_code)
        for k in range(3):
            b = bufs[k]
            p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
            rc = L.vr_complex_to_host(ctypes.c_void_p(c.handle), k, p(b[0]), p(b[1]), p(b[2]), p(b[3]))
            assert rc == 0, vr.vr_last_error()
        _, ng = vr.vr_complex_grade_values(c.handle)
        if gv is None:
            gv = torch.empty(ng, dtype=torch.float64).pin_memory()
        L.vr_complex_grade_values_to_host(ctypes.c_void_p(c.handle), ctypes.c_void_p(gv.data_ptr()))
        del c

    e2e_val = None
    if not args.no_e2e:
        for _ in range(W):
            e2e_step()
        torch.cuda.synchronize()
        with NoGC():
            t0 = time.perf_counter()
            for _ in range(args.steps):
                e2e_step()
            torch.cuda.synchronize()
            e2e_s = time.perf_counter() - t0
        d2h += gv.numel() * 8
        e2e_val = simplices * args.steps * world / e2e_s

    # ---- roofline of the dominant kernel: its region timed by the library's
    # CUDA events on the build stream inside the timed region.
    hbm, src = peaks()
    roof = None
    if dom and dom in timed_phases:
        tp = timed_phases[dom]
        per_launch_ms = tp["ms_per_call"] if dom.endswith(".pass") else \
            tp["ms_per_call"] / max(tp["launches_per_call"], 1)
        ach = per_launch_bytes[dom] / (per_launch_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": recorded_traffic(dom, args.config), "peak_source": src,
                "algorithmic_bytes_per_launch": per_launch_bytes[dom],
                "launch_ms": per_launch_ms, "launches_timed": tp["calls"]}

    line = {"metric": METRIC, "value": value, "unit": "simplices/s", "n_gpus": world, "steps": args.steps,
            "warmup": W, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype_name, "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": cloud.n, "d": cloud.d, "maxdim": cloud.maxdim,
                       "maxrad": cloud.maxrad, "simplices_per_step": simplices,
                       "counts": counts, "l2": "flushed between steps (256 MB write)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "e2e": {"value": e2e_val, "unit": "simplices/s",
                    "h2d_bytes_per_step": cloud.points.nbytes,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "roofline": roof,
            "phases_ms": {k: round(v["ms_per_call"], 4) for k, v in phases.items()},
            "phases_note": "ms per call, from an untimed calibration pass before the timed region",
            "phase_launches": {k: v["launches_per_call"] for k, v in phases.items()},
            "clocks": clk.summary()}
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        r, reps, el = oracle_rate(cloud, args.cpu_seconds)
        line["cpu_baseline"] = {"value": r, "unit": "simplices/s", "cores": 1, "kind": "oracle",
                                "sample": f"{reps} full builds of the workload in {el:.1f} s, single-threaded"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ranks.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
