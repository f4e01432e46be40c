"""Benchmark: VR filtered-complex build throughput (simplices/s), with the
batched and served forms nested in the same line.

Workload (default): 4000 points in R^32, float32, a mixture of 8 isotropic
Gaussians (centres uniform in [-5, 5]^32, sigma 1), radius cap at the 5th
percentile of pairwise squared distance, simplices up to dimension 2
(vertices, edges, triangles: 19.76M triangles per build).

One step = one complete vr_build (distances, cap, ranking, enumeration,
(grade, lex) order, boundary CSC) from device-resident points; its result is
freed after the step's end event.  L2 is flushed (256 MB write) between timed
steps, outside the per-step events.  e2e repeats the step through the same
C-ABI call with the points in pinned host memory and copies every output
array back to pinned host memory inside the timed region.

Nested in the default line (skip with --no-nested):
  batched: 4096 uneven sphere clouds (n ~ U[32, 512], int8, maxdim 2) in one
           vr_build_batch per step, against one vr_build per cloud on every
           cloud, and the oracle run across clouds on all host cores;
  served:  a Poisson stream of 20000 mixed requests through the continuous-
           batching server at 0.8x its closed-loop capacity (p50/p99 latency,
           clouds/s), against one vr_build per request in arrival order, and
           the oracle across requests on all host cores on a bounded sample.

--impl reference times the plain CPU oracle (the correctness reference) on
the host cores on the same workload; it is a deliberately slow program.
Multi-GPU (torchrun): the single-cloud build does not shard, so every rank
builds its own replica ("replicas only"); value = all ranks' simplices / the
slowest rank's time.  Batches and streams shard by cloud.
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
DEFAULT_CONFIG = "gauss32"


def method_bytes_per_step(cloud, counts):
    """Bytes the method must move per build: the input, 76 B per kept edge
    (key 8 written + 8 read; outputs verts 8, grade 4, rowidx 8, colptr 8;
    neighbour CSR 16 written + 16 read), 36 B per triangle (verts 12,
    grade 4, rowidx 12, colptr 8) and 44 B per tetrahedron (verts 16, grade 4,
    rowidx 16, colptr 8)."""
    E = counts[1] if len(counts) > 1 else 0
    T = counts[2] if len(counts) > 2 else 0
    T4 = counts[3] if len(counts) > 3 else 0
    return int(cloud.points.nbytes) + 76 * E + 36 * T + 44 * T4


def roofline_bytes(cloud, E, T, T4=0, ngrades=0, tri_order=1):
    """Per launch of each single-kernel phase: (method bytes, intermediate
    bytes).  Method bytes are the per-unit figures of method_bytes_per_step
    that the kernel moves; intermediates (sort keys, bitmaps) are listed
    apart and never counted in `achieved`.  tri_order is the build's
    triangle path (vr_build_stats): 1 lex keys, 8 B; 2 max-edge keys, 4 B
    when the edge indices fit beside the vertex in 32 bits, else 8 B; 3
    max-edge third vertices in claimed space, 2 B per triangle plus each
    edge's count and run start."""
    tet_read = 8 if (ngrades - 1).bit_length() <= 12 else 16
    n = cloud.n
    Wd = (n + 31) // 32
    if tri_order == 3:
        key, key_e = 2, 8
    else:
        key, key_e = (8 if tri_order == 1 or E > 1 << (32 - max(1, (n - 1).bit_length())) else 4), 0
    return {
        "tri_final": (36 * T, key * T),        # outputs 36 B; reads one key (or third vertex)
        "tri_emit": (36 * T, 0),               # outputs 36 B, emitted at their final position
        "tri_lex_gen": (0, 8 * T),             # writes one 8 B key
        "tri_gen": (0, key * T + key_e * E),   # max-edge order: one key (or third vertex) per triangle
        "tri_sort.pass": (0, 16 * T),          # one digit pass over the keys
        "tri_sort.hist": (0, 8 * T),
        "edge_sort.pass": (16 * E, 0),         # the edge key: 8 B written + 8 B read
        "edge_sort.hist": (0, 8 * E),
        "edge_keys": (8 * E, 0),               # writes the edge key
        "distance": (int(cloud.points.nbytes), 4 * n * Wd),  # reads the points, writes the bitmap
        "tet_final": (44 * T4, tet_read * T4),
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


def host_cores():
    """Cores this process may run on (the box's usable host cores)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


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


def oracle_parallel_rate(clouds, seconds: float, threads: int):
    """The oracle as it stands, one whole build per cloud, clouds taken in
    order by `threads` host threads (the C call releases the interpreter
    lock, so the builds run in parallel).  Stops taking new clouds after
    `seconds`; returns (clouds built, elapsed seconds, threads)."""
    import ctypes
    import oracle
    oracle.build()
    lib = oracle._load()
    lock = threading.Lock()
    state = {"next": 0, "done": 0}
    t0 = time.perf_counter()

    def worker():
        while True:
            with lock:
                i = state["next"]
                if i >= len(clouds) or time.perf_counter() - t0 > seconds:
                    return
                state["next"] += 1
            c = clouds[i]
            pts = np.ascontiguousarray(c.points)
            out = oracle._Complex()
            rc = lib.vro_build(pts.ctypes.data, c.n, c.d, oracle._dtype_code(pts), c.maxdim, float(c.maxrad),
                               ctypes.byref(out))
            if rc:
                raise RuntimeError(f"oracle failed on cloud {i}: {rc}")
            lib.vro_free(ctypes.byref(out))
            with lock:
                state["done"] += 1

    th = [threading.Thread(target=worker) for _ in range(threads)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    return state["done"], time.perf_counter() - t0, threads


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
            "config": {"workload": WORKLOAD, "n": cloud.n, "d": cloud.d, "maxdim": cloud.maxdim,
                       "maxrad": cloud.maxrad},
            "cpu_baseline": {"value": v, "unit": "simplices/s", "cores": 1, "nproc": host_cores(), "kind": "oracle",
                             "sample": f"{args.steps} full builds of the workload, single-threaded C oracle"},
            "e2e": {"value": v, "unit": "simplices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# Bytes of one cloud's descriptor in the batch path (struct CloudDesc of the
# batch source: 14 eight-byte fields and 8 four-byte ones); the library sends it
# to the device twice per batch and reads it back twice.
CLOUD_DESC_BYTES = 144

BATCH_WORKLOAD = "4096 sphere clouds n~U[32,512] d=3 int8 (scale 100, noise 0.02), cap 40, maxdim 2"


def batch_leg(args, ranks, local):
    """Batched clouds/s: all clouds of the uneven sphere workload in one
    vr_build_batch call per step, against the per-cloud path (one vr_build per
    cloud, plain launches, same GPU) on every cloud.  Returns the result
    dict and this rank's clouds (for the CPU baseline)."""
    import ctypes
    import torch
    import paper_1809_04424_b300 as vr
    world = ranks.world
    lo, hi = ranks.shard(args.n_clouds)  # this rank's clouds of the batch
    clouds = synth.config4(args.n_clouds)[lo:hi]
    pts = np.concatenate([c.points for c in clouds], axis=0)
    off = np.concatenate([[0], np.cumsum([c.n for c in clouds])]).astype(np.int64)
    dev = torch.from_numpy(pts).cuda()
    L = vr.lib()
    W = max(args.warmup, 3)
    for _ in range(W):
        b = vr.vr_build_batch(dev, off, 2, 40.0)
        info = b.info()
        tot = info["total_simplices"]
        if info["n_failed"]:
            raise RuntimeError("batch build failed on some clouds")
        del b
    torch.cuda.synchronize()
    L.vr_profile_reset()
    L.vr_profile_enable(1)
    launches0 = L.vr_launch_count()
    steps = max(args.batch_steps, 1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    stream = torch.cuda.current_stream()
    ranks.barrier()
    torch.cuda.synchronize()
    with NoGC(), Clocks(local) as clk:
        t0 = time.perf_counter()
        for k in range(steps):
            ev[k][0].record(stream)
            b = vr.vr_build_batch(dev, off, 2, 40.0)
            ev[k][1].record(stream)
            del b
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    L.vr_profile_enable(0)
    launches = L.vr_launch_count() - launches0
    dev_ms = ranks.max(sum(a.elapsed_time(b) for a, b in ev))
    phases = {}
    for i in range(L.vr_profile_phases()):
        nm, ms, calls, nl = ctypes.c_char_p(), ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        L.vr_profile_phase(i, ctypes.byref(nm), ctypes.byref(ms), ctypes.byref(calls), ctypes.byref(nl))
        phases[nm.value.decode()] = round(ms.value / max(calls.value, 1), 4)
    batched = whole_job_rate(args.n_clouds * steps, dev_ms / 1e3)
    tot = ranks.sum(tot)
    # The launch shape the tuner picked for this class, its candidates, and
    # the default shape (every CTA the launch allows per SM, largest cloud
    # first) timed the same way.
    shape = vr.vr_batch_get_shape()
    cands = shape["candidates"]
    default = (max(c[0] for c, _ in cands), 0) if cands else None
    default_rate = None
    if default is not None:
        vr.vr_batch_set_shape(*default)
        for _ in range(2):
            del_b = vr.vr_build_batch(dev, off, 2, 40.0)
            del del_b
        torch.cuda.synchronize()
        evd = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            evd[k][0].record(stream)
            b = vr.vr_build_batch(dev, off, 2, 40.0)
            evd[k][1].record(stream)
            del b
        torch.cuda.synchronize()
        vr.vr_batch_set_shape(0)
        default_rate = whole_job_rate(args.n_clouds * steps, ranks.max(sum(a.elapsed_time(b) for a, b in evd)) / 1e3)
    # per-cloud path: one vr_build per cloud, every cloud of this rank
    devs = [torch.from_numpy(c.points).cuda() for c in clouds]
    for dp in devs[:16]:
        vr.vr_build(dp, 2, 40.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for dp in devs:
        x = vr.vr_build(dp, 2, 40.0)
        del x
    torch.cuda.synchronize()
    per_cloud = whole_job_rate(args.n_clouds, ranks.max(time.perf_counter() - t0))
    # e2e: host points in, each cloud's descriptor back, the complexes stay on the device
    host = torch.from_numpy(pts).pin_memory()
    t0 = time.perf_counter()
    for _ in range(steps):
        b = vr.vr_build_batch(host.numpy(), off, 2, 40.0)
        if b.info()["n_failed"]:
            raise RuntimeError("batch build failed on some clouds")
        del b
    torch.cuda.synchronize()
    e2e = whole_job_rate(args.n_clouds * steps, ranks.max(time.perf_counter() - t0))
    out = {"metric": "batched clouds/s", "value": batched, "unit": "clouds/s", "steps": steps, "warmup": W,
           "ms_per_step": dev_ms / steps, "wall_ms_per_step": 1e3 * wall / steps,
           "workload": BATCH_WORKLOAD, "clouds": args.n_clouds, "simplices_per_step": tot,
           "simplices_per_s": tot * steps / (dev_ms / 1e3),
           "l2": "inputs and outputs larger than L2 per step",
           "per_cloud_path": {"value": per_cloud, "unit": "clouds/s", "clouds": args.n_clouds,
                              "how": "one vr_build per cloud, plain launches, same GPU, every cloud"},
           "speedup_vs_per_cloud": batched / per_cloud,
           "launch_shape": {"tuned": shape["used"], "default": default,
                            "default_clouds_per_s": default_rate,
                            "tuner_candidates_ms": [[list(c), round(ms, 4)] for c, ms in cands],
                            "what": "CTAs per SM of the one persistent launch, work-list order (0 largest first)"},
           "e2e": {"value": e2e, "unit": "clouds/s",
                   "h2d_bytes_per_step": int(pts.nbytes) + len(clouds) * (2 * CLOUD_DESC_BYTES + 4),
                   "d2h_bytes_per_step": len(clouds) * 2 * CLOUD_DESC_BYTES,
                   "read_back": "each cloud's descriptor (sizes, status, grade count); the complexes stay on "
                                "the device"},
           "gpu_launches": launches, "phases_ms": phases, "clocks": clk.summary()}
    return out, clouds


def cpu_batch_baseline(clouds, seconds, threads):
    done, el, th = oracle_parallel_rate(clouds, seconds, threads)
    return {"value": done / el, "unit": "clouds/s", "cores": th, "nproc": host_cores(), "kind": "oracle",
            "sample": f"{done} of {len(clouds)} clouds in {el:.1f} s, one whole oracle build per cloud, "
                      f"{th} host threads across clouds"}


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


SERVE_WORKLOAD = ("Poisson stream of {N} requests, n log-uniform [50,5000], half int8 d=3 torus/sphere, "
                  "half f32 d=16 Gaussian mixtures, maxdim {{1,2}}, per-request cap")


def _gen_requests(n):
    return synth.config5(n)[1]


class RequestsAhead:
    """The serving workload's requests drawn in a spawned process (about a
    millisecond of numpy per request) while the GPU legs run."""

    def __init__(self, n):
        import multiprocessing as mp
        self.pool = mp.get_context("spawn").Pool(1)
        self.res = self.pool.apply_async(_gen_requests, (n,))

    def get(self):
        out = self.res.get()
        self.pool.close()
        self.pool.join()
        return out


def serve_leg(args, ranks, local, reqs_all):
    """Serving: a Poisson stream of mixed requests (n log-uniform in
    [50, 5000]; half int8 d=3 torus/sphere, half float32 d=16 mixtures;
    maxdim in {1, 2}; per-request cap) through the continuous-batching server
    at 0.8x its measured capacity: p50/p99 latency and clouds/s, against the
    per-cloud path (one vr_build per request, FIFO) on the same arrival rate.
    Returns the result dict and this rank's requests."""
    import paper_1809_04424_b300 as vr
    world = ranks.world
    lo, hi = ranks.shard(len(reqs_all))  # this rank's share of the stream
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
        M = min(N, args.sweep_requests)
        a = np.cumsum(synth.rng(1809 + 51).exponential(1.0 / (f * cap), size=M))
        l2, w2 = _open_loop(submit, poll, reqs[:M], a)
        sweep[str(f)] = {"p50_ms": 1e3 * float(np.percentile(l2, 50)), "p99_ms": 1e3 * float(np.percentile(l2, 99)),
                         "clouds_per_s": M / w2, "requests": M}
    srv.close()
    # per-cloud path: one vr_build per request in arrival order, one worker
    M = min(N, 2000)
    import threading
    lock = threading.Lock()

    def per_poll(r):
        with lock:  # a single FIFO worker: plain launches, one cloud at a time
            x = vr.vr_build(r.points, r.maxdim, r.maxrad)
            del x
    t0 = time.perf_counter()
    for r in reqs[:200]:
        per_poll(r)
    per_cap = 200 / (time.perf_counter() - t0)
    a = np.cumsum(synth.rng(1809 + 52).exponential(1.0 / lam, size=M))
    lp, wp = _open_loop(lambda r: r, per_poll, reqs[:M], a, n_pollers=1)
    out = {"metric": "served clouds/s", "value": whole_job_rate(len(reqs_all), wall_all), "unit": "clouds/s",
           "requests": len(reqs_all), "workload": SERVE_WORKLOAD.format(N=len(reqs_all)),
           "arrival_rate_per_s": lam, "capacity_closed_loop": cap,
           "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)), "p99": 1e3 * float(np.percentile(lat, 99)),
                          "mean": 1e3 * float(lat.mean())},
           "rate_sweep": sweep,
           "per_cloud_path": {"capacity_clouds_per_s": per_cap, "requests": M,
                              "arrival_rate_per_s": lam,
                              "p50_ms": 1e3 * float(np.percentile(lp, 50)),
                              "p99_ms": 1e3 * float(np.percentile(lp, 99)), "clouds_per_s": M / wp,
                              "how": "one vr_build per request, one FIFO worker, same arrival rate"},
           "e2e": {"value": N / wall, "unit": "clouds/s",
                   "h2d_bytes_per_step": int(np.mean([r.points.nbytes for r in reqs])),
                   "d2h_bytes_per_step": 2 * CLOUD_DESC_BYTES,
                   "read_back": "per request its descriptor (batched requests, twice) or the status word the "
                                "device writes to mapped host memory (large ones); the complexes stay on the "
                                "device"},
           "clocks": clk.summary()}
    return out, reqs


def cpu_serve_baseline(reqs, seconds, threads):
    done, el, th = oracle_parallel_rate(reqs, seconds, threads)
    return {"value": done / el, "unit": "clouds/s", "cores": th, "nproc": host_cores(), "kind": "oracle",
            "sample": f"the first {done} requests of the stream in arrival order in {el:.1f} s, one whole oracle "
                      f"build per request, {th} host threads across requests"}


def run_batch_bench(args):
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    ranks = Ranks()
    out, clouds = batch_leg(args, ranks, local)
    line = {"metric": out["metric"], "value": out["value"], "unit": "clouds/s", "n_gpus": ranks.world,
            "steps": out["steps"], "warmup": out["warmup"], "ms_per_step": out["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": out["workload"], "simplices_per_step": out["simplices_per_step"],
                                            "l2": out["l2"]}}
    line.update({k: v for k, v in out.items() if k not in line and k not in ("workload",)})
    if rank == 0 and args.cpu_seconds > 0:
        line["cpu_baseline"] = cpu_batch_baseline(clouds, args.cpu_seconds, host_cores())
    if rank == 0:
        print(json.dumps(line), flush=True)
    ranks.close()
    return 0


def run_serve_bench(args):
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    ranks = Ranks()
    reqs_all = synth.config5(args.n_requests)[1]
    out, reqs = serve_leg(args, ranks, local, reqs_all)
    line = {"metric": out["metric"], "value": out["value"], "unit": "clouds/s", "n_gpus": ranks.world,
            "steps": len(reqs_all), "warmup": 64, "ms_per_step": 1e3 / out["value"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "mixed int64/f64", "data": "synthetic",
            "config": {"workload": out["workload"], "arrival_rate_per_s": out["arrival_rate_per_s"],
                       "capacity_closed_loop": out["capacity_closed_loop"]}}
    line.update({k: v for k, v in out.items() if k not in line and k not in ("workload",)})
    if rank == 0 and args.cpu_seconds > 0:
        line["cpu_baseline"] = cpu_serve_baseline(reqs, args.cpu_seconds, host_cores())
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


def gram_accuracy(cloud, pts_dev, step, read_phases, L, flush):
    """The float tensor-core distance tiles against the canonical FP64 values
    (every pair; untimed): max relative error in d over the kept pairs, the
    normalised error and its bound beta, the pairs left to the exact FP64
    decision; for the two-way split (the build's) and the three-way split,
    with the distance phase's time in builds under each."""
    import torch
    import paper_1809_04424_b300 as vr
    out = {"what": "max |d_tc - d_fp64| / d_fp64 over kept pairs; split 2 = hi+lo (3 products, used), "
                   "3 = hi+mid+lo (6 products)"}
    for split in (2, 3):
        a = vr.vr_gram_accuracy_check(pts_dev, cloud.maxrad, split=split)
        vr.vr_set_gram_split(split)
        L.vr_profile_select(None)
        L.vr_profile_reset()
        L.vr_profile_enable(1)
        for _ in range(10):
            flush.zero_()
            c = step()
            del c
        torch.cuda.synchronize()
        L.vr_profile_enable(0)
        ph = read_phases()
        vr.vr_set_gram_split(2)
        out[f"split{split}"] = {"max_rel_d_err": a["max_rel_d_err"], "max_norm_err": a["max_norm_err"],
                                "beta": a["beta"], "kept_pairs": a["kept_pairs"], "band_pairs": a["band_pairs"],
                                "distance_phase_ms": round(ph["distance"]["ms_per_call"], 4) if "distance" in ph
                                else None}
    return out


def single_cloud_leg(args, ranks, local):
    """One vr_build per step of the chosen single-cloud workload; returns the
    contract's line (without the CPU baseline) and the cloud."""
    import ctypes
    import torch
    import paper_1809_04424_b300 as vr
    world, rank = ranks.world, ranks.rank
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
        st = c.stats()
        ngrades = st["ngrades"]
        tri_order = st["tri_order"]
        del c
    torch.cuda.synchronize()
    simplices = sum(counts)

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
    per_launch_bytes = roofline_bytes(cloud, counts[1] if len(counts) > 1 else 0,
                                      counts[2] if len(counts) > 2 else 0,
                                      counts[3] if len(counts) > 3 else 0, ngrades, tri_order)
    # The roofline kernel: the longest single-kernel region that moves bytes
    # of the method's own (a sort's digit passes: several launches of the
    # same kernel, each timed).
    single = {k: v for k, v in phases.items() if k in per_launch_bytes and per_launch_bytes[k][0] > 0
              and (v["launches_per_call"] == 1 or k.endswith(".pass"))}
    dom = max(single, key=lambda k: single[k]["ms_per_call"]) if single else None

    # ---- timed region: K steps, per-step CUDA events, L2 flushed between;
    # inside it the library times only the roofline kernel's region.
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
    ndims = len(counts)
    bufs = []
    for k in range(ndims):
        m = counts[k]
        bufs.append([torch.empty(m * (k + 1), dtype=torch.int32).pin_memory(),
                     torch.empty(m, dtype=torch.int32).pin_memory(),
                     torch.empty(m + 1, dtype=torch.int64).pin_memory() if k else None,
                     torch.empty(m * (k + 1), dtype=torch.int32).pin_memory() if k else None])
    d2h = sum(b.numel() * b.element_size() for bb in bufs for b in bb if b is not None)
    gv = torch.empty(ngrades, dtype=torch.float64).pin_memory()

    def e2e_step():
        c = gpu_build(cloud, host_pts.data_ptr(), n=cloud.n, d=cloud.d, dtype=cloud.dtype_code)
        for k in range(ndims):
            b = bufs[k]
            p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
            rc = L.vr_complex_to_host(ctypes.c_void_p(c.handle), k, p(b[0]), p(b[1]), p(b[2]), p(b[3]))
            assert rc == 0, vr.vr_last_error()
        L.vr_complex_grade_values_to_host(ctypes.c_void_p(c.handle), ctypes.c_void_p(gv.data_ptr()))
        del c

    e2e_val = None
    if not args.no_e2e:
        for _ in range(W):
            e2e_step()
        torch.cuda.synchronize()
        ranks.barrier()
        with NoGC():
            t0 = time.perf_counter()
            for _ in range(args.steps):
                e2e_step()
            torch.cuda.synchronize()
            e2e_s = ranks.max(time.perf_counter() - t0)
        d2h += gv.numel() * 8
        e2e_val = simplices * args.steps * world / e2e_s

    # ---- roofline of the dominant kernel: its region timed by the library's
    # CUDA events on the build stream inside the timed region; and the whole
    # build against the bytes the method must move.
    hbm, src = peaks()
    roof = None
    ms_step = total_ms / args.steps
    build_bytes = method_bytes_per_step(cloud, counts)
    if dom and dom in timed_phases:
        tp = timed_phases[dom]
        per_launch_ms = tp["ms_per_call"] if dom.endswith(".pass") else \
            tp["ms_per_call"] / max(tp["launches_per_call"], 1)
        alg, inter = per_launch_bytes[dom]
        ach = alg / (per_launch_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": recorded_traffic(dom, args.config), "peak_source": src,
                "algorithmic_bytes_per_launch": alg, "intermediate_bytes_per_launch": inter,
                "launch_ms": per_launch_ms, "launches_timed": tp["calls"],
                "build_bytes_per_step": build_bytes,
                "build_achieved": build_bytes / (ms_step / 1e3) / 1e9,
                "build_frac": build_bytes / (ms_step / 1e3) / 1e9 / hbm,
                "note": "achieved counts only the bytes the method must move (outputs, input, edge keys, "
                        "neighbour lists); intermediates are listed apart; of measured HBM copy bandwidth"}

    line = {"metric": METRIC, "value": value, "unit": "simplices/s", "n_gpus": world, "steps": args.steps,
            "warmup": W, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
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
    for k in ("max_rel_dist_err", "near_tie_edges"):
        if k in st:
            line.setdefault("accuracy", {})[k] = st[k]
    if cloud.points.dtype == np.float32 and 16 < cloud.d <= 64 and not isinstance(cloud, synth.Matrix):
        line.setdefault("accuracy", {})["gram"] = gram_accuracy(cloud, pts_dev, step, read_phases, L, flush)
    del flush
    torch.cuda.empty_cache()
    return line, cloud


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="length of each CPU-oracle baseline sample (0 skips them)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--config", default=DEFAULT_CONFIG, choices=sorted(WORKLOADS) + ["batch", "serve"],
                    help="workload (default: the 4000-point float Gaussian-mixture cloud)")
    ap.add_argument("--no-nested", action="store_true",
                    help="skip the batched and served legs nested in the single-cloud line")
    ap.add_argument("--n-clouds", type=int, default=4096, help="clouds of the batch workload")
    ap.add_argument("--batch-steps", type=int, default=10, help="timed batches of the batch workload")
    ap.add_argument("--n-requests", type=int, default=20000, help="requests of the serving workload")
    ap.add_argument("--sweep-requests", type=int, default=4000, help="requests per point of the rate sweep")
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

    nested = not args.no_nested
    ahead = RequestsAhead(args.n_requests) if nested else None  # spawned before any CUDA call

    import torch
    world, rank, local = dist_env()
    assert torch.cuda.is_available(), "bench needs a CUDA device"
    torch.cuda.set_device(local)
    ranks = Ranks()

    line, cloud = single_cloud_leg(args, ranks, local)
    if nested:
        bat, clouds4 = batch_leg(args, ranks, local)
        reqs_all = ahead.get()
        srv, reqs = serve_leg(args, ranks, local, reqs_all)
        line["batched"], line["served"] = bat, srv
    # CPU baselines last, with the GPU legs and the request generator done.
    if rank == 0 and args.cpu_seconds > 0:
        r, reps, el = oracle_rate(cloud, args.cpu_seconds)
        line["cpu_baseline"] = {"value": r, "unit": "simplices/s", "cores": 1, "nproc": host_cores(),
                                "kind": "oracle",
                                "sample": f"{reps} full builds of the workload in {el:.1f} s, single-threaded"}
        if nested:
            line["batched"]["cpu_baseline"] = cpu_batch_baseline(clouds4, args.cpu_seconds, host_cores())
            line["served"]["cpu_baseline"] = cpu_serve_baseline(reqs, args.cpu_seconds, host_cores())
    if rank == 0:
        print(json.dumps(line), flush=True)
    ranks.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
