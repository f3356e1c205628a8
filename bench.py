#!/usr/bin/env python3
"""Benchmark: batched LiDAR ray casting, 4096 environments x 1M triangles.

Workload (one "step" = one simulation step of every environment): the
1,000,300-triangle indoor mesh, 4,096 environments each at its own pose of a
seeded SE(3) random walk, 16 x 360 rays per environment = 23,592,960 rays per
step, max range 120 m.  A step copies that step's poses into the
device-resident pose state and replays one CUDA graph (work-queue table copy +
one persistent kernel).  L2 is flushed (256 MiB write) between timed steps.

Printed JSON line (rank 0):
  value            Grays/s of the batched persistent kernel, inputs in HBM
  e2e              same metric through fgl_cast_batched_host with pinned host
                   buffers (poses H2D and ranges+ids D2H inside the timed region)
  per_env_launch   the plain form: one fgl_cast launch per environment
  roofline         the dominant kernel's bound, instruction issue: executed warp
                   instructions per ray (ncu capture of the same sources) x
                   rays / kernel time against 4 warp schedulers x SMs x the
                   sampled SM clock; beside it the cost model of eq. cost(r_j)
                   as bytes against the measured HBM copy bandwidth (node and
                   triangle bytes are served by L1/L2, so it can exceed 1), the
                   measured DRAM and L2 rates, and `limiter`
  cpu_baseline     the FP64 oracle on the host cores over a bounded sample

--impl reference times the FP64 CPU oracle (the only reference this method
has) on the same workload and metric.  With --gpus N under torchrun every
rank runs its own replica (the path needs no exchange between GPUs).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Grays/s @4096 envs x 1M tris; p50/p99 scan latency, served vs per-env launch"
UNIT = "Grays/s"
WORKLOAD = ("batched_walk: 4096 envs x (16 beams -15..+15 deg x 360 az) = 23,592,960 rays/step "
            "on the 1,000,300-tri seeded indoor mesh (20x15x4 m room, 2000 icospheres, 834 "
            "boxes), per-env seeded SE(3) random walk 0.1 m / 2 deg per step, max range 120 m")
# the sources each profiled kernel is built from: a committed ncu figure is
# used only while its kernel's sources are unchanged
KERNEL_SOURCES = {
    # the wide kernel's work per ray also depends on the tree its builder makes
    "k_persistent": ["paper_2509_17390_gb300/csrc/trace.cuh", "paper_2509_17390_gb300/csrc/kernels.cu",
                     "paper_2509_17390_gb300/csrc/bvh_build.cpp"],
    "k_lbvh_cast": ["paper_2509_17390_gb300/csrc/trace.cuh", "paper_2509_17390_gb300/csrc/lbvh.cu"],
}


def kernel_hash(name: str = "k_persistent") -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES[name]:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    return h.hexdigest()[:16]


def read_peaks():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def read_profile(name: str, field: str, entry: str = None):
    """A per-launch figure from the committed ncu summary (profiles/traffic.json),
    if it was taken on the current kernel sources.  `entry` names a workload's
    own capture of kernel `name` (default: the kernel's entry itself)."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        e = d.get(entry or name)
        if e and e.get("kernel_hash") == kernel_hash(name) and e.get(field) is not None:
            return float(e[field])
    except Exception:
        pass
    return None


def issue_roofline(kernel, entry, rays_per_s, clocks, dev, extra=None):
    """The ray-casting kernels' bound: instruction issue.  Executed warp
    instructions per ray (ncu smsp__inst_executed.sum of a committed capture
    on the current sources) x rays/s, against the issue rate of the unit
    counts and the clock: 4 warp schedulers per SM, one instruction each per
    cycle, x SMs x the median SM clock sampled in the timed region.  None
    when no capture matches the sources."""
    import torch
    ipr = read_profile(kernel, "warp_inst_per_ray", entry)
    if ipr is None:
        return None
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = 4.0 * sms * mhz * 1e6 / 1e9
    ach = ipr * rays_per_s / 1e9
    out = {"bound": "alu", "kernel": kernel, "achieved": round(ach, 1), "peak": round(peak, 1),
           "unit": "G warp-inst/s", "frac": round(ach / peak, 4),
           "traffic": read_profile(kernel, "dram_bytes_per_launch", entry),
           "warp_inst_per_ray": ipr, "peak_source": "derived",
           "peak_basis": f"4 warp schedulers x {sms} SMs x {mhz:.0f} MHz (median SM clock of the timed region)",
           "basis": "instruction issue: executed warp instructions per ray (ncu, same kernel sources) "
                    "x rays / kernel time; the kernel's nodes and triangles come from L1/L2, and "
                    "its issue slots, not HBM, bound it"}
    if extra:
        out.update(extra)
    return out


def read_traffic(name: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources."""
    return read_profile(name, "dram_bytes_per_launch")


def _nvtx(push: bool):
    try:
        import torch
        if push:
            torch.cuda.nvtx.range_push("bench_timed")
        else:
            torch.cuda.nvtx.range_pop()
    except Exception:
        pass


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region: the sampler
    is started and seen writing before the region opens (nvidia-smi takes a
    while to start), samples every 50 ms with nvidia-smi's own timestamp, and
    the summary keeps the samples taken between entering and leaving the
    region (all of them, flagged, if the region was shorter than a sample).
    The region is also an NVTX range named "bench_timed", so that a profiler
    can take its launches alone (ncu --nvtx --nvtx-include bench_timed/)."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    TS = "%Y/%m/%d %H:%M:%S.%f"

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def __enter__(self):
        import datetime
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            deadline = time.time() + 5.0
            while time.time() < deadline and self.proc.poll() is None and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
        except Exception:
            self.proc = None
        self.t0 = datetime.datetime.now()
        _nvtx(True)
        return self

    def __exit__(self, *a):
        import datetime
        _nvtx(False)
        self.t1 = datetime.datetime.now()
        if self.proc:
            time.sleep(0.06)                       # the sample in flight at the end
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        import datetime
        if not self.path or not os.path.exists(self.path):
            return None
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], self.TS)
                rows.append((ts, float(f[2]), float(f[3]), [n for n, v in zip(names, f[6:10])
                                                            if v.lower() == "active"]))
            except ValueError:
                continue
        os.unlink(self.path)
        inside = [r for r in rows if self.t0 and self.t1 and self.t0 <= r[0] <= self.t1]
        use = inside or rows
        if not use:
            return None
        return {"sm_mhz": float(np.median([r[1] for r in use])), "sm_max_mhz": max(r[2] for r in use),
                "reasons": sorted({n for r in use for n in r[3]}), "samples": len(use),
                "samples_in_timed_region": len(inside), "interval_ms": 50}


def dist_setup(n_gpus: int):
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return ws, rank, local


def barrier_max(x: float, ws: int) -> float:
    """Maximum of x over the ranks (the slowest rank's time)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, seconds: float, ws: int) -> float:
    """Whole-job throughput of identical replicas: every rank's units over
    the slowest rank's time."""
    return ws * units_per_rank / barrier_max(seconds, ws)


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(w, step_poses, n_env_sample: int, seed: int = 0, osc=None):
    import oracle
    if osc is None:
        osc = oracle.Scene(w.verts, w.tris, bvh=True)
    rng = np.random.default_rng(seed)
    envs = np.sort(rng.choice(step_poses.shape[0], n_env_sample, replace=False))
    dirs = oracle.sensor_dirs(w.sensor.elev, w.sensor.azim)
    o, d = oracle.world_rays(dirs, step_poses[envs])
    return osc, o, d, envs


def counted_bytes(fgl, items, stream, opts=None):
    """Algorithmic bytes of casting `items` once (eq. cost(r_j) as bytes): a
    counting pass per item (node visits x its scene's node size + triangle
    tests x 48 B + 24 B of direction and result per ray).  Returns (bytes,
    rays, node visits, triangle tests)."""
    tot_b = tot_r = tot_n = tot_t = 0
    for it in items:
        sc, se = it[0], it[1]
        copts = fgl.BatchOpts(count_work=1, packet_rays=opts.packet_rays if opts else 0,
                              block_threads=opts.block_threads if opts else 0)
        fgl.work_counters()
        fgl.cast_batched([it], copts, stream=stream)
        fgl.sync(stream)
        r, n, t = fgl.work_counters()
        tot_b += n * sc.stats()["node_stride"] + t * 48 + r * 24
        tot_r, tot_n, tot_t = tot_r + r, tot_n + n, tot_t + t
    return tot_b, tot_r, tot_n, tot_t


def hbm_roofline(bytes_, seconds, rays, nodes, tris, kernel="k_persistent"):
    peak, kind = read_peaks()
    achieved = bytes_ / seconds / 1e9
    return {"bound": "hbm", "kernel": kernel, "achieved": round(achieved, 1), "peak": peak,
            "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None, "peak_source": kind,
            "bytes_per_ray": round(bytes_ / max(1, rays), 1),
            "node_visits_per_ray": round(nodes / max(1, rays), 2),
            "tri_tests_per_ray": round(tris / max(1, rays), 2),
            "basis": "algorithmic bytes of eq. cost(r_j) from a counting pass"}


def l2_read_peak(dev, mib: int = 32, reps: int = 20):
    """L2 read bandwidth measured here: the library's probe reads a {mib} MiB
    device buffer (resident in the 129 MB L2 after a warm-up pass) `reps`
    times with 16-byte L1-bypassing loads on 4 x 512 threads per SM, timed
    with CUDA events; best of 5."""
    import torch
    import paper_2509_17390_gb300 as fgl
    a = torch.ones(mib << 18, dtype=torch.float32, device=dev)
    sink = torch.zeros(1, dtype=torch.int32, device=dev)
    fgl.probe_l2_read(a, 2, sink)
    best = None
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fgl.probe_l2_read(a, reps, sink)
        e1.record()
        e1.synchronize()
        gbs = (mib << 20) * reps / (e0.elapsed_time(e1) / 1e3) / 1e9
        best = gbs if best is None else max(best, gbs)
    del a
    return {"gbs": round(best, 1), "basis": f"fgl_probe_l2_read: {mib} MiB resident buffer read {reps} "
                                            f"times with 16-byte L2 loads, best of 5 (read bytes)"}


def time_oracle(osc, o, d, max_range, nthreads: int = 0):
    t0 = time.perf_counter()
    osc.cast(o, d, max_range, flags=False, nthreads=nthreads)
    return time.perf_counter() - t0


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine)."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


# ---------------------------------------------------------------------------
# serving: trace replay
# ---------------------------------------------------------------------------
class OutputArena:
    """Page-locked result space reused in arrival order: a request takes the
    next slice; when the arena wraps onto slices still in use, the replayer
    first waits for those requests (back-pressure, counted in latency)."""

    def __init__(self, nbytes: int):
        import torch
        self.buf = torch.empty(nbytes // 4, dtype=torch.int32).pin_memory()
        self.n = self.buf.numel()
        self.head = 0

    def take(self, n_vals: int):
        if n_vals * 2 > self.n:
            raise ValueError("request larger than the output arena")
        if self.head + 2 * n_vals > self.n:
            self.head = 0
        a = self.head
        self.head += 2 * n_vals
        r = self.buf[a:a + n_vals].view(dtype=__import__("torch").float32)
        i = self.buf[a + n_vals:a + 2 * n_vals]
        return (a, a + 2 * n_vals), r, i


def make_trace(rng, rate: float, window_s: float, max_env: int, pose_pool, n_scenes: int,
               sensor_pick, n_req_cap: int = 10 ** 9):
    """Poisson arrivals (rate per second) over a window; n_env log-uniform on
    [1, max_env]; poses drawn from pose_pool[scene] ([m, 3, 4])."""
    t, out = 0.0, []
    while len(out) < n_req_cap:
        t += rng.exponential(1.0 / rate)
        if t > window_s:
            break
        sc = int(rng.integers(n_scenes))
        n_env = int(np.exp(rng.uniform(0.0, np.log(max_env))))
        pool = pose_pool[sc]
        P = pool[rng.integers(len(pool), size=n_env)]
        out.append((t, sc, sensor_pick(rng, sc), np.ascontiguousarray(P, np.float32)))
    return out


def scale_to_load(trace, window_s: float, n_rays_of, rays_per_s: float):
    """The trace (arrival, scene, sensor, poses, ...) with its arrival times
    stretched so that it offers rays_per_s over its stretched window:
    (scaled trace, new window in s)."""
    offered = sum(e[3].shape[0] * n_rays_of[e[2]] for e in trace) / window_s
    f = offered / rays_per_s
    return [(e[0] * f,) + tuple(e[1:]) for e in trace], window_s * f


class SlotPlan:
    """Device-resident pose state for a trace: each scene owns a ring of
    `per_scene` server environment slots, and each request takes the next
    n_env slots of its scene's ring and overwrites them first with n_env
    consecutive poses of a device-resident pose source (standing in for a
    simulator that keeps its state on the GPU): no pose byte crosses to or
    from the host."""

    def __init__(self, server, sources, per_scene: int, seed: int = 0):
        import torch
        self.sources = sources                      # scene -> CUDA tensor [m, 3, 4]
        self.per = per_scene
        self.first = []
        for sc in range(len(sources)):
            src = sources[sc]
            reps = -(-per_scene // src.shape[0])
            init = src.cpu().numpy()
            init = np.ascontiguousarray(np.concatenate([init] * reps)[:per_scene], np.float32)
            self.first.append(server.add_envs(init))
        self.rng = np.random.default_rng(seed)
        self.next = [0] * len(sources)
        self.torch = torch

    def take(self, sc: int, n_env: int):
        """(env_first, device pose view) of the next request on scene sc."""
        n_env = min(n_env, self.per)
        a = self.next[sc]
        if a + n_env > self.per:
            a = 0
        self.next[sc] = a + n_env
        src = self.sources[sc]
        if n_env > src.shape[0]:
            raise ValueError("a request needs more environments than its pose source holds")
        off = int(self.rng.integers(0, src.shape[0] - n_env + 1))
        return self.first[sc] + a, src[off:off + n_env]


def slot_trace(trace, plan: SlotPlan):
    """The same arrivals, scenes, sensors and sizes with the poses replaced by
    slot ranges that the request overwrites from device memory."""
    out = []
    for (ta, sc, se, P) in trace:
        first, view = plan.take(sc, P.shape[0])
        out.append((ta, sc, se, None, (first, view)))
    return out


def replay(server, trace, scene_ids, sensor_ids, n_rays_of, arena, max_range, timeout_s=600):
    """Submit each request at its arrival time; latency = arrival -> results
    in host memory.  A trace entry is (arrival, scene, sensor, host poses)
    or (arrival, scene, sensor, None, (env_first, device pose view)) for a
    request on resident slots.  Returns stats."""
    live = []     # (ticket, submission delay behind the arrival time in ms, slice)
    lat, rays = [], 0
    t0 = time.perf_counter()

    def retire(k):
        tk, delay_ms, _ = live.pop(k)
        info = server.wait(tk, int(timeout_s * 1000))
        lat.append(info["latency_ms"] + delay_ms)    # arrival -> results in host memory

    for entry in trace:
        ta, sc, se, P = entry[:4]
        slot = entry[4] if len(entry) > 4 else None
        n_env = P.shape[0] if P is not None else slot[1].shape[0]
        n = n_env * n_rays_of[se]
        now = time.perf_counter() - t0
        if now < ta:
            time.sleep(ta - now)
        sl, r, i = arena.take(n)
        while live and any(not (sl[1] <= a or b <= sl[0]) for _, _, (a, b) in live):
            retire(0)
        delay_ms = max(0.0, (time.perf_counter() - t0 - ta) * 1e3)
        if slot is None:
            tk = server.submit(scene_ids[sc], sensor_ids[se], P, max_range, r, i)
        else:
            tk = server.submit(scene_ids[sc], sensor_ids[se], slot[1], max_range, r, i,
                               env_first=slot[0])
        live.append((tk, delay_ms, sl))
        rays += n
    while live:
        retire(0)
    busy = time.perf_counter() - t0
    lat = np.asarray(lat)
    return {"requests": len(trace), "rays": rays, "wall_s": round(busy, 3),
            "rays_per_s": rays / busy, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean())}


def replay_runs(server, trace, scene_ids, sensor_ids, n_rays_of, arena, max_range, runs: int = 3):
    """The same trace replayed `runs` times on one server: per-run figures,
    and p50 / p99 / rays/s as the median over runs with their spread
    (largest / smallest)."""
    res = [replay(server, trace, scene_ids, sensor_ids, n_rays_of, arena, max_range)
           for _ in range(runs)]
    med = lambda k: float(np.median([r[k] for r in res]))
    spread = lambda k: round(max(r[k] for r in res) / max(1e-9, min(r[k] for r in res)), 2)
    return {"requests": res[0]["requests"], "runs": runs,
            "p50_ms": med("p50_ms"), "p99_ms": med("p99_ms"), "rays_per_s": med("rays_per_s"),
            "p50_spread": spread("p50_ms"), "p99_spread": spread("p99_ms"),
            "per_run": [{"p50_ms": round(r["p50_ms"], 2), "p99_ms": round(r["p99_ms"], 2),
                         "Grays_s": round(r["rays_per_s"] / 1e9, 4)} for r in res]}


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-env", type=int, default=4096)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-per-env", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--packet", type=int, default=0)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--sdepth", type=int, default=0)
    ap.add_argument("--refill", type=int, default=0)
    ap.add_argument("--postpone", type=int, default=0)
    ap.add_argument("--width", type=int, default=8)
    ap.add_argument("--tri", type=int, default=0)
    ap.add_argument("--tile", type=str, default="")
    ap.add_argument("--workload", default="walk",
                    choices=["walk", "hetero", "serve", "occupancy", "walk_instances", "lbvh", "mesh"])
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-poses", default="slots", choices=["slots", "request"],
                    help="served walk: poses in device-resident slots (default) or carried by each request")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    from synth import workloads

    n_steps = args.warmup + args.steps
    if args.impl == "reference":
        return run_reference(args, n_steps)
    if args.workload == "hetero":
        return run_hetero(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "occupancy":
        return run_occupancy(args)
    if args.workload == "walk_instances":
        return run_walk_instances(args)
    if args.workload == "lbvh":
        return run_lbvh(args)
    if args.workload == "mesh":
        return run_mesh(args)

    import torch
    import paper_2509_17390_gb300 as fgl

    ws, rank, local = dist_setup(args.gpus)
    w = workloads.batched_walk(2, n_env=args.n_env, n_steps=min(n_steps, 100))
    n_env = args.n_env
    walk = w.poses                                    # [S, n_env, 3, 4]
    S = walk.shape[0]
    scene = fgl.Scene(w.verts, w.tris, width=args.width)
    tr, tc = (int(x) for x in args.tile.split("x")) if args.tile else (0, 0)
    sensor = fgl.Sensor.from_table(w.sensor, tr, tc)
    n_rays = n_env * sensor.n_rays
    dev = torch.device("cuda", torch.cuda.current_device())
    walk_d = torch.from_numpy(walk).to(dev)          # all steps' poses resident
    pose_state = torch.empty((n_env, 3, 4), dtype=torch.float32, device=dev)
    out_r = torch.empty(n_rays, dtype=torch.float32, device=dev)
    out_i = torch.empty(n_rays, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    opts = fgl.BatchOpts(packet_rays=args.packet, block_threads=args.block, stack_smem=args.sdepth,
                         refill_min=args.refill, postpone_pct=args.postpone, use_graph=1,
                         tri_mode=args.tri)
    items = [(scene, sensor, pose_state, w.max_range, out_r, out_i)]
    arr = fgl.make_items(items)

    def step(s):
        with torch.cuda.stream(stream):
            pose_state.copy_(walk_d[s % S])
        fgl.cast_batched(items, opts, stream=stream, arr=arr)

    # warm-up (graph capture happens on the first call)
    for s in range(args.warmup):
        step(s)
    fgl.sync(stream)

    # work counters for the roofline (one step, outside the timed region)
    copts = fgl.BatchOpts(packet_rays=args.packet, block_threads=args.block, stack_smem=args.sdepth,
                          refill_min=args.refill, postpone_pct=args.postpone, count_work=1,
                          tri_mode=args.tri)
    fgl.work_phase_counters()
    with torch.cuda.stream(stream):
        pose_state.copy_(walk_d[args.warmup % S])
    fgl.cast_batched(items, copts, stream=stream)
    fgl.sync(stream)
    phases = fgl.work_phase_counters()
    c_rays, c_nodes, c_tris = phases["rays"], phases["node_visits"], phases["tri_tests"]
    st = scene.stats()
    # eq. cost(r_j) as bytes: S_io = 8 B of output per ray (pose and direction
    # reads are broadcast across the rays of an environment and not counted)
    b_ray = (c_nodes * st["node_stride"] + c_tris * 48) / max(1, c_rays) + 8

    # timed region: per step flush L2 (untimed), then events around the step
    barrier(ws)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
                ev[k][0].record(stream)
            step(args.warmup + k)
            with torch.cuda.stream(stream):
                ev[k][1].record(stream)
        torch.cuda.synchronize()
    fgl.sync(stream)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = barrier_max(sum(step_ms) / 1e3, ws)
    ms = total_s * 1e3 / args.steps
    value = aggregate_rate(n_rays * args.steps, sum(step_ms) / 1e3, ws) / 1e9
    clocks = clk.summary()

    # kernel-only time for the roofline: graph = 1 tiny memcpy + 1 kernel
    kern_ms = float(np.mean(step_ms))
    peak, peak_kind = read_peaks()
    achieved = b_ray * n_rays / (kern_ms / 1e3) / 1e9
    # eq. cost(r_j) as bytes against HBM (the cost model's figure; above 1
    # because the node and triangle bytes are served by L1/L2, not HBM)
    cost_model = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                  "frac": round(achieved / peak, 4), "peak_source": peak_kind,
                  "bytes_per_ray": round(b_ray, 1),
                  "basis": "node visits x node size + triangle tests x 48 B + 8 B of output per "
                           "ray (counted in a pass outside the timing), as if each came from HBM",
                  "node_visits_per_ray": round(c_nodes / max(1, c_rays), 2),
                  "tri_tests_per_ray": round(c_tris / max(1, c_rays), 2),
                  "phases_per_ray": {k: round(v / max(1, c_rays), 4) for k, v in phases.items() if k != "rays"}}
    # measured traffic beside the cost model: DRAM bytes of one full launch and
    # L2 (lts__t_bytes) bytes per ray from the committed ncu captures, as rates;
    # the L2 rate against an L2 copy bandwidth measured here
    traffic = read_traffic("k_persistent")
    measured = {"dram_bytes_per_launch": traffic}
    if traffic is not None:
        measured["dram_gbs"] = round(traffic / (kern_ms / 1e3) / 1e9, 1)
        measured["dram_frac"] = round(traffic / (kern_ms / 1e3) / 1e9 / peak, 4)
    lpr = read_profile("k_persistent", "lts_bytes_per_ray")
    l2pk = l2_read_peak(dev)
    l2 = {"achieved": None, "peak": l2pk["gbs"], "unit": "GB/s", "peak_basis": l2pk["basis"]}
    if lpr is not None:
        l2a = lpr * n_rays / (kern_ms / 1e3) / 1e9
        l2.update({"achieved": round(l2a, 1), "frac": round(l2a / l2pk["gbs"], 4), "bytes_per_ray": lpr})
    # the bound: instruction issue (executed warp instructions per ray from the
    # committed capture of these sources); without a matching capture the
    # line falls back to the cost model
    rps = n_rays / (kern_ms / 1e3)
    roofline = issue_roofline("k_persistent", None, rps, clocks, dev,
                              {"cost_model": cost_model, "dram": measured, "l2": l2})
    if roofline is None:
        roofline = dict(cost_model, traffic=traffic, dram=measured, l2=l2,
                        note="no ncu capture of the current kernel sources: the issue bound is unmeasured")
    fr = {"issue": roofline["frac"] if roofline["bound"] == "alu" else None,
          "l2": l2.get("frac"), "dram": measured.get("dram_frac")}
    fr = {k: v for k, v in fr.items() if v is not None}
    roofline["limiter"] = {"kind": max(fr, key=fr.get) if fr else "unknown",
                           "fractions": {**fr, "hbm_cost_model": cost_model["frac"]}}

    # the optional sensor effects (dropout 5%, range noise 1 cm + 0.1%) on one
    # step's returns, timed alone: an HBM-bound pass, 8 B read + 8 B written a
    # return (the noise and the dropout decisions are drawn per hit)
    ev_fx = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    fx_ms = []
    for k in range(4):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)
            ev_fx[0].record(stream)
        fgl.apply_sensor_effects(out_r, out_i, n_env, seed=7, step=k, drop_prob=0.05, sigma0=0.01,
                                 sigma1=0.001, max_range=w.max_range, stream=stream)
        with torch.cuda.stream(stream):
            ev_fx[1].record(stream)
        ev_fx[1].synchronize()
        if k:
            fx_ms.append(ev_fx[0].elapsed_time(ev_fx[1]))
    fx_s = float(np.mean(fx_ms)) / 1e3
    effects = {"kernel": "k_effects", "ms": round(fx_s * 1e3, 4), "bound": "hbm",
               "achieved": round(16 * n_rays / fx_s / 1e9, 1), "peak": peak, "unit": "GB/s",
               "frac": round(16 * n_rays / fx_s / 1e9 / peak, 4),
               "basis": "at most 8 B read + 8 B written per return (misses: 4 B read), L2 flushed before each pass"}

    # per-env launch (plain form): one fgl_cast per environment
    per_env = None
    if not args.no_per_env:
        L = fgl.lib()
        sh = stream.cuda_stream
        base_p = pose_state.data_ptr()
        base_r, base_i = out_r.data_ptr(), out_i.data_ptr()
        nr = sensor.n_rays
        reps = 2
        torch.cuda.synchronize()
        tot = 0.0
        for k in range(reps):
            with torch.cuda.stream(stream):
                pose_state.copy_(walk_d[(args.warmup + k) % S])
                flush.fill_(k & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for e in range(n_env):
                st_ = L.fgl_cast(scene.handle, sensor.handle, base_p + 48 * e, 1, w.max_range,
                                 base_r + 4 * nr * e, base_i + 4 * nr * e, sh)
                if st_:
                    raise RuntimeError(L.fgl_last_error())
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        fgl.sync(stream)
        pms = tot / reps
        per_env = {"value": round(n_rays / (pms / 1e3) / 1e9, 4), "unit": UNIT,
                   "ms_per_step": round(pms, 3), "launches_per_step": n_env}

    # end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        hp = torch.empty((n_env, 3, 4), dtype=torch.float32).pin_memory()
        hr = torch.empty(n_rays, dtype=torch.float32).pin_memory()
        hi = torch.empty(n_rays, dtype=torch.int32).pin_memory()
        hitems = [(scene, sensor, hp, w.max_range, hr, hi)]
        for s in range(2):
            hp.copy_(torch.from_numpy(walk[s % S]))
            fgl.cast_batched_host(hitems, opts, stream=stream)
        ksteps = max(3, min(args.steps, 10))
        tot = 0.0
        for k in range(ksteps):
            hp.copy_(torch.from_numpy(walk[(args.warmup + k) % S]))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fgl.cast_batched_host(hitems, opts, stream=stream)
            tot += time.perf_counter() - t0
        tot = barrier_max(tot, ws)
        e2e = {"value": round(ws * n_rays * ksteps / tot / 1e9, 4), "unit": UNIT,
               "h2d_bytes_per_step": n_env * 48, "d2h_bytes_per_step": n_rays * 8,
               "ms_per_step": round(tot * 1e3 / ksteps, 3)}

    # served: continuous batching vs one launch per env on Poisson traces
    served = None
    if not args.no_serve:
        served = served_walk(fgl, scene, sensor, walk, walk_d, w.max_range, value, rank,
                             slots=args.serve_poses == "slots")

    # CPU oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        osc, o, d, envs = oracle_sample(w, walk[args.warmup % S], 1024)
        t = time_oracle(osc, o, d, w.max_range)
        n1 = len(o) // 16                                   # one core on a sixteenth of the sample
        t1 = time_oracle(osc, o[:n1], d[:n1], w.max_range, nthreads=1)
        cpu = {"value": round(len(o) / t / 1e9, 6), "unit": UNIT, "cores": os.cpu_count(),
               "kind": "oracle", "cpu_model": cpu_model(),
               "single_core_value": round(n1 / t1 / 1e9, 7),
               "sample": f"{len(envs)} of {n_env} envs x {sensor.n_rays} rays (one step), FP64 "
                         f"median-split BVH, no ambiguity flags, {t:.1f} s on all cores; "
                         f"{n1} rays on one core, {t1:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
            "ms_per_step_median": round(float(np.median(step_ms)), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "parallelism": f"replicas x{ws}", "l2": "flushed "
                       "between timed steps (256 MiB write)", "bvh_width": st["width"],
                       "opts": opts.as_dict(), "scene_tris": st["n_tris"],
                       "rays_per_step": n_rays, "frames_per_s": round(ws * n_env / (ms / 1e3), 1)},
            "gpu_launches": args.steps, "roofline": roofline,
            "sensor_effects": effects, "e2e": e2e,
            "per_env_launch": per_env, "served": served, "cpu_baseline": cpu, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def served_walk(fgl, scene, sensor, walk, walk_d, max_range, grays, rank, slots=True):
    """Poisson requests of 1-4096 walk environments (log-uniform) through
    the continuous-batching server, the environments' poses kept on the
    device (each request overwrites its slots from the device-resident walk,
    then scans them): first at twice the kernel's batched capacity for 1 s,
    which saturates the server and measures its sustained rate, then at 70%
    of that sustained rate for 2 s, replayed three times; the first requests
    of the same trace also through the server that issues one launch per
    environment, and again through the batched server."""
    rng = np.random.default_rng(11 + rank)
    pool = {0: walk.reshape(-1, 3, 4)}
    mean_env = (4096 - 1) / np.log(4096)
    # result space and environment slots sized so that neither wraps onto a
    # request still in flight within about 300 ms at this load (a wrap makes
    # the replayer or the server wait, which would add to the measured tail)
    arena = OutputArena(8 << 30)
    srv = fgl.Server(tick_rays=16 << 20, env_capacity=262144)
    sid, tid = srv.add_scene(scene), srv.add_sensor(sensor)
    plan = SlotPlan(srv, [walk_d.reshape(-1, 3, 4)], 262144, seed=12 + rank)
    conv = (lambda tr: slot_trace(tr, plan)) if slots else (lambda tr: tr)
    sat_rate = 2.0 * grays * 1e9 / (mean_env * sensor.n_rays)
    sat_trace = conv(make_trace(rng, sat_rate, 1.0, 4096, pool, 1, lambda r, sc: 0))
    sat = replay(srv, sat_trace, [sid], [tid], [sensor.n_rays], arena, max_range)
    n_env_of = lambda tr: tr[3].shape[0] if tr[3] is not None else tr[4][1].shape[0]
    mean_rays = float(np.mean([n_env_of(tr) * sensor.n_rays for tr in sat_trace]))
    rate = 0.7 * sat["rays_per_s"] / mean_rays
    trace = conv(make_trace(rng, rate, 2.0, 4096, pool, 1, lambda r, sc: 0))
    out = {"load": "Poisson, 70% of the server's sustained rate (measured at twice the kernel's "
                   "capacity over 1 s), 2 s window; n_env log-uniform 1-4096",
           "poses": "device-resident environment slots (262,144), each request overwrites its "
                    "slots from the device-resident walk: 0 pose bytes host->device" if slots else
                    "carried by each request from host memory (n_env x 48 B host->device)",
           "saturated": {"requests": sat["requests"], "Grays_s": round(sat["rays_per_s"] / 1e9, 4)},
           "rate_req_per_s": round(rate, 1)}
    strace = trace
    res = replay_runs(srv, strace, [sid], [tid], [sensor.n_rays], arena, max_range)
    out.update({"requests": res["requests"], "p50_ms": round(res["p50_ms"], 2),
                "p99_ms": round(res["p99_ms"], 2), "value": round(res["rays_per_s"] / 1e9, 4),
                "unit": "Grays/s", "runs": res["runs"], "p50_spread": res["p50_spread"],
                "p99_spread": res["p99_spread"], "per_run": res["per_run"]})
    # the same trace prefix through both servers (the plain server falls behind)
    pre, acc = [], 0
    for tr in strace:
        acc += n_env_of(tr) * sensor.n_rays
        pre.append(tr)
        if acc > 2.5e8:
            break
    resb = replay(srv, pre, [sid], [tid], [sensor.n_rays], arena, max_range)
    srv.close()
    srvp = fgl.Server(mode=1, env_capacity=262144)
    sid, tid = srvp.add_scene(scene), srvp.add_sensor(sensor)
    SlotPlan(srvp, [walk_d.reshape(-1, 3, 4)], 262144)     # same slot ids
    resp = replay(srvp, pre, [sid], [tid], [sensor.n_rays], arena, max_range)
    srvp.close()
    f = lambda r: {"p50_ms": round(r["p50_ms"], 2), "p99_ms": round(r["p99_ms"], 2),
                   "Grays_s": round(r["rays_per_s"] / 1e9, 4)}
    out["same_prefix"] = {"requests": len(pre), "batched": f(resb), "per_env_launch": f(resp)}
    return out


def hetero_setup(fgl, seed=4, n_env=256, ladder=None):
    """Meshes, scenes (width picked per mesh by timing), sensors and the
    batched items of the heterogeneous workload."""
    import torch
    from synth import workloads
    t0 = time.perf_counter()
    meshes = workloads.hetero_meshes(gpu_mesher, seed, ladder)
    t_mesh = time.perf_counter() - t0
    tables = workloads.hetero_sensors(seed)
    envs = workloads.hetero_envs(seed, meshes, n_env)
    groups = {}
    for m, sidx, P in envs:
        groups.setdefault((m, sidx), []).append(P)
    keys = sorted(groups)
    sensors = {k: fgl.Sensor.from_table(tables[k]) for k in sorted({s for _, s in keys})}
    t0 = time.perf_counter()
    scenes = {m: {W: fgl.Scene(spec.verts, spec.tris, width=W) for W in (8, 4)}
              for m, spec in enumerate(meshes)}
    t_build = time.perf_counter() - t0
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)
    poses = {k: torch.from_numpy(np.stack(groups[k])).to(dev) for k in keys}
    outs = {k: (torch.empty(poses[k].shape[0] * sensors[k[1]].n_rays, dtype=torch.float32, device=dev),
                torch.empty(poses[k].shape[0] * sensors[k[1]].n_rays, dtype=torch.int32, device=dev))
            for k in keys}

    def items_for(widths, only_mesh=None):
        return [(scenes[k[0]][widths[k[0]]], sensors[k[1]], poses[k], 30.0, outs[k][0], outs[k][1])
                for k in keys if only_mesh is None or k[0] == only_mesh]

    widths = {}
    for m in range(len(meshes)):            # BVH width per mesh, by timing its own items
        best = None
        for W in (8, 4):
            its = items_for({mm: W for mm in range(len(meshes))}, only_mesh=m)
            if not its:
                continue
            _, res = fgl.autotune(its, fgl.BatchOpts(use_graph=1), reps=2, passes=1, stream=stream)
            if best is None or res["best_ms"] < best[1]:
                best = (W, res["best_ms"])
        widths[m] = best[0] if best else 8
    # mixed widths cost one launch (and one drain) per width: keep the mix only
    # if it beats a single width over the whole batch
    def batch_ms(ws_, reps=3):
        its = items_for(ws_)
        arr_ = fgl.make_items(its)
        o = fgl.BatchOpts(use_graph=1)
        for _ in range(2):
            fgl.cast_batched(its, o, stream=stream, arr=arr_)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fgl.cast_batched(its, o, stream=stream, arr=arr_)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps
    if len(set(widths.values())) > 1:
        cands = {"mixed": dict(widths), "all 8": {m: 8 for m in widths}, "all 4": {m: 4 for m in widths}}
        timed = {k: batch_ms(v) for k, v in cands.items()}
        widths = cands[min(timed, key=timed.get)]
        width_choice = {k: round(v, 3) for k, v in timed.items()}
    else:
        width_choice = None
    items = items_for(widths)
    opts, tune = fgl.autotune(items, fgl.BatchOpts(use_graph=1), reps=3, passes=2, stream=stream)
    info = {"meshes": [{"tris": int(len(sp.tris)), "gaussians": sp.n_gauss, "voxel_m": sp.voxel,
                        "width": widths[m]} for m, sp in enumerate(meshes)],
            "mesher_s": round(t_mesh, 2), "bvh_build_s": round(t_build, 1),
            "width_choice_ms": width_choice,
            "autotune": {"opts": opts.as_dict(), "best_ms": round(tune["best_ms"], 3),
                         "start_ms": round(tune["start_ms"], 3), "trials": tune["trials"]}}
    return meshes, tables, envs, groups, scenes, sensors, widths, items, opts, stream, info


def run_walk_instances(args):
    """The batched walk with four rigid instances per environment (an
    icosphere, two boxes and a pillar), each moving on its own seeded walk:
    every step casts the static mesh and the moved instances, with the
    world-frame return points."""
    import torch
    import paper_2509_17390_gb300 as fgl
    from synth import workloads
    ws, rank, local = dist_setup(args.gpus)
    n_steps = args.warmup + args.steps
    wi = workloads.walk_instances(2, args.n_env, min(n_steps, 100))
    w, meshes, IP = wi.walk, wi.meshes, wi.poses
    n_env, S = args.n_env, w.poses.shape[0]
    K = len(meshes)
    dev = torch.device("cuda", torch.cuda.current_device())
    scene = fgl.Scene(w.verts, w.tris, width=args.width)
    inst = [fgl.Scene(v, t, width=args.width) for v, t in meshes]
    sensor = fgl.Sensor.from_table(w.sensor)
    n_rays = n_env * sensor.n_rays
    walk_d = torch.from_numpy(w.poses).to(dev)
    ip_d = torch.from_numpy(IP).to(dev)
    pose_state = torch.empty((n_env, 3, 4), dtype=torch.float32, device=dev)
    ip_state = torch.empty((n_env, K, 3, 4), dtype=torch.float32, device=dev)
    out_r = torch.empty(n_rays, dtype=torch.float32, device=dev)
    out_i = torch.empty(n_rays, dtype=torch.int32, device=dev)
    out_k = torch.empty(n_rays, dtype=torch.int32, device=dev)
    out_p = torch.empty((n_rays, 3), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    opts = fgl.BatchOpts(use_graph=1)
    ex = {"instances": inst, "instance_poses": ip_state, "out_instance": out_k, "points": out_p}
    items = [(scene, sensor, pose_state, w.max_range, out_r, out_i, 0.0, ex)]
    arr = fgl.make_items(items)
    items0 = [(scene, sensor, pose_state, w.max_range, out_r, out_i)]
    arr0 = fgl.make_items(items0)

    def step(s, with_inst=True):
        with torch.cuda.stream(stream):
            pose_state.copy_(walk_d[s % S])
            ip_state.copy_(ip_d[s % S])
        if with_inst:
            fgl.cast_batched(items, opts, stream=stream, arr=arr)
        else:
            fgl.cast_batched(items0, opts, stream=stream, arr=arr0)

    def timed(with_inst):
        for k in range(args.warmup):
            step(k, with_inst)
        fgl.sync(stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        barrier(ws)
        torch.cuda.synchronize()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
                ev[k][0].record(stream)
            step(args.warmup + k, with_inst)
            with torch.cuda.stream(stream):
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        fgl.sync(stream)
        return barrier_max(sum(a.elapsed_time(b) for a, b in ev) / 1e3, ws)

    with ClockSampler(local) as clk:
        tot = timed(True)
    clocks = clk.summary()
    tot0 = timed(False)
    seen = float((out_k >= 0).float().mean().item())
    # end to end through the host-buffer entry: the step's sensor and instance
    # poses from page-locked host memory in, ranges, ids, instances and points out
    e2e = None
    if not args.no_e2e:
        hp = torch.empty((n_env, 3, 4), dtype=torch.float32).pin_memory()
        hip = torch.empty((n_env, K, 3, 4), dtype=torch.float32).pin_memory()
        hr = torch.empty(n_rays, dtype=torch.float32).pin_memory()
        hi = torch.empty(n_rays, dtype=torch.int32).pin_memory()
        hk = torch.empty(n_rays, dtype=torch.int32).pin_memory()
        hpt = torch.empty((n_rays, 3), dtype=torch.float32).pin_memory()

        hitems = [(scene, sensor, hp, w.max_range, hr, hi, 0.0,
                   {"instances": inst, "instance_poses": hip, "out_instance": hk, "points": hpt})]

        def e2e_step(s):                # fgl_cast_batched_host: chunked, copies overlap the casts
            hp.copy_(torch.from_numpy(w.poses[s % S]))
            hip.copy_(torch.from_numpy(IP[s % S]))
            fgl.cast_batched_host(hitems, opts, stream=stream)

        for k in range(2):
            e2e_step(k)
        ksteps = max(3, min(args.steps, 10))
        t_e = 0.0
        for k in range(ksteps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step(args.warmup + k)
            t_e += time.perf_counter() - t0
        fgl.sync(stream)
        t_e = barrier_max(t_e, ws)
        e2e = {"value": round(ws * n_rays * ksteps / t_e / 1e9, 4), "unit": UNIT,
               "h2d_bytes_per_step": n_env * 48 * (1 + K), "d2h_bytes_per_step": n_rays * 24,
               "ms_per_step": round(t_e * 1e3 / ksteps, 3)}
    # the dominant kernel is the scene cast (k_persistent): its cost-model
    # bytes from a counting pass, over its own time (the step without instances)
    with torch.cuda.stream(stream):
        pose_state.copy_(walk_d[args.warmup % S])
    cb, cr, cn, ct = counted_bytes(fgl, items0, stream, opts)
    cost = hbm_roofline(cb, tot0 / args.steps, cr, cn, ct, kernel="k_persistent (the scene cast)")
    roofline = issue_roofline("k_persistent", "k_persistent@walk_instances", n_rays * args.steps / tot0,
                              clocks, torch.device("cuda"), {"cost_model": cost,
                              "note": "the scene cast, over its own time (the step without instances)"})
    if roofline is None:
        roofline = dict(cost, note="no ncu capture of the current kernel sources on this workload: "
                                   "the issue bound is unmeasured")
    if rank == 0:
        line = {"metric": "Grays/s @4096 envs x 1M tris + 4 moving instances per env (with return points)",
                "value": round(ws * n_rays * args.steps / tot / 1e9, 4), "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot * 1e3 / args.steps, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": "walk_instances: batched_walk plus 4 rigid instances per environment "
                                       "(an icosphere of radius 0.3 m, two boxes, a 1.8 m pillar) on "
                                       "per-step poses 0.6-1.2 m from each sensor",
                           "rays_per_step": n_rays, "instance_tris": [int(len(t)) for _, t in meshes],
                           "returns_on_instances": round(seen, 4),
                           "l2": "flushed between timed steps (256 MiB write)"},
                "without_instances_ms_per_step": round(tot0 * 1e3 / args.steps, 3),
                "gpu_launches": args.steps * 3,   # scene cast, fused instance pass, return points
                "e2e": e2e, "roofline": roofline, "clocks": clocks}
        print(json.dumps(line), flush=True)


def run_lbvh(args):
    """The paper's route on the batched walk: a triangle LBVH built on the GPU
    and cast one thread per beam, against the host-built wide SAH BVH and its
    persistent batched kernel; plus a dynamic-scene step (every vertex moved,
    the LBVH rebuilt, then cast)."""
    import torch
    import paper_2509_17390_gb300 as fgl
    from synth import workloads
    ws, rank, local = dist_setup(args.gpus)
    n_steps = args.warmup + args.steps
    w = workloads.batched_walk(2, n_env=args.n_env, n_steps=min(n_steps, 100))
    n_env, S = args.n_env, w.poses.shape[0]
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)
    vd = torch.from_numpy(w.verts).to(dev)
    td = torch.from_numpy(w.tris).to(dev)
    # builds: GPU LBVH (synchronised, median of 5) vs host SAH + collapse
    lb = fgl.Lbvh(vd, td, stream=stream)
    bms = []
    for _ in range(5):
        lb.rebuild(vd, td, stream=stream)
        bms.append(lb.stats()["build_ms"])
    wide = fgl.Scene(w.verts, w.tris, width=args.width)
    sensor = fgl.Sensor.from_table(w.sensor)
    n_rays = n_env * sensor.n_rays
    walk_d = torch.from_numpy(w.poses).to(dev)
    pose = torch.empty((n_env, 3, 4), dtype=torch.float32, device=dev)
    out_r = torch.empty(n_rays, dtype=torch.float32, device=dev)
    out_i = torch.empty(n_rays, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    opts = fgl.BatchOpts(use_graph=1)
    items = [(wide, sensor, pose, w.max_range, out_r, out_i)]
    arr = fgl.make_items(items)
    shift = torch.tensor([0.0, 0.0, 0.0], device=dev)

    def cast_lbvh(s):
        with torch.cuda.stream(stream):
            pose.copy_(walk_d[s % S])
        lb.cast(sensor, pose, w.max_range, out_range=out_r, out_tri=out_i, stream=stream)

    def cast_wide(s):
        with torch.cuda.stream(stream):
            pose.copy_(walk_d[s % S])
        fgl.cast_batched(items, opts, stream=stream, arr=arr)

    def dynamic(s):
        with torch.cuda.stream(stream):
            pose.copy_(walk_d[s % S])
            vd.add_(0.001)                      # every vertex moves
        lb.rebuild(vd, td, stream=stream)
        lb.cast(sensor, pose, w.max_range, out_range=out_r, out_tri=out_i, stream=stream)

    def timed(fn):
        for k in range(args.warmup):
            fn(k)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        barrier(ws)
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
                ev[k][0].record(stream)
            fn(args.warmup + k)
            with torch.cuda.stream(stream):
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        return barrier_max(sum(a.elapsed_time(b) for a, b in ev) / 1e3, ws)

    with ClockSampler(local) as clk:
        t_lbvh = timed(cast_lbvh)
    clocks = clk.summary()
    t_wide = timed(cast_wide)
    t_dyn = timed(dynamic)
    # the LBVH cast is bound by instruction issue like the wide kernel: warp
    # instructions per ray (ncu, committed with its sources' hash) x rays/s
    # against 4 warp instructions per SM per cycle at the sampled clock
    roofline = None
    ipr = read_profile("k_lbvh_cast", "warp_inst_per_ray")
    if ipr is not None:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = (clocks or {}).get("sm_mhz") or 2070.0
        ach = ipr * n_rays * args.steps / t_lbvh / 1e9
        pk = 4.0 * sms * mhz * 1e6 / 1e9
        roofline = {"bound": "alu", "kernel": "k_lbvh_cast", "achieved": round(ach, 1), "peak": round(pk, 1),
                    "unit": "G warp-inst/s", "frac": round(ach / pk, 4), "warp_inst_per_ray": ipr,
                    "traffic": read_profile("k_lbvh_cast", "dram_bytes_per_launch"),
                    "peak_source": "derived",
                    "peak_basis": f"4 warp schedulers x {sms} SMs x {mhz:.0f} MHz (instruction issue)"}
    if rank == 0:
        line = {"metric": "Grays/s @4096 envs x 1M tris, GPU-built triangle LBVH cast one thread per beam",
                "value": round(ws * n_rays * args.steps / t_lbvh / 1e9, 4), "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(t_lbvh * 1e3 / args.steps, 3), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "batched_walk (4096 envs x 5760 rays, 1,000,300 tris)",
                           "l2": "flushed between timed steps (256 MiB write)"},
                "lbvh_build_ms_median": round(float(np.median(bms)), 2),
                "lbvh_depth": lb.stats()["depth"],
                "wide_sah_build_ms_host": round(wide.stats()["build_ms"], 1),
                "wide_batched": {"value": round(ws * n_rays * args.steps / t_wide / 1e9, 4), "unit": UNIT,
                                 "ms_per_step": round(t_wide * 1e3 / args.steps, 3)},
                "dynamic_rebuild_and_cast": {"ms_per_step": round(t_dyn * 1e3 / args.steps, 3),
                                             "value": round(ws * n_rays * args.steps / t_dyn / 1e9, 4),
                                             "unit": UNIT},
                "gpu_launches": args.steps, "roofline": roofline, "clocks": clocks}
        print(json.dumps(line), flush=True)


def occupancy_setup(torch):
    """The heterogeneous ladder's Gaussian sets (same seeds as the meshes of
    hetero_batch) on grids covering each room plus 0.3 m, at the ladder's
    voxel sizes."""
    from synth import gaussians, workloads
    sets = []
    for k, (room, nb, ns, ng, h) in enumerate(workloads.HETERO_LADDER):
        gs = gaussians.gaussian_room(4 * 100 + k, room, ng, nb, ns)
        L = np.asarray(room, np.float64)
        origin = (-0.3, -0.3, -0.3)
        dims = tuple(int(np.ceil((L[a] + 0.6) / h)) for a in range(3))
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        sets.append({"gs": gs, "h": h, "origin": origin, "dims": dims,
                     "dev": (t(gs.mu), t(gs.scale), t(gs.quat), t(gs.alpha)), "n": len(gs)})
    return sets


def run_occupancy(args):
    """Gaussian-to-occupancy conversion (Sec. IV-A) over the 8 ladder sets."""
    import torch
    import paper_2509_17390_gb300 as fgl
    ws, rank, local = dist_setup(args.gpus)
    sets = occupancy_setup(torch)
    dev = torch.device("cuda", torch.cuda.current_device())
    outs = []
    for S in sets:
        nx, ny, nz = S["dims"]
        outs.append((torch.empty((nz, ny, nx), dtype=torch.float32, device=dev),
                     torch.empty((nz, ny, nx), dtype=torch.uint8, device=dev),
                     torch.empty((nz, ny, nx), dtype=torch.uint8, device=dev)))
    theta = 0.5
    ss = SetStreams(torch, dev, [int(np.prod(S["dims"])) for S in sets], MESH_STREAMS)
    stream = ss.main

    def one(i, st, timing=False):
        S = sets[i]
        D, O, U = outs[i]
        return fgl.gaussian_density(*S["dev"], S["origin"], S["h"], S["dims"], theta=theta, out_density=D,
                                    out_occ=O, out_surf=U, stream=st, timing=timing)[3]

    for _ in range(args.warmup):
        ss.run(one)
    torch.cuda.synchronize()
    # per-kernel event times: untimed passes, one set at a time on one stream
    passes = [[one(i, stream, timing=True) for i in range(len(sets))] for _ in range(3)]
    stats = passes[0]
    evals = sum(st["n_pairs"] * 512 for st in stats)   # 8^3 voxel evaluations per candidate pair
    voxels = sum(st["n_voxels"] for st in stats)
    dens_ms = [sum(st["ms_density"] for st in p_) for p_ in passes]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
                ev[k][0].record(stream)
            ss.run(one)
            with torch.cuda.stream(stream):
                ev[k][1].record(stream)
        torch.cuda.synchronize()
    tot = barrier_max(sum(a.elapsed_time(b) for a, b in ev) / 1e3, ws)
    value = ws * evals * args.steps / tot / 1e9
    clocks = clk.summary()
    # the density kernel: one ex2 per (voxel, candidate) evaluation.  ex2 issues
    # at 16 per SM per cycle: at 4.9e12 ex2/s (2.07 GHz, 152 SMs) ncu shows the
    # XU pipe at 50% of its instruction peak with math-pipe throttle as the top
    # stall, i.e. ex2 takes two of the pipe's issue slots
    kern_s = float(np.median(dens_ms)) / 1e3
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    peak = 16.0 * sms * mhz * 1e6 / 1e9
    achieved = evals / kern_s / 1e9
    roofline = {"bound": "alu", "achieved": round(achieved, 1), "peak": round(peak, 1),
                "unit": "G ex2/s", "frac": round(achieved / peak, 4),
                "peak_basis": f"ex2: 16 per SM per cycle x {sms} SMs x {mhz:.0f} MHz", "kernel": "k_density<8>",
                "kernel_ms_per_step": round(kern_s * 1e3, 3)}
    # end to end: Gaussians from pinned host memory, surface masks back
    e2e = None
    if not args.no_e2e:
        host = []
        for S in sets:
            g = S["gs"]
            host.append([torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                         for a in (g.mu, g.scale, g.quat, g.alpha)])
        hsurf = [torch.empty(o[2].shape, dtype=torch.uint8).pin_memory() for o in outs]
        bi = sum(sum(t.numel() * t.element_size() for t in h) for h in host)
        bo = sum(t.numel() for t in hsurf)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)

        def e2e_set(i, st):                            # on stream st (the current stream)
            for d_, h_ in zip(sets[i]["dev"], host[i]):
                d_.copy_(h_, non_blocking=True)
            one(i, st)
            hsurf[i].copy_(outs[i][2], non_blocking=True)

        ss.run(e2e_set)
        e1.record(stream)
        e1.synchronize()
        e_s = e0.elapsed_time(e1) / 1e3
        e2e = {"value": round(evals / e_s / 1e9, 3), "unit": "Geval/s", "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "ms_per_step": round(e_s * 1e3, 3)}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        import oracle
        S = sets[3]                                    # the 250k-Gaussian set: about 1.5 s on 16 cores
        g = S["gs"]
        t_ = time.perf_counter()
        oracle.density(g.mu, g.scale, g.quat, g.alpha, S["origin"], S["h"], S["dims"], 8)
        el = time.perf_counter() - t_
        cpu = {"value": round(stats[3]["n_pairs"] * 512 / el / 1e9, 5), "unit": "Geval/s",
               "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"the {len(g.mu) // 1000}k-Gaussian set ({S['dims'][0]}x{S['dims'][1]}x{S['dims'][2]} voxels), FP64 brute force, {el:.1f} s"}
    if rank == 0:
        line = {"metric": "Geval/s Gaussian-to-occupancy (voxel x candidate evaluations of eq. D(v), 8 sets of 50k-2M Gaussians)",
                "value": round(value, 3), "unit": "Geval/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(tot * 1e3 / args.steps, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": "occupancy: the hetero ladder's Gaussian sets (50k-2M Gaussians on procedural rooms), grids = room + 0.3 m at 5-2 cm voxels, 8^3 tiles, theta 0.5",
                           "voxels_per_step": voxels, "evaluations_per_step": evals,
                           "pairs": [st["n_pairs"] for st in stats],
                           "l2": "flushed between timed steps (256 MiB write)",
                           "sets": [{"gaussians": S["n"], "voxel_m": S["h"], "dims": S["dims"]} for S in sets]},
                "gpu_launches": args.steps * sum(st["n_launches"] for st in stats), "roofline": roofline, "e2e": e2e,
                "cpu_baseline": cpu, "Mvoxels_per_s": round(ws * voxels * args.steps / tot / 1e6, 1),
                "clocks": clocks}
        print(json.dumps(line), flush=True)


MESH_STREAMS = 4  # streams (and host threads) the 8 sets of the mesh and occupancy workloads share


class SetStreams:
    """A workload's sets spread over n streams driven by n host threads
    (largest set first, each to the least-loaded stream), so one set's host
    synchronisations overlap the others' kernels; run() brackets all of
    them on the `main` stream."""

    def __init__(self, torch, dev, sizes, n):
        import concurrent.futures
        self.torch = torch
        self.main = torch.cuda.Stream(device=dev)
        self.streams = [torch.cuda.Stream(device=dev) for _ in range(n)]
        self.assign = [[] for _ in range(n)]
        load = [0] * n
        for i in sorted(range(len(sizes)), key=lambda i: -sizes[i]):
            k = int(np.argmin(load))
            self.assign[k].append(i)
            load[k] += sizes[i]
        self.pool = concurrent.futures.ThreadPoolExecutor(n)

    def run(self, per_set):
        """per_set(i, stream) for every set, with `stream` current in its
        thread (allocations follow it); returns once everything is enqueued."""
        torch = self.torch
        start = torch.cuda.Event()
        start.record(self.main)

        def work(k):
            st = self.streams[k]
            st.wait_event(start)
            with torch.cuda.stream(st):
                for i in self.assign[k]:
                    per_set(i, st)
            done = torch.cuda.Event()
            done.record(st)
            return done

        for done in self.pool.map(work, range(len(self.streams))):
            self.main.wait_event(done)


def gpu_mesher(gs, origin, h, dims):
    """The library's 3DGS-to-mesh pipeline (Sec. IV-A, IV-B) on one Gaussian
    set: the heterogeneous workload's meshes."""
    import torch
    import paper_2509_17390_gb300 as fgl
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    v, tr, _ = fgl.mesh_from_gaussians(t(gs.mu), t(gs.scale), t(gs.quat), t(gs.alpha), origin, h, dims)
    return v.cpu().numpy(), tr.cpu().numpy()


def mesh_setup(torch):
    """The hetero ladder's Gaussian sets on their grids (room plus
    MESH_MARGIN, so the level set never meets the grid's faces)."""
    from synth import gaussians, workloads
    sets = []
    for k, (room, nb, ns, ng, h) in enumerate(workloads.HETERO_LADDER):
        gs = gaussians.gaussian_room(4 * 100 + k, room, ng, nb, ns)
        origin, dims = workloads.hetero_grid(room, h)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        sets.append({"gs": gs, "h": h, "origin": origin, "dims": dims, "n": len(gs),
                     "dev": (t(gs.mu), t(gs.scale), t(gs.quat), t(gs.alpha))})
    return sets


def mesh_group_roofline(voxels, caps, stages_ms, peak_gbs):
    """The Sec. IV-B group's HBM figure on the largest set alone: its
    algorithmic bytes (11 B a voxel, 12 B a vertex and a triangle) over its
    event-timed denoise + TSDF + marching-tetrahedra stages (stages_ms[i] =
    [density, denoise, tsdf, marching tetrahedra] of set i), where launch
    gaps weigh least."""
    i = int(np.argmax(voxels))
    nbytes = 11 * voxels[i] + 12 * (caps[i][0] + caps[i][1])
    ms = float(sum(stages_ms[i][1:]))
    gbs = nbytes / (ms / 1e3) / 1e9
    return {"voxels": int(voxels[i]), "bytes": int(nbytes), "ms": round(ms, 3), "achieved": round(gbs, 1),
            "frac": round(gbs / peak_gbs, 4)}


def run_mesh(args):
    """3DGS to mesh on the GPU (Sec. IV-A then IV-B) over the 8 ladder sets:
    density and surface shell, denoising (sigma = h / 2, tau = 1/2), the
    narrow-band TSDF (r = 0.06 m) and marching tetrahedra.  The sets run on
    MESH_STREAMS streams from as many host threads (largest set first, each to
    the least-loaded stream), so one mesh's host synchronisations (sizing the
    pair buffers, reading the mesh counts) overlap other meshes' kernels."""
    import concurrent.futures
    import torch
    import paper_2509_17390_gb300 as fgl
    ws, rank, local = dist_setup(args.gpus)
    sets = mesh_setup(torch)
    dev = torch.device("cuda", torch.cuda.current_device())
    theta, trunc = 0.5, 0.06
    ss = SetStreams(torch, dev, [int(np.prod(S["dims"])) for S in sets], MESH_STREAMS)
    stream = ss.main
    all_sets = ss.run

    def one(S, cap, st=None, ev=None):
        st = stream if st is None else st
        h = S["h"]
        if ev:
            ev[0].record(st)
        _, _, surf, dst = fgl.gaussian_density(*S["dev"], S["origin"], h, S["dims"], theta=theta,
                                               stream=st, timing=bool(ev))
        if ev:
            ev[1].record(st)
        mask, _, _ = fgl.denoise(surf, h, 0.5 * h, tau=0.5, stream=st)
        if ev:
            ev[2].record(st)
        phi, _, _, tst = fgl.tsdf(mask, h, trunc, stream=st)
        if ev:
            ev[3].record(st)
        v, t, _ = fgl.marching_tets(phi, S["origin"], h, capacity=cap, stream=st)
        if ev:
            ev[4].record(st)
        return v, t, dst, tst

    caps = [None] * len(sets)
    for i, S in enumerate(sets):                          # counts, to size the outputs once
        v, t, _, _ = one(S, None)
        caps[i] = (len(v), len(t))
    for _ in range(args.warmup):
        all_sets(lambda i, st: one(sets[i], caps[i], st))
    torch.cuda.synchronize()
    # per-stage event times (an untimed pass, one set at a time on one stream)
    stage = np.zeros(4)
    launches = 0
    voxels = 0
    evals, dens_ms = 0, 0.0
    per_set_ms, per_set_stages = [], []
    for S, c in zip(sets, caps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        _, _, dst, tst = one(S, c, ev=ev)
        torch.cuda.synchronize()
        st4 = [ev[i].elapsed_time(ev[i + 1]) for i in range(4)]
        stage += st4
        per_set_ms.append(round(sum(st4), 3))
        per_set_stages.append(st4)
        evals += dst["n_pairs"] * 512
        dens_ms += dst["ms_density"]
        nx, ny, nz = S["dims"]
        voxels += nx * ny * nz
        # density; the fused blur (sigma = h/2: 2 taps a side) thresholds in the
        # same launch; TSDF; marching tetrahedra: pack, count (with the offsets
        # within chunks), chunk offsets, list, vertices, triangles
        launches += dst["n_launches"] + 1 + tst["n_launches"] + 6
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
                evs[k][0].record(stream)
            all_sets(lambda i, st: one(sets[i], caps[i], st))
            with torch.cuda.stream(stream):
                evs[k][1].record(stream)
        torch.cuda.synchronize()
    tot = barrier_max(sum(a.elapsed_time(b) for a, b in evs) / 1e3, ws)
    value = ws * voxels * args.steps / tot / 1e6
    clocks = clk.summary()
    peak, peak_src = read_peaks()
    # the Sec. IV-B steps as one HBM-bound group: the surface grid read and the
    # mask written (1 + 1 B a voxel), mask read and phi written (1 + 4), phi
    # read (4) and the mesh written (12 B a vertex, 12 B a triangle)
    nvt = sum(c[0] + c[1] for c in caps)
    mesh_bytes = 11 * voxels + 12 * nvt
    mesh_s = float(stage[1:].sum()) / 1e3
    roof_mesh = {"bound": "hbm", "achieved": round(mesh_bytes / mesh_s / 1e9, 1), "peak": round(peak, 1),
                 "unit": "GB/s", "frac": round(mesh_bytes / mesh_s / 1e9 / peak, 4),
                 "peak_source": peak_src, "bytes_per_step": int(mesh_bytes),
                 "basis": "11 B per voxel + 12 B per vertex and per triangle over denoise + TSDF + marching tetrahedra",
                 "largest_set": mesh_group_roofline([int(np.prod(S["dims"])) for S in sets], caps,
                                                    per_set_stages, peak)}
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    e2e = None
    if not args.no_e2e:
        host = [[torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                 for a in (S["gs"].mu, S["gs"].scale, S["gs"].quat, S["gs"].alpha)] for S in sets]
        hv = [torch.empty((c[0], 3), dtype=torch.float32).pin_memory() for c in caps]
        ht = [torch.empty((c[1], 3), dtype=torch.int32).pin_memory() for c in caps]
        bi = sum(sum(t.numel() * t.element_size() for t in h) for h in host)
        bo = sum(12 * (c[0] + c[1]) for c in caps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)

        def e2e_set(i, st):                            # on stream st (the current stream)
            for d_, h_ in zip(sets[i]["dev"], host[i]):
                d_.copy_(h_, non_blocking=True)
            v, t, _, _ = one(sets[i], caps[i], st)
            hv[i].copy_(v, non_blocking=True)
            ht[i].copy_(t, non_blocking=True)

        all_sets(e2e_set)
        e1.record(stream)
        e1.synchronize()
        e_s = e0.elapsed_time(e1) / 1e3
        e2e = {"value": round(voxels / e_s / 1e6, 1), "unit": "Mvoxels/s", "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "ms_per_step": round(e_s * 1e3, 3)}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        import oracle
        S = sets[2]                                    # the 145k-Gaussian set: about 1 s on 16 cores
        g = S["gs"]
        h = S["h"]
        t_ = time.perf_counter()
        D, _ = oracle.density(g.mu, g.scale, g.quat, g.alpha, S["origin"], h, S["dims"], 8)
        _, surf = oracle.occupancy(D, theta)
        sv = np.float64(np.float32(0.5 * h)) / np.float64(np.float32(h))
        M, _ = oracle.rethreshold(oracle.blur(surf, sv), "fixed", 0.5)
        phi, _, _ = oracle.tsdf(M, h, trunc)
        oracle.marching_tets(phi, S["origin"], h)
        el = time.perf_counter() - t_
        nx, ny, nz = S["dims"]
        cpu = {"value": round(nx * ny * nz / el / 1e6, 3), "unit": "Mvoxels/s", "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": f"the {len(g.mu) // 1000}k-Gaussian set ({nx}x{ny}x{nz} voxels): FP64 brute-force density, blur, TSDF, marching tetrahedra, {el:.1f} s"}
    if rank == 0:
        line = {"metric": "Mvoxels/s 3DGS-to-mesh on the GPU (density, denoise, narrow-band TSDF, marching tetrahedra; 8 sets of 50k-2M Gaussians)",
                "value": round(value, 1), "unit": "Mvoxels/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(tot * 1e3 / args.steps, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": "mesh: the hetero ladder's Gaussian sets (50k-2M Gaussians on procedural open-topped rooms), grids = room + 0.75 m at 5-2 cm voxels, theta 0.5, blur sigma h/2 with tau 1/2, TSDF r = 0.06 m, iso 0, mc_step 1",
                           "streams": len(ss.streams),
                           "voxels_per_step": voxels, "meshes_per_step": len(sets),
                           "l2": "flushed between timed steps (256 MiB write)",
                           "sets": [{"gaussians": S["n"], "voxel_m": S["h"], "dims": S["dims"],
                                     "verts": c[0], "tris": c[1], "ms_3dgs_to_mesh": m}
                                    for S, c, m in zip(sets, caps, per_set_ms)],
                           "stage_ms": {"density": round(stage[0], 3), "denoise": round(stage[1], 3),
                                        "tsdf": round(stage[2], 3), "marching_tets": round(stage[3], 3)}},
                "gpu_launches": args.steps * launches,
                "roofline": {"bound": "alu", "kernel": "k_density<8>",
                             "achieved": round(evals / (dens_ms / 1e3) / 1e9, 1),
                             "peak": round(16.0 * sms * mhz * 1e6 / 1e9, 1), "unit": "G ex2/s",
                             "frac": round(evals / (dens_ms / 1e3) / (16.0 * sms * mhz * 1e6), 4),
                             "peak_basis": f"ex2: 16 per SM per cycle x {sms} SMs x {mhz:.0f} MHz",
                             "kernel_ms_per_step": round(dens_ms, 3),
                             "note": "the Sec. IV-A density dominates the step; the Sec. IV-B kernels are in roofline_mesh_steps"},
                "roofline_mesh_steps": roof_mesh, "e2e": e2e, "cpu_baseline": cpu,
                "meshes_per_s": round(ws * len(sets) * args.steps / tot, 2), "clocks": clocks}
        print(json.dumps(line), flush=True)


def run_hetero(args):
    import torch
    import paper_2509_17390_gb300 as fgl
    ws, rank, local = dist_setup(args.gpus)
    meshes, tables, envs, groups, scenes, sensors, widths, items, opts, stream, info = hetero_setup(fgl)
    n_rays = sum(it[2].shape[0] * it[1].n_rays for it in items)
    arr = fgl.make_items(items)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        fgl.cast_batched(items, opts, stream=stream, arr=arr)
    fgl.sync(stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
                ev[k][0].record(stream)
            fgl.cast_batched(items, opts, stream=stream, arr=arr)
            with torch.cuda.stream(stream):
                ev[k][1].record(stream)
        torch.cuda.synchronize()
    fgl.sync(stream)
    tot = barrier_max(sum(a.elapsed_time(b) for a, b in ev) / 1e3, ws)
    value = ws * n_rays * args.steps / tot / 1e9
    clocks = clk.summary()
    cb, cr, cn, ct = counted_bytes(fgl, items, stream, opts)
    cost = hbm_roofline(cb, tot / args.steps, cr, cn, ct)
    roofline = issue_roofline("k_persistent", "k_persistent@hetero", n_rays * args.steps / tot,
                              clocks, torch.device("cuda"), {"cost_model": cost})
    if roofline is None:
        roofline = dict(cost, note="no ncu capture of the current kernel sources on this workload: "
                                   "the issue bound is unmeasured")
    # the plain form: one fgl_cast launch per environment
    L = fgl.lib()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for sc, se, P, R, r, i in items:
        for e in range(P.shape[0]):
            st = L.fgl_cast(sc.handle, se.handle, P.data_ptr() + 48 * e, 1, R,
                            r.data_ptr() + 4 * se.n_rays * e, i.data_ptr() + 4 * se.n_rays * e,
                            stream.cuda_stream)
            assert st == 0, L.fgl_last_error()
    e1.record(stream)
    e1.synchronize()
    per_env = {"value": round(n_rays / (e0.elapsed_time(e1) / 1e3) / 1e9, 4), "unit": UNIT,
               "launches_per_step": len(envs)}
    # end to end through the host-buffer entry point: every item's poses from
    # page-locked host memory in, its ranges and ids out, inside the timing
    e2e = None
    if not args.no_e2e:
        hitems = []
        for sc, se, P, R, r, i in items:
            hitems.append((sc, se, P.cpu().pin_memory(), R, torch.empty(r.numel()).pin_memory(),
                           torch.empty(i.numel(), dtype=torch.int32).pin_memory()))
        for _ in range(2):
            fgl.cast_batched_host(hitems, opts, stream=stream)
        ksteps = max(3, min(args.steps, 10))
        t_e = 0.0
        for _ in range(ksteps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fgl.cast_batched_host(hitems, opts, stream=stream)
            t_e += time.perf_counter() - t0
        t_e = barrier_max(t_e, ws)
        same = all(torch.equal(h[4], it[4].cpu()) and torch.equal(h[5], it[5].cpu())
                   for h, it in zip(hitems, items))
        e2e = {"value": round(ws * n_rays * ksteps / t_e / 1e9, 4), "unit": UNIT,
               "h2d_bytes_per_step": sum(it[2].numel() * 4 for it in items),
               "d2h_bytes_per_step": n_rays * 8, "ms_per_step": round(t_e * 1e3 / ksteps, 3),
               "results_equal_device_path": bool(same)}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        import oracle
        rng = np.random.default_rng(5)
        tot_r, tot_t = 0, 0.0
        oscs = {}                                       # one FP64 BVH per mesh (built untimed)
        for (m, sidx) in sorted(groups)[:24]:
            tab = tables[sidx]
            o, d = oracle.world_rays(oracle.sensor_dirs(tab.elev, tab.azim), np.stack(groups[(m, sidx)][:32]))
            idx = rng.choice(len(o), min(len(o), 600_000), replace=False)
            if m not in oscs:
                oscs[m] = oracle.Scene(meshes[m].verts, meshes[m].tris, bvh=True)
            t_ = time.perf_counter()
            oscs[m].cast(o[idx], d[idx], 30.0, flags=False)
            tot_t += time.perf_counter() - t_
            tot_r += len(idx)
        cpu = {"value": round(tot_r / tot_t / 1e9, 6), "unit": UNIT, "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": f"{tot_r} rays from 24 (mesh, sensor) groups (up to 32 envs each), FP64 BVH, {tot_t:.1f} s"}
    if rank == 0:
        line = {"metric": "Grays/s, heterogeneous batch (8 meshes 90k-5.2M tris, 256 envs, mixed sensors)",
                "value": round(value, 4), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(tot * 1e3 / args.steps, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": "hetero_batch: 8 meshes from the library's GPU 3DGS-to-mesh pipeline "
                                       "(density, denoise, TSDF, marching tetrahedra) over 50k-2M seeded "
                                       "Gaussians (voxels 5->2 cm, grids = room + 0.75 m), 256 envs "
                                       "round-robin, sensors 16/32/64/128 beams x 360-2048 az or a 20k "
                                       "rosette, max range 30 m", "rays_per_step": n_rays,
                           "l2": "flushed between timed steps (256 MiB write)", **info},
                "gpu_launches": args.steps * len(set(widths.values())), "per_env_launch": per_env,
                "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks}
        print(json.dumps(line), flush=True)


def run_serve(args):
    """Serving workload: Poisson requests (mean 2,000/s over a 0.25 s window,
    then about 1,000 requests -- so that the p99 rests on about ten of them --
    whose arrival times are scaled to offer 70% of the capacity measured
    there, that trace replayed three times) of 1-4096 environments (log-uniform) over the 8 resident
    heterogeneous scenes with mixed sensors, 150 GiB budget.  Environment
    poses stay on the device: each scene owns a ring of 8,192 server slots
    and each request overwrites its slots from a device-resident pose pool
    before they are scanned.  The first requests also go through the server
    that issues one launch per environment."""
    import torch
    import paper_2509_17390_gb300 as fgl
    from synth import poses as _poses
    ws, rank, local = dist_setup(args.gpus)
    meshes, tables, envs, groups, scenes, _, widths, items, opts, stream, info = hetero_setup(fgl)
    rng = np.random.default_rng(21)
    all_sensors = [fgl.Sensor.from_table(t) for t in tables]
    pool = {m: _poses.sample_free_pose(rng, spec.obstacles, 2048, margin=0.25)
            for m, spec in enumerate(meshes)}
    dev = torch.device("cuda", torch.cuda.current_device())
    # device pose sources, the 2,048 free poses of each scene repeated to 8,192
    # so that a request of up to 4,096 environments takes a contiguous slice
    pool_d = [torch.from_numpy(np.ascontiguousarray(np.concatenate([pool[m]] * 4))).to(dev)
              for m in range(len(meshes))]
    n_rays_of = [s.n_rays for s in all_sensors]
    pick = lambda r, sc: int(r.integers(len(all_sensors)))
    # result space that wraps about every 2 s at this load, well after the
    # slowest request of a replay finished (a wrap onto a request still in
    # flight makes the replayer wait, which would add to the measured latency)
    arena = OutputArena(48 << 30)
    opts.use_graph = 0
    per_scene = 32768                               # slots per scene: a ring that wraps every few seconds
    srv = fgl.Server(hbm_budget_bytes=150 << 30, tick_rays=32 << 20, opts=opts,
                     env_capacity=per_scene * len(meshes))
    sids = [srv.add_scene(scenes[m][widths[m]]) for m in range(len(meshes))]
    tids = [srv.add_sensor(s) for s in all_sensors]
    plan = SlotPlan(srv, pool_d, per_scene, seed=22)
    sat_trace = slot_trace(make_trace(rng, 2000.0, 0.25, 4096, pool, len(meshes), pick), plan)
    sat = replay(srv, sat_trace, sids, tids, n_rays_of, arena, 30.0)
    mean_rays = float(np.mean([t[4][1].shape[0] * n_rays_of[t[2]] for t in sat_trace]))
    rate = 0.7 * sat["rays_per_s"] / mean_rays
    srv.reset_stats()
    # the arrival times scaled so that this trace itself offers 70% of the
    # sustained rate (request sizes are heavy-tailed: the rate above, set
    # from the saturation trace's mean size, offers more or less than that)
    raw = make_trace(rng, rate, 8.0, 4096, pool, len(meshes), pick)
    raw, window = scale_to_load(raw, 8.0, n_rays_of, 0.7 * sat["rays_per_s"])
    cal_trace = slot_trace(raw, plan)
    rate = len(raw) / window
    with ClockSampler(local) as clk:
        cal = replay_runs(srv, cal_trace, sids, tids, n_rays_of, arena, 30.0, runs=3)
    clocks = clk.summary()
    st = srv.stats()
    pre, acc = [], 0
    for tr in cal_trace:
        acc += tr[4][1].shape[0] * n_rays_of[tr[2]]
        pre.append(tr)
        if acc > 2.5e8:
            break
    preb = replay(srv, pre, sids, tids, n_rays_of, arena, 30.0)
    srv.close()
    srvp = fgl.Server(mode=1, hbm_budget_bytes=150 << 30, env_capacity=per_scene * len(meshes))
    sidp = [srvp.add_scene(scenes[m][widths[m]]) for m in range(len(meshes))]
    tidp = [srvp.add_sensor(s) for s in all_sensors]
    SlotPlan(srvp, pool_d, per_scene)                        # same slot ids
    prep = replay(srvp, pre, sidp, tidp, n_rays_of, arena, 30.0)
    srvp.close()
    if rank == 0:
        f = lambda r: {"requests": r["requests"], "Grays_s": round(r["rays_per_s"] / 1e9, 4),
                       "p50_ms": round(r["p50_ms"], 2), "p99_ms": round(r["p99_ms"], 2)}
        line = {"metric": "served Grays/s and p50/p99 scan latency (8 resident scenes, mixed sensors)",
                "value": round(cal["rays_per_s"] / 1e9, 4), "unit": UNIT, "n_gpus": ws,
                "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                "p50_ms": round(cal["p50_ms"], 2), "p99_ms": round(cal["p99_ms"], 2),
                "saturation_2000rps": f(sat),
                "at_70pct": {**f(cal), "rate_req_per_s": round(rate, 2),
                             "offered_Grays_s": round(0.7 * sat["rays_per_s"] / 1e9, 4), "runs": cal["runs"],
                             "p50_spread": cal["p50_spread"], "p99_spread": cal["p99_spread"],
                             "per_run": cal["per_run"]},
                "same_prefix": {"batched": f(preb), "per_env_launch": f(prep)},
                "server": {"evictions": st["evictions"], "uploads": st["uploads"], "ticks": st["ticks"]},
                "e2e": {"value": round(cal["rays_per_s"] / 1e9, 4), "unit": UNIT,
                        "h2d_bytes_per_step": 0, "d2h_bytes_per_step": "all results (8 B a ray)",
                        "note": "served latency and rate are end to end: arrival -> results in host memory"},
                "clocks": clocks,
                "config": {"workload": "serve: Poisson arrivals of 1-4096 environments (log-uniform) over "
                                       "the 8 heterogeneous scenes, 21 sensors, 150 GiB budget, 32 Mi-ray "
                                       "ticks; poses in device-resident slots (32,768 a scene) updated "
                                       "from device memory by each request", **info}}
        print(json.dumps(line), flush=True)


def run_reference(args, n_steps):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from synth import workloads
    w = workloads.batched_walk(2, n_env=args.n_env, n_steps=min(n_steps, 100))
    S = w.poses.shape[0]
    n_sample = 512
    times, nrays = [], 0
    osc = None
    for k in range(n_steps):
        osc, o, d, envs = oracle_sample(w, w.poses[k % S], n_sample, seed=k, osc=osc)
        t = time_oracle(osc, o, d, w.max_range)
        if k >= args.warmup:
            times.append(t)
            nrays = len(o)
    tot = sum(times)
    v = nrays * len(times) / tot / 1e9
    # a whole step is args.n_env environments; each timed step casts a sample
    # of n_sample of them, so the step time is the sample's scaled by rays
    full_rays = args.n_env * w.sensor.n_rays
    line = {"metric": METRIC, "value": round(v, 6), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(full_rays / (v * 1e9) * 1e3, 3),
            "sample_ms_per_step": round(tot * 1e3 / len(times), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "parallelism": "host cores"},
            "cpu_baseline": {"value": round(v, 6), "unit": UNIT, "kind": "oracle",
                             "cores": os.cpu_count(),
                             "sample": f"per step {n_sample} of {args.n_env} envs x "
                                       f"{w.sensor.n_rays} rays, FP64 median-split BVH"},
            "e2e": {"value": round(v, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
