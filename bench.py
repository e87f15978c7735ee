#!/usr/bin/env python3
"""Throughput of the RBSM per-fragment path on one GB300 (or N replicas).

Workload (the 3840x2160 configuration): 32 frames of a moving light, each
frame an 8192^2 float32 shadow map rasterised from 200 occluders and
3840x2160 light-space fragments of a static camera.  One step evaluates every
fragment of every frame against its frame's map, giving each fragment both
answers of the method: the revectorised hard shadow (silhouette recovery,
Listing 4) and the RSMSS fake penumbra (filtering, Listing 5), in ONE
persistent batched launch (rbsm_batch_run, mode BOTH).  Inputs are larger
than L2 (about 11 GB per step), so no L2 flush is needed between steps.

Printed: one JSON line with the metric (Gfragments/s, whole job), the
roofline of the batched kernel against the measured HBM copy bandwidth, an
end-to-end figure through the public API with host buffers, and the CPU
oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gfragments/s visibility at 3840x2160"
UNIT = "Gfragments/s"
BYTES_PER_FRAGMENT = 12 + 4 + 4     # x, y, z in; silhouette and filter visibility out
BYTES_PER_TEXEL = 4                 # each unique centre texel read once
FALLBACK_HBM_GBS = 6800.0
KERNEL_SOURCES = ["paper_1711_07793_gb300/csrc/rbsm_device.cuh", "paper_1711_07793_gb300/csrc/rbsm_batch_kernel.cuh",
                  "paper_1711_07793_gb300/csrc/rbsm_batch.cu"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "batch_kernel_c5_traffic.md")


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--frames", type=int, default=32, help="frames per step (32 = the full workload)")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--e2e-steps", type=int, default=10)
    p.add_argument("--skip-e2e", action="store_true", help="profiling runs only")
    p.add_argument("--skip-cpu", action="store_true", help="profiling runs only")
    p.add_argument("--skip-learned", action="store_true", help="profiling runs only")
    p.add_argument("--skip-rpcf", action="store_true", help="profiling runs only")
    p.add_argument("--skip-light", action="store_true", help="profiling runs only")
    p.add_argument("--skip-gbuffer", action="store_true", help="profiling runs only")
    p.add_argument("--skip-sweep", action="store_true", help="profiling runs only")
    p.add_argument("--only", default="", help="with --configs: comma-separated workloads (C1,C2,C3,C4)")
    p.add_argument("--configs", action="store_true",
                   help="one line per workload C1-C4 (GPU rate, roofline, oracle on 1 and all threads)")
    p.add_argument("--guard-tau", type=float, default=0.01, help="surrogate guard (largest accepted error estimate)")
    p.add_argument("--texture", choices=["on", "off"], default="on",
                   help="read each map's four-neighbourhood with texture gathers (rbsm_map_texture_create)")
    p.add_argument("--graph", choices=["on", "off"], default="on",
                   help="replay the batched launch as a CUDA graph (rbsm_batch_graph_*)")
    p.add_argument("--autotune", choices=["on", "off"], default="on",
                   help="pick the launch shape with rbsm_batch_autotune before timing")
    p.add_argument("--tile-threads", type=int, default=0)
    p.add_argument("--ctas-per-sm", type=int, default=0)
    return p.parse_args(argv)


# ------------------------------------------------------------ distributed --

def dist_env():
    """(rank, world, local_rank) from torchrun's environment (1 process: 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value, world):
    """Largest value over all ranks (the whole job ends with its slowest rank)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ peaks --

def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(frames):
    """DRAM bytes per launch from the committed ncu summary, scaled to
    `frames`, or None when the summary is missing or the kernel changed."""
    try:
        text = open(TRAFFIC_FILE).read()
    except OSError:
        return None
    src = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    per = re.search(r"dram_bytes_per_frame:\s*([0-9.eE+]+)", text)
    if not src or not per or src.group(1) != kernel_source_hash():
        return None
    return float(per.group(1)) * frames


# ----------------------------------------------------------------- clocks --

class ClockSampler:
    """nvidia-smi samples (every 200 ms) of one GPU while a region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.samples.append((time.time(), parts))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self, t0, t1):
        sel = [p for t, p in self.samples if t0 - 0.2 <= t <= t1 + 0.2]
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(p[0]) for p in sel if num(p[0]) is not None]
        mx = [num(p[1]) for p in sel if num(p[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for p in sel for k in range(4) if p[4 + k].lower() == "active"})
        power = [num(p[2]) for p in sel if num(p[2]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sel), "power_w_max": max(power) if power else None}


def smi_gpu_id(local_rank):
    """An id nvidia-smi accepts for this process's GPU: its UUID when torch
    reports one, else the CUDA_VISIBLE_DEVICES entry, else the index."""
    import torch
    try:
        u = str(torch.cuda.get_device_properties(local_rank).uuid)
        if re.fullmatch(r"(GPU-)?[0-9a-fA-F-]{36}", u):
            return u if u.startswith("GPU-") else "GPU-" + u
    except (AttributeError, RuntimeError):
        pass
    cvd = [s.strip() for s in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if s.strip()]
    if local_rank < len(cvd):
        return cvd[local_rank]
    return str(local_rank)


# --------------------------------------------------------------- workload --

def unique_texels(x, y, size):
    """Number of distinct centre texels the fragments land on (float32
    texel coordinates, clamp-to-edge), for the algorithmic map bytes."""
    import numpy as np
    u = np.clip(np.floor(x * np.float32(size)), 0, size - 1).astype(np.int64)
    v = np.clip(np.floor(y * np.float32(size)), 0, size - 1).astype(np.int64)
    seen = np.zeros(size * size, dtype=bool)
    seen[v * size + u] = True
    return int(seen.sum())


def make_workload(frames, seed, pin=True):
    """Host tensors (pinned) of `frames` frames of the 8192^2 / 3840x2160
    moving-light workload, plus per-frame unique-texel counts."""
    import numpy as np
    import torch
    import rbsm_scenes as sc
    c5 = sc.Config5(seed)
    n = c5.screen[0] * c5.screen[1]
    out = []
    for f in range(frames):
        depth = torch.empty((c5.size, c5.size), dtype=torch.float32, pin_memory=pin)
        xyz = torch.empty((3, n), dtype=torch.float32, pin_memory=pin)
        dn, xn = depth.numpy(), xyz.numpy()
        fr = c5.frame(f, out_depth=dn, out_xyz=(xn[0], xn[1], xn[2]))
        out.append({"depth": depth, "xyz": xyz, "U": unique_texels(xn[0], xn[1], c5.size),
                    "sphere_fraction": fr.meta["sphere_fraction"]})
    return c5, out


# ------------------------------------------------------------ CPU oracle --

def oracle_throughput(host_frames, min_seconds=10.0):
    """The oracle as it stands, chunked over every host core (ctypes releases
    the GIL), on whole frames of the workload, cycling through them until
    min_seconds have passed: Gfragments/s where a fragment gets both answers
    (silhouette and filtering)."""
    import numpy as np
    from concurrent.futures import ThreadPoolExecutor
    from oracle import rbsm as orc
    cores = os.cpu_count() or 1
    done = 0
    frames_done = 0
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        while time.perf_counter() - t0 < min_seconds:
            fr = host_frames[frames_done % len(host_frames)]
            depth = fr["depth"].numpy()
            xyz = fr["xyz"].numpy()
            n = xyz.shape[1]
            bounds = np.linspace(0, n, cores + 1).astype(np.int64)

            def work(k):
                a, b = bounds[k], bounds[k + 1]
                for mode in (orc.MODE_SILHOUETTE, orc.MODE_FILTER):
                    orc.evaluate(depth, xyz[0, a:b], xyz[1, a:b], xyz[2, a:b], mode)
                return b - a

            done += sum(ex.map(work, range(cores)))
            frames_done += 1
    dt = time.perf_counter() - t0
    return {"value": done / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d frames (cycling through the %d frames of the workload), every fragment, "
                      "both visibility functions, %.1f s" % (frames_done, len(host_frames), dt)}


def edge_statistics(host_frames, per_frame=65536, max_dist=16, seed=11):
    """The workload's edge-fragment fraction and traversal-length histogram
    (reported next to the CPU baseline; untimed): the oracle's four walks of
    the edge fragments of a uniform sample of every frame.  A walk's length
    is |rd| texels (the fragment's texel included); `capped` counts walks
    that reached max_dist without an end."""
    import numpy as np
    from oracle import rbsm as orc
    rng = np.random.default_rng(seed)
    edge = total = 0
    found = np.zeros(max_dist + 2, np.int64)
    open_ = np.zeros(max_dist + 2, np.int64)
    for fr in host_frames:
        xyz = fr["xyz"].numpy()
        idx = np.sort(rng.choice(xyz.shape[1], min(per_frame, xyz.shape[1]), replace=False))
        r = orc.evaluate(fr["depth"].numpy(), xyz[0, idx], xyz[1, idx], xyz[2, idx], orc.MODE_FILTER,
                         max_dist=max_dist, want_rd=True)
        walked = (r["codes"] & (1 << 9)) != 0
        total += idx.size
        edge += int(walked.sum())
        rd = r["rd"][walked].ravel()
        found += np.bincount(rd[rd > 0], minlength=max_dist + 2)[:max_dist + 2]
        open_ += np.bincount(-rd[rd < 0], minlength=max_dist + 2)[:max_dist + 2]
    return {"fraction": edge / max(total, 1), "sample_fragments": total,
            "walk_length_histogram": {
                "length": list(range(1, max_dist + 2)),
                "end_found": found[1:].tolist(),
                "no_end": open_[1:].tolist()},
            "capped_walks": int(open_[max_dist + 1]),
            "walks": int(found.sum() + open_.sum()),
            "sample": "%d fragments per frame of every frame, oracle walks, max_dist %d" % (per_frame, max_dist)}


# ------------------------------------------------------------------- ours --

def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1711_07793_gb300 import api
    from paper_1711_07793_gb300 import build as lib_build
    lib_build.build()

    torch.cuda.set_device(local_rank)
    device = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)

    c5, host = make_workload(args.frames, args.seed + 1000 * rank)
    n_frag = c5.screen[0] * c5.screen[1]
    frames = len(host)
    maps = [h["depth"].to(device, non_blocking=True) for h in host]
    xyz = [h["xyz"].to(device, non_blocking=True) for h in host]
    jobs = [api.Job(k, xyz[k][0], xyz[k][1], xyz[k][2], mode=3) for k in range(frames)]
    texs = [api.MapTexture(m) for m in maps] if args.texture == "on" else None
    batch = api.Batch(texs or maps, jobs, tile_threads=args.tile_threads, ctas_per_sm=args.ctas_per_sm)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    tuning = None
    if args.autotune == "on" and not args.tile_threads and not args.ctas_per_sm:
        tuning = api.rbsm_batch_autotune(batch, repeats=3, cache=None)
        torch.cuda.synchronize()
    graph = api.BatchGraph(batch) if args.graph == "on" else None

    def step():
        if graph is not None:
            graph.launch()
        else:
            api.rbsm_batch_run(batch)

    # warm-up, then exactly K timed steps, one CUDA event pair per launch
    for _ in range(args.warmup):
        step()
    sampler = ClockSampler(smi_gpu_id(local_rank))
    sampler.start()
    time.sleep(0.5)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.time()
    for k in range(args.steps):
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    barrier(world)
    sampler.stop()
    clocks = sampler.summary(t0, t1)
    assert api.rbsm_batch_status(batch) == 0
    launch_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = starts[0].elapsed_time(ends[-1])
    total_ms = max_over_ranks(total_ms, world)
    ms_per_step = total_ms / args.steps

    # roofline of the batched kernel (the only kernel of a step)
    peak, peak_kind = load_peaks()
    bytes_per_launch = sum(BYTES_PER_FRAGMENT * n_frag + BYTES_PER_TEXEL * h["U"] for h in host)
    mean_launch_ms = statistics.mean(launch_ms)
    achieved = bytes_per_launch / (mean_launch_ms * 1e-3) / 1e9
    traffic = recorded_traffic(frames)

    # end to end through the public API: maps, fragment planes and answers
    # in page-locked host memory, one rbsm_stager_run per step (copies in of
    # the fragment planes and of each map's window, the batched kernel,
    # copies out of the answers, overlapped across frames on the stager's
    # streams); the bytes are the stager's own count of what it copied
    e2e = None
    if not args.skip_e2e:
        stager = api.Stager(max_fragments=n_frag, max_width=max(h["depth"].shape[1] for h in host),
                            max_height=max(h["depth"].shape[0] for h in host), texture=args.texture == "on")
        host_jobs = [api.Job(k, host[k]["xyz"][0], host[k]["xyz"][1], host[k]["xyz"][2], mode=3)
                     for k in range(frames)]
        host_maps = [h["depth"] for h in host]
        shape = {"tile_threads": batch.desc.tile_threads, "ctas_per_sm": batch.desc.ctas_per_sm}

        def e2e_step():
            stager.run(host_maps, host_jobs, **shape)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        in0, out0 = stager.stats()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.e2e_steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.e2e_steps, world)
        in1, out1 = stager.stats()
        assert stager.status() == 0
        h2d = (in1 - in0) // args.e2e_steps
        d2h = (out1 - out0) // args.e2e_steps
        # the answers of the last step equal the device-resident batch's
        for k in (0, frames - 1):
            assert torch.equal(host_jobs[k].vis_filter, jobs[k].vis_filter.cpu())
            assert torch.equal(host_jobs[k].vis_silhouette, jobs[k].vis_silhouette.cpu())
        stager.close()
        e2e = {"value": world * frames * n_frag / (e2e_ms * 1e-3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
               "path": "rbsm_stager_run: pinned host maps/fragments/answers; fragment planes and map windows in"}

    light = None
    if not args.skip_light:
        light = measure_light_pass(api, c5, maps, frames, n_frag, step, stream)
        assert api.rbsm_batch_status(batch) == 0

    sweep = None
    if not args.skip_sweep:
        sweep = measure_maxdist(api, texs or maps, xyz, frames, n_frag, args, stream,
                                (batch.desc.tile_threads, batch.desc.ctas_per_sm))

    gbuf = None
    if not args.skip_gbuffer:
        gbuf = measure_gbuffer(api, c5, texs or maps, host, frames, n_frag, stream)

    rpcf = None
    if not args.skip_rpcf:
        rpcf = measure_rpcf(api, texs or maps, xyz, frames, n_frag, args, stream)

    learned = None
    if not args.skip_learned:
        learned = compare_learned(api, texs or maps, xyz, frames, n_frag, args, stream)
        learned["training"] = measure_training(api, maps, xyz, args, stream)

    cpu = None
    edges = {}
    if rank == 0 and world == 1 and not args.skip_cpu:
        cpu = oracle_throughput(host)
        edges = edge_statistics(host)

    line = {
        "metric": METRIC, "value": world * frames * n_frag / (ms_per_step * 1e-3) / 1e9, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "C5: %d frames x 3840x2160 fragments, 8192^2 fp32 maps, moving light, "
                               "silhouette + RSMSS per fragment" % frames,
                   "frames": frames, "screen": list(c5.screen), "map": c5.size, "mode": "both",
                   "batched": "one persistent launch per step (rbsm_batch_run)", "max_dist": 16,
                   "l2": "inputs larger than L2 (%.1f GB per step), no flush" % (
                       sum(h["depth"].numel() * 4 + h["xyz"].numel() * 4 for h in host) / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "tile_threads": batch.desc.tile_threads or 256,
                   "ctas_per_sm": batch.desc.ctas_per_sm or "occupancy",
                   "autotune": tuning, "cuda_graph": graph is not None,
                   "neighbourhood": "texture gathers" if texs else "plain loads"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind if peak_kind == "measured"
                     else "fallback 6800 GB/s",
                     "traffic": traffic, "kernel": "rbsm::batch_kernel",
                     "algorithmic_bytes_per_launch": bytes_per_launch,
                     "mean_launch_ms": mean_launch_ms, "min_launch_ms": min(launch_ms)},
        "e2e": e2e,
        "cpu_baseline": cpu,
        "learned": learned,
        "rpcf": rpcf,
        "gbuffer": gbuf,
        "maxdist_sweep": sweep,
        "light_pass": light["light_pass"] if light else None,
        "frame_pipeline": light["frame_pipeline"] if light else None,
        "gpu_launches": args.steps,
        "clocks": clocks,
        "edge": dict({"unique_texels_per_frame": statistics.mean(h["U"] for h in host)}, **edges),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------- learned --

CHECKPOINT = os.path.join(ROOT, "paper_1711_07793_gb300", "weights", "surrogate_c4.npz")
# the surrogate's stated bound on the answers it gives (|error| against the
# exact Listing 5 answer) at guard_tau = 0.01
SURROGATE_BOUND = {"mean": 0.01, "p99": 0.03, "max": 0.1}


def compare_learned(api, maps, xyz, frames, n_frag, args, stream):
    """Plain RSMSS against the surrogate with its guard, both batched over
    the same frames in one persistent launch per step (filtering mode): time
    per step, the surrogate's share of edge fragments, and the error of the
    learned answers against the plain ones (over every fragment and over the
    fragments the surrogate answered)."""
    import torch
    from paper_1711_07793_gb300.surrogate import Surrogate
    if not os.path.exists(CHECKPOINT):
        return {"unavailable": "no surrogate checkpoint (run python -m paper_1711_07793_gb300.train_surrogate)"}
    net = Surrogate.from_checkpoint(CHECKPOINT)
    # both timed arms write the same outputs (the filtering answers); the
    # codes, whose bit 10 marks a surrogate answer, come from an untimed run
    # for the statistics
    plain_jobs = [api.Job(k, xyz[k][0], xyz[k][1], xyz[k][2], mode=2) for k in range(frames)]
    timed_jobs = [api.Job(k, xyz[k][0], xyz[k][1], xyz[k][2], mode=2) for k in range(frames)]
    net_jobs = [api.Job(k, xyz[k][0], xyz[k][1], xyz[k][2], mode=2, codes=True) for k in range(frames)]
    plain = api.Batch(maps, plain_jobs, tile_threads=args.tile_threads, ctas_per_sm=args.ctas_per_sm)
    learned = api.Batch(maps, timed_jobs, tile_threads=args.tile_threads, ctas_per_sm=args.ctas_per_sm,
                        surrogate=net, guard_tau=args.guard_tau)
    with_codes = api.Batch(maps, net_jobs, tile_threads=args.tile_threads, ctas_per_sm=args.ctas_per_sm,
                           surrogate=net, guard_tau=args.guard_tau)
    steps = max(3, min(args.steps, 200))

    def timed(batch):
        for _ in range(3):
            api.rbsm_batch_run(batch)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            api.rbsm_batch_run(batch)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    ms_plain = timed(plain)
    ms_learned = timed(learned)
    api.rbsm_batch_run(with_codes)
    torch.cuda.synchronize()
    same = all(torch.equal(a.vis_filter, b.vis_filter) for a, b in zip(timed_jobs, net_jobs))
    acc, fb = api.rbsm_batch_surrogate_counts(with_codes)
    errs, errs_net = [], []
    for pj, lj in zip(plain_jobs, net_jobs):
        d = (lj.vis_filter - pj.vis_filter).abs()
        errs.append(d)
        answered = ((lj.codes.to(torch.int32) >> 10) & 1) == 1
        errs_net.append(d[answered])
    d = torch.cat(errs).double()
    dn = torch.cat(errs_net).double()
    def q(t, p):
        if t.numel() == 0:
            return None
        k = max(1, int(round(p * t.numel())))
        return float(torch.kthvalue(t.cpu(), k).values)
    fps = lambda ms: frames * n_frag / (ms * 1e-3) / 1e9
    answered = {"mean": float(dn.mean()) if dn.numel() else None, "p99": q(dn, 0.99),
                "max": float(dn.max()) if dn.numel() else None}
    met = all(answered[k] is not None and answered[k] <= v for k, v in SURROGATE_BOUND.items())
    return {"metric": "Gfragments/s RSMSS (filtering) visibility, same frames, one batched launch per step",
            "plain": {"value": fps(ms_plain), "ms_per_step": ms_plain},
            "learned": {"value": fps(ms_learned), "ms_per_step": ms_learned, "guard_tau": args.guard_tau,
                        "outputs": "filtering answers only, as the plain arm; codes from an untimed run",
                        "same_answers_as_the_run_with_codes": same},
            "speedup": ms_plain / ms_learned,
            "edge_fragments": acc + fb, "surrogate_answers": acc, "fallbacks": fb,
            "fallback_frac": fb / max(1, acc + fb),
            "error_vs_plain_all": {"mean": float(d.mean()), "p99": q(d, 0.99), "max": float(d.max())},
            "error_vs_plain_answered": answered,
            "stated_bound": dict(SURROGATE_BOUND, guard_tau=0.01,
                                 guards="walks inside the 5x5 window, trusted pattern (calibrated bitmap), "
                                        "error estimate <= guard_tau"),
            "bound_met": met if args.guard_tau <= 0.01 else None,
            "checkpoint": {k: net.header.get(k) for k in ("samples", "epochs", "data", "loss_per_epoch")}}


def measure_training(api, maps, xyz, args, stream, batch=8192):
    """The surrogate's training step on the tensor cores (rbsm_mlp_step: the
    tcgen05 gradient kernel, then the fixed-order reduction fused with Adam)
    over minibatches of edge fragments of the first two frames, and its
    forward pass over every sample: time per step with CUDA events, samples
    per second and the products' useful FLOP rate."""
    import torch
    from paper_1711_07793_gb300.surrogate import Surrogate
    import rbsm_scenes as sc
    data = [(maps[k], xyz[k][0], xyz[k][1], xyz[k][2]) for k in range(min(2, len(maps)))]
    samples, count = Surrogate.dataset(data, capacity=1 << 20)
    net = Surrogate(sc.mlp_init(0))
    steps = max(20, min(args.steps, 400))
    per_epoch = count // batch
    perm = torch.randperm(count, generator=torch.Generator().manual_seed(3)).to(torch.int32).cuda()
    orders = [perm[(s % per_epoch) * batch:(s % per_epoch + 1) * batch] for s in range(steps)]
    for s in range(3):
        net.train_step(samples, orders[s], 1e-3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for s in range(steps):
        net.train_step(samples, orders[s], 1e-3)
    e1.record(stream)
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / steps
    for _ in range(3):
        net.forward(samples, count)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(20):
        net.forward(samples, count)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_us = e0.elapsed_time(e1) * 1e3 / 20
    # useful products per sample: forward 32x64 + 64x64 + 64x2, backward-data 2x64 + 64x64,
    # weight gradients 32x64 + 64x64 + 64x2 multiply-adds
    flops = 2 * (32 * 64 + 64 * 64 + 64 * 2) * 2 + 2 * (2 * 64 + 64 * 64)
    return {"kernel": "rbsm::mlp::surrogate_tc_kernel (tcgen05, 128-sample tiles) + reduce_kernel (fixed order, Adam)",
            "batch": batch, "samples": count, "steps_timed": steps, "us_per_step": us,
            "samples_per_s": batch / (us * 1e-6), "useful_tflops": flops * batch / (us * 1e-6) / 1e12,
            "forward": {"samples": count, "us": fwd_us, "gsamples_per_s": count / (fwd_us * 1e-6) / 1e9}}


def measure_rpcf(api, maps, xyz, frames, n_frag, args, stream, k=3):
    """RPCF (PCF over the RSMSS answer, rbsm_rpcf) on the same frames, one
    launch per frame: time per 32-frame step next to rsmss_filter's, and
    the algorithmic-byte rate of its launches (the same bytes per fragment
    as RSMSS: the k x k samples re-read texels that are already on chip)."""
    import torch
    outs = [torch.empty(n_frag, dtype=torch.float32, device=xyz[0].device) for _ in range(frames)]
    ws = torch.zeros(2, dtype=torch.int64, device=xyz[0].device)     # the tile counter of rbsm_rpcf_ws
    steps = max(3, min(args.steps // 20, 20))

    def timed(fn):
        for _ in range(2):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    def rpcf():
        for f in range(frames):
            api.rbsm_rpcf(maps[f], xyz[f][0], xyz[f][1], xyz[f][2], k=k, vis=outs[f], workspace=ws)

    def rsmss():
        for f in range(frames):
            api.rsmss_filter(maps[f], xyz[f][0], xyz[f][1], xyz[f][2], vis=outs[f])

    ms = timed(rpcf)
    ms_rsmss = timed(rsmss)
    fps = lambda t: frames * n_frag / (t * 1e-3) / 1e9
    # the other filter sizes on the first 8 frames (one launch per frame)
    few = min(frames, 8)
    by_k = {}
    for kk in (1, 5, 7):
        def rpcf_k(kk=kk):
            for f in range(few):
                api.rbsm_rpcf(maps[f], xyz[f][0], xyz[f][1], xyz[f][2], k=kk, vis=outs[f], workspace=ws)
        by_k[str(kk)] = few * n_frag / (timed(rpcf_k) * 1e-3) / 1e9
    return {"metric": "Gfragments/s RPCF visibility (k x k PCF over RSMSS), same frames, one launch per frame "
                      "(rbsm_rpcf_ws)",
            "k": k, "value": fps(ms), "ms_per_step": ms, "launches_per_step": frames,
            "rsmss_same_launches": {"value": fps(ms_rsmss), "ms_per_step": ms_rsmss},
            "samples_per_fragment": k * k,
            "other_k_gfrag_s": {"frames": few, **by_k}}


def measure_light_pass(api, c5, maps, frames, n_frag, step_fn, stream):
    """The light pass on the GPU (rbsm_shadow_maps, one call for the
    frames): the frames' 8192^2 maps rasterised from their analytic
    occluders into the bench's own map buffers (the kernel writes the
    generator's bytes, checked here on one frame with rbsm_shadow_map),
    alone and followed by the visibility step: the per-frame pipeline with
    maps made on the device."""
    import torch
    occs = [api.DeviceOccluders(o.rects, o.rect_depth, o.spheres)
            for o in (c5.occluders(f) for f in range(frames))]
    size = c5.size
    probe = api.rbsm_shadow_map(occs[frames - 1], size, size, float(size))
    same = bool(torch.equal(probe, maps[frames - 1]))
    del probe
    steps = 5

    def light():
        api.rbsm_shadow_maps(occs, size, size, float(size), outs=maps)

    def pipeline():
        light()
        step_fn()

    def timed(fn):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    ms_light = timed(light)
    ms_pipe = timed(pipeline)
    texels = frames * size * size
    return {"light_pass": {"metric": "Gtexels/s shadow maps from analytic occluders (rbsm_shadow_maps)",
                           "value": texels / (ms_light * 1e-3) / 1e9, "ms_per_step": ms_light, "maps": frames,
                           "map": size, "occluders_per_map": len(c5.base.rects) + len(c5.base.spheres),
                           "bytes_equal_to_generator": same,
                           "write_gbs": texels * 4 / (ms_light * 1e-3) / 1e9},
            "frame_pipeline": {"metric": "Gfragments/s with the maps rasterised on the device in the step",
                               "value": frames * n_frag / (ms_pipe * 1e-3) / 1e9, "ms_per_step": ms_pipe}}


def measure_gbuffer(api, c5, maps, host, frames, n_frag, stream):
    """The depth-buffer path (rbsm_visibility_gbuffer): the frames' camera
    written as one depth plane and a 4 x 4 matrix each, p projected in the
    kernel; one call (one launch per frame) per step, mode BOTH."""
    import torch
    dev = maps[0].depth.device if hasattr(maps[0], "depth") else maps[0].device
    jobs = []
    for f in range(frames):
        d, m = c5.gbuffer(host[f]["xyz"][2].numpy())
        jobs.append(api.GBufferJob(maps[f], torch.from_numpy(d).to(dev), m, mode=3))
    steps = 10

    def run():
        api.rbsm_visibility_gbuffer(jobs)

    for _ in range(3):
        run()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return {"metric": "Gfragments/s visibility from depth buffers (p projected in the kernel), mode both",
            "value": frames * n_frag / (ms * 1e-3) / 1e9, "ms_per_step": ms, "launches_per_step": frames,
            "input_bytes_per_fragment": 4}


def measure_maxdist(api, maps, xyz, frames, n_frag, args, stream, shape, caps=(8, 16, 32, 64)):
    """The traversal cap as an accuracy / speed knob: for each cap, the
    batched C5 step's rate and the largest filtering error against the
    closed-form ramp on staircase edges of run lengths 8..64."""
    import numpy as np
    import torch
    from rbsm_scenes import shapes
    n = 512
    offs = [((a + 0.5) / 16, (b + 0.5) / 16) for a in range(16) for b in range(16)]
    stairs = []
    for run_len in (8, 16, 32, 64):
        depth = np.where(shapes.staircase_mask(n, run_len, 8, 40), shapes.BLOCKER, shapes.LIT).astype(np.float32)
        X, Y = shapes.fragment_grid(80, n - 80, 34, n - 34, offs)
        margin = (Y - 40) - (X - 8) / run_len
        keep = (np.abs(margin) < 2.0) & (np.abs(margin) > 1e-6)
        x, y = shapes.to_texcoords(X[keep], Y[keep], n, n)
        stairs.append((run_len, torch.from_numpy(depth).to(xyz[0].device),
                       [torch.from_numpy(np.ascontiguousarray(a)).to(xyz[0].device) for a in (x, y, np.ones_like(x))],
                       np.clip(1.0 + margin[keep], 0.0, 1.0)))
    out = []
    for cap in caps:
        jobs = [api.Job(k, xyz[k][0], xyz[k][1], xyz[k][2], mode=3) for k in range(frames)]
        b = api.Batch(maps, jobs, max_dist=cap, tile_threads=shape[0], ctas_per_sm=shape[1])
        for _ in range(3):
            api.rbsm_batch_run(b)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(20):
            api.rbsm_batch_run(b)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 20
        errs = {}
        for run_len, d, (xs, ys, zs), ramp in stairs:
            fil, _ = api.rsmss_filter(d, xs, ys, zs, max_dist=cap)
            errs[str(run_len)] = float(np.max(np.abs(fil.cpu().numpy().astype(np.float64) - ramp)))
        out.append({"max_dist": cap, "value": frames * n_frag / (ms * 1e-3) / 1e9, "ms_per_step": ms,
                    "staircase_filter_max_err_by_run_length": errs})
    return {"metric": "Gfragments/s (C5 step, mode both) and closed-form error per traversal cap", "caps": out}


# ----------------------------------------------------------- per config --

def oracle_rate(cases, threads, min_seconds):
    """The oracle on `threads` host threads over (depth, x, y, z) cases, both
    answers per fragment, cycling until min_seconds have passed."""
    import numpy as np
    from concurrent.futures import ThreadPoolExecutor
    from oracle import rbsm as orc
    done, k = 0, 0
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        while time.perf_counter() - t0 < min_seconds:
            depth, x, y, z = cases[k % len(cases)]
            k += 1
            n = min(x.shape[0], 2_000_000)
            bounds = np.linspace(0, n, threads + 1).astype(np.int64)

            def work(t):
                a, b = bounds[t], bounds[t + 1]
                for mode in (orc.MODE_SILHOUETTE, orc.MODE_FILTER):
                    orc.evaluate(depth, x[a:b], y[a:b], z[a:b], mode)
                return b - a

            done += sum(ex.map(work, range(threads)))
    return done / (time.perf_counter() - t0) / 1e9


def run_configs(args):
    """One JSON line per workload C1-C4 (the C5 line is the default run):
    the batched launch's rate and roofline fraction (autotuned shape, CUDA
    graph, map textures, mode BOTH), the oracle's rate on 1 and on all host
    threads (bounded samples of the same inputs) and, for C4, plain RSMSS
    against the guarded surrogate."""
    import numpy as np
    import torch
    from paper_1711_07793_gb300 import api
    from paper_1711_07793_gb300 import build as lib_build
    import rbsm_scenes as sc
    lib_build.build()
    device = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    peak, peak_kind = load_peaks()
    cores = os.cpu_count() or 1
    workloads = [("C1 256^2, 320x240", lambda: [sc.config1(0)]),
                 ("C2 2048^2, 1920x1080", lambda: [sc.config2(0)]),
                 ("C3 16 maps (512^2..4096^2) x 8 views (720p..4K), 4 lights", lambda: sc.Config3(0)),
                 ("C4 4096^2, 3840x2160", lambda: [sc.config4(0)])]
    only = [o.strip().upper() for o in args.only.split(",") if o.strip()]
    for name, make in workloads:
        if only and name.split()[0] not in only:
            continue
        w = make()
        if isinstance(w, sc.Config3):
            maps_np = w.maps
            parts = [(j.map_index, j.x, j.y, j.z) for j in w.jobs]
        else:
            maps_np = [f.depth for f in w]
            parts = [(0, f.x, f.y, f.z) for f in w]
        dmaps = [torch.from_numpy(m).to(device) for m in maps_np]
        texs = [api.MapTexture(m) for m in dmaps]
        planes = [(k, *(torch.from_numpy(np.ascontiguousarray(a)).to(device) for a in (x, y, z)))
                  for k, x, y, z in parts]
        jobs = [api.Job(k, x, y, z, mode=3) for k, x, y, z in planes]
        batch = api.Batch(texs, jobs)
        tuning = None
        if args.autotune == "on":
            tuning = api.rbsm_batch_autotune(batch, repeats=3, cache=None)
        graph = api.BatchGraph(batch)
        for _ in range(5):
            graph.launch()
        steps = 50
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            graph.launch()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        n = sum(x.shape[0] for _, x, _, _ in parts)
        texels = sum(unique_texels(x, y, maps_np[k].shape[0]) for k, x, y, _ in parts)
        nbytes = BYTES_PER_FRAGMENT * n + BYTES_PER_TEXEL * texels
        cases = [(maps_np[k], x, y, z) for k, x, y, z in parts]
        line = {"workload": name, "fragments": n, "unit": UNIT,
                "gpu": {"value": n / (ms * 1e-3) / 1e9, "ms_per_launch": ms,
                        "hbm_frac": nbytes / (ms * 1e-3) / 1e9 / peak, "peak_gbs": peak,
                        "launch": {"tile_threads": batch.desc.tile_threads, "ctas_per_sm": batch.desc.ctas_per_sm,
                                   "chunk_tiles": batch.desc.chunk_tiles, "flags": batch.desc.flags},
                        "autotune": tuning}}
        if not args.skip_cpu:
            line["cpu_oracle"] = {"threads_1": oracle_rate(cases, 1, 3.0),
                                  "threads_all": oracle_rate(cases, cores, 3.0), "cores": cores}
        if name.startswith("C4") and not args.skip_learned:
            line["learned"] = compare_learned(api, texs, [torch.stack([p[1], p[2], p[3]]) for p in planes],
                                              1, n, args, stream)
        graph.close()
        for t in texs:
            t.close()
        print(json.dumps(line), flush=True)


# -------------------------------------------------------------- reference --

def run_reference(args, rank, world):
    """The oracle as it stands on the host cores: each step is one frame of
    the workload (every fragment, both visibility functions)."""
    if rank != 0:
        return
    import numpy as np
    from concurrent.futures import ThreadPoolExecutor
    from oracle import rbsm as orc
    import rbsm_scenes as sc
    c5 = sc.Config5(args.seed)
    fr = c5.frame(0)
    cores = os.cpu_count() or 1
    bounds = np.linspace(0, fr.n, cores + 1).astype(np.int64)

    def work(k):
        a, b = bounds[k], bounds[k + 1]
        for mode in (orc.MODE_SILHOUETTE, orc.MODE_FILTER):
            orc.evaluate(fr.depth, fr.x[a:b], fr.y[a:b], fr.z[a:b], mode)

    with ThreadPoolExecutor(max_workers=cores) as ex:
        for _ in range(args.warmup):
            list(ex.map(work, range(cores)))
        t0 = time.perf_counter()
        for _ in range(args.steps):
            list(ex.map(work, range(cores)))
        dt = time.perf_counter() - t0
    ms = dt * 1e3 / args.steps
    value = fr.n / (ms * 1e-3) / 1e9
    sample = "frame 0 of 32 (3840x2160 fragments, 8192^2 map) per step, both visibility functions"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "C5: 32 frames x 3840x2160 fragments, 8192^2 fp32 maps, moving light, "
                                   "silhouette + RSMSS per fragment", "sampled": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main(argv=None):
    args = parse_args(argv)
    rank, world, local_rank = dist_env()
    if world != args.gpus and world == 1 and args.gpus > 1:
        raise SystemExit("--gpus %d needs torchrun with %d processes" % (args.gpus, args.gpus))
    if args.warmup < 0 or args.steps < 1:
        raise SystemExit("--steps must be >= 1 and --warmup >= 0")
    if args.configs:
        run_configs(args)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
