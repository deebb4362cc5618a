"""Benchmark of the CrowdSplat crowd-synthesis hot path on GB300.

One step = one animated frame of the paper-scale crowd: new joint poses for
every instance (cs_set_instances) followed by cs_render (forward kinematics,
distance LoD + cull, LBS + EWA projection + SH colour, tile binning, depth
and tile radix sorts, compositing) at 1920x1080.  Workload: 14 procedural
templates x 65,536 Gaussians (SH degree 3), 3,500 instances on a jittered
grid, 3 distance LoD levels (100/25/6 %, 10 m / 30 m), camera 3 m from the
first row (synthetic stand-ins for the paper's avatars and motions).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores instead (a bounded pixel sample of the same frame).
"""
from __future__ import annotations

import argparse
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "crowd FPS @3,500 inst 1080p; learned vs plain LoD FPS at equal PSNR"
UNIT = "frames/s"
PAPER_FPS = 31.0  # RTX4090, resolution not stated: context only, not this workload


def aggregate(ms_local: float, steps: int, world: int, dist=None, device=None):
    """Max of the per-rank timed milliseconds over ranks and the whole-job
    throughput: all ranks' steps divided by the slowest rank's time."""
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * steps / (ms_max / 1e3)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=float(d["hbm_gbs"]), src="measured", sm_max_mhz=float(d.get("sm_max_mhz", 2070)))
    return dict(hbm_gbs=6800.0, src="fallback", sm_max_mhz=2070.0)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic bytes per stage (per frame): the bytes each stage must move at
# least, from the frame statistics (splats, live splats, pairs, passes)
# ---------------------------------------------------------------------------

def stage_bytes(st, n_inst, tpl_bytes, pixels):
    S, P = st["splats"], st["pairs"]
    live = st.get("splats_live", S) or S
    V = st["instances_visible"]
    # radix passes: ceil(bits / 9) (digits of at most 9 bits)
    passes_depth = max(1, math.ceil(max(1, st.get("depth_key_bits", 32)) / 9))
    tile_bits = max(1, math.ceil(math.log2(max(2, st["tiles_x"] * st["tiles_y"]))))
    passes_tile = math.ceil(tile_bits / 9)
    return {
        "fk": n_inst * (4 + 72 * 4 + 24 * 48),
        "cull_lod": n_inst * (4 + 48 + 48 + 16 + 4),
        # template attributes once (shared, L2-resident across a group) +
        # per-instance transforms + per-splat key and bin word + the 48 B
        # record of every live splat
        "skin_project": tpl_bytes + V * (24 * 48 + 64) + S * (4 + 4) + live * 48,
        # per pass: keys read by the histogram, key+value read and written;
        # the first pass reads no values (they are the indices), the last
        # writes the bin words in depth order (gathered)
        "depth_sort": S * (passes_depth * (4 + 8 + 8) - 4 + 8),
        # block sums of the pair counts: bin words read; emission (with the
        # scan's down-sweep): bin words and order read, 6 B per pair written
        "pair_emit": S * (4 + 4 + 4) + P * 6,
        "tile_sort": P * passes_tile * (2 + 6 + 6),
        "tile_ranges": P * 2 * 2,
        # each pair: splat id + 48 B record; each pixel: 16 B written
        "blend": P * (4 + 48) + pixels * 16,
    }


def workload_name(sc):
    t = sc.templates[0]
    return (f"crowd_{len(sc.templates)}x{int(t.n)}g_sh{int(t.sh_degree)}_{sc.instances.n}inst_"
            f"{sc.camera.width}x{sc.camera.height}_lod{len(sc.lod.fractions)}_animated")


def bench_config(sc, args, world=1):
    """The config object of both arms' JSON lines (same keys)."""
    return {"workload": workload_name(sc), "templates": len(sc.templates),
            "gaussians_per_template": int(sc.templates[0].n), "sh_degree": int(sc.templates[0].sh_degree),
            "instances": int(sc.instances.n), "width": sc.camera.width, "height": sc.camera.height,
            "lod": {"thresholds_m": [float(x) for x in sc.lod.thresholds],
                    "fractions": [round(float(x), 4) for x in sc.lod.fractions]},
            "l2": "inputs larger than L2 (templates 231 MB, splat records > 1 GB per frame)",
            "parallelism": f"replicas{world}" if world > 1 else "single",
            "template_storage": args.storage}


def project_scope_bytes(st, tpl_bytes):
    """Algorithmic bytes of the fused skinning + projection kernel as the
    hot-path scope table counts them: the shared templates read once, the
    24 skinning transforms (48 B each) of every visible instance, and one
    40-byte splat record written per Gaussian-instance."""
    return tpl_bytes + st["instances_visible"] * 24 * 48 + st["splats"] * 40


def profile_figures():
    """Per-kernel figures taken from the committed ncu summaries (DRAM
    traffic per launch, pipe utilisation); an entry is null once its kernel
    has changed since the capture."""
    p = os.path.join(ROOT, "profiles", "ncu_metrics.json")
    return json.load(open(p)) if os.path.exists(p) else {}


def template_bytes(sc, storage="fp32"):
    """Device bytes of the uploaded templates (the library's layout)."""
    tot = 0
    for t in sc.templates:
        k = (t.sh_degree + 1) ** 2
        if storage == "bf16":
            tot += t.means.shape[0] * (16 + 16 + ((k * 3 + 7) // 8) * 16)
        else:
            tot += t.means.shape[0] * (16 + 16 + 8 + 16 + 4 + ((k * 3 + 3) // 4) * 16)
    return tot


# ---------------------------------------------------------------------------
# oracle on the host cores (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------

def oracle_sample(os_, sc, stride=16, offset=(0, 0)):
    """One bounded sample of the oracle's frame: the FP64 projection of
    every instance (a one-pixel render) and the composite of every
    `stride`-th pixel in x and y from `offset` (1/stride^2 of the pixels).
    Returns (seconds the sample took, full-frame seconds extrapolated as
    projection + stride^2 x the lattice's compositing time, details)."""
    import oracle
    W, H = sc.camera.width, sc.camera.height
    t0 = time.perf_counter()
    oracle.render(os_, lattice=(W // 2, H // 2, 1, 1, 1, 1))
    t_proj = time.perf_counter() - t0
    ox, oy = offset
    nx, ny = (W - ox + stride - 1) // stride, (H - oy + stride - 1) // stride
    t0 = time.perf_counter()
    oracle.render(os_, lattice=(ox, oy, stride, stride, nx, ny))
    t_lat = time.perf_counter() - t0
    full = t_proj + max(t_lat - t_proj, 0.0) * (W * H) / (nx * ny)
    return t_proj + t_lat, full, dict(project_s=round(t_proj, 3), lattice_s=round(t_lat, 3), stride=stride,
                                      lattice_px=nx * ny, cores=oracle.num_threads())


def run_reference(args, sc, rank, world):
    """The reference arm: the FP64 CPU oracle (there is no reference code;
    the reference is the paper's text).  Each step is one bounded sample of
    the frame (projection of all instances + one 1/256 pixel lattice, the
    lattice offset moving from step to step); ms_per_step is the measured
    wall time of a step, value the median full-frame rate the samples
    extrapolate to.  Rank 0 only."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    os_ = oracle.OracleScene(sc)
    st = args.oracle_stride
    for w in range(min(args.warmup, 1)):  # the oracle has no warm state: one untimed sample
        oracle_sample(os_, sc, st, (w % st, w % st))
    wall, full, info = [], [], {}
    for k in range(args.steps):
        wt, ft, info = oracle_sample(os_, sc, st, ((5 * k) % st, (11 * k) % st))
        wall.append(wt)
        full.append(ft)
    fps = 1.0 / statistics.median(full)
    sample = (f"per step: FP64 projection of all {sc.instances.n} instances + every {st}th pixel in x and y "
              f"({info['lattice_px']} px, offset moving per step); full frame = projection + {st}^2 x lattice "
              f"compositing time (median over steps {statistics.median(full):.1f} s)")
    line = {"impl": "reference", "metric": METRIC, "value": fps, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(wall) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(sc, args, world),
            "cpu_baseline": {"value": fps, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
                             "sample": sample, "frame_s_extrapolated": round(statistics.median(full), 2),
                             "sample_s": round(statistics.mean(wall), 3)},
            "e2e": {"value": fps, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_ours(args, sc, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_2501_17792_gb300 import binding, build
    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    storage = binding.CS_STORE_BF16 if args.storage == "bf16" else binding.CS_STORE_FP32
    r = binding.Renderer(device=local_rank, stream=stream, stage_timing=True, template_storage=storage)
    r.upload_templates(sc.templates)
    r.set_lod(sc.lod)
    n = sc.instances.n
    from paper_2501_17792_gb300 import scene as S
    frames = args.warmup + args.steps
    # per-frame poses resident in HBM before the timed region (animated crowd)
    poses = torch.stack([torch.from_numpy(S.random_poses(100 + 1000 * rank + f, n)) for f in range(frames)]).to(dev)
    tid = torch.from_numpy(sc.instances.template_id).to(dev)
    root = torch.from_numpy(sc.instances.root.reshape(n, 12)).to(dev)
    out = torch.empty((sc.camera.height, sc.camera.width, 4), dtype=torch.float32, device=dev)
    torch.cuda.synchronize()

    def step(f, stats=False):
        with torch.cuda.stream(stream):
            r.set_instances(tid, root, poses[f])
            return r.render(sc.camera, out=out, stats=stats)

    _, st0 = step(0, stats=True)
    for f in range(args.warmup):
        step(f)
    torch.cuda.synchronize()
    r.stage_times(average=True)  # restart the stage means at the timed region
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local_rank) if rank == 0 else None
    if clk:
        clk.start()
        time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for f in range(args.warmup, frames):
        step(f)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_total = e0.elapsed_time(e1)
    stage_ms, stage_frames = r.stage_times(average=True)
    clocks = clk.stop() if clk else None
    ms_max, value = aggregate(ms_total, args.steps, world, dist, dev)
    if world > 1:
        dist.barrier()
    ms_per_step = ms_max / args.steps

    # end to end through the C ABI with host buffers: every step's inputs
    # (template ids, roots, that step's poses) resident in pinned host memory
    # before the timed region, copied host -> device inside it; image out
    h_img = torch.empty((sc.camera.height, sc.camera.width, 4), dtype=torch.float32).pin_memory()
    h_tid = torch.from_numpy(sc.instances.template_id.copy()).pin_memory()
    h_root = torch.from_numpy(sc.instances.root.reshape(n, 12).copy()).pin_memory()
    h_poses = [torch.from_numpy(S.random_poses(100 + 1000 * rank + f, n)).pin_memory()
               for f in range(args.e2e_steps + 2)]
    import ctypes as C
    cam = binding.camera_struct(sc.camera)
    L = binding.load()

    def e2e_step(f):
        rc = L.cs_set_instances(r.h, n, h_tid.data_ptr(), h_root.data_ptr(), h_poses[f].data_ptr(), 0)
        assert rc == 0, L.cs_last_error(r.h)
        rc = L.cs_render_to_host(r.h, C.byref(cam), h_img.data_ptr(), None)
        assert rc == 0, L.cs_last_error(r.h)

    for f in range(2):
        e2e_step(f)
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for f in range(args.e2e_steps):
        e2e_step(f + 2)
    _, e2e_value = aggregate((time.perf_counter() - t0) * 1e3, args.e2e_steps, world, dist, dev)
    h2d = n * (4 + 48 + 24 * 3 * 4)
    d2h = sc.camera.width * sc.camera.height * 16

    if rank != 0:
        r.close()
        return
    pk = peaks()
    pixels = sc.camera.width * sc.camera.height
    tpl_b = template_bytes(sc, args.storage)
    sb = stage_bytes(st0, n, tpl_b, pixels)
    prof = profile_figures()
    stages = {}
    for name, ms in stage_ms.items():
        if name not in sb:
            stages[name] = {"ms": round(ms, 4)}
            continue
        gbs = sb[name] / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
        stages[name] = {"ms": round(ms, 4), "algo_bytes": int(sb[name]), "GB/s": round(gbs, 1),
                        "frac_of_measured_hbm": round(gbs / pk["hbm_gbs"], 4)}
    if "blend" in stages:
        # compositing is bound by FP32 issue and the exp unit, not DRAM: its
        # fraction is the FMA-pipe utilisation of the committed capture
        bl = prof.get("k_blend", {})
        stages["blend"] = {"ms": stages["blend"]["ms"], "bound": "fp32 issue",
                           "fp32_pipe_frac": bl.get("fma_pipe_frac"), "source": bl.get("source")}
    # the roofline kernel: k_project, the largest single kernel of the frame,
    # with the scope table's algorithmic bytes (templates once, transforms,
    # 40 B per splat record); its measured DRAM traffic is the committed
    # one-pass capture's, null once the kernel has changed since
    top_ms = stage_ms["skin_project"]
    algo = project_scope_bytes(st0, tpl_b)
    achieved = algo / (top_ms * 1e-3) / 1e9
    kp = prof.get("k_project", {})
    traffic = kp.get("dram_bytes_per_launch")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.storage == "fp32" else "f32 compute, bf16/fp16 template storage", "data": "synthetic",
        "config": bench_config(sc, args, world),
        "frame": {"visible_instances": st0["instances_visible"], "per_level": st0["instances_per_level"][:3],
                  "splats": st0["splats"], "pairs": st0["pairs"],
                  "gaussians_per_s": st0["splats"] * value},
        "stages": stages,
        "roofline": {"bound": "hbm", "kernel": "k_project", "achieved": round(achieved, 1), "peak": pk["hbm_gbs"],
                     "unit": "GB/s", "frac": round(achieved / pk["hbm_gbs"], 4), "traffic": traffic,
                     "algorithmic_bytes": int(algo),
                     "traffic_over_algorithmic": round(traffic / algo, 3) if traffic else None,
                     "ms": round(top_ms, 4),
                     "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if pk["src"] == "measured" else "fallback"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        # the statistics frame st0 runs one kernel more than a timed frame
        # (the live-splat count behind splats_live)
        "gpu_launches": (int(st0["kernel_launches"]) - (1 if st0["splats"] > 0 else 0)) * args.steps,
        "clocks": clocks,
        "paper_context": {"fps": PAPER_FPS, "hardware": "RTX4090 + i9-13900", "note": "different workload, context only"},
    }
    r.close()
    del poses, out
    torch.cuda.empty_cache()
    if not args.no_learned_lod:
        line["learned_lod"] = learned_lod_summary(learned_lod_eval(args, reduced=True))
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        os_ = oracle.OracleScene(sc)
        wall, full, t0, k = [], [], time.perf_counter(), 0
        st = args.oracle_stride
        while k < 3 or (time.perf_counter() - t0 < args.cpu_baseline_s and k < st * st):
            wt, ft, info = oracle_sample(os_, sc, st, ((5 * k) % st, (11 * k) % st))
            wall.append(wt)
            full.append(ft)
            k += 1
        line["cpu_baseline"] = {"value": 1.0 / statistics.median(full), "unit": UNIT, "cores": info["cores"],
                                "kind": "oracle",
                                "sample": (f"{k} samples, each the FP64 projection of all {n} instances + every "
                                           f"{st}th pixel in x and y ({info['lattice_px']} px, offset moving per "
                                           f"sample); full frame = projection + {st}^2 x lattice compositing time "
                                           f"(median {statistics.median(full):.1f} s); {sum(wall):.1f} s of CPU "
                                           f"wall time"),
                                "frame_s_extrapolated": round(statistics.median(full), 2)}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# CrowdSplat Table 1 / Table 2 sweep (1280x720, one template size per row)
# ---------------------------------------------------------------------------

PAPER_TABLE2 = {  # Table 2 FPS on RTX4090, (w/o motion, w/ motion); context only
    202738: {1: (728, 617), 100: (50, 18.2), 400: (22.2, None)},
    12661: {1: (1612, 1370), 100: (586, 312), 400: (251, 76), 1000: (125, 34), 5000: (10.3, 6.1)},
    3176: {1: (1703, 1347), 100: (1240, 804), 400: (673, 298), 1000: (275, 121), 5000: (38.6, 23.2)},
}
PAPER_TABLE1 = {  # Table 1 GPU memory MiB on RTX4090, (plain, shared); context only
    202738: {1: (651, 651), 100: (7929, 7075)},
    12661: {1: (567, 567), 100: (1005, 953), 400: (2335, 2121), 1000: (5127, 4593), 5000: (21340, 19625)},
    3176: {1: (557, 557), 100: (675, 639), 400: (993, 937), 1000: (1695, 1541), 5000: (5995, 5329)},
}


def run_sweep(args):
    """FPS without motion (same poses every frame) and with motion (new poses
    every frame), and device memory, for one template of each paper size
    duplicated to the paper's character counts on a 1.2 m grid starting 3 m
    from the camera, 1280x720, full detail (the paper's rows use a single
    template size).  Memory: the library always shares template attributes;
    the unshared figure adds a template copy per extra character.  One more
    row per template size measures the plain (unshared) layout itself at the
    largest character count the library can hold as separate templates
    (CS_MAX_TEMPLATES = 63): every character its own uploaded copy."""
    import torch
    from paper_2501_17792_gb300 import binding, build
    from paper_2501_17792_gb300 import scene as S
    build.build()
    cam = S.look_camera((0.0, 1.6, 0.0), 10.0, 1280, 720)
    rows_out = []

    def measure(tpls, tid, root, count):
        r = binding.Renderer(device=0)
        r.upload_templates(tpls)
        out = torch.empty((720, 1280, 4), dtype=torch.float32, device="cuda")
        fps = {}
        dtid = torch.from_numpy(np.ascontiguousarray(tid, np.int32)).cuda()
        droot = torch.from_numpy(np.ascontiguousarray(root.reshape(count, 12))).cuda()
        for motion in (False, True):
            poses = [torch.from_numpy(S.random_poses(100 + (f if motion else 0), count)).cuda()
                     for f in range(args.steps + args.warmup)]
            for f in range(args.warmup):
                r.set_instances(dtid, droot, poses[f])
                r.render(cam, out=out)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for f in range(args.warmup, args.warmup + args.steps):
                r.set_instances(dtid, droot, poses[f])
                r.render(cam, out=out)
            e1.record()
            torch.cuda.synchronize()
            fps["motion" if motion else "static"] = args.steps / (e0.elapsed_time(e1) / 1e3)
        _, st = r.render(cam, out=out, stats=True)
        mem = r.memory_stats()
        r.close()
        return fps, st, (mem["total_bytes"] + out.numel() * 4) / 2 ** 20

    for n_gauss, cells in PAPER_TABLE2.items():
        tpl = S.make_template(1000, n_gauss, 3)
        tbytes = template_bytes(S.Scene([tpl], None, cam, S.single_lod(), ""))
        for count in list(cells) + [63]:
            cols = min(50, int(math.ceil(math.sqrt(count))))
            nrows = int(math.ceil(count / cols))
            inst = S.crowd_instances(1, cols, nrows)
            tid, root = inst.template_id[:count], inst.root[:count]
            fps, st, shared_mib = measure([tpl], tid, root, count)
            row = dict(gaussians=n_gauss, characters=count, fps_static=round(fps["static"], 1),
                       fps_motion=round(fps["motion"], 1), splats=st["splats"], pairs=st["pairs"],
                       mem_shared_mib=round(shared_mib, 1),
                       mem_unshared_mib=round(shared_mib + (count - 1) * tbytes / 2 ** 20, 1),
                       paper_fps=PAPER_TABLE2[n_gauss].get(count), paper_mib=PAPER_TABLE1[n_gauss].get(count))
            if count == 63:
                # the plain layout measured: character k renders its own copy k
                pfps, pst, plain_mib = measure([tpl] * count, np.arange(count, dtype=np.int32), root, count)
                row.update(plain_measured=dict(fps_static=round(pfps["static"], 1),
                                               fps_motion=round(pfps["motion"], 1),
                                               mem_mib=round(plain_mib, 1), splats=pst["splats"],
                                               pairs=pst["pairs"]))
            rows_out.append(row)
            print(json.dumps(row), flush=True)
    return rows_out


def _fps(r, cam, tid, root, poses, out, warmup, steps):
    """Frames per second of animated frames (new device-resident poses per
    frame), CUDA events on the default stream."""
    import torch
    for f in range(warmup):
        r.set_instances(tid, root, poses[f % len(poses)])
        r.render(cam, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for f in range(steps):
        r.set_instances(tid, root, poses[(warmup + f) % len(poses)])
        r.render(cam, out=out)
    e1.record()
    torch.cuda.synchronize()
    return steps / (e0.elapsed_time(e1) / 1e3)


def learned_lod_eval(args, reduced=False):
    """Ranked (learned) LoD against the distance LoD with prefix subsets, at
    10,000 instances and 3840x2160.  PSNR against the full-detail frame is
    the mean over `frames` animated frames (different poses); the learned
    ranking is timed at the smallest budget whose mean PSNR matches the
    distance LoD's.  Returns the JSON object of the comparison."""
    import numpy as np
    import torch
    from paper_2501_17792_gb300 import binding, build
    from paper_2501_17792_gb300 import lod as LOD
    from paper_2501_17792_gb300 import scene as S
    build.build()
    small = args.small
    W, H = (960, 540) if small else (3840, 2160)
    cols, rows = (30, 30) if small else (100, 100)
    n_tpl, n_g = (4, 16384) if small else (14, 65536)
    views = 8 if small else 34
    frames = 5
    t_all = time.time()
    tpls = [S.make_template(1000 + t, n_g, 3) for t in range(n_tpl)]
    cam = S.look_camera((0.0, 1.6, 0.0), 10.0, W, H)
    r = binding.Renderer(device=0)
    r.upload_templates(tpls)
    sizes = r.template_sizes
    # 1. training data: contributions of every Gaussian per distance band
    torch.cuda.synchronize()
    t0 = time.time()
    feat = r.lod_features()
    contrib = LOD.collect_contributions(r, n_tpl, cam, views_per_band=views, instances_per_view=100, seed=5)
    targets = r.lod_targets(contrib)
    torch.cuda.synchronize()
    t_collect = time.time() - t0
    # 2. the ranking MLP
    t0 = time.time()
    mlp = binding.Mlp(device=0, seed=1)
    hist = LOD.train_ranker(mlp, feat, targets, steps=args.lod_steps, log_every=max(1, args.lod_steps // 5))
    scores = LOD.band_scores(mlp, feat, 3)
    torch.cuda.synchronize()
    t_train = time.time() - t0

    def spearman(a, b):
        ra = np.argsort(np.argsort(a)).astype(np.float64)
        rb = np.argsort(np.argsort(b)).astype(np.float64)
        return float(np.corrcoef(ra, rb)[0, 1])
    tg = targets.cpu().numpy()
    sc_np = scores.cpu().numpy()
    rho = [round(spearman(sc_np[b], tg[b]), 4) for b in range(3)]

    base = S.paper_lod()
    f = np.asarray(base.fractions, np.float64)

    def lod_cfg(scale=1.0, expo=0.5):
        fr = np.array([1.0, f[1] * scale, f[2] * scale])
        return S.LodConfig(thresholds=base.thresholds, fractions=fr.astype(np.float32),
                           scale_mult=(fr ** -expo).astype(np.float32)), fr

    def apply(lod, subs):
        LOD.clear_subsets(r, n_tpl)
        r.set_lod(lod)
        if subs is not None:
            LOD.apply_subsets(r, subs)

    r2 = None  # a second renderer holding templates stored in learned order

    def prefix_renderer(fr):
        """r2 with every template re-uploaded in the nested learned order for
        level fractions fr, so each level renders a prefix (no gather)."""
        nonlocal r2
        if r2 is None:
            r2 = binding.Renderer(device=0)
        orders = LOD.prefix_orders(scores, fr, sizes)
        r2.upload_templates([LOD.permute_template(tp, o) for tp, o in zip(tpls, orders)])
        return r2

    def prepare(cfg):
        """Renderer of a config (name, lod, subsets, prefix-order fractions)."""
        name, lod, subs, pfr = cfg
        rr = prefix_renderer(pfr) if pfr is not None else r
        if pfr is None:
            LOD.clear_subsets(rr, n_tpl)
        rr.set_lod(lod)
        if subs is not None:
            LOD.apply_subsets(rr, subs)
        return rr

    def mean_psnr(inst, pose_list, configs):
        """{name: (mean PSNR vs full detail over the frames, splats of frame 0)}."""
        tid = torch.from_numpy(inst.template_id).cuda()
        root = torch.from_numpy(inst.root.reshape(-1, 12)).cuda()
        refs = []
        apply(S.single_lod(), None)
        for pose in pose_list:
            r.set_instances(tid, root, pose)
            img, st = r.render(cam, stats=True)
            refs.append(img)
        res = {}
        img = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
        for cfg in configs:
            rr = prepare(cfg)
            ps, spl = [], None
            for pose, ref in zip(pose_list, refs):
                rr.set_instances(tid, root, pose)
                _, st2 = rr.render(cam, out=img, stats=True)
                ps.append(LOD.psnr(img, ref))
                spl = st2["splats"] if spl is None else spl
            res[cfg[0]] = (float(np.mean(ps)), int(spl))
        del refs
        return res, int(st["splats"])

    # 3. scale-multiplier exponent, tuned on a training crowd (other layout
    # and poses) for both methods
    tr_inst = S.crowd_instances(n_tpl, cols, rows, layout_seed=8, pose_seed=300)
    expos = (0.0, 0.25, 0.5)
    cfgs = []
    for e in expos:
        lod, fr = lod_cfg(1.0, e)
        cfgs.append((f"plain_{e}", lod, None, None))
        cfgs.append((f"learned_{e}", lod, LOD.ranked_subsets(r, scores, fr, sizes, levels=(1, 2)), None))
    tune, _ = mean_psnr(tr_inst, [torch.from_numpy(tr_inst.pose).cuda()], cfgs)
    e_plain = max(expos, key=lambda e: tune[f"plain_{e}"][0])
    e_learn = max(expos, key=lambda e: tune[f"learned_{e}"][0])

    # 4. evaluation crowd: PSNR vs full detail (mean over frames), budgets, FPS
    inst = S.crowd_instances(n_tpl, cols, rows, layout_seed=7, pose_seed=100)
    n = inst.n
    poses = [torch.from_numpy(S.random_poses(100 + k, n)).cuda() for k in range(max(frames, args.warmup + args.steps))]
    tid = torch.from_numpy(inst.template_id).cuda()
    root = torch.from_numpy(inst.root.reshape(n, 12)).cuda()
    lod_plain, _ = lod_cfg(1.0, 0.5)
    lod_plain_t, _ = lod_cfg(1.0, e_plain)
    scales = ((1.0, 0.5, 0.25, 0.18, 0.12, 0.08, 0.05, 0.03) if reduced else
              (1.0, 0.7, 0.5, 0.35, 0.25, 0.18, 0.12, 0.08, 0.05, 0.03, 0.02))
    cfgs = [("plain", lod_plain, None, None), ("plain_tuned", lod_plain_t, None, None)]
    learned = {}
    for s_ in scales:
        lod, fr = lod_cfg(s_, e_learn)
        learned[s_] = (f"learned_{s_}", lod, LOD.ranked_subsets(r, scores, fr, sizes, levels=(1, 2)), None)
        cfgs.append(learned[s_])
    # the same ranking with nested levels stored as template prefixes
    prefix = {s_: (f"prefix_{s_}", lod_cfg(s_, e_learn)[0], None, lod_cfg(s_, e_learn)[1]) for s_ in scales}
    cfgs.extend(prefix.values())
    if not reduced:
        cfgs.append(("direct", lod_cfg(1.0, e_learn)[0],
                     LOD.ranked_subsets(r, contrib, lod_cfg(1.0)[1], sizes, levels=(1, 2)), None))
    res, full_splats = mean_psnr(inst, poses[:frames], cfgs)

    def equal_budget(kind, target_psnr):
        eq = [s_ for s_ in scales if res[f"{kind}_{s_}"][0] >= target_psnr]
        return min(eq) if eq else None

    s_eq = equal_budget("learned", res["plain"][0])
    s_eq_t = equal_budget("learned", res["plain_tuned"][0])
    p_eq = equal_budget("prefix", res["plain"][0])
    out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")

    def fps_of(cfg):
        rr = prepare(cfg)
        return _fps(rr, cam, tid, root, poses, out, args.warmup, args.steps)

    fps_full = fps_of(("full", S.single_lod(), None, None))
    fps_plain = fps_of(cfgs[0])
    fps_plain_t = fps_of(cfgs[1])
    fps_same = fps_of(learned[1.0])
    fps_eq = fps_of(learned[s_eq]) if s_eq is not None else None
    fps_eq_t = fps_of(learned[s_eq_t]) if s_eq_t is not None else None
    fps_pre_same = fps_of(prefix[1.0])
    fps_pre_eq = fps_of(prefix[p_eq]) if p_eq is not None else None
    r.close()
    if r2 is not None:
        r2.close()
    mlp.close()
    rd = lambda x: round(x, 3)  # noqa: E731
    line = {
        "metric": "learned vs distance LoD: FPS at equal PSNR vs full detail",
        "value": round(fps_eq, 2) if fps_eq else None, "unit": "frames/s",
        "higher_is_better": True, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "dtype": "f32 render, bf16 MLP", "data": "synthetic",
        "config": {"workload": f"crowd_{n_tpl}x{n_g}g_sh3_{n}inst_{W}x{H}_lod3_animated",
                   "bands_m": [10, 30], "fractions": [1.0, 0.25, 0.06],
                   "psnr": f"mean over {frames} animated frames (poses from seeds 100..{99 + frames}) "
                           "against the full-detail frame of the same poses"},
        "distance_lod": {"fps": round(fps_plain, 2), "psnr_db": rd(res["plain"][0]),
                         "splats": res["plain"][1], "scale_mult_exponent": 0.5},
        "learned_lod_equal_psnr": {"budget_scale": s_eq, "fps": round(fps_eq, 2) if fps_eq else None,
                                   "psnr_db": rd(res[f"learned_{s_eq}"][0]) if s_eq else None,
                                   "splats": res[f"learned_{s_eq}"][1] if s_eq else None},
        "speedup_at_equal_psnr": round(fps_eq / fps_plain, 3) if fps_eq else None,
        "learned_prefix_equal_psnr": {"budget_scale": p_eq, "fps": round(fps_pre_eq, 2) if fps_pre_eq else None,
                                      "psnr_db": rd(res[f"prefix_{p_eq}"][0]) if p_eq else None,
                                      "splats": res[f"prefix_{p_eq}"][1] if p_eq else None,
                                      "speedup": round(fps_pre_eq / fps_plain, 3) if fps_pre_eq else None,
                                      "same_budget_fps": round(fps_pre_same, 2),
                                      "same_budget_psnr_db": rd(res["prefix_1.0"][0]),
                                      "note": "levels nested and re-uploaded as template prefixes (no gather)"},
        "learned_lod_same_budget": {"fps": round(fps_same, 2), "psnr_db": rd(res["learned_1.0"][0]),
                                    "splats": res["learned_1.0"][1], "scale_mult_exponent": e_learn},
        "vs_tuned_distance_lod": {"fps": round(fps_plain_t, 2), "psnr_db": rd(res["plain_tuned"][0]),
                                  "splats": res["plain_tuned"][1], "tuned_exponent": e_plain,
                                  "learned_budget_scale": s_eq_t,
                                  "learned_fps": round(fps_eq_t, 2) if fps_eq_t else None,
                                  "speedup": round(fps_eq_t / fps_plain_t, 3) if fps_eq_t else None},
        "learned_psnr_by_budget": {str(s_): rd(res[f"learned_{s_}"][0]) for s_ in scales},
        "prefix_psnr_by_budget": {str(s_): rd(res[f"prefix_{s_}"][0]) for s_ in scales},
        "learned_splats_by_budget": {str(s_): res[f"learned_{s_}"][1] for s_ in scales},
        "full_detail": {"fps": round(fps_full, 2), "splats": full_splats},
        "training": {"instance_views": 3 * views * 100, "rows": int(targets.numel()), "steps": args.lod_steps,
                     "loss": [(int(a), round(b, 4)) for a, b in hist], "spearman_by_band": rho,
                     "collect_s": round(t_collect, 2), "train_s": round(t_train, 2),
                     "cost_s": round(t_collect + t_train, 2)},
        "tuning_psnr_db": {k: rd(v[0]) for k, v in tune.items()},
        "wall_s": round(time.time() - t_all, 1),
    }
    if "direct" in res:
        line["direct_contribution_ranking_psnr_db"] = rd(res["direct"][0])
    return line


def learned_lod_summary(d):
    """The part of the learned-LoD comparison the default bench line carries."""
    keys = ("config", "distance_lod", "learned_lod_equal_psnr", "speedup_at_equal_psnr", "learned_prefix_equal_psnr",
            "learned_lod_same_budget", "vs_tuned_distance_lod", "full_detail", "wall_s")
    out = {k: d[k] for k in keys}
    out["training_cost_s"] = d["training"]["cost_s"]
    out["training"] = {k: d["training"][k] for k in ("instance_views", "rows", "steps", "spearman_by_band",
                                                     "collect_s", "train_s")}
    return out


def run_learned_lod(args):
    line = learned_lod_eval(args, reduced=False)
    print(json.dumps(line), flush=True)
    return line


def run_grad(args):
    """Forward (training) + backward of the differentiable path on 1
    template of 65,536 Gaussians (SH degree 3), 64 instances, 512x512:
    steps per second of render_train + backward (loss gradient = random
    weights per pixel), CUDA events on the default stream."""
    import numpy as np
    import torch
    from paper_2501_17792_gb300 import binding, build
    from paper_2501_17792_gb300 import scene as S
    build.build()
    tpl = S.make_template(2100, 65536, 3)
    rng = np.random.default_rng(9)
    roots = [S.yaw_root(rng.uniform(0, 2 * math.pi), (col - 3.5) * 0.9, 0.0, 3.0 + row * 0.9)
             for row in range(8) for col in range(8)]
    n = 64
    cam = S.look_camera((0.0, 1.4, 0.0), 12.0, 512, 512, vfov_deg=60.0)
    r = binding.Renderer(device=0)
    r.upload_templates([tpl])
    frames = args.warmup + args.steps
    poses = [torch.from_numpy(S.random_poses(77 + f, n)).cuda() for f in range(frames)]
    tid = torch.zeros(n, dtype=torch.int32, device="cuda")
    root = torch.from_numpy(np.stack(roots).astype(np.float32).reshape(n, 12)).cuda()
    dl = torch.from_numpy(rng.normal(0, 1, (512, 512, 4)).astype(np.float32)).cuda()
    out = torch.empty((512, 512, 4), dtype=torch.float32, device="cuda")
    G = r.n_gauss_total
    grads = dict(means=torch.zeros((G, 3), device="cuda"), scales=torch.zeros((G, 3), device="cuda"),
                 quats=torch.zeros((G, 4), device="cuda"), opacity=torch.zeros(G, device="cuda"),
                 sh=torch.zeros((G, 16, 3), device="cuda"), pose=torch.zeros((n, 24, 3), device="cuda"))

    def step(f, ev=None):
        r.set_instances(tid, root, poses[f])
        r.render_train(cam, out=out)
        if ev is not None:
            ev.record()
        r.backward(dl, n, grads)

    r.set_instances(tid, root, poses[0])
    _, st = r.render_train(cam, out=out, stats=True)
    for f in range(args.warmup):
        step(f)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    mids = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e0.record()
    for k in range(args.steps):
        starts[k].record()
        step(args.warmup + k, mids[k])
    e1.record()
    torch.cuda.synchronize()
    total = e0.elapsed_time(e1)
    fwd = sum(s_.elapsed_time(m) for s_, m in zip(starts, mids)) / args.steps
    line = {"metric": "differentiable render: forward + backward steps per second", "value": args.steps / (total / 1e3),
            "unit": "steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total / args.steps, "ms_forward": fwd, "ms_backward": total / args.steps - fwd,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "grad_1x65536g_sh3_64inst_512x512", "splats": st["splats"], "pairs": st["pairs"]}}
    print(json.dumps(line), flush=True)
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--oracle-stride", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-baseline-s", type=float, default=12.0,
                    help="seconds of oracle samples for cpu_baseline (at least 3 samples)")
    ap.add_argument("--no-learned-lod", action="store_true",
                    help="skip the learned-vs-distance LoD comparison of the default run")
    ap.add_argument("--small", action="store_true", help="small crowd (debugging)")
    ap.add_argument("--sweep", action="store_true",
                    help="paper Table 1/2 sweep at 1280x720 (one JSON line per cell)")
    ap.add_argument("--storage", choices=["fp32", "bf16"], default="fp32",
                    help="template storage precision (bf16: BF16 attributes, FP16 SH, tensor-core skinning)")
    ap.add_argument("--grad", action="store_true",
                    help="forward + backward of the differentiable path (65,536 Gaussians, 64 instances, 512x512)")
    ap.add_argument("--learned-lod", action="store_true",
                    help="learned vs distance LoD at 10,000 instances, 3840x2160 (one JSON line)")
    ap.add_argument("--lod-steps", type=int, default=1500, help="MLP training steps for --learned-lod")
    ap.add_argument("--profile-case", nargs="?", const="crowd540", default=None, choices=["crowd540", "lod4k"],
                    help="frames for ncu captures: crowd540 (default) the quarter crowd, 875 instances at 960x540; "
                         "lod4k the 10,000-instance 3840x2160 crowd at the learned LoD's equal-PSNR budget "
                         "(levels 1 and 2 at 0.08 of their distance-LoD sizes)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.sweep:
        run_sweep(args)
        return
    if args.learned_lod:
        run_learned_lod(args)
        return
    if args.grad:
        run_grad(args)
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    from paper_2501_17792_gb300 import scene as S
    if args.small:
        sc = S.crowd(n_templates=2, n_gauss=4096, cols=10, rows=10, width=640, height=360)
    elif args.profile_case == "crowd540":
        sc = S.crowd(cols=25, rows=35, width=960, height=540)
    elif args.profile_case == "lod4k":
        base = S.paper_lod()
        fr = np.asarray(base.fractions, np.float64) * np.array([1.0, 0.08, 0.08])
        sc = S.crowd(cols=100, rows=100, width=3840, height=2160,
                     lod=S.LodConfig(thresholds=base.thresholds, fractions=fr.astype(np.float32),
                                     scale_mult=np.ones(3, np.float32)))
    else:
        sc = S.crowd()
    if args.impl == "reference":
        run_reference(args, sc, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_ours(args, sc, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
