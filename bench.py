#!/usr/bin/env python
"""Benchmark of the manifold-walk hot path on GB300.

A step is one pass of the whole hot path over one batch: guided seed chains
(Eq. deduction with the alpha-mixture of Sec. 5.5), Newton manifold walks,
contributions T = kappa G L_o with Bernoulli-trial reciprocal probabilities
(Sec. 5.8, reciprocal probability estimation) and the irradiance estimate (Eq. ThroughputMC), then the guide
records and histogram update (Eq. eq_weight).  The workload is the refractive
caustic through a glass sphere (radius 1, IOR 1.5, k = 2, 0.2 x 0.2 area light
at z = 4, 256 x 256 receiver points x 16 seeds = 1,048,576 chains, guide of
16 x 16 cells x 64 x 64 bins trained by one untimed p_0 pass).

Metric: converged manifold walks per second (every Newton walk that reached
max|C| < tol: the first walks and the Bernoulli trial walks).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank runs its own batch (weak scaling, no collective on
the data path); rank 0 prints one JSON line.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "converged manifold walks/sec and FP32 % of peak at 1 GB300, batched vs plain, at oracle tol"
UNIT = "walks/s"
WORKLOAD = "glass_sphere_k2_guided: r=1 IOR 1.5, 256x256 points x 16 seeds = 1,048,576 chains, 16x16x64x64 guide"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256, help="receiver points per side")
    ap.add_argument("--spq", type=int, default=16)
    ap.add_argument("--mode", default="batched", choices=["batched", "plain"])
    ap.add_argument("--no-flush", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the K3/K6, mixed-batch and adjoint measurements")
    ap.add_argument("--no-graph", action="store_true", help="batched mode without graph capture")
    ap.add_argument("--no-pipeline", action="store_true", help="one batch per graph replay (no double buffering)")
    ap.add_argument("--in-flight", type=int, default=4, help="batches advanced by one graph replay (own contexts)")
    ap.add_argument("--no-autotune", action="store_true", help="library default schedule instead of the autotuned one")
    ap.add_argument("--part", choices=list(PARTS), help="run one secondary measurement only")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                try:
                    rows.append((float(f[1]), float(f[2]), f[5:9]))
                except ValueError:
                    pass
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def unit_flops():
    with open(os.path.join(ROOT, "paper_2311_12818_gb300", "unit_flops.json")) as f:
        return json.load(f)["flops"]


def algorithmic_flops(st, F, surface="sphere"):
    """Flops of the work a kernel family did, from its counters and the
    per-primitive operation counts of the counted-scalar oracle."""
    frame = F["frame_" + surface]
    normal = F["normal_" + surface]
    return (st["full_evals"] * (frame + F["vertex_blocks"]) + st["c_evals"] * (normal + F["vertex_constraint"])
            + st["newton_steps"] * F["thomas_first_row"] + (st["thomas_rows"] - st["newton_steps"]) * F["thomas_row"]
            + st["ggt_rows"] * F["ggt_row"] + st["sphere_tests"] * F["ray_sphere"]
            + st["plane_tests"] * F["ray_rect"] + st["tri_tests"] * F["ray_triangle"] + st["node_tests"] * F["ray_box"])


def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    from paper_2311_12818_gb300 import inputs as I
    from paper_2311_12818_gb300 import mpg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    wl = I.glass_sphere(n=args.n, spq=args.spq)
    B, Q = wl.B, wl.Q
    off = rank * B  # each rank draws its own seeds (weak scaling)
    mode = mpg.WALK_BATCHED if args.mode == "batched" else mpg.WALK_PLAIN
    P = mpg.params_from(wl.params, walk_mode=mode, k_uniform=2)
    graph_mode = args.mode == "batched" and not args.no_graph
    # Batched mode replays a graph that advances two batches at once on two
    # contexts and two streams (double buffering): consecutive steps are
    # independent (each samples the trained guide and builds its own), so the
    # latency-bound ends of one batch's kernels overlap the other batch's work.
    n_buf = max(1, args.in_flight) if graph_mode and not args.no_pipeline else 1
    ctxs = [mpg.Context(local) for _ in range(n_buf)]

    def buffers(c):
        return dict(sc=mpg.Scene(c, wl), ch=mpg.Chains(wl, device=dev), out=mpg.Contribution.empty(B, Q, device=dev),
                    rec=(torch.zeros(B, dtype=torch.int32, device=dev),
                         torch.zeros((3, B), dtype=torch.float32, device=dev),
                         torch.zeros(B, dtype=torch.float32, device=dev), torch.zeros(4, dtype=torch.int32, device=dev)),
                    nxt=mpg.Guide(wl.n_cells, I.guide_edges(), device=dev))
    bufs = [buffers(c) for c in ctxs]
    ctx, sc, ch, out, rec = ctxs[0], bufs[0]["sc"], bufs[0]["ch"], bufs[0]["out"], bufs[0]["rec"]
    guide = mpg.Guide(wl.n_cells, I.guide_edges(), device=dev)

    # untimed fixture: one p_0 training pass builds the guide
    mpg.mpg_sample_seeds(ctx, sc, None, ch, P, wl.rng_seed, off + (1 << 40))
    mpg.mpg_manifold_walk(ctx, sc, ch, P)
    mpg.mpg_chain_contribution(ctx, sc, None, ch, P, wl.rng_seed, off + (1 << 40), out=out)
    mpg.mpg_guide_records(ctx, sc, ch, out.contrib, out=rec)
    mpg.mpg_guide_update(ctx, guide, rec[0], rec[1], rec[2], R=B, R_dev=rec[3], weight_shift=wl.params.weight_shift)
    ctx.sync()
    tune_s = None
    if args.mode == "batched" and not args.no_autotune:
        # the batched schedule chosen once by the library's autotuner (untimed),
        # on a guided batch of this workload
        t0 = time.perf_counter()
        P, _ = mpg.mpg_autotune(ctx, sc, guide, ch, P, wl.rng_seed, off + (1 << 41), repeats=2)
        tune_s = time.perf_counter() - t0

    def step_on(j, i, stream=None):
        c, bf = ctxs[j], bufs[j]
        o = off + i * B * world
        mpg.mpg_sample_seeds(c, bf["sc"], guide, bf["ch"], P, wl.rng_seed, o, stream=stream)
        mpg.mpg_manifold_walk(c, bf["sc"], bf["ch"], P, stream=stream)
        mpg.mpg_chain_contribution(c, bf["sc"], guide, bf["ch"], P, wl.rng_seed, o, out=bf["out"], stream=stream)
        mpg.mpg_guide_records(c, bf["sc"], bf["ch"], bf["out"].contrib, out=bf["rec"], stream=stream)
        mpg.mpg_guide_clear(c, bf["nxt"], stream=stream)
        r = bf["rec"]
        mpg.mpg_guide_update(c, bf["nxt"], r[0], r[1], r[2], R=B, R_dev=r[3], weight_shift=wl.params.weight_shift,
                             stream=stream)

    def step(i):
        step_on(0, i)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MiB > L2
    stream = torch.cuda.current_stream()
    for j in range(n_buf):
        for i in range(args.warmup):  # uncaptured: sizes each context's buffers
            step_on(j, 1000 + 16 * i + j)
    torch.cuda.synchronize()
    graph = None
    plan = [1] * args.steps  # batches advanced by each timed launch (sum = steps, exactly)
    if graph_mode:
        def capture(nb, base):
            # replay r of an nb-batch graph draws at the offsets of steps base + nb r + j
            g = mpg.Graph(ctx, rng_advance=nb * B * world, join=ctxs[1:nb])
            side = [torch.cuda.Stream(device=dev) for _ in range(nb)]
            with g:
                for j in range(nb):
                    side[j].wait_stream(g.stream)
                    step_on(j, base + j, stream=side[j])
                for j in range(nb):
                    g.stream.wait_stream(side[j])
            return g
        graph = capture(n_buf, 2000)
        rem = args.steps % n_buf
        graph_rem = capture(rem, 1 << 20) if rem else None
        for i in range(args.warmup):
            graph.launch()
            if graph_rem is not None:
                graph_rem.launch()
        torch.cuda.synchronize()
        plan = [n_buf] * (args.steps // n_buf) + ([rem] if rem else [])
    n_launch = len(plan)
    steps_run = sum(plan)
    per_launch = max(plan)

    def run(i):
        if graph is None:
            step(i)
        elif plan[i] == n_buf:
            graph.launch()
        else:
            graph_rem.launch()

    def all_stats():
        tot = None
        for c in ctxs:
            st = c.stats()
            tot = st if tot is None else {k: tot[k] + st[k] for k in tot}
        return tot

    def reset_all():
        for c in ctxs:
            c.reset_stats()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---- device-timed steps (inputs resident in HBM)
    reset_all()
    n_launch0 = ctx.launches()
    clocks = Clocks(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.5)  # let the sampler come up before the timed region
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_launch)]
    for i in range(n_launch):
        if not args.no_flush:
            flush.zero_()
        ev[i][0].record(stream)
        run(i)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    for c in ctxs:
        c.sync()
    step_ms = [a.elapsed_time(b) / nb for (a, b), nb in zip(ev, plan) for _ in range(nb)]
    launches = ctx.launches() - n_launch0
    total = all_stats()
    conv = total["converged"]
    t_ms = sum(step_ms)
    from paper_2311_12818_gb300 import dist as D
    t_ms, conv_all = D.job_throughput(t_ms, float(conv), device=dev)  # max time, summed walks
    value = conv_all / (t_ms * 1e-3)
    # irradiance throughput: receiver points and admissible contributions (the
    # records of each context's last timed step) per second, all ranks
    contrib_step = sum(int(bf["rec"][3][0].item()) for bf in bufs) / len(bufs)
    irr = {"shading_points_per_s": world * Q * steps_run / (t_ms * 1e-3),
           "contributions_per_s": world * contrib_step * steps_run / (t_ms * 1e-3),
           "contributions_per_step": contrib_step}

    # ---- attribution: the same steps uncaptured, each launch bracketed by
    # CUDA events on its own stream (per-family time, counters and flops)
    ctx.reset_stats()
    ctx.profile(reset=True)
    ctx.set_profile(True)
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        if not args.no_flush:
            flush.zero_()
        ev2[i][0].record(stream)
        step(3000 + i)
        ev2[i][1].record(stream)
    torch.cuda.synchronize()
    ctx.set_profile(False)
    ctx.sync()
    attr_ms = sum(a.elapsed_time(b) for a, b in ev2)
    fam = {}
    F = unit_flops()
    for k, name in enumerate(mpg.KERNEL_NAMES):
        ms, n = ctx.profile(k)
        st = ctx.stats(k)
        fam[name] = dict(ms=ms, launches=n, stats=st, flops=algorithmic_flops(st, F))
    # first walks alone: one more uncaptured step, its statuses read after the walk
    c0, bf0 = ctxs[0], bufs[0]
    mpg.mpg_sample_seeds(c0, bf0["sc"], guide, bf0["ch"], P, wl.rng_seed, off + 7777 * B * world)
    mpg.mpg_manifold_walk(c0, bf0["sc"], bf0["ch"], P)
    c0.sync()
    primary_per_step = int((bf0["ch"].status == 1).sum().item())

    # ---- end to end through the public API with host buffers
    pin = lambda a: torch.as_tensor(a).pin_memory()  # noqa: E731
    host_in = []
    for bf in bufs:
        c_ = bf["ch"]
        host_in += [(c_.xD, pin(np.ascontiguousarray(wl.xD.T, np.float32))),
                    (c_.nD, pin(np.ascontiguousarray(wl.nD.T, np.float32))),
                    (c_.cell, pin(wl.cell.astype(np.int32))), (c_.xL, pin(np.ascontiguousarray(wl.xL.T, np.float32))),
                    (c_.k, pin(wl.k.astype(np.uint8))), (c_.tau, pin(wl.tau.astype(np.uint8))),
                    (c_.pn, pin(wl.pn.astype(np.float32)))]
    h2d = sum(h.numel() * h.element_size() for _, h in host_in) // per_launch
    E_host = [torch.empty(Q, dtype=torch.float32).pin_memory() for _ in bufs]
    n_host = [torch.empty(4, dtype=torch.int32).pin_memory() for _ in bufs]
    d2h = (E_host[0].numel() * 4 + n_host[0].numel() * 4) * len(bufs) // per_launch
    e2e_conv = 0
    e2e_ms = 0.0
    for i in range(max(1, n_launch // 2)):
        if not args.no_flush:
            flush.zero_()
        reset_all()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for d, h in host_in:
            d.copy_(h, non_blocking=True)
        if graph is not None:
            graph.launch()
        else:
            step(500 + i)
        for j, bf in enumerate(bufs[:per_launch]):
            E_host[j].copy_(bf["out"].E, non_blocking=True)
            n_host[j].copy_(bf["rec"][3], non_blocking=True)
        b.record(stream)
        b.synchronize()
        e2e_ms += a.elapsed_time(b)
        e2e_conv += all_stats()["converged"]
    e2e_value = e2e_conv / (e2e_ms * 1e-3) if world == 1 else None

    # ---- roofline of the dominant kernel family (FP32 ALU bound)
    dom = max((n for n in fam if n != "aux"), key=lambda n: fam[n]["ms"])
    d = fam[dom]
    achieved = d["flops"] / (d["ms"] * 1e-3) if d["ms"] > 0 else 0.0
    props = torch.cuda.get_device_properties(dev)
    sm_max = clk.get("sm_max_mhz") or 2070.0
    peak_nominal = props.multi_processor_count * 128 * 2 * sm_max * 1e6
    peak_ffma = ctx.fp32_peak()
    peak_dfma = ctx.fp64_peak()
    kname = {"walk": "k_walk_p" if args.mode == "batched" else "k_walk", "bernoulli": "k_bern_round"}.get(dom, "k_" + dom)
    traffic = profiled_traffic("k_walk_p__glass_sphere_1M.md") if kname == "k_walk_p" else None
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved / 1e12, "peak": peak_nominal / 1e12,
                "unit": "TFLOP/s", "frac": achieved / peak_nominal, "traffic": traffic,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one primary-walk launch"
                                  " (profiles/k_walk_p__glass_sphere_1M.md); null when the kernels changed since",
                "peak_source": "derived: %d SMs x 128 FP32 lanes x 2 flop x %.0f MHz" % (props.multi_processor_count, sm_max),
                "peak_ffma_measured": peak_ffma / 1e12, "frac_of_ffma_measured": achieved / peak_ffma if peak_ffma else None,
                "peak_fp64_dfma_measured": peak_dfma / 1e12,
                "algorithmic_flops_per_launch": d["flops"] / max(1, d["launches"]),
                "avg_launch_ms": d["ms"] / max(1, d["launches"]),
                "timing": "per-launch CUDA events in an uncaptured pass of the same steps"}
    step_flops = sum(f["flops"] for f in fam.values())
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps_run,
        "warmup": args.warmup, "ms_per_step": t_ms / steps_run, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded procedural scene, no dataset)",
        "config": {"workload": WORKLOAD, "chains_per_step": B, "receiver_points": Q, "seeds_per_point": wl.spq,
                   "k": 2, "walk_mode": args.mode, "graph": graph is not None,
                   "batches_in_flight": per_launch,
                   "schedule": {f: getattr(P, f) for f in mpg.SCHEDULE_FIELDS}, "autotune_s": tune_s,
                   "l2": "flushed between steps (256 MiB write)" if not args.no_flush else "not flushed",
                   "parallelism": "replicas x%d" % world,
                   "counted_walks": "walks that converged: the first walks and the trial walks of each chain's"
                                    " sequential Bernoulli loop up to its first recurrence"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": roofline,
        "clocks": clk,
        "detail": {"irradiance_throughput": irr,
                   "converged_per_step": conv / steps_run, "walks_per_step": total["walks"] / steps_run,
                   "primary_converged_per_step": primary_per_step,
                   "primary_converged_walks_per_s": world * primary_per_step * steps_run / (t_ms * 1e-3),
                   "trials_per_step": total["trials"] / steps_run,
                   "fp64_geometry_terms_per_step": total["ggt_fp64"] / steps_run,
                   "step_ms": [round(x, 4) for x in step_ms],
                   "graph_kernels_per_step": graph.kernels() if graph is not None else None,
                   "uncaptured_profiled_ms_per_step": attr_ms / args.steps,
                   "step_fp32_tflops": step_flops / (attr_ms * 1e-3) / 1e12 if world == 1 else None,
                   "timed_step_fp32_tflops": algorithmic_flops(total, F) / (sum(step_ms) * 1e-3) / 1e12,
                   "timed_step_fp32_frac": algorithmic_flops(total, F) / (sum(step_ms) * 1e-3) / peak_nominal,
                   "families": {n: {"ms_per_step": f["ms"] / args.steps, "launches": f["launches"],
                                    "gflop_per_step": f["flops"] / args.steps / 1e9,
                                    "tflops": f["flops"] / (f["ms"] * 1e-3) / 1e12 if f["ms"] > 0 else None}
                                for n, f in fam.items() if f["launches"]}},
    }
    del graph
    if rank == 0 and not args.no_secondary:
        line["configs"] = other_configs(args, dev, flush, torch, peak_nominal)
        line["secondary"] = secondary(args, dev, flush, torch, peak_nominal)
    if rank == 0:
        line["cpu_baseline"] = cpu_baseline(wl)
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def timed_loop(fn, steps, warmup, flush, stream, torch):
    """Mean ms of fn(i) over `steps` calls after `warmup`, L2 flushed before each."""
    for i in range(warmup):
        fn(10_000 + i)
    torch.cuda.synchronize()
    ms = 0.0
    for i in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn(i)
        b.record(stream)
        b.synchronize()
        ms += a.elapsed_time(b)
    return ms / steps


def kernel_digest():
    """sha256 over the CUDA sources (file names and contents, sorted) and the build script."""
    import glob
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2311_12818_gb300", "csrc")
    files = sorted(glob.glob(os.path.join(d, "*.cu")) + glob.glob(os.path.join(d, "*.cuh")))
    for f in files + [os.path.join(ROOT, "paper_2311_12818_gb300", "build.py")]:  # sources and flags
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(summary):
    """DRAM bytes per launch from a committed ncu summary under profiles/, or
    None when the summary was taken on other kernel sources than these.  A
    summary may list later source digests at which the profiled kernel's own
    code (the kernel and every function it calls) is unchanged, one per line
    as "Kernel unchanged at digest: <sha256> (<the change>)"."""
    import re
    try:
        with open(os.path.join(ROOT, "profiles", summary)) as f:
            text = f.read()
    except OSError:
        return None
    dg = re.search(r"Kernel source digest[^:]*: ([0-9a-f]{64})", text)
    tb = re.search(r"dram_bytes_per_launch: (\d+)", text)
    if not dg or not tb:
        return None
    valid = {dg.group(1)} | set(re.findall(r"Kernel unchanged at digest: ([0-9a-f]{64})", text))
    if kernel_digest() not in valid:
        return None
    return int(tb.group(1))


def profiled_fraction(summary):
    """The executed-FP32 fraction a committed ncu summary states ('= F of the
    derived 80.5 TFLOP/s'), or None when it was taken on other kernel sources
    (same digest rule as profiled_traffic)."""
    import re
    if profiled_traffic(summary) is None:
        return None
    with open(os.path.join(ROOT, "profiles", summary)) as f:
        m = re.search(r"= ([0-9.]+) of the derived", f.read())
    return float(m.group(1)) if m else None


def measured_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


PARTS = ("plain", "k3", "k6", "mixed", "adjoint", "vmf", "repeats", "progressive", "selective", "glossy", "mixed_group",
         "mixed_step", "stree",
         "configs", "glossy_chains")
# measured by default beside the headline; "mixed" and "adjoint" are covered
# by the configuration lines (other_configs) and run only with --part
DEFAULT_PARTS = ("plain", "k3", "k6", "vmf", "repeats", "progressive", "selective", "glossy", "glossy_chains")


def other_configs(args, dev, flush, torch, peak_fp32):
    """The other configurations of the benchmark as lines of their own (see
    config_line): the mirror sphere (k = 1, point light), the water
    heightfield (BVH, k = 1..2), the mixed-length batch (k = 1..8, 2^22 chains:
    batched vs plain on identical inputs) and the adjoint on the water scene."""
    from paper_2311_12818_gb300 import inputs as I
    from paper_2311_12818_gb300 import mpg
    stream = torch.cuda.current_stream()
    F = unit_flops()
    steps = max(3, min(10, args.steps // 4))
    ctx = mpg.Context(dev.index or 0)
    out = {}
    out["mirror_sphere"] = config_line(
        ctx, dev, flush, torch, stream, I.mirror_sphere(),
        "mirror_sphere_k1: r=1, point light (0,3,2), 64x64 points x 16 seeds from p_0 = 65,536 chains",
        steps, args.warmup, F, peak_fp32, cpu_wl=I.mirror_sphere(), cpu_note="the whole workload")
    out["water"] = config_line(
        ctx, dev, flush, torch, stream, I.water(),
        "water_heightfield: 128x128 heights (32,258 triangles, BVH), IOR 1.33, 512x512 floor points x 4 seeds"
        " = 1,048,576 chains, k = 1 (T) or 2 (RT, TR)",
        steps, args.warmup, F, peak_fp32, cpu_wl=I.water(n=128, spq=4),
        cpu_note="1/16 sample: 128x128 floor points over the same extent x 4 seeds")
    out["mixed"] = config_line(
        ctx, dev, flush, torch, stream, I.mixed(),
        "mixed_k1to8: nested spheres + 4 lenses + mirror, 1024x512 points x 8 seeds = 4,194,304 chains,"
        " k ~ Geometric(0.35) on 1..8, random types",
        steps, args.warmup, F, peak_fp32, cpu_wl=I.mixed(nx=256, ny=128, spq=8),
        cpu_note="1/16 sample: 256x128 points over the same extent x 8 seeds")
    out["adjoint"] = part_adjoint(ctx, dev, flush, torch, stream, steps)
    return out


def secondary(args, dev, flush, torch, peak_fp32, parts=DEFAULT_PARTS):
    """The other configurations, measured beside the headline:
    - k3: the standalone BVH ray batch on the water heightfield (GB/s);
    - k6: the guide-histogram update of one glass-sphere pass (GB/s);
    - mixed: the mixed-length batch (k = 1..8, 2^22 chains) plain (one launch
      per k), batched (one graph replay) and batched with the autotuned schedule;
    - adjoint: the adjoint of the water irradiance with respect to the heights;
    - vmf: the vMF mixture guide with sampled chain lengths on the mixed batch;
    - repeats: four Bernoulli estimates per chain in rendering (R x 4) or in
      training and rendering (TR x 4) on the guided glass-sphere step;
    - selective: the guided glass-sphere step with selective activation;
    - glossy: product importance sampling with a glossy separator (mixed batch);
    - progressive: the online training schedule and rendering of a
      64-seed-per-point budget on the glass sphere, as one captured graph."""
    import numpy as np
    from paper_2311_12818_gb300 import inputs as I
    from paper_2311_12818_gb300 import mpg
    stream = torch.cuda.current_stream()
    hbm, hbm_src = measured_hbm()
    steps = max(2, args.steps // 2)
    F = unit_flops()
    out = {}
    ctx = mpg.Context(dev.index or 0)
    if "plain" in parts:
        out["glass_plain"] = part_plain(ctx, dev, flush, torch, stream, steps, F, peak_fp32)
    if "k3" in parts:
        out["k3_bvh_trace"] = part_k3(ctx, dev, flush, torch, stream, steps, F, hbm, hbm_src)
    if "k6" in parts:
        out["k6_guide_update"] = part_k6(ctx, dev, flush, torch, stream, steps, hbm, hbm_src)
    if "mixed" in parts:
        out["mixed_batch"] = part_mixed(ctx, dev, flush, torch, stream, steps, F, peak_fp32)
    if "adjoint" in parts:
        out["adjoint"] = part_adjoint(ctx, dev, flush, torch, stream, steps)
    if "vmf" in parts:
        out["vmf_guide"] = part_vmf(ctx, dev, flush, torch, stream, steps, F, peak_fp32)
    if "repeats" in parts:
        out["repeated_estimates"] = part_repeats(ctx, dev, flush, torch, stream, steps)
    if "glossy" in parts:
        out["glossy_separator"] = part_glossy(ctx, dev, flush, torch, stream, steps)
    if "glossy_chains" in parts:
        out["glossy_chains"] = part_glossy_chains(ctx, dev, flush, torch, stream, steps, F, peak_fp32)
    if "selective" in parts:
        out["selective_activation"] = part_selective(ctx, dev, flush, torch, stream, steps)
    if "progressive" in parts:
        out["progressive"] = part_progressive(ctx, dev, flush, torch, stream, max(2, steps // 5))
    if "mixed_group" in parts and parts == ("mixed_group",):
        out["mixed_group"] = part_mixed_group(ctx, dev, flush, torch, stream, steps)
    return out


def part_mixed_group(ctx, dev, flush, torch, stream, steps):
    """The mixed-length step with one chain per lane group in walks and
    parallel rounds (first parallel batch 4), uncaptured: for profiling the
    group kernels (run alone with --part mixed_group)."""
    from paper_2311_12818_gb300 import inputs as I
    from paper_2311_12818_gb300 import mpg
    wl = I.mixed()
    sc = mpg.Scene(ctx, wl)
    ch = mpg.Chains(wl, device=dev)
    res = mpg.Contribution.empty(wl.B, wl.Q, device=dev)
    P = mpg.params_from(wl.params, walk_mode=mpg.WALK_BATCHED, tau_random=True, walk_group=3, trial_batch=4)

    def step(i):
        mpg.mpg_sample_seeds(ctx, sc, None, ch, P, wl.rng_seed, i * wl.B)
        mpg.mpg_manifold_walk(ctx, sc, ch, P)
        mpg.mpg_chain_contribution(ctx, sc, None, ch, P, wl.rng_seed, i * wl.B, out=res)
    ms = timed_loop(step, steps, 1, flush, stream, torch)
    return {"workload": "mixed_k1to8, 4,194,304 chains, walk_group 3, trial_batch 4", "ms_per_step": ms}


def part_plain(ctx, dev, flush, torch, stream, steps, F, peak_fp32):
    """The benchmark step (seeds -> walk -> contribution with Bernoulli trials)
    on the same glass-sphere inputs in plain mode: one launch per chain length,
    one thread per chain, each chain's trials as a sequential loop; no graph."""
    from paper_2311_12818_gb300 import inputs as I
    from paper_2311_12818_gb300 import mpg
    wl = I.glass_sphere()
    sc = mpg.Scene(ctx, wl)
    ch = mpg.Chains(wl, device=dev)
    res = mpg.Contribution.empty(wl.B, wl.Q, device=dev)
    out = {"workload": "glass_sphere_k2 (p_0 seeds), 1,048,576 chains: seeds -> walk -> contribution + trials"}
    for name, mode in (("plain", mpg.WALK_PLAIN), ("batched", mpg.WALK_BATCHED)):
        P = mpg.params_from(wl.params, walk_mode=mode, k_uniform=2)

        def step(i, P=P):
            mpg.mpg_sample_seeds(ctx, sc, None, ch, P, wl.rng_seed, i * wl.B)
            mpg.mpg_manifold_walk(ctx, sc, ch, P)
            mpg.mpg_chain_contribution(ctx, sc, None, ch, P, wl.rng_seed, i * wl.B, out=res)
        step(0)
        ctx.sync()
        ctx.reset_stats()
        ms = timed_loop(step, steps, 2, flush, stream, torch)
        st = ctx.stats()
        per = steps + 2
        fl = algorithmic_flops(st, F) / per
        out[name] = {"ms_per_step": ms, "converged_walks_per_s": st["converged"] / per / (ms * 1e-3),
                     "fp32_tflops": fl / (ms * 1e-3) / 1e12, "fp32_frac": fl / (ms * 1e-3) / peak_fp32}
    out["batched_over_plain"] = out["batched"]["converged_walks_per_s"] / out["plain"]["converged_walks_per_s"]
    return out


def part_k3(ctx, dev, flush, torch, stream, steps, F, hbm, hbm_src):
    import numpy as np
    from paper_2311_12818_gb300 import inputs as I
    from paper_2311_12818_gb300 import mpg
    wl = I.water()
    sc = mpg.Scene(ctx, wl)
    n = 1 << 22
    o, d = I.water_rays(n)
    o = torch.as_tensor(o.T.astype(np.float32), device=dev).contiguous()
    d = torch.as_tensor(d.T.astype(np.float32), device=dev).contiguous()
    res = (torch.empty(n, dtype=torch.float32, device=dev), torch.empty(n, dtype=torch.int32, device=dev),
           torch.empty(n, dtype=torch.int32, device=dev), torch.empty((2, n), dtype=torch.float32, device=dev))
    mpg.mpg_trace_rays(ctx, sc, o, d, out=res)
    ctx.reset_stats()
    ms = timed_loop(lambda i: mpg.mpg_trace_rays(ctx, sc, o, d, out=res), steps, 2, flush, stream, torch)
    st = ctx.stats(mpg.KERNEL_TRACE)
    per = steps + 2
    nodes, tris = st["node_tests"] / per, st["tri_tests"] / per
    byts = n * (24 + 20) + nodes * 32 + tris * 48
    nn, nt = sc.info(0)
    return {
        "workload": "water heightfield 128x128 (%d triangles, %d BVH nodes), %d rays" % (nt, nn, n),
        "ms": ms, "rays_per_s": n / (ms * 1e-3), "node_tests_per_ray": nodes / n, "tri_tests_per_ray": tris / n,
        "algorithmic_bytes": byts, "gbs": byts / (ms * 1e-3) / 1e9, "hbm_peak_gbs": hbm, "peak_source": hbm_src,
        "frac": byts / (ms * 1e-3) / 1e9 / hbm,
        "bytes_rule": "44 B of ray in/out + 32 B per child-box test + 48 B per triangle test (nodes and triangles are"
                      " L2-resident: the figure is L2+DRAM traffic against the HBM peak)",
        "fp32_tflops": algorithmic_flops(st, F, "sphere") / per / (ms * 1e-3) / 1e12}


def part_k6(ctx, dev, flush, torch, stream, steps, hbm, hbm_src):
    from paper_2311_12818_gb300 import inputs as I
    from paper_2311_12818_gb300 import mpg
    wl = I.glass_sphere()
    sc = mpg.Scene(ctx, wl)
    ch = mpg.Chains(wl, device=dev)
    P = mpg.params_from(wl.params, walk_mode=mpg.WALK_BATCHED, k_uniform=2)
    res = mpg.Contribution.empty(wl.B, wl.Q, device=dev)
    mpg.mpg_sample_seeds(ctx, sc, None, ch, P, wl.rng_seed, 0)
    mpg.mpg_manifold_walk(ctx, sc, ch, P)
    mpg.mpg_chain_contribution(ctx, sc, None, ch, P, wl.rng_seed, 0, out=res)
    rec = (torch.zeros(wl.B, dtype=torch.int32, device=dev), torch.zeros((3, wl.B), dtype=torch.float32, device=dev),
           torch.zeros(wl.B, dtype=torch.float32, device=dev), torch.zeros(4, dtype=torch.int32, device=dev))
    mpg.mpg_guide_records(ctx, sc, ch, res.contrib, out=rec)
    g = mpg.Guide(wl.n_cells, I.guide_edges(), device=dev)
    R = int(rec[3][0].item())

    def upd(i):
        mpg.mpg_guide_clear(ctx, g)
        mpg.mpg_guide_update(ctx, g, rec[0], rec[1], rec[2], R=wl.B, R_dev=rec[3], weight_shift=wl.params.weight_shift)
    ms = timed_loop(upd, steps, 2, flush, stream, torch)
    hist = g.counts.numel() * 8
    byts = R * (4 + 12 + 4 + 8) + 2 * hist + 2 * hist  # records + atomics, clear, prefix-sum read + write
    return {
        "workload": "glass sphere pass: %d records into 256 cells x 64x64 bins (uint64)" % R,
        "ms": ms, "records_per_s": R / (ms * 1e-3), "algorithmic_bytes": byts, "gbs": byts / (ms * 1e-3) / 1e9,
        "hbm_peak_gbs": hbm, "peak_source": hbm_src, "frac": byts / (ms * 1e-3) / 1e9 / hbm,
        "bytes_rule": "20 B per record + 8 B atomic, clear of counts and prefix sums (16 B/bin), prefix sums"
                      " (8 B/bin read + 8 B/bin written)"}


def part_mixed(ctx, dev, flush, torch, stream, steps, F, peak_fp32):
    from paper_2311_12818_gb300 import inputs as I
    from paper_2311_12818_gb300 import mpg
    wl = I.mixed()
    ctx2 = mpg.Context(dev.index or 0)
    parts = [(c, mpg.Scene(c, wl), mpg.Chains(wl, device=dev), mpg.Contribution.empty(wl.B, wl.Q, device=dev))
             for c in (ctx, ctx2)]
    mixed = {"workload": "mixed_k1to8: nested spheres + 4 lenses + mirror, 1024x512 points x 8 = 4,194,304 chains"}

    def measure(P, use_graph, in_flight=1):
        def step_on(j, o, s=None):
            c, sc, ch, res = parts[j]
            mpg.mpg_sample_seeds(c, sc, None, ch, P, wl.rng_seed, o, stream=s)
            mpg.mpg_manifold_walk(c, sc, ch, P, stream=s)
            mpg.mpg_chain_contribution(c, sc, None, ch, P, wl.rng_seed, o, out=res, stream=s)
        for j in range(in_flight):
            step_on(j, j * wl.B)
        torch.cuda.synchronize()
        fn = lambda i: step_on(0, i * wl.B)  # noqa: E731
        if use_graph:
            gr = mpg.Graph(ctx, rng_advance=in_flight * wl.B, join=[p[0] for p in parts[1:in_flight]])
            side = [torch.cuda.Stream(device=dev) for _ in range(in_flight)]
            with gr:
                for j in range(in_flight):
                    side[j].wait_stream(gr.stream)
                    step_on(j, (7 << 32) + j * wl.B, side[j])
                for sd in side:
                    gr.stream.wait_stream(sd)
            fn = lambda i: gr.launch()  # noqa: E731
        for p in parts:
            p[0].reset_stats()
        n0 = ctx.launches()
        ms = timed_loop(fn, steps, 2, flush, stream, torch) / in_flight  # per batch
        st = {k: parts[0][0].stats()[k] + parts[1][0].stats()[k] for k in ("converged", "walks")}
        fam = [p[0].stats() for p in parts]
        tot = {k: fam[0][k] + fam[1][k] for k in fam[0]}
        per = (steps + 2) * in_flight
        fl = algorithmic_flops(tot, F) / per
        return {"ms_per_step": ms, "converged_walks_per_s": st["converged"] / per / (ms * 1e-3),
                "walks_per_s": st["walks"] / per / (ms * 1e-3), "fp32_tflops": fl / (ms * 1e-3) / 1e12,
                "fp32_frac": fl / (ms * 1e-3) / peak_fp32, "launches_per_step": (ctx.launches() - n0) / per,
                "graph": use_graph, "batches_in_flight": in_flight}

    base = mpg.params_from(wl.params, walk_mode=mpg.WALK_BATCHED, tau_random=True, k_uniform=0)
    mixed["plain"] = measure(mpg.params_from(wl.params, walk_mode=mpg.WALK_PLAIN, tau_random=True, k_uniform=0), False)
    mixed["batched"] = measure(base, True)
    t0 = time.perf_counter()
    tuned, tms = mpg.mpg_autotune(ctx, parts[0][1], None, parts[0][2], base, wl.rng_seed, 0, repeats=1)
    tune_s = time.perf_counter() - t0
    mixed["batched_autotuned"] = measure(tuned, True)
    mixed["batched_autotuned"]["schedule"] = {f: getattr(tuned, f) for f in mpg.SCHEDULE_FIELDS}
    mixed["batched_autotuned"]["tuning_s"] = tune_s
    mixed["batched_autotuned_2_in_flight"] = measure(tuned, True, in_flight=2)
    best = max(mixed[k]["converged_walks_per_s"] for k in ("batched", "batched_autotuned", "batched_autotuned_2_in_flight"))
    mixed["batched_over_plain"] = best / mixed["plain"]["converged_walks_per_s"]
    return mixed


def config_line(ctx, dev, flush, torch, stream, wl, describe, steps, warmup, F, peak_fp32, autotune=True,
                cpu_wl=None, cpu_note=""):
    """One configuration measured like the headline: the batched step (seeds
    -> walk -> contribution with Bernoulli trials -> irradiance) replayed from
    a captured graph with the autotuned schedule, against the plain mode (one
    launch per chain length, sequential trial loops, no graph) on identical
    inputs (the same random-number offsets, so the same seeds and trials);
    converged walks per second with and without the Bernoulli trial walks;
    the irradiance throughput; the roofline of the dominant kernel family from
    per-launch CUDA events of an uncaptured pass of the same steps; the same
    metric end to end with host inputs; and the oracle on the host cores."""
    import numpy as np
    from paper_2311_12818_gb300 import mpg
    B, Q = wl.B, wl.Q
    uniform = int(wl.k[0]) if (wl.k == wl.k[0]).all() else 0
    sc = mpg.Scene(ctx, wl)
    ch = mpg.Chains(wl, device=dev)
    res = mpg.Contribution.empty(B, Q, device=dev)
    base = mpg.params_from(wl.params, walk_mode=mpg.WALK_BATCHED, tau_random=wl.tau_random, k_uniform=uniform)
    plain = mpg.params_from(wl.params, walk_mode=mpg.WALK_PLAIN, tau_random=wl.tau_random, k_uniform=uniform)

    def step(P, o, s=None):
        mpg.mpg_sample_seeds(ctx, sc, None, ch, P, wl.rng_seed, o, stream=s)
        mpg.mpg_manifold_walk(ctx, sc, ch, P, stream=s)
        mpg.mpg_chain_contribution(ctx, sc, None, ch, P, wl.rng_seed, o, out=res, stream=s)

    step(base, 1 << 44)
    ctx.sync()
    tune_s, P = None, base
    if autotune:
        t0 = time.perf_counter()
        P, _ = mpg.mpg_autotune(ctx, sc, None, ch, base, wl.rng_seed, 1 << 45, repeats=1)
        tune_s = time.perf_counter() - t0
    BASE = 1 << 40
    offs = [BASE + (warmup + j) * B for j in range(steps)]  # graph replay warmup + j draws here
    step(P, BASE)
    ctx.sync()
    g = mpg.Graph(ctx, rng_advance=B)
    with g:
        step(P, BASE, g.stream)
    for _ in range(warmup):
        g.launch()
    torch.cuda.synchronize()

    def timed(fn):
        ctx.reset_stats()
        ms, prim = [], 0
        for j in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn(j)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        ctx.sync()
        return sum(ms) / steps, ctx.stats()

    ms_b, st_b = timed(lambda j: g.launch())
    n_launch = g.kernels()
    adm_b = int((res.contrib > 0).sum().item())
    # plain mode on the same offsets
    ms_p, st_p = timed(lambda j: step(plain, offs[j]))
    # attribution: the batched schedule uncaptured at the same offsets, every
    # launch bracketed by events on its own stream; primary convergences
    ctx.reset_stats()
    ctx.profile(reset=True)
    ctx.set_profile(True)
    prim_b = 0
    for j in range(steps):
        flush.zero_()
        mpg.mpg_sample_seeds(ctx, sc, None, ch, P, wl.rng_seed, offs[j])
        mpg.mpg_manifold_walk(ctx, sc, ch, P)
        ctx.sync()
        prim_b += int((ch.status == 1).sum().item())
        mpg.mpg_chain_contribution(ctx, sc, None, ch, P, wl.rng_seed, offs[j], out=res)
    ctx.sync()
    ctx.set_profile(False)
    fam = {}
    for kind, fname in enumerate(mpg.KERNEL_NAMES):
        fms, nl = ctx.profile(kind)
        fst = ctx.stats(kind)
        fam[fname] = dict(ms=fms, launches=nl, flops=algorithmic_flops(fst, F))
    ctx.profile(reset=True)
    dom = max((n for n in fam if n not in ("aux", "trace")), key=lambda n: fam[n]["ms"])
    d = fam[dom]
    kernels = {"walk": "k_walk_g" if P.walk_group & 1 else "k_walk_p",
               "bernoulli": "k_bern_round_g" if P.walk_group & 2 else "k_bern_round",
               "contrib": "k_contrib", "seed": "k_seed"}[dom]
    achieved = d["flops"] / (d["ms"] * 1e-3) if d["ms"] > 0 else 0.0
    roofline = {"bound": "alu", "kernel": kernels, "family": dom, "achieved": achieved / 1e12,
                "peak": peak_fp32 / 1e12, "unit": "TFLOP/s", "frac": achieved / peak_fp32, "traffic": None,
                "algorithmic_flops_per_launch": d["flops"] / max(1, d["launches"]),
                "avg_launch_ms": d["ms"] / max(1, d["launches"]),
                "timing": "per-launch CUDA events in an uncaptured pass of the same steps (family: %d launches)"
                          % d["launches"]}
    # end to end: pinned host inputs copied in, the irradiance image read back
    pin = lambda a: torch.as_tensor(a).pin_memory()  # noqa: E731
    host_in = [(ch.xD, pin(np.ascontiguousarray(wl.xD.T, np.float32))),
               (ch.nD, pin(np.ascontiguousarray(wl.nD.T, np.float32))), (ch.cell, pin(wl.cell.astype(np.int32))),
               (ch.xL, pin(np.ascontiguousarray(wl.xL.T, np.float32))), (ch.k, pin(wl.k.astype(np.uint8))),
               (ch.tau, pin(wl.tau.astype(np.uint8))), (ch.pn, pin(wl.pn.astype(np.float32)))]
    E_host = torch.empty(Q, dtype=torch.float32).pin_memory()

    def e2e_step(j):
        for dd, hh in host_in:
            dd.copy_(hh, non_blocking=True)
        g.launch()
        E_host.copy_(res.E, non_blocking=True)
    n_e2e = max(2, steps // 2)
    ctx.reset_stats()
    ms_e = 0.0
    for j in range(n_e2e):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_step(j)
        b.record(stream)
        b.synchronize()
        ms_e += a.elapsed_time(b)
    ctx.sync()
    ms_e /= n_e2e
    e2e_conv = ctx.stats()["converged"] / n_e2e
    h2d = sum(h.numel() * h.element_size() for _, h in host_in)
    out = {
        "workload": describe, "metric": METRIC, "unit": UNIT,
        "value": st_b["converged"] / steps / (ms_b * 1e-3), "ms_per_step": ms_b, "steps": steps,
        "warmup": warmup, "chains_per_step": B, "same_inputs_as_plain": True,
        "primary_converged_walks_per_s": prim_b / steps / (ms_b * 1e-3),
        "converged_per_step": st_b["converged"] / steps, "primary_converged_per_step": prim_b / steps,
        "trials_per_step": st_b["trials"] / steps,
        "irradiance_throughput": {"shading_points_per_s": Q / (ms_b * 1e-3),
                                  "contributions_per_s": adm_b / (ms_b * 1e-3), "contributions_per_step": adm_b},
        "fp32_tflops_step": algorithmic_flops(st_b, F) / steps / (ms_b * 1e-3) / 1e12,
        "fp32_frac_step": algorithmic_flops(st_b, F) / steps / (ms_b * 1e-3) / peak_fp32,
        "graph_kernels_per_step": n_launch,
        "schedule": {f: getattr(P, f) for f in mpg.SCHEDULE_FIELDS}, "autotune_s": tune_s,
        "plain": {"ms_per_step": ms_p, "converged_walks_per_s": st_p["converged"] / steps / (ms_p * 1e-3),
                  "converged_per_step": st_p["converged"] / steps,
                  "fp32_frac_step": algorithmic_flops(st_p, F) / steps / (ms_p * 1e-3) / peak_fp32},
        "roofline": roofline,
        "families_uncaptured_ms_per_step": {n: f["ms"] / steps for n, f in fam.items() if f["launches"]},
        "e2e": {"value": e2e_conv / (ms_e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": Q * 4},
    }
    out["batched_over_plain"] = out["value"] / out["plain"]["converged_walks_per_s"]
    if cpu_wl is not None:
        out["cpu_baseline"] = cpu_line(cpu_wl, cpu_note)
    del g
    return out


def cpu_line(wl, note):
    """The oracle (as it stands) on all host cores over a sample workload:
    seeds -> walk -> contribution -> Bernoulli trials -> irradiance."""
    import numpy as np

    from oracle import oracle as O
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    sc = O.Scene(wl)
    s = O.sample_seeds(wl, sc, None, threads=threads)
    c = O.walk(wl, sc, s, threads=threads)
    k = O.contribution(wl, sc, c, threads=threads)
    tw = np.zeros(wl.B, np.uint32)
    N, _ = O.bernoulli(wl, sc, c, k["admissible"], None, threads=threads, trial_walks=tw)
    O.irradiance(wl, k["T"], N, k["admissible"])
    dt = time.perf_counter() - t0
    conv = int((c["status"] == 1).sum() + tw.sum())
    return {"value": conv / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%s: %d chains, one step, %.1f s" % (note, wl.B, dt)}


def part_adjoint(ctx, dev, flush, torch, stream, steps):
    from paper_2311_12818_gb300 import inputs as I
    from paper_2311_12818_gb300 import mpg
    wl = I.water()
    sc = mpg.Scene(ctx, wl)
    ch = mpg.Chains(wl, device=dev)
    P = mpg.params_from(wl.params, walk_mode=mpg.WALK_BATCHED)
    res = mpg.run(ctx, sc, ch, wl, params=P)
    dLdE = torch.as_tensor(I.upstream_grad(wl.Q), dtype=torch.float32, device=dev)
    gr = torch.zeros(wl.hf_heights.size, dtype=torch.float32, device=dev)
    n_adj = int((res.contrib > 0).sum().item())

    def adj(i):
        gr.zero_()
        mpg.mpg_walk_adjoint(ctx, sc, ch, res.T, res.contrib, dLdE, gr)
    ms = timed_loop(adj, steps, 2, flush, stream, torch)
    return {"workload": "water_heightfield: 128x128 heights, 512x512 points x 4 = 1,048,576 chains",
            "differentiated_chains": n_adj, "ms": ms, "chains_per_s": n_adj / (ms * 1e-3),
            "roofline": {"bound": "alu", "kernel": "k_adjoint<1>",
                         "executed_fp32_frac": profiled_fraction("k_adjoint__water_1M.md"),
                         "source": "executed FP32 flops (ncu per-opcode counts, FFMA = 2) over the ncu duration of one"
                                   " launch, profiles/k_adjoint__water_1M.md; null when the kernels changed since"}}


def part_vmf(ctx, dev, flush, torch, stream, steps, F, peak_fp32):
    """The paper's guiding distribution (Sec. 5.5) on the mixed-length batch.
    A p_0 training pass gives the records (cell, w_D, w, n, tau) of its
    admissible chains; the vMF lobes are built from them (timed); the guided
    step draws n from alpha P_0 + (1 - alpha) P_e(n | cell) and (w_D, tau)
    from alpha p_0 + (1 - alpha) p_e, walks and forms the contributions with
    Bernoulli trials from the same mixture.  Both steps replay captured
    graphs, each with the schedule the library's autotuner picks for it (the
    default schedule walks every length in the one-thread form, which at k >= 3
    takes about three times as long on this batch)."""
    import numpy as np
    from paper_2311_12818_gb300 import inputs as I
    from paper_2311_12818_gb300 import mpg
    wl = I.mixed()
    sc = mpg.Scene(ctx, wl)
    P = mpg.params_from(wl.params, walk_mode=mpg.WALK_BATCHED, tau_random=True, k_uniform=0)
    ch0, chv = mpg.Chains(wl, device=dev), mpg.Chains(wl, device=dev)
    res0 = mpg.Contribution.empty(wl.B, wl.Q, device=dev)
    resv = mpg.Contribution.empty(wl.B, wl.Q, device=dev)
    p0w = I.GEOMETRIC_K_WEIGHTS
    # training pass with p_0 and its records
    mpg.mpg_sample_seeds(ctx, sc, None, ch0, P, wl.rng_seed, 1 << 40)
    mpg.mpg_manifold_walk(ctx, sc, ch0, P)
    mpg.mpg_chain_contribution(ctx, sc, None, ch0, P, wl.rng_seed, 1 << 40, out=res0)
    rec = mpg.mpg_guide_records(ctx, sc, ch0, res0.contrib, with_types=True)
    g = mpg.VmfGuide(wl.n_cells, wl.B)

    def build(i):
        mpg.mpg_vmf_build(ctx, g, rec[0], rec[1], rec[2], rec[3], rec[4], R=wl.B, R_dev=rec[5],
                          weight_shift=wl.params.weight_shift)
    build(0)
    ctx.sync()
    R = int(rec[5][0].item())
    L = g.n_lobes
    keys = (rec[0][:R].long().cpu().numpy() << 11) | ((rec[3][:R].long().cpu().numpy() - 1) << 8) | \
        rec[4][:R].long().cpu().numpy()
    sizes = np.unique(keys, return_counts=True)[1].astype(np.float64)
    pairs = float((sizes * (sizes - 1)).sum())
    b_ms = timed_loop(build, steps, 2, flush, stream, torch)
    out = {"workload": "mixed_k1to8, 4,194,304 chains; vMF lobes from the %d records of a p_0 training pass" % R,
           "lobes": L, "groups": int(sizes.size), "largest_group": int(sizes.max()),
           "nearest_neighbour_pair_tests": pairs,
           "build": {"ms": b_ms, "lobes_per_s": L / (b_ms * 1e-3), "pair_tests_per_s": pairs / (b_ms * 1e-3),
                     "launches": 1 + 3 * 3 + 5}}

    def measure(guided):
        ch, res = (chv, resv) if guided else (ch0, res0)
        gg = g if guided else None
        if guided:
            mpg.mpg_sample_lengths(ctx, g, ch, p0w, P, wl.rng_seed, 0, out=(ch.k, ch.pn))
        Ps, _ = mpg.mpg_autotune(ctx, sc, gg, ch, P, wl.rng_seed, 1 << 45, repeats=1)

        def step(o, s=None):
            if guided:
                mpg.mpg_sample_lengths(ctx, g, ch, p0w, Ps, wl.rng_seed, o, out=(ch.k, ch.pn), stream=s)
            mpg.mpg_sample_seeds(ctx, sc, gg, ch, Ps, wl.rng_seed, o, stream=s)
            mpg.mpg_manifold_walk(ctx, sc, ch, Ps, stream=s)
            mpg.mpg_chain_contribution(ctx, sc, gg, ch, Ps, wl.rng_seed, o, out=res, stream=s)
        step(0)
        torch.cuda.synchronize()
        gr = mpg.Graph(ctx, rng_advance=wl.B)
        with gr:
            step(3 << 32)
        ctx.reset_stats()
        ms = timed_loop(lambda i: gr.launch(), steps, 2, flush, stream, torch)
        st = ctx.stats()
        per = steps + 2
        fl = algorithmic_flops(st, F) / per
        # per-family launch time (events around each launch on its stream; the
        # per-length streams overlap) in an uncaptured pass of the same step
        ctx.profile(reset=True)
        ctx.set_profile(True)
        step(9 << 32)
        ctx.sync()
        ctx.set_profile(False)
        fam = {mpg.KERNEL_NAMES[kind]: ctx.profile(kind)[0] for kind in range(len(mpg.KERNEL_NAMES))}
        ctx.profile(reset=True)
        c = res.contrib
        adm = int((c > 0).sum().item())
        return {"ms_per_step": ms, "converged_walks_per_s": st["converged"] / per / (ms * 1e-3),
                "walks_per_s": st["walks"] / per / (ms * 1e-3), "fp32_tflops": fl / (ms * 1e-3) / 1e12,
                "fp32_frac": fl / (ms * 1e-3) / peak_fp32, "trials_per_step": st["trials"] / per,
                "admissible_per_step": adm, "capped_per_step": int(res.capped.sum().item()),
                "mean_E": float(res.E.double().mean().item()),
                "mean_E_std_err": float(res.E.double().std().item() / np.sqrt(wl.Q)),
                "graph_kernels": gr.kernels(), "family_ms_uncaptured": fam,
                "schedule": {f: getattr(Ps, f) for f in mpg.SCHEDULE_FIELDS}}
    out["p0_step"] = measure(False)
    out["vmf_step"] = measure(True)
    out["admissible_chains_per_ms"] = {k: out[k]["admissible_per_step"] / out[k]["ms_per_step"]
                                       for k in ("p0_step", "vmf_step")}
    return out


def part_repeats(ctx, dev, flush, torch, stream, steps):
    """The repeated reciprocal-probability estimate of the paper's performance
    analysis on the benchmark's guided glass-sphere step: one estimate per
    chain, four in rendering only (R x 4), four in training and rendering
    (TR x 4).  Per configuration: a p_0 training pass builds the histogram
    guide, the guided step replays a captured graph (ms, converged walks/s),
    and two independent guided steps give the per-point variance of E as half
    the mean squared difference of their images."""
    import dataclasses
    from paper_2311_12818_gb300 import inputs as I
    from paper_2311_12818_gb300 import mpg
    wl = I.glass_sphere()
    sc = mpg.Scene(ctx, wl)
    ch = mpg.Chains(wl, device=dev)
    res = mpg.Contribution.empty(wl.B, wl.Q, device=dev)
    rec = (torch.zeros(wl.B, dtype=torch.int32, device=dev), torch.zeros((3, wl.B), dtype=torch.float32, device=dev),
           torch.zeros(wl.B, dtype=torch.float32, device=dev), torch.zeros(4, dtype=torch.int32, device=dev))
    g = mpg.Guide(wl.n_cells, I.guide_edges(), device=dev)

    def params(r):
        return mpg.params_from(dataclasses.replace(wl.params, bern_repeats=r), walk_mode=mpg.WALK_BATCHED,
                               k_uniform=2)
    out = {"workload": "glass_sphere_k2 guided, 1,048,576 chains per step; histogram guide from a p_0 pass"}
    for name, r_train, r_render in (("single", 1, 1), ("R_x4", 1, 4), ("TR_x4", 4, 4)):
        Pt, Pr = params(r_train), params(r_render)
        mpg.mpg_sample_seeds(ctx, sc, None, ch, Pt, wl.rng_seed, 1 << 40)
        mpg.mpg_manifold_walk(ctx, sc, ch, Pt)
        mpg.mpg_chain_contribution(ctx, sc, None, ch, Pt, wl.rng_seed, 1 << 40, out=res)
        mpg.mpg_guide_records(ctx, sc, ch, res.contrib, out=rec)
        mpg.mpg_guide_clear(ctx, g)
        mpg.mpg_guide_update(ctx, g, rec[0], rec[1], rec[2], R=wl.B, R_dev=rec[3], weight_shift=wl.params.weight_shift)

        def step(o, P=Pr):
            mpg.mpg_sample_seeds(ctx, sc, g, ch, P, wl.rng_seed, o)
            mpg.mpg_manifold_walk(ctx, sc, ch, P)
            mpg.mpg_chain_contribution(ctx, sc, g, ch, P, wl.rng_seed, o, out=res)
        images = []
        for o in (5 << 32, 6 << 32):
            step(o)
            ctx.sync()
            images.append(res.E.double().clone())
        var = float(((images[0] - images[1]) ** 2).mean().item() / 2)
        gr = mpg.Graph(ctx, rng_advance=wl.B)
        with gr:
            step(7 << 32)
        ctx.reset_stats()
        ms = timed_loop(lambda i: gr.launch(), steps, 2, flush, stream, torch)
        st = ctx.stats()
        per = steps + 2
        out[name] = {"train_repeats": r_train, "render_repeats": r_render, "ms_per_step": ms,
                     "converged_walks_per_s": st["converged"] / per / (ms * 1e-3),
                     "trials_per_step": st["trials"] / per, "mean_E": float(images[0].mean().item()),
                     "per_point_variance_of_E": var}
    for name in ("R_x4", "TR_x4"):
        out[name]["variance_vs_single"] = out[name]["per_point_variance_of_E"] / out["single"]["per_point_variance_of_E"]
        out[name]["time_vs_single"] = out[name]["ms_per_step"] / out["single"]["ms_per_step"]
    return out


def part_glossy(ctx, dev, flush, torch, stream, steps):
    """Glossy separators (Sec. 5.7) on the mixed batch: the receivers carry a
    normalised Phong lobe (exponent 20) around the mirror direction of rays
    from a camera at (0, -3, 1).  A p_0 pass gives the records; one histogram
    guide takes their weights as they are (Eq. eq_weight), the other multiplied
    by the separator's BSDF (product importance sampling, Eq. eq_weight_pis).
    Per guide: the guided step's time, and the per-point variance of the
    radiance toward the camera from two independent steps."""
    from paper_2311_12818_gb300 import inputs as I
    from paper_2311_12818_gb300 import mpg
    wl = I.mixed()
    cam, e = (0.0, -3.0, 1.0), 20.0
    sc = mpg.Scene(ctx, wl)
    ch = mpg.Chains(wl, device=dev)
    res = mpg.Contribution.empty(wl.B, wl.Q, device=dev)
    P = mpg.params_from(wl.params, walk_mode=mpg.WALK_BATCHED, tau_random=True, k_uniform=0)
    mpg.mpg_sample_seeds(ctx, sc, None, ch, P, wl.rng_seed, 1 << 40)
    mpg.mpg_manifold_walk(ctx, sc, ch, P)
    mpg.mpg_chain_contribution(ctx, sc, None, ch, P, wl.rng_seed, 1 << 40, out=res)
    rec = mpg.mpg_guide_records(ctx, sc, ch, res.contrib, with_chain=True)
    guides = {}
    tree = mpg.STree(ctx, ch, rec[5], R=wl.B, R_dev=rec[6])  # over the p_0 pass's samples
    for name in ("plain_weights", "product_weights"):
        w = rec[2].clone()
        if name == "product_weights":
            mpg.mpg_records_bsdf(ctx, ch, rec[5], rec[1], w, cam, e, R=wl.B, R_dev=rec[6])
        g = mpg.Guide(wl.n_cells, I.guide_edges(), device=dev)
        mpg.mpg_guide_update(ctx, g, rec[0], rec[1], w, R=wl.B, R_dev=rec[6], weight_shift=wl.params.weight_shift)
        guides["cell_histogram_" + name] = (g, None)
        lr = tree.records((rec[0], rec[1], w, rec[3], rec[4]), wl.B)
        v = mpg.VmfGuide(tree.n_leaves, max(tree.n_members, 1))
        mpg.mpg_vmf_build(ctx, v, *lr[:5], R=lr[0].numel(), R_dev=lr[5], weight_shift=wl.params.weight_shift)
        guides["tree_vmf_" + name] = (v, tree)
    leaves = tree.query(ch)
    out = {"workload": "mixed_k1to8, 4,194,304 chains; Phong separator (exponent %g), camera at %s; tree of %d "
                       "leaves" % (e, cam, tree.n_leaves)}
    for name, (g, t) in guides.items():
        def step(o, g=g, t=t):
            ch.chain_cell = leaves if t is not None else None
            mpg.mpg_sample_seeds(ctx, sc, g, ch, P, wl.rng_seed, o)
            mpg.mpg_manifold_walk(ctx, sc, ch, P)
            mpg.mpg_chain_contribution(ctx, sc, g, ch, P, wl.rng_seed, o, out=res)
        imgs = []
        for o in (5 << 36, 6 << 36):
            step(o)
            _, L = mpg.mpg_separator_bsdf(ctx, ch, res.contrib, cam, e)
            ctx.sync()
            imgs.append(L.double().clone())
        ms = timed_loop(lambda i: step((7 << 36) + i * wl.B), max(2, steps // 5), 1, flush, stream, torch)
        out[name] = {"ms_per_step": ms, "mean_radiance": float(imgs[0].mean().item()),
                     "per_point_variance": float(((imgs[0] - imgs[1]) ** 2).mean().item() / 2)}
    ch.chain_cell = None
    for kind in ("cell_histogram_", "tree_vmf_"):
        out[kind + "product_over_plain_variance"] = (out[kind + "product_weights"]["per_point_variance"]
                                                     / out[kind + "plain_weights"]["per_point_variance"])
    return out


def part_glossy_chains(ctx, dev, flush, torch, stream, steps, F, peak_fp32):
    """Glossy chains (Sec. 5.7) on the glass sphere with a rough surface
    (Beckmann alpha = 0.05): seeds, offset normals, walks to C = o and the
    estimate W with Bernoulli trials walked with the chain's offsets (the
    plain kernels), beside the specular plain step on the same seeds."""
    import dataclasses
    from paper_2311_12818_gb300 import inputs as I
    from paper_2311_12818_gb300 import mpg
    alpha = 0.05
    wl = I.glass_sphere()
    wl = dataclasses.replace(wl, params=dataclasses.replace(wl.params, roughness=alpha))
    sc = mpg.Scene(ctx, wl)
    ch = mpg.Chains(wl, device=dev)
    res = mpg.Contribution.empty(wl.B, wl.Q, device=dev)
    off = torch.zeros((8, 2, wl.B), dtype=torch.float32, device=dev)
    P = mpg.params_from(wl.params, walk_mode=mpg.WALK_PLAIN, k_uniform=2)
    out = {"workload": "glass_sphere_k2 with rough interfaces (Beckmann alpha %.2f), 1,048,576 chains, p_0 seeds"
                       % alpha}
    for name, glossy in (("specular_plain", False), ("glossy", True)):
        def step(i, glossy=glossy):
            ch.offset = None
            mpg.mpg_sample_seeds(ctx, sc, None, ch, P, wl.rng_seed, i * wl.B)
            if glossy:
                mpg.mpg_sample_offsets(ctx, ch, alpha, wl.rng_seed, i * wl.B, out=off)
                ch.offset = off
            mpg.mpg_manifold_walk(ctx, sc, ch, P)
            mpg.mpg_chain_contribution(ctx, sc, None, ch, P, wl.rng_seed, i * wl.B, out=res)
        step(0)
        ctx.sync()
        ctx.reset_stats()
        ms = timed_loop(step, steps, 2, flush, stream, torch)
        st = ctx.stats()
        per = steps + 2
        fl = algorithmic_flops(st, F) / per
        out[name] = {"ms_per_step": ms, "converged_walks_per_s": st["converged"] / per / (ms * 1e-3),
                     "contributions_per_step": int((res.T > 0).sum().item()),
                     "mean_E": float(res.E.double().mean().item()),
                     "fp32_tflops": fl / (ms * 1e-3) / 1e12, "fp32_frac": fl / (ms * 1e-3) / peak_fp32}
    ch.offset = None
    return out


def part_selective(ctx, dev, flush, torch, stream, steps):
    """Selective activation (Sec. 5.8) on the benchmark's guided glass-sphere
    step: points whose guide cell holds no weight after the p_0 training pass
    draw no seed.  Step time and active fraction with and without it; the
    image of the active points is unchanged (same seeds)."""
    import dataclasses
    from paper_2311_12818_gb300 import inputs as I
    from paper_2311_12818_gb300 import mpg
    wl = I.glass_sphere()
    sc = mpg.Scene(ctx, wl)
    ch = mpg.Chains(wl, device=dev)
    res = mpg.Contribution.empty(wl.B, wl.Q, device=dev)
    g = mpg.Guide(wl.n_cells, I.guide_edges(), device=dev)
    P = mpg.params_from(wl.params, walk_mode=mpg.WALK_BATCHED, k_uniform=2)
    mpg.mpg_sample_seeds(ctx, sc, None, ch, P, wl.rng_seed, 1 << 40)
    mpg.mpg_manifold_walk(ctx, sc, ch, P)
    mpg.mpg_chain_contribution(ctx, sc, None, ch, P, wl.rng_seed, 1 << 40, out=res)
    rec = mpg.mpg_guide_records(ctx, sc, ch, res.contrib)
    mpg.mpg_guide_update(ctx, g, rec[0], rec[1], rec[2], R=wl.B, R_dev=rec[3], weight_shift=wl.params.weight_shift)
    ctx.sync()
    active_cells = (g.counts.sum(dim=1) > 0).cpu()
    active = float(active_cells[torch.as_tensor(wl.cell.astype("int64"))].float().mean().item())
    out = {"workload": "glass_sphere_k2 guided, 1,048,576 chains", "active_point_fraction": active}
    images = {}
    for name, sel in (("off", 0), ("on", 1)):
        Ps = mpg.params_from(dataclasses.replace(wl.params, selective=sel), walk_mode=mpg.WALK_BATCHED, k_uniform=2)

        def step(o, Ps=Ps):
            mpg.mpg_sample_seeds(ctx, sc, g, ch, Ps, wl.rng_seed, o)
            mpg.mpg_manifold_walk(ctx, sc, ch, Ps)
            mpg.mpg_chain_contribution(ctx, sc, g, ch, Ps, wl.rng_seed, o, out=res)
        step(3 << 32)
        ctx.sync()
        images[name] = res.E.clone()
        gr = mpg.Graph(ctx, rng_advance=wl.B)
        with gr:
            step(3 << 32)
        ctx.reset_stats()
        ms = timed_loop(lambda i: gr.launch(), steps, 2, flush, stream, torch)
        st = ctx.stats()
        out[name] = {"ms_per_step": ms, "seeds_per_step": st["seeds"] / (steps + 2),
                     "converged_per_step": st["converged"] / (steps + 2)}
    pts = torch.as_tensor(active_cells.numpy()[wl.cell.astype("int64")], device=dev)
    out["image_equal_on_active_points"] = bool(torch.equal(images["off"][pts], images["on"][pts]))
    out["on"]["time_vs_off"] = out["on"]["ms_per_step"] / out["off"]["ms_per_step"]
    return out


def part_progressive(ctx, dev, flush, torch, stream, steps):
    """Online training and rendering (Sec. 5.8) of the glass-sphere image with
    a budget of 64 seeds per receiver point (256 x 256 points): training
    iterations of 1, 2, 4 and 12 seeds per point, each building the next guide
    from its own records, then 45 seeds per point of rendering; the whole
    schedule is one captured graph.  Two replays at independent random numbers
    give the per-point variance of the image (half the mean squared
    difference), against the same for 64 seeds per point from p_0 alone."""
    from paper_2311_12818_gb300 import inputs as I
    from paper_2311_12818_gb300 import mpg
    from paper_2311_12818_gb300 import progressive as PG
    out = {"workload": "glass_sphere_k2, 256 x 256 points, 64 seeds per point in total"}

    def variance(a, b):
        return float(((a - b) ** 2).mean().item() / 2)
    for kind in ("histogram", "vmf", "vmf_tree", "vmf_tree_levels"):
        pr = PG.Progressive(ctx, PG.glass_sphere_stages(n=256), total_spp=64, guide=kind.replace("_levels", ""),
                            device=dev, tree_method=mpg.STREE_LEVELS if kind.endswith("_levels") else mpg.STREE_RECURSIVE)
        pr.run(0)
        ctx.sync()
        if kind.startswith("vmf_tree"):  # tree builds synchronise with the host: timed uncaptured
            run = lambda i: pr.run((1 << 44) + (i << 40))  # noqa: E731
            gr = None
        else:
            gr = pr.capture(offset=1 << 44, advance=1 << 40)
            run = lambda i: gr.launch()  # noqa: E731
        ctx.reset_stats()
        ms = timed_loop(run, steps, 2, flush, stream, torch)
        st = ctx.stats()
        per = steps + 2
        run(100)
        ctx.sync()
        a = pr.image.double().clone()
        run(101)
        ctx.sync()
        out[kind] = {"plan_spp": pr.plan, "render_spp": pr.render_spp, "chains": pr.total_chains(),
                     "ms_per_schedule": ms, "converged_walks_per_s": st["converged"] / per / (ms * 1e-3),
                     "graph_kernels": gr.kernels() if gr is not None else None, "captured": gr is not None,
                     "mean_E": float(a.mean().item()), "per_point_variance_of_E": variance(a, pr.image.double())}
        if kind.startswith("vmf_tree"):
            out[kind]["leaves_last_training_iteration"] = pr.trees[(len(pr.plan) - 1) % 2].n_leaves
            out[kind]["tree_build"] = "level by level on the device" if kind.endswith("_levels") else \
                "depth first on the host (positions gathered on the device)"
        del gr, pr
    wl = I.glass_sphere(n=256, spq=64)
    sc = mpg.Scene(ctx, wl)
    ch = mpg.Chains(wl, device=dev)
    res = mpg.Contribution.empty(wl.B, wl.Q, device=dev)
    P = mpg.params_from(wl.params, walk_mode=mpg.WALK_BATCHED, k_uniform=2)
    imgs = []
    for o in (1 << 44, (1 << 44) + (1 << 40)):
        mpg.mpg_sample_seeds(ctx, sc, None, ch, P, wl.rng_seed, o)
        mpg.mpg_manifold_walk(ctx, sc, ch, P)
        mpg.mpg_chain_contribution(ctx, sc, None, ch, P, wl.rng_seed, o, out=res)
        ctx.sync()
        imgs.append(res.E.double().clone())
    out["p0_only"] = {"spp": 64, "chains": wl.B, "mean_E": float(imgs[0].mean().item()),
                      "per_point_variance_of_E": variance(imgs[0], imgs[1])}
    for kind in ("histogram", "vmf", "vmf_tree", "vmf_tree_levels"):
        out[kind]["variance_vs_p0_only"] = out[kind]["per_point_variance_of_E"] / out["p0_only"]["per_point_variance_of_E"]
    return out


def run_part(args):
    """One secondary measurement alone (--part), for profiling a single kernel."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    props = torch.cuda.get_device_properties(dev)
    peak = props.multi_processor_count * 128 * 2 * 2070.0 * 1e6
    if args.part == "configs":
        print(json.dumps({"part": args.part, **other_configs(args, dev, flush, torch, peak)}))
        return
    if args.part == "mixed_step":
        print(json.dumps({"part": args.part, **part_mixed_step(args, dev, torch)}))
        return
    if args.part == "stree":
        print(json.dumps({"part": args.part, **part_stree(args, dev, torch)}))
        return
    print(json.dumps({"part": args.part, **secondary(args, dev, flush, torch, peak, parts=(args.part,))}))


def part_mixed_step(args, dev, torch):
    """Uncaptured steps of the mixed-length batch (4 n x 2 n receiver points x 8
    seeds; n = 256 is the full configuration) with the schedule the autotuner
    usually picks for it (lane-group walks and rounds, refills every 4 passes,
    one synchronous round, first parallel batch of 16): a short program whose
    launches ncu can list or capture one by one."""
    from paper_2311_12818_gb300 import inputs as I
    from paper_2311_12818_gb300 import mpg
    ctx = mpg.Context(dev.index or 0)
    wl = I.mixed(nx=4 * args.n, ny=2 * args.n)
    P = mpg.params_from(wl.params, walk_mode=mpg.WALK_BATCHED, tau_random=wl.tau_random, walk_group=3,
                        refill_every=4, trial_sync_rounds=1, trial_batch=16)
    sc = mpg.Scene(ctx, wl)
    ch = mpg.Chains(wl, device=dev)
    out = mpg.Contribution.empty(wl.B, wl.Q, device=dev)
    ms = []
    for j in range(max(2, args.steps)):
        o = (1 << 40) + j * wl.B
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        mpg.mpg_sample_seeds(ctx, sc, None, ch, P, wl.rng_seed, o)
        mpg.mpg_manifold_walk(ctx, sc, ch, P)
        mpg.mpg_chain_contribution(ctx, sc, None, ch, P, wl.rng_seed, o, out=out)
        b.record()
        b.synchronize()
        ms.append(a.elapsed_time(b))
    ctx.sync()
    return {"chains": wl.B, "ms_per_step_uncaptured": ms}


def part_stree(args, dev, torch):
    """The spatial tree (Sec. 5.6) over the records of one p_0 pass of the
    glass sphere (n x n points x 16 seeds): the level-by-level device build and
    the depth-first host build timed, and the query of every chain's leaf."""
    from paper_2311_12818_gb300 import inputs as I
    from paper_2311_12818_gb300 import mpg
    ctx = mpg.Context(dev.index or 0)
    wl = I.glass_sphere(n=args.n)
    P = mpg.params_from(wl.params, walk_mode=mpg.WALK_BATCHED, k_uniform=2)
    sc = mpg.Scene(ctx, wl)
    ch = mpg.Chains(wl, device=dev)
    mpg.mpg_sample_seeds(ctx, sc, None, ch, P, wl.rng_seed, 1 << 40)
    mpg.mpg_manifold_walk(ctx, sc, ch, P)
    res = mpg.mpg_chain_contribution(ctx, sc, None, ch, P, wl.rng_seed, 1 << 40)
    rec = mpg.mpg_guide_records(ctx, sc, ch, res.contrib, with_chain=True)
    ctx.sync()
    out = {"chains": wl.B, "records": int(rec[6][0].item())}
    for name, method in (("levels", mpg.STREE_LEVELS), ("recursive", mpg.STREE_RECURSIVE)):
        ms = []
        for _ in range(max(2, args.steps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tree = mpg.STree(ctx, ch, rec[5], R=wl.B, R_dev=rec[6], method=method)
            torch.cuda.synchronize()
            ms.append((time.perf_counter() - t0) * 1e3)
        out[name] = {"build_ms": ms, "leaves": tree.n_leaves, "members": tree.n_members}
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    tree.query(ch)
    b.record()
    b.synchronize()
    out["query_ms"] = a.elapsed_time(b)
    return out


def cpu_sample(n=256, spq=16):
    """Sample of the same workload for the oracle: an n x n receiver grid over
    the same extent with 16 seeds per point (n = 256 is the whole workload)."""
    from paper_2311_12818_gb300 import inputs as I
    return I.glass_sphere(n=n, spq=spq)


def oracle_step(wl, threads):
    """One oracle pass of the hot path (guide trained untimed first); returns
    (seconds, converged walks)."""
    import numpy as np

    from oracle import oracle as O
    from paper_2311_12818_gb300 import inputs as I
    sc = O.Scene(wl)
    s0 = O.sample_seeds(wl, sc, None, threads=threads, rng_offset=1 << 40)
    c0 = O.walk(wl, sc, s0, threads=threads)
    k0 = O.contribution(wl, sc, c0, threads=threads)
    N0, _ = O.bernoulli(wl, sc, c0, k0["admissible"], threads=threads, rng_offset=1 << 40)
    g = O.Guide(wl.n_cells, I.guide_edges())
    g.update(*O.records(wl, c0, k0["T"], N0, k0["admissible"]), wl.params.weight_shift)
    t0 = time.perf_counter()
    s = O.sample_seeds(wl, sc, g, threads=threads)
    c = O.walk(wl, sc, s, threads=threads)
    k = O.contribution(wl, sc, c, threads=threads)
    tw = np.zeros(wl.B, np.uint32)
    N, _ = O.bernoulli(wl, sc, c, k["admissible"], g, threads=threads, trial_walks=tw)
    E = O.irradiance(wl, k["T"], N, k["admissible"])
    g2 = O.Guide(wl.n_cells, I.guide_edges())
    g2.update(*O.records(wl, c, k["T"], N, k["admissible"]), wl.params.weight_shift)
    dt = time.perf_counter() - t0
    conv = int((c["status"] == 1).sum() + tw.sum())
    del E
    return dt, conv


def cpu_baseline(wl_full):
    """The oracle on all host cores (the whole workload) and on one core (a
    64 x 64-point sample of it, same extent and seeds per point)."""
    threads = os.cpu_count() or 1
    wl = cpu_sample()
    dt, conv = oracle_step(wl, threads)
    w1 = cpu_sample(n=64)
    dt1, conv1 = oracle_step(w1, 1)
    return {"value": conv / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "the whole workload (%d chains), one guided step after an untimed training pass, %.1f s"
                      % (wl.B, dt),
            "single_core": {"value": conv1 / dt1, "unit": UNIT, "cores": 1,
                            "sample": "64 x 64 receiver points x 16 seeds (%d chains), one guided step, %.1f s"
                                      % (w1.B, dt1)}}


def run_reference(args, rank, world):
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    wl = cpu_sample(n=128)
    times, convs = [], []
    for i in range(args.warmup + args.steps):
        dt, conv = oracle_step(wl, threads)
        if i >= args.warmup:
            times.append(dt)
            convs.append(conv)
    value = sum(convs) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded procedural scene, no dataset)",
            "config": {"workload": WORKLOAD, "sample": "%d chains per step (128x128 points x 16 seeds over the same "
                                                       "receiver extent)" % wl.B},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "%d chains per step, %d steps" % (wl.B, args.steps)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.part:
        run_part(args)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
