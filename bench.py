"""Benchmark of the GAVIS hot path on GB300: one step = visibility-field
construction over every training view + uncertainty scoring of every
candidate view + argmax, on the batched workload (1M Gaussians in three rooms,
200 training views at 1280x720, 256 candidate views at 640x480, colour and
field coefficients in float16, compositing in float32).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gavis|reference]

Prints one JSON line (rank 0).  `value` is candidate views scored per second
of device time with inputs resident in HBM; `e2e` is the same metric through
the C ABI with the scene copied from pinned host memory and the scores read
back inside the timed region.  Under torchrun every rank runs an independent
replica of the workload (the path has no exchange step): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic float32 operations per (pixel, Gaussian) pair, counted
# operation by operation from the algorithms (an FMA counts 2, any other
# float32 add, multiply or compare 1; exp and log go to the special-function
# unit and are listed apart):
#   footprint q = A dx^2 + 2B dx dy + C dy^2 from dx, dy:        9
#   overlap test q <= q_cut:                                      1
#   alpha = o exp(-q/2): scale + multiply (+ 1 exp):              2
# single-view particle visibility (Alg. visibility):
#   sum_T += T, T *= 1 - alpha (FMA), T < eps_T:                  4   -> 16 + 1 exp
# uncertainty + colour (Alg. UQ with eq:alpha_comp, eq:huber, eq:orig_vr):
#   alpha* = a1 alpha + a0 (FMA), w = alpha* T, wv = w V:         4
#   H += -wv ln wv + wv k_c (multiply, add, FMA; + 1 log):        4
#   w0 += w (1 - V) (FMA), T *= 1 - alpha* (FMA), T < eps_T:      5
#   colour: wc = alpha Tc, rgb += wc c (3 FMA), Tc *= 1 - alpha
#   (FMA), Tc < eps_T:                                            10  -> 35 + 1 exp + 1 log
FLOPS_PER_PAIR_UA = 35
FLOPS_PER_PAIR_VIS = 16
FP32_LANES_PER_SM = 128
# warp instructions a Blackwell SM issues per clock (4 schedulers x 1)
ISSUE_PER_SM_CLK = 4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gavis", choices=["gavis", "reference"])
    ap.add_argument("--workload", type=int, default=3, help="workload shape 1..4 (3 = the batched 1M case)")
    ap.add_argument("--n", type=int, default=None, help="override Gaussian count (profiling runs)")
    ap.add_argument("--n-train", type=int, default=None)
    ap.add_argument("--n-cand", type=int, default=None)
    ap.add_argument("--views-per-batch", type=int, default=0)
    ap.add_argument("--tile", type=int, default=0, help="tile edge 8/16/32; 0 = autotune per path")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-views", type=int, default=16,
                    help="cpu_baseline: training and candidate views of the oracle sample (about 10 s of CPU work)")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain unbatched f32 comparison step")
    ap.add_argument("--no-graph", action="store_true", help="skip the CUDA-graph scoring comparison")
    ap.add_argument("--no-precision", action="store_true", help="skip the storage-precision errors vs the oracle")
    ap.add_argument("--precision-views", type=int, default=8,
                    help="precision_err: sampled training and candidate views (about 30 s of CPU work)")
    ap.add_argument("--serving", action="store_true", help="serving workload: Poisson requests over 4 resident scenes")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: mean request rate (req/s)")
    ap.add_argument("--rates", default="", help="serving: comma-separated request rates, one line each")
    ap.add_argument("--serving-budget-gb", type=float, default=120.0, help="serving: HBM admission budget (GB)")
    ap.add_argument("--requests", type=int, default=300, help="serving: number of requests")
    ap.add_argument("--workers", type=int, default=4, help="serving: worker streams")
    ap.add_argument("--batch-views", type=int, default=128, help="serving: views per batch")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(args):
    import scenegen as sg
    return sg.config(args.workload, n=args.n, n_train=args.n_train, n_cand=args.n_cand)


def config_json(c, args, extra=None):
    sc = c["scene"]
    d = {
        "workload": c["name"],
        "gaussians": sc.n,
        "train_views": len(c["train"]),
        "train_wh": [c["train"][0].W, c["train"][0].H],
        "candidate_views": len(c["cand"]),
        "candidate_wh": [c["cand"][0].W, c["cand"][0].H],
        "sh_degree": sc.sh_degree,
        "vf_degree": c["vf_degree"],
        "coeff_storage": c["coeff_dtype"],
        "compositing": "f32",
        "tile": args.tile if args.tile else "autotuned",
        "l2": "inputs and per-view records larger than L2 (no flush needed)",
        "parallelism": "replicas" if args.gpus > 1 else "single",
    }
    if extra:
        d.update(extra)
    return d


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "power_w_max": max(pw),
                "samples": len(sm), "reasons": sorted(reasons)}


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over the ranks of the default process group (x when
    there is none): the job's time is its slowest replica's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, ms: float) -> float:
    """Whole-job units per second: every replica processes units_per_rank in
    the max-over-ranks time ms (weak scaling)."""
    return world * units_per_rank / (ms / 1e3)


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(math.ceil(q / 100.0 * len(xs))) - 1))
    return xs[k]


# ----------------------------------------------------------------------------
# the oracle arm (reference) and the CPU baseline
# ----------------------------------------------------------------------------

def oracle_sample(c, n_views=1):
    """Time the oracle on a bounded sample of the step: `n_views` training
    views (particle visibility + field accumulation) and `n_views` candidate
    views (field query + uncertainty rendering), extrapolated to the full step."""
    import numpy as np
    import oracle
    sc = c["scene"]
    L = c["vf_degree"]
    t0 = time.perf_counter()
    gamma, _, _ = oracle.vf_build(c["train"][:n_views], sc, L)
    t1 = time.perf_counter()
    for cam in c["cand"][:n_views]:
        V, _ = oracle.vf_query(gamma, L, n_views, cam, sc.means)
        rgb, unc, amb, used = oracle.render_view(cam, sc, V)
    t2 = time.perf_counter()
    per_train = (t1 - t0) / n_views
    per_cand = (t2 - t1) / n_views
    step_s = per_train * len(c["train"]) + per_cand * len(c["cand"])
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return dict(step_s=step_s, per_train_s=per_train, per_cand_s=per_cand, cores=cores,
                sample=f"{n_views} training + {n_views} candidate view(s) of the full workload, "
                       f"extrapolated to {len(c['train'])} + {len(c['cand'])} views per step",
                work_s=t2 - t0)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    c = workload(args)
    n_cand = len(c["cand"])
    for _ in range(args.warmup):
        oracle_sample(c, 1)
    times = []
    info = None
    for _ in range(args.steps):
        info = oracle_sample(c, 1)
        times.append(info["step_s"])
    step_s = sum(times) / len(times)
    value = n_cand / step_s
    line = {
        "impl": "reference", "metric": "uncertainty-render views/s at 1M Gaussians (VF build + scoring per step)",
        "value": value, "unit": "views/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": config_json(c, args),
        "cpu_baseline": {"value": value, "unit": "views/s", "cores": info["cores"], "kind": "oracle",
                         "sample": info["sample"]},
        "e2e": {"value": value, "unit": "views/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# the CUDA arm
# ----------------------------------------------------------------------------

def run_gavis(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    import __graft_entry__ as ge
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    if world == 1 or rank == 0:
        ge.build()
    if world > 1:
        dist.barrier(device_ids=[local]) if torch.cuda.is_available() else dist.barrier()
    import paper_2605_30342_gb300 as gv
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    c = workload(args)
    sc = c["scene"]
    cdt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[c["coeff_dtype"]]
    L = c["vf_degree"]
    train, cand = c["train"], c["cand"]
    n_cand = len(cand)

    # inputs: pinned host copies (e2e) and resident device copies (value)
    host = {
        "means": torch.as_tensor(sc.means).pin_memory(),
        "scales": torch.as_tensor(sc.scales).pin_memory(),
        "rots": torch.as_tensor(sc.rots).pin_memory(),
        "opac": torch.as_tensor(sc.opac).pin_memory(),
        "sh": torch.as_tensor(sc.sh).to(cdt).pin_memory(),
    }
    devt = {k: v.to(dev, non_blocking=True) for k, v in host.items()}
    torch.cuda.synchronize()
    gs = gv.Gaussians(devt["means"], devt["scales"], devt["rots"], devt["opac"], devt["sh"], sc.sh_degree)
    ctx = gv.Context(local)
    prm = gv.Params(vf_degree=L, tile=args.tile, views_per_batch=args.views_per_batch)
    vf = gv.VisibilityField(torch.zeros((sc.n, (L + 1) ** 2), dtype=cdt, device=dev), L, 0, 1.0)
    prm_vf, prm_sc = prm, prm
    tuned = None
    if args.tile == 0:
        # autotuner: tile edge per path, timed on 64 training / 64 candidate views (untimed here)
        prm_vf, ms_vf = ctx.autotune(gs, train[:64], None, gv.Params(vf_degree=L, views_per_batch=args.views_per_batch))
        ctx.vf_build(gs, train, degree=L, params=prm_vf, out=vf)
        prm_sc, ms_sc = ctx.autotune(gs, cand[:64], vf, gv.Params(vf_degree=L, views_per_batch=args.views_per_batch))
        tuned = {"vf_build_tile": prm_vf.tile, "score_tile": prm_sc.tile}
    W, H = cand[0].W, cand[0].H
    outs = {"rgb": torch.empty((n_cand, 3, H, W), device=dev), "unc": torch.empty((n_cand, H, W), device=dev),
            "score": torch.empty(n_cand, device=dev), "best_dev": torch.empty(1, dtype=torch.int32, device=dev)}

    def step_host():   # the chain sized on the host: gavis_vf_build + gavis_score_views
        ctx.vf_build(gs, train, degree=L, params=prm_vf, out=vf)
        return ctx.score_views(gs, vf, cand, params=prm_sc, out=outs, sync_best=False)

    for _ in range(max(args.warmup, 0)):
        step_host()
    torch.cuda.synchronize()

    # The scoring chain captured once as a CUDA graph (gavis_plan_*), sized
    # from an instrumented pass; the timed step replays it after the field
    # build.  Its outputs are bit-identical to gavis_score_views (checked
    # below, in graph_scoring).
    recs = gv.camera_records(cand)
    plan, plan_batch, plan_err = None, 0, None
    if not args.no_graph:
        ctx.prof_enable(True)
        ctx.score_views(gs, vf, cand, params=prm_sc, out=outs, sync_best=False)
        r0 = ctx.prof_read()
        ctx.prof_enable(False)
        plan, plan_batch, plan_err = make_plan(gv, ctx, gs, vf, cand, recs, W, H, prm_sc, r0["visible"], r0["keys"])
    use_plan = False
    if plan is not None:
        ms_plan, ms_sv = faster_scoring(ctx, plan, recs, gs, vf, cand, prm_sc, outs)
        use_plan = ms_plan <= ms_sv

    def step():
        ctx.vf_build(gs, train, degree=L, params=prm_vf, out=vf)
        if use_plan:
            plan.launch(recs)
        else:
            ctx.score_views(gs, vf, cand, params=prm_sc, out=outs, sync_best=False)

    res_out = {"score": plan.score, "best_dev": plan.best_dev} if use_plan else outs
    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()

    # ---------------- device-timed region (inputs resident) ----------------
    # value: plain steps, no instrumentation; then the same number of steps
    # with stage events (per-stage device times for the roofline)
    ctx.prof_enable(False)
    launches0 = ctx.prof_read()["total_launches"]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier(device_ids=[local])
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record(stream)
    for k in range(args.steps):
        step()
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier(device_ids=[local])
    clocks = sampler.stop()
    step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    total_ms = evs[0].elapsed_time(evs[-1])
    launches = ctx.prof_read()["total_launches"] - launches0
    best = int(res_out["best_dev"].item())
    # stage events over the same number of steps of the host-sized chain
    # (the same kernels; a graph replay records no per-stage events)
    ctx.prof_enable(True)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for k in range(args.steps):
        step_host()
    p1.record(stream)
    torch.cuda.synchronize()
    prof = ctx.prof_read()
    ctx.prof_enable(False)
    instrumented_ms = p0.elapsed_time(p1) / args.steps

    total_ms = max_over_ranks(total_ms, dev)
    ms_per_step = total_ms / args.steps
    value = job_throughput(n_cand, world, ms_per_step)

    # ---------------- per-call work counts (one untimed instrumented pass) ----------------
    # (the composited pairs are counted here, with the device counters on; the
    # timed steps record stage events only)
    ctx.prof_enable(True, pairs=True)
    ctx.vf_build(gs, train, degree=L, params=prm_vf, out=vf)
    r_vf = ctx.prof_read()
    vis_vf, keys_vf, pairs_vis = r_vf["visible"], r_vf["keys"], r_vf["pairs"][1]
    sorted_vf = r_vf["sorted_keys"]
    ctx.prof_enable(True, pairs=True)
    ctx.score_views(gs, vf, cand, params=prm_sc, out=outs, sync_best=False)
    r_sc = ctx.prof_read()
    vis_sc, keys_sc, pairs_ua = r_sc["visible"], r_sc["keys"], r_sc["pairs"][0]
    sorted_sc = r_sc["sorted_keys"]
    ctx.prof_enable(False)
    b = torch.tensor([], dtype=cdt).element_size()
    K, Kc = (L + 1) ** 2, (sc.sh_degree + 1) ** 2
    # per-view byte model: centres of every Gaussian for culling, the rest of
    # the record for visible ones, outputs (visibility sums, or rgb + unc)
    bytes_vf = len(train) * sc.n * 12 + vis_vf * (32 + 8) + sc.n * K * b
    bytes_sc = n_cand * sc.n * 12 + vis_sc * (32 + Kc * 3 * b + K * b) + n_cand * W * H * 16
    model_bytes = bytes_vf + bytes_sc
    hbm = {"model_bytes_per_step": int(model_bytes), "achieved_gbs": model_bytes / (ms_per_step / 1e3) / 1e9,
           "peak_gbs": peaks()[0].get("hbm_gbs"),
           "frac": model_bytes / (ms_per_step / 1e3) / 1e9 / peaks()[0].get("hbm_gbs", 6800.0),
           "visible_records": {"vf_build": int(vis_vf), "score": int(vis_sc)},
           "note": "per-view algorithmic bytes (Gaussian data counted once per view; the batched chain "
                   "reads it once per batch), divided by the device time of the step"}

    # ---------------- the plain unbatched f32 path, for comparison ----------------
    plain = None
    if not args.no_plain:
        sh32 = devt["sh"].float().contiguous()
        gs32 = gv.Gaussians(devt["means"], devt["scales"], devt["rots"], devt["opac"], sh32, sc.sh_degree)
        vf32 = gv.VisibilityField(torch.zeros((sc.n, (L + 1) ** 2), device=dev), L, 0, 1.0)
        pp = gv.Params(vf_degree=L, tile=16, views_per_batch=1)

        def plain_step():
            ctx.vf_build(gs32, train, degree=L, params=pp, out=vf32)
            return ctx.score_views(gs32, vf32, cand, params=pp, out=outs, sync_best=False)

        plain_step()
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        plain_step()
        p1.record(stream)
        torch.cuda.synchronize()
        plain_ms = p0.elapsed_time(p1)
        plain = {"ms_per_step": plain_ms, "views_per_s": n_cand / (plain_ms / 1e3),
                 "speedup_of_batched": plain_ms / ms_per_step,
                 "what": "f32 colour and field coefficients, one view per kernel chain, tile 16, one step; "
                         "both paths pass the same oracle parity gate"}
        del sh32, gs32, vf32
        # restore the benchmark's field (the plain step overwrote the outputs only)
        ctx.score_views(gs, vf, cand, params=prm_sc, out=outs, sync_best=False)

    # ---------------- scoring replayed as one CUDA graph, against the host-sized call ----------------
    graph = {"skipped": plan_err} if plan_err else None
    if plan is not None:
        for _ in range(3):
            plan.launch(recs)
            ctx.score_views(gs, vf, cand, params=prm_sc, out=outs, sync_best=False)
        torch.cuda.synchronize()
        same = bool(torch.equal(plan.score, outs["score"])) and int(plan.best_dev.item()) == int(outs["best_dev"].item())
        g0, g1, g2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        g0.record(stream)
        for _ in range(args.steps):
            plan.launch(recs)
        g1.record(stream)
        for _ in range(args.steps):
            ctx.score_views(gs, vf, cand, params=prm_sc, out=outs, sync_best=False)
        g2.record(stream)
        torch.cuda.synchronize()
        graph = {"ms_per_scoring": g0.elapsed_time(g1) / args.steps,
                 "score_views_ms": g1.elapsed_time(g2) / args.steps, "identical_to_score_views": same,
                 "overflowed": plan.overflowed()[0], "kernels_per_launch": plan.kernels,
                 "views_per_batch": plan_batch or n_cand,
                 "timed_step_uses_plan": use_plan,
                 "what": "the candidate-scoring chain captured once (gavis_plan_create) and replayed per step"}

    # ---------------- end to end through host buffers ----------------
    e2e_steps = max(1, args.e2e_steps)
    h2d = sum(v.numel() * v.element_size() for v in host.values()) + gv.camera_records(train)._length_ * 96 \
        + gv.camera_records(cand)._length_ * 96
    d2h = n_cand * 4 + 4
    score_h = torch.empty(n_cand).pin_memory()
    best_h = torch.empty(1, dtype=torch.int32).pin_memory()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier(device_ids=[local])
    # The geometry (centres, scales, rotations, opacities) is copied on the
    # step's stream ahead of the field build; the colour coefficients, read
    # only by the scoring chain, are copied on a second stream while the field
    # is built, and the scoring waits for that copy.
    side = torch.cuda.Stream()
    geo_keys = [k for k in host if k != "sh"]
    sh_done = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(e2e_steps + 1)]

    def e2e_step(k_, ev_k=None):
        if ev_k is not None:
            ev_k[0].record(stream)
        for k in geo_keys:
            devt[k].copy_(host[k], non_blocking=True)
        side.wait_stream(stream)   # the previous step's scoring has read the coefficients
        with torch.cuda.stream(side):
            sh_done[k_][0].record(side)
            devt["sh"].copy_(host["sh"], non_blocking=True)
            sh_done[k_][1].record(side)
        if ev_k is not None:
            ev_k[1].record(stream)
        ctx.vf_build(gs, train, degree=L, params=prm_vf, out=vf)
        stream.wait_event(sh_done[k_][1])
        if use_plan:
            plan.launch(recs)
        else:
            ctx.score_views(gs, vf, cand, params=prm_sc, out=outs, sync_best=False)
        if ev_k is not None:
            ev_k[2].record(stream)
        score_h.copy_(res_out["score"], non_blocking=True)
        best_h.copy_(res_out["best_dev"], non_blocking=True)
        if ev_k is not None:
            ev_k[3].record(stream)

    # untimed warm-up of the end-to-end loop (the first copy after the legs
    # above pays a one-time cost of the driver)
    for _ in range(max(args.warmup, 1)):
        e2e_step(e2e_steps)
    torch.cuda.synchronize()
    # events between the parts of each step (device time of the copies and of the step)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(e2e_steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_host0 = time.perf_counter()
    e0.record(stream)
    for k_ in range(e2e_steps):
        e2e_step(k_, ev[k_])
    e1.record(stream)
    torch.cuda.synchronize()
    t_host = (time.perf_counter() - t_host0) * 1e3 / e2e_steps
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / e2e_steps, dev)
    e2e_value = job_throughput(n_cand, world, e2e_ms)
    e2e_parts = {"h2d_ms_each": [round(e[0].elapsed_time(e[1]), 3) for e in ev],
                 "step_ms_each": [round(e[1].elapsed_time(e[2]), 3) for e in ev],
                 "h2d_ms": sum(e[0].elapsed_time(e[1]) for e in ev) / e2e_steps,
                 "step_ms": sum(e[1].elapsed_time(e[2]) for e in ev) / e2e_steps,
                 "d2h_ms": sum(e[2].elapsed_time(e[3]) for e in ev) / e2e_steps,
                 "sh_h2d_ms_overlapped": sum(sh_done[k][0].elapsed_time(sh_done[k][1]) for k in range(e2e_steps))
                                         / e2e_steps,
                 "what": "h2d_ms: the geometry copies on the step's stream; the colour coefficients are copied "
                         "on a second stream during the field build (sh_h2d_ms_overlapped) and the scoring "
                         "waits for them; step_ms: field build + scoring incl. that wait",
                 "host_wall_ms": t_host}

    # ---------------- roofline of the dominant kernel ----------------
    st = prof["stages"]
    pk, pk_kind = peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    work = dict(steps=args.steps, workload=args.workload, pairs_ua=pairs_ua, pairs_vis=pairs_vis,
                tile_sc=prm_sc.tile, tile_vf=prm_vf.tile, n_cand=n_cand, n_train=len(train), W=W, H=H,
                vis_vf=vis_vf, vis_sc=vis_sc, sorted_vf=sorted_vf, sorted_sc=sorted_sc, n=sc.n, K=K, Kc=Kc, b=b)
    roof = stage_roofline(st, work, pk, pk_kind, n_sm)

    # ---------------- storage precision against the float64 oracle ----------------
    prec = None
    if rank == 0 and world == 1 and not args.no_precision and cdt != torch.float32:
        prec = precision_errors(gv, ctx, c, gs, cdt, prm_vf, prm_sc, args.precision_views)

    # ---------------- CPU baseline (rank 0, N = 1) ----------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        info = oracle_sample(c, args.cpu_sample_views)
        cpu = {"value": n_cand / info["step_s"], "unit": "views/s", "cores": info["cores"], "kind": "oracle",
               "sample": info["sample"], "work_s": info["work_s"]}

    if rank == 0:
        line = {
            "metric": "uncertainty-render views/s at 1M Gaussians (VF build + scoring per step)",
            "value": value, "unit": "views/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": config_json(c, args, dict({"autotuned": tuned} if tuned else {}, scoring_path=(
                "gavis_plan_launch: the scoring chain (the uncertainty pass one persistent launch per batch) "
                "captured once as a CUDA graph and replayed" if use_plan else
                "gavis_score_views (the chain sized on the host)") + "; the faster of the two, measured before "
                "the timed steps (both in graph_scoring)", field_path="gavis_vf_build")),
            "e2e": {"value": e2e_value, "unit": "views/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms, "steps": e2e_steps, "parts": e2e_parts},
            "gpu_launches": int(launches),
            "roofline": roof,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "latency_ms": {"p50": percentile(step_ms, 50), "p99": percentile(step_ms, 99), "what": "one step"},
            "stages_ms_per_step": {k: v[0] / args.steps for k, v in st.items()},
            "stages_note": ("device time per stage from CUDA events on the launching stream, over a second "
                            f"run of {args.steps} steps with the stage events on ({instrumented_ms:.3f} ms per step "
                            "there; value is timed without them)"),
            "pairs_per_step": {"uncertainty": pairs_ua, "visibility": pairs_vis},
            "pairs_per_s": {"uncertainty": pairs_ua * args.steps / (st["composite_ua"][0] / 1e3)
                            if st["composite_ua"][0] else None,
                            "visibility": pairs_vis * args.steps / (st["composite_vis"][0] / 1e3)
                            if st["composite_vis"][0] else None,
                            "what": "pixel-Gaussian pairs composited per second of the composite kernels"},
            "tile_keys_per_step": prof["keys"] // args.steps,
            "hbm": hbm,
            "plain_unbatched_f32": plain,
            "graph_scoring": graph,
            "precision_err": prec,
            "best_view": best,
        }
        print(json.dumps(line), flush=True)
    if plan is not None:
        plan.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def stage_roofline(st, w, pk, pk_kind, n_sm):
    """Roofline of the step's dominant stage.  st: stage -> (device ms over
    the timed steps, launches); w: the work counts of one step (pairs
    composited, visible records, tile entries whose lists were sorted, view
    and Gaussian counts, tiles, coefficient sizes) and the number of timed
    steps; pk: measured peaks (hbm_gbs, sm_max_mhz).  The composites report
    FP32 work per pair against the FP32 FMA peak (plus the issue roofline
    when a capture of the current kernel gives its instructions per pair),
    the sort and the projection algorithmic bytes against the HBM peak; any
    other stage reports its time only."""
    dom = max(st, key=lambda k: st[k][0])
    sm_mhz = float(pk.get("sm_max_mhz", 2070.0))
    fp32_peak = 2.0 * n_sm * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12   # TFLOP/s, FMA = 2 flops
    hbm_pk = pk.get("hbm_gbs", 6800.0)
    ms, nl = st[dom]
    steps = w["steps"]
    if dom in ("composite_ua", "composite_vis"):
        # pairs of the timed steps: the instrumented step's count (the same
        # work every step) times the steps
        pairs = (w["pairs_ua"] if dom == "composite_ua" else w["pairs_vis"]) * steps
        fpp = FLOPS_PER_PAIR_UA if dom == "composite_ua" else FLOPS_PER_PAIR_VIS
        achieved = pairs * fpp / (ms / 1e3) / 1e12
        tile = w["tile_sc"] if dom == "composite_ua" else w["tile_vf"]
        prof_k = profile_for("k_" + dom, tile, w["workload"])
        roof = {"kernel": "k_" + dom, "bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak,
                "traffic": prof_k.get("bytes_per_launch") if prof_k else None,
                "peak_source": f"FP32 FMA: {n_sm} SMs x {FP32_LANES_PER_SM} lanes x 2 x {sm_mhz:.0f} MHz "
                               f"(sm_max_mhz of {pk_kind} peaks file)",
                "units_per_launch": pairs / max(nl, 1), "unit_name": "pixel-Gaussian pairs",
                "flops_per_unit": fpp, "avg_launch_ms": ms / max(nl, 1), "launches": nl}
        ipp = prof_k.get("warp_inst_per_pair") if prof_k else None
        if ipp:
            # the kernel is issue-bound: its ceiling is the SMs' warp-instruction
            # issue rate divided by the instructions it issues per pair
            peak_pairs = n_sm * ISSUE_PER_SM_CLK * sm_mhz * 1e6 / ipp
            roof["issue"] = {"warp_inst_per_pair": ipp, "peak_pairs_per_s": peak_pairs,
                             "achieved_pairs_per_s": pairs / (ms / 1e3),
                             "frac": pairs / (ms / 1e3) / peak_pairs,
                             "source": "warp instructions per pair from the ncu capture in profiles/"}
        return roof
    if dom == "sort":
        # the sort stage (histogram, scan and scatter launches of both binning
        # levels): 16 B per item per 8-bit pass (key and value read once and
        # written once; histogram reads not counted), 4 passes for stage A's
        # 32-bit record keys, 2 for stage B's 16-bit tile keys where the tile
        # lists were sorted (counted lists have no sort), 1 for the tile order
        # of the scoring pass (one 8-byte item per view tile)
        tiles_sc = w["n_cand"] * (-(-w["W"] // w["tile_sc"])) * (-(-w["H"] // w["tile_sc"])) \
            if w["tile_sc"] <= 16 else 0
        sort_bytes = ((w["vis_vf"] + w["vis_sc"]) * 4 * 16 + (w["sorted_vf"] + w["sorted_sc"]) * 2 * 16
                      + tiles_sc * 16) * steps
        achieved = sort_bytes / (ms / 1e3) / 1e9
        return {"kernel": "sort", "bound": "hbm", "achieved": achieved, "peak": hbm_pk, "unit": "GB/s",
                "frac": achieved / hbm_pk, "traffic": None,
                "algorithmic_bytes_per_step": sort_bytes / steps,
                "what": "the sort stage's device time (all its launches); 16 B per item per 8-bit pass, 4 passes "
                        "per visible record, 2 per sorted tile entry, 1 per scoring view tile",
                "avg_launch_ms": ms / max(nl, 1), "launches": nl}
    if dom == "project":
        # the projection stage (the field build's geometry-only launches and
        # the scoring launches): every Gaussian's record read once per group
        # of 32 views (centre, scale, rotation, opacity; colour and field
        # coefficients for scoring), one visibility bit per (view, Gaussian),
        # and per visible record its 32 B geometry (+ 32 B appearance for
        # scoring), 8 B rectangle and 4 B depth written
        coeff = (w["Kc"] * 3 + w["K"]) * w["b"]
        groups_vf, groups_sc = -(-w["n_train"] // 32), -(-w["n_cand"] // 32)
        proj_bytes = (groups_vf * w["n"] * 44 + groups_sc * w["n"] * (44 + coeff)
                      + (w["n_train"] + w["n_cand"]) * w["n"] / 8 + w["vis_vf"] * 44 + w["vis_sc"] * 76) * steps
        achieved = proj_bytes / (ms / 1e3) / 1e9
        return {"kernel": "k_project", "bound": "hbm", "achieved": achieved, "peak": hbm_pk, "unit": "GB/s",
                "frac": achieved / hbm_pk, "traffic": None,
                "algorithmic_bytes_per_step": proj_bytes / steps,
                "what": "the projection stage's device time (all its launches); Gaussian records read once per "
                        "group of 32 views, a visibility bit per (view, Gaussian), 44 B (field build) or 76 B "
                        "(scoring) written per visible record",
                "avg_launch_ms": ms / max(nl, 1), "launches": nl}
    return {"kernel": dom, "bound": "hbm", "achieved": None, "peak": pk.get("hbm_gbs"), "unit": "GB/s",
            "frac": None, "traffic": None, "avg_launch_ms": ms / max(nl, 1), "launches": nl}


def make_plan(gv, ctx, gs, vf, cand, recs, W, H, prm_sc, visible, keys):
    """The scoring plan for the candidate set: all views in one batch when
    their records fit, else the largest of 256, 128 or 64 views per batch
    that fits.  A first plan with generous capacities is launched once; the
    plan kept is then sized from that launch's largest batch (+2%: the
    candidate set is fixed, and the grids are sized by the capacities).
    Returns (plan or None, views per batch (0 = all), error text or None)."""
    n_cand = len(cand)
    err = None
    for batch in (0, 256, 128, 64):
        if batch and batch >= n_cand:
            continue
        nb = 1 if batch == 0 else (n_cand + batch - 1) // batch
        pb = gv.Params(**{f: getattr(prm_sc, f) for f, _ in prm_sc._fields_})
        pb.views_per_batch = batch
        grow = 1.25 if batch == 0 else 2.0
        try:
            plan = ctx.plan(gs, vf, n_cand, W, H, int(keys / nb * grow) + 1024,
                            record_capacity=int(visible / nb * grow) + 1024, params=pb, want_rgb=True, want_unc=True)
            plan.launch(recs)
            _, rec_need, ent_need = plan.overflowed()
            plan.close()
            plan = ctx.plan(gs, vf, n_cand, W, H, int(ent_need * 1.02) + 1024,
                            record_capacity=int(rec_need * 1.02) + 1024, params=pb, want_rgb=True, want_unc=True)
            return plan, batch, None
        except gv.GavisError as e:
            err = str(e)
    return None, 0, err


def faster_scoring(ctx, plan, recs, gs, vf, cand, prm_sc, outs, reps=3):
    """Device time of the plan replay and of gavis_score_views for the same
    candidates (after one warm call each); the timed step uses the faster."""
    import torch
    plan.launch(recs)
    ctx.score_views(gs, vf, cand, params=prm_sc, out=outs, sync_best=False)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record()
    for _ in range(reps):
        plan.launch(recs)
    e[1].record()
    for _ in range(reps):
        ctx.score_views(gs, vf, cand, params=prm_sc, out=outs, sync_best=False)
    e[2].record()
    torch.cuda.synchronize()
    return e[0].elapsed_time(e[1]) / reps, e[1].elapsed_time(e[2]) / reps


def precision_errors(gv, ctx, c, gs, cdt, prm_vf, prm_sc, k):
    """Error of every output of the stored-precision path against the oracle
    fed the float32 inputs (float64 field, float32 colour) on k sampled
    views: the field of k training views (gamma/|P|), and k candidate views
    scored with that oracle field rounded to the storage type (rgb, unc,
    score, V).  Max-abs and 99th percentile per output."""
    import numpy as np
    import torch
    import oracle
    oracle.build()
    sc = c["scene"]
    L = c["vf_degree"]
    spread = lambda n: [int(round(i * (n - 1) / (k - 1))) for i in range(k)]
    train = [c["train"][i] for i in spread(len(c["train"]))]
    cands = [c["cand"][i] for i in spread(len(c["cand"]))]
    t0 = time.perf_counter()
    g_o, _, _ = oracle.vf_build(train, sc, L)
    P = len(train)
    g_dev = ctx.vf_build(gs, train, degree=L, params=prm_vf, dtype=cdt).coeffs.double().cpu().numpy()

    def st(e):
        e = np.abs(np.asarray(e, np.float64)).ravel()
        return {"max_abs": float(e.max(initial=0.0)), "p99": float(np.percentile(e, 99)) if e.size else 0.0}

    res = {"gamma_over_P": st((g_dev - g_o) / P)}
    vf = gv.VisibilityField(torch.as_tensor(g_o.astype(np.float32)).to("cuda", cdt).contiguous(), L, P, 1.0)
    out = ctx.score_views(gs, vf, cands, params=prm_sc)
    Vg = ctx.vf_query(gs, vf, cands).double().cpu().numpy()
    unc, rgb, score = out["unc"].cpu().numpy(), out["rgb"].cpu().numpy(), out["score"].cpu().numpy()
    e_rgb, e_unc, e_V, e_s = [], [], [], []
    for v, cam in enumerate(cands):
        V64, _ = oracle.vf_query(g_o, L, P, cam, sc.means)
        r = oracle.render_view(cam, sc, V64)
        e_rgb.append((rgb[v] - r[0]).ravel())
        e_unc.append((unc[v] - r[1]).ravel())
        e_V.append(Vg[v] - V64)
        e_s.append(score[v] - r[1].mean())
    res.update(rgb=st(np.concatenate(e_rgb)), unc=st(np.concatenate(e_unc)), V=st(np.concatenate(e_V)),
               score=st(e_s))
    res["what"] = (f"stored {str(cdt).split('.')[-1]} coefficients vs the float64 oracle on float32 inputs: field "
                   f"of {P} sampled training views, {len(cands)} sampled candidate views scored with that field")
    res["oracle_s"] = time.perf_counter() - t0
    return res


def kernel_source_sha(path, kernel):
    """sha256 (16 hex digits) of a kernel's definition: from the line that
    names it with '(CompositeArgs' or '(' up to its closing brace."""
    import hashlib
    text = open(path).read()
    i = text.find(kernel + "(")
    while i >= 0 and text.find("{", i) > text.find(";", i):   # skip declarations and calls
        i = text.find(kernel + "(", i + 1)
    if i < 0:
        return None
    start = text.rfind("\n", 0, text.rfind("template", 0, i)) + 1 if "template" in text[max(0, i - 200):i] else \
        text.rfind("\n", 0, i) + 1
    j = text.find("{", i)
    depth = 0
    for k in range(j, len(text)):
        depth += {"{": 1, "}": -1}.get(text[k], 0)
        if depth == 0:
            return hashlib.sha256(text[start:k + 1].encode()).hexdigest()[:16]
    return None


def profile_for(kernel, tile, workload):
    """The committed ncu figures of a kernel (DRAM bytes per launch, warp
    instructions per pair), when they were taken on the current source of
    the kernel, at the same tile size, for this workload (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        with open(p) as f:
            d = json.load(f)
        e = d.get(f"{kernel}/tile{tile}")
        if not e or e.get("workload") != workload:
            return None
        src = os.path.join(ROOT, "paper_2605_30342_gb300", "csrc", e["source"])
        return e if kernel_source_sha(src, kernel) == e.get("kernel_sha") else None
    except Exception:
        return None


def run_serving(args):
    """Serving workload: 4 resident scenes of 100k, 500k, 1M and 2M Gaussians
    built as in the room workload (one room, fields from 100 training views at
    800x800 along a walk), Poisson arrivals, 8-512 candidate views per request
    (log-uniform) at one of four resolutions, f16 coefficients, f32
    compositing, a 120 GB admission budget.  One line per request rate."""
    import numpy as np
    import torch
    import scenegen as sg
    import __graft_entry__ as ge
    ge.build()
    import paper_2605_30342_gb300 as gv
    ctx = gv.Context(0)
    scenes = []
    t_build = time.perf_counter()
    for k, n in enumerate((100_000, 500_000, 1_000_000, 2_000_000)):
        sc = sg.multi_room_scene(n, 1, 1, seed=k, sh_degree=3)
        gs = gv.Gaussians.from_numpy(sc, sh_dtype=torch.float16)
        train = sg.walk_cameras(100, sc, 800, 800, seed=k + 1, x_frac=(0.0, 0.5))
        vf = ctx.vf_build(gs, train, degree=3, dtype=torch.float16)
        scenes.append((sc, gs, vf))
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t_build
    ctx.close()
    res = [(160, 120), (320, 240), (640, 480), (800, 600)]
    budget = int(args.serving_budget_gb * 1e9)
    rates = [float(r) for r in args.rates.split(",")] if args.rates else [args.rate]
    for rate in rates:
        rng = np.random.default_rng(7)
        reqs = []
        t = 0.0
        for r in range(args.requests):
            t += rng.exponential(1.0 / rate)
            sid = int(rng.integers(4))
            nv = int(round(np.exp(rng.uniform(np.log(8), np.log(512)))))
            W, H = res[int(rng.integers(4))]
            cams = sg.se2_cameras(nv, scenes[sid][0], W, H, seed=1000 + r)
            reqs.append((t, sid, cams))
        srv = gv.Server(0, budget_bytes=budget, n_workers=args.workers, max_views_per_batch=args.batch_views)
        ids = [srv.add_scene(gs, vf) for _, gs, vf in scenes]
        prm = gv.Params(vf_degree=3)
        # warm-up: one request per (scene, resolution), untimed
        for sid in range(4):
            for (W, H) in res:
                srv.wait(srv.submit(ids[sid], sg.se2_cameras(8, scenes[sid][0], W, H, seed=99), params=prm))
        st0 = srv.stats()
        sampler = ClockSampler(0)
        sampler.start()
        t0 = time.perf_counter()
        rids = []
        for (ta, sid, cams) in reqs:
            now = time.perf_counter() - t0
            if ta > now:
                time.sleep(ta - now)
            rids.append(srv.submit(ids[sid], cams, params=prm))
        out = [srv.wait(r) for r in rids]
        wall = time.perf_counter() - t0
        clocks = sampler.stop()
        lat = [o["latency_ms"] for o in out]
        views = sum(len(c) for _, _, c in reqs)
        st = srv.stats()
        st["views_scored"] -= st0["views_scored"]
        st["batches"] -= st0["batches"]
        srv.close()
        offered = views / reqs[-1][0]
        line = {
            "metric": "serving: views/s and p50/p99 request latency (4 resident scenes 100k-2M Gaussians)",
            "value": views / wall, "unit": "views/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "serving: Poisson arrivals over 4 resident room scenes (100k, 500k, 1M, 2M "
                                   "Gaussians; fields from 100 training views at 800x800)",
                       "rate_req_s": rate, "requests": args.requests, "views": views,
                       "views_per_request": "log-uniform 8..512", "resolutions": res, "coeff_storage": "f16",
                       "workers": args.workers, "batch_views": args.batch_views, "budget_bytes": budget},
            "latency_ms": {"p50": percentile(lat, 50), "p99": percentile(lat, 99), "max": max(lat)},
            "offered_views_per_s": offered, "achieved_over_offered": (views / wall) / offered,
            "wall_s": wall, "scene_build_s": t_build, "server": st, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.serving:
        run_serving(args)
    else:
        run_gavis(args)


if __name__ == "__main__":
    main()
