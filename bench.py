#!/usr/bin/env python
"""Benchmark: Mcell-updates/s per RK stage of the immersed-boundary solver.

Workload (default): M=2, Re=1e4 flow over a 15 deg wedge (3-vertex polyline,
chord 1) on a 768x384 grid over [-1,3]x[-1,1], WENO5 + LDFSS + RK3, CFL 0.5,
FP32-bulk arithmetic (FP64 state accumulation).  One benchmark step is one
full SSP-RK3 time step of the hot path: time-step reduction, three rounds of
IB / ghost reconstruction, domain halos and the fused residual + stage
update (the body is static, so classification and stencils are built once
before timing).  The same step in plain FP64 is timed beside it.

value  = active (non-solid) cells x 3 stages x K steps / device time, all ranks
e2e    = the same metric through the C ABI from pinned host memory: every step
         uploads the FP64 state, steps, and reads the forces back.

Multi-GPU (torchrun): each rank runs its own replica of the workload (weak
scaling, no data-path collective); ranks are timed between barriers and the
maximum time is used.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the request loop runs up to --serve-slots cases on their own streams: give them
# that many hardware work queues (read when the CUDA context is created)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

WORKLOADS = {
    "wedge_768x384": "wedge_m2_re1e4",
    "cylinder_160x80": "cylinder_m02_re40",
    "osc_cylinder_1024x512": "oscillating_cylinder_m02_re185",
    "naca_dual_2048x1024": "naca0012_a5_m0001",
    "shock_driven_656x656": "shock_driven_cylinder",
}
# algorithmic DRAM bytes per cell and stage of the fused residual kernel
# (each stage reads its input planes and tags once and writes its output once;
# halos are re-read from L2/shared memory, not counted)
BYTES_PER_CELL_STAGE = {"fp32_bulk": 179.0 / 3.0, "fp64": 259.0 / 3.0}
# algorithmic floating-point operations per cell and stage (counted from the
# formulas, FMA = 2): WENO5 per variable and direction 91 (x 4 x 2), LDFSS
# 110 per face (x 2), viscous 40 per face (x 2), primitives 25, update 20
FLOPS_PER_CELL_STAGE = 91 * 8 + 110 * 2 + 40 * 2 + 25 + 20
# dual time, FP32-bulk: algorithmic DRAM bytes per cell and pseudo stage (FP32 tile 16 + tag 1 + FP64 iterate
# 32 + primitives of the sub-iteration start 32 (written at stage 1, read at stages 2 and 3) + the physical step's
# BDF part 32 + FP64 output 32 + FP32 mirror 16) and FP64 flops per cell and pseudo stage of the point-implicit
# update (counted from the formulas, FMA = 2, a division = 1: BDF2 term 13, conversion to primitives 32, enthalpy
# 10, structured solve 26, stage combination 16, conversion back 28, misc 1)
# 3-D FP64 flow (sphere): floating-point operations per cell and stage of the 3-D kernels, counted from their
# formulas as above (FMA = 2, a division or square root = 1): per face WENO5 72 (x 5 variables x 2 sides), LDFSS
# 119, viscous 62, three faces per cell; primitives 17 and the stage update 60 per cell
FLOPS3D_PER_CELL_STAGE = 3 * (72 * 10 + 119 + 62) + 17 + 60
DUAL_BYTES_PER_CELL_STAGE = 161.0
DUAL_FP64_FLOPS_PER_CELL = 126
L2_FLUSH_BYTES = 512 << 20


def measure_fma_peaks(ibm, smi_index, seconds=1.0):
    """FP32 and FP64 FMA rates of this GPU (ibm_fma_peak: independent FMA recurrences on every SM), each from
    one launch of about `seconds`, calibrated by a short launch; SM clocks sampled during both."""
    out = {}
    with ClockSampler(smi_index) as clk:
        for name, fp64, probe in (("fp32", 0, 200000), ("fp64", 1, 20000)):
            rate, ms = ibm.fma_peak(fp64, probe)
            iters = max(probe, int(probe * seconds * 1e3 / max(ms, 1e-3)))
            rate, ms = ibm.fma_peak(fp64, iters)
            out[name] = {"tflops": rate / 1e12, "launch_ms": ms, "iters": iters}
    out["clocks"] = clk.summary()
    out["how"] = ("ibm_fma_peak: 8 independent FMA recurrences per thread, 4 x 256 threads per SM, one launch of "
                  "about %.1f s per precision timed with CUDA events (FMA = 2 flop)" % seconds)
    return out


def _spec(name, precision, grid=None):
    from paper_1912_11908_gb300 import workloads as W
    fn = getattr(W, WORKLOADS[name])
    kw = {}
    if grid:
        kw["nx"], kw["ny"] = (int(v) for v in grid.lower().split("x"))
    return fn(precision=W.PREC_FP32_BULK if precision == "fp32_bulk" else W.PREC_FP64, **kw)


def _pre_stage_in_graph(step_ms, prof, nsteps=10):
    """Pre-stage time of a captured step: the graph-replayed step time less the stage launches and the end of
    the step, those timed by events around their own (device-bound) launches over `nsteps` profiled steps."""
    return step_ms - (prof["residual_stage"][0] + prof["step_end"][0]) / nsteps


def _active_cells(case):
    import numpy as np
    return int((case.tags() != 1).sum())


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def source_sha256(files):
    """sha256 over the concatenated kernel sources (paper_1912_11908_gb300/csrc)."""
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_1912_11908_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def _traffic(summary, grid, stage_launch=None):
    """DRAM bytes per launch from a committed ncu summary (profiles/*.json), if the kernel source is unchanged
    and the summary covers this grid and the launch form in use."""
    p = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("source_sha256") != source_sha256(d.get("sources", [])):
        return None
    if list(d.get("grid", [])) != list(grid):
        return None
    if stage_launch is not None and "stage_launch" in d and (d["stage_launch"] > 0) != (stage_launch > 0):
        return None
    return d.get("dram_bytes_per_launch")


class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", "bench_clocks_%d.csv" % os.getpid())

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def max_over_ranks(value, dist, device):
    """Largest value over the ranks of the process group (a replica job takes as long as its slowest rank);
    the value itself when there is no process group."""
    if not dist:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Aggregate throughput of a weak-scaling replica run: the units of all ranks over the slowest rank's time."""
    return units_per_rank * world / seconds


def _time_steps(case, torch, flush, K, stream):
    """Device time of K steps, one CUDA-event pair per step on the case stream, L2 flushed in between."""
    total = 0.0
    for _ in range(K):
        flush.add_(1)  # writes more than L2 between timed steps (outside the events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        case.step(1)
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    return total


def run_ours(args, rank, world):
    import numpy as np
    import torch

    from paper_1912_11908_gb300 import _build, ibm

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if local == 0:
        _build.build()  # the other ranks wait for it in the process-group rendezvous
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    flush = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    spec = _spec(args.workload, args.precision, args.grid)
    case = ibm.Case(spec, stream=stream.cuda_stream)
    if "shock" in spec:  # a planar shock set up across the domain (shock-driven cylinder)
        from paper_1912_11908_gb300 import workloads as W
        case.set_state(W.shock_initial_state(spec))
    if args.stage_launch is not None and args.precision == "fp32_bulk":
        case.stage_launches(args.stage_launch)
    case.classify()
    cells = _active_cells(case)
    case.step(args.warmup)
    torch.cuda.synchronize()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    dev_index = torch.cuda.current_device()
    phys = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
    smi_index = phys[dev_index] if phys and phys[0] not in ("",) else dev_index
    n0 = case.launches()
    barrier()
    with ClockSampler(smi_index) as clk:
        t_dev_ms = _time_steps(case, torch, flush, args.steps, stream)
    barrier()
    launches = case.launches() - n0
    t_dev_ms = max_over_ranks(t_dev_ms, dist, "cuda")
    is_dual = spec["time_scheme"] == 1
    stages_per_step = 3 * spec["subiters"] if is_dual else 3
    value = whole_job_rate(cells * stages_per_step * args.steps, world, t_dev_ms * 1e-3) / 1e6

    # live kernel timing for the roofline: the same steps with CUDA events around every kernel group
    case.profile(True)
    nprof = min(args.steps, 50)
    case.profile_read()
    case.step(nprof)
    prof = case.profile_read()
    case.profile(False)
    stage_ms, stage_launches = prof["residual_stage"]
    stage_avg_ms = stage_ms / max(1, stage_launches)
    launch_timing = "CUDA events around every stage launch (direct launches, %d timed)" % stage_launches
    if args.precision == "fp32_bulk" and not is_dual and spec["motion"] == 0:
        # a static-body FP32-bulk step is exactly three stage launches (the time-step reduction rides in
        # stage 3): the stage's average duration is the graph-replayed step time / 3, programmatic overlap kept
        stage_avg_ms = t_dev_ms / args.steps / 3.0
        launch_timing = "graph-replayed timed steps: step time / 3 (%d steps, three stage launches each)" % args.steps
        stage_launches = 3 * args.steps
    bpc = DUAL_BYTES_PER_CELL_STAGE if is_dual else BYTES_PER_CELL_STAGE[args.precision]
    bytes_per_launch = bpc * spec["nx"] * spec["ny"]
    achieved = bytes_per_launch / (stage_avg_ms * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    if args.precision == "fp32_bulk":
        grid = (spec["nx"], spec["ny"])
        traffic = (_traffic("k_dual_f32_naca1024x512.json", grid, case.stage_launch()) if is_dual
                   else _traffic("k_stage_f32_wedge768x384.json", grid, case.stage_launch()))
    else:
        traffic = None
    flops_per_launch = (DUAL_FP64_FLOPS_PER_CELL if is_dual else FLOPS_PER_CELL_STAGE) * spec["nx"] * spec["ny"]
    achieved_tf = flops_per_launch / (stage_avg_ms * 1e-3) / 1e12
    fma = measure_fma_peaks(ibm, smi_index) if not args.skip_peaks else None
    if fma is None:  # profiling runs: the peaks of the last measured run are not needed
        fma = {"fp32": {"tflops": float("nan")}, "fp64": {"tflops": float("nan")}, "clocks": None, "how": "skipped"}
    if is_dual:
        # the FP64 point-implicit update bounds the pseudo stage
        rl_bound, rl_peak = "fp64", fma["fp64"]["tflops"]
        rl_kernel = ("k_dual_f32_batch_one (block table of this case alone: plain and body tiles in one launch per "
                     "pseudo stage)" if case.stage_launch() > 0
                     else "k_dual_f32 (plain + body tiles)")
        rl_src = "measured: FP64 FMA rate (ibm_fma_peak)"
    elif args.precision == "fp32_bulk":
        rl_bound, rl_peak = "alu", fma["fp32"]["tflops"]
        rl_kernel = ("k_stage_f32_one (plain and body tiles in one launch per stage)" if case.stage_launch() > 0
                     else "k_stage_f32 (plain + body tiles)")
        rl_src = "measured: FP32 FMA rate (ibm_fma_peak)"
    else:
        rl_bound, rl_peak = "fp64", fma["fp64"]["tflops"]
        rl_kernel = "k_stage_f64"
        rl_src = "measured: FP64 FMA rate (ibm_fma_peak)"

    # plain FP64 path on the same workload and GPU
    fp64 = None
    if args.precision == "fp32_bulk" and not args.skip_fp64:
        c64 = ibm.Case(_spec(args.workload, "fp64", args.grid), stream=stream.cuda_stream)
        c64.classify()
        c64.step(max(3, args.warmup // 4))
        k64 = max(3, min(args.steps, 40))
        t64 = _time_steps(c64, torch, flush, k64, stream)
        v64 = cells * 3 * k64 / (t64 * 1e-3) / 1e6
        fp64 = {"value": v64, "ms_per_step": t64 / k64, "steps": k64,
                "fp32_bulk_speedup": value / world / v64}
        c64.close()

    # dual time (NACA0012 at 5 deg, M = 0.001, 2048x1024, 30 sub-iterations of three pseudo stages): FP32-bulk
    # (FP32 residual, FP64 point-implicit update) and plain FP64
    dual = None
    if not args.skip_dual:
        from paper_1912_11908_gb300 import workloads as W
        dual = {}
        for prec, pname, kd in ((W.PREC_FP32_BULK, "fp32_bulk", 4), (W.PREC_FP64, "fp64", 2)):
            dspec = W.naca0012_a5_m0001(precision=prec)
            cd = ibm.Case(dspec, stream=stream.cuda_stream)
            cd.classify()
            dcells = _active_cells(cd)
            cd.step(1)
            td = _time_steps(cd, torch, flush, kd, stream)
            nst = 3 * dspec["subiters"]
            dual[pname] = {"workload": dspec["name"], "subiters": dspec["subiters"], "pseudo_stages_per_step": nst,
                           "value": dcells * nst * kd / (td * 1e-3) / 1e6,
                           "unit": "Mcell-updates/s per pseudo stage", "ms_per_physical_step": td / kd, "steps": kd}
            cd.close()
        dual["fp32_bulk_speedup"] = dual["fp32_bulk"]["value"] / dual["fp64"]["value"]

    # moving body (oscillating cylinder, 1024x512, FP32-bulk): re-classification and stencils every step
    moving = None
    if not args.skip_moving:
        from paper_1912_11908_gb300 import workloads as W
        mspec = W.oscillating_cylinder_m02_re185(precision=W.PREC_FP32_BULK)
        cm = ibm.Case(mspec, stream=stream.cuda_stream)
        cm.classify()
        mcells = _active_cells(cm)
        cm.step(5)
        km = 50
        tm = _time_steps(cm, torch, flush, km, stream)
        cm.profile(True)
        cm.profile_read()
        cm.step(10)
        mprof = cm.profile_read()
        cm.profile(False)
        moving = {"workload": mspec["name"], "precision": "fp32_bulk", "value": mcells * 3 * km / (tm * 1e-3) / 1e6,
                  "unit": "Mcell-updates/s", "ms_per_step": tm / km, "steps": km,
                  "pre_stage_ms_per_step": mprof["geometry"][0] / 10, "stage_ms_per_step": mprof["residual_stage"][0] / 10,
                  "pre_stage_in_graph_ms_per_step": _pre_stage_in_graph(tm / km, mprof),
                  "pre_stage": "re-classification, tags, lists and stencils of the new pose, the force of a body "
                               "under the fluid force and dt, up to the start of stage 1 (the stencils and the "
                               "force run on side streams beside the rest); pre_stage_ms_per_step: CUDA events "
                               "around directly launched kernels (host launch time included); "
                               "pre_stage_in_graph_ms_per_step: the graph-replayed step time less the stage "
                               "launches and the end of step timed the same way"}
        cm.close()
        # cylinder crossing gas at rest at M_D = 1.2 (Re 300, 80 x 16 diameters at D/40, FP32-bulk): the
        # supersonic moving-body pressure condition in every stage's node rebuild
        sspec = W.moving_cylinder_supersonic(1.2, precision=W.PREC_FP32_BULK)
        cs = ibm.Case(sspec, stream=stream.cuda_stream)
        cs.classify()
        scells = _active_cells(cs)
        cs.step(5)
        ks = 50
        ts = _time_steps(cs, torch, flush, ks, stream)
        cs.profile(True)
        cs.profile_read()
        cs.step(10)
        sprof = cs.profile_read()
        cs.profile(False)
        moving["supersonic"] = {"workload": sspec["name"], "precision": "fp32_bulk",
                                "value": scells * 3 * ks / (ts * 1e-3) / 1e6, "unit": "Mcell-updates/s",
                                "ms_per_step": ts / ks, "steps": ks,
                                "pre_stage_ms_per_step": sprof["geometry"][0] / 10,
                                "pre_stage_in_graph_ms_per_step": _pre_stage_in_graph(ts / ks, sprof),
                                "stage_ms_per_step": sprof["residual_stage"][0] / 10}
        cs.close()
        # planar shock (Mach 1.5) driving a cylinder free to translate (Sec. 8.2.6, 656 x 656, FP32-bulk): force
        # and body update every step on top of the re-classification
        kspec = W.shock_driven_cylinder(precision=W.PREC_FP32_BULK)
        ck = ibm.Case(kspec, stream=stream.cuda_stream)
        ck.set_state(W.shock_initial_state(kspec))
        ck.classify()
        kcells = _active_cells(ck)
        ck.step(5)
        kk = 50
        tk = _time_steps(ck, torch, flush, kk, stream)
        ck.profile(True)
        ck.profile_read()
        ck.step(10)
        kprof = ck.profile_read()
        ck.profile(False)
        moving["shock_driven"] = {"workload": kspec["name"], "precision": "fp32_bulk",
                                  "value": kcells * 3 * kk / (tk * 1e-3) / 1e6, "unit": "Mcell-updates/s",
                                  "ms_per_step": tk / kk, "steps": kk,
                                  "pre_stage_ms_per_step": kprof["geometry"][0] / 10,
                                  "pre_stage_in_graph_ms_per_step": _pre_stage_in_graph(tk / kk, kprof),
                                  "stage_ms_per_step": kprof["residual_stage"][0] / 10}
        ck.close()

    # serving mix through the request loop: Poisson arrivals (latency) and all at once (throughput)
    serving = None
    if not args.skip_serving and rank == 0:
        from paper_1912_11908_gb300 import workloads as W
        mix0 = W.serving_mix(args.serve_requests)
        ndual = sum(1 for r in mix0 if r["spec"]["time_scheme"] == W.TIME_DUAL)
        serving = {"workload": "serving mix: %d seeded requests (cylinder / NACA00xx / wedge, static or oscillating, "
                               "M 0.001-2, Re 40-1e4, grids 64x64-1024x512, FP32-bulk; %d explicit requests of 500 "
                               "SSP-RK3 steps, %d at M <= 0.01 of 10 dual-time steps x 30 sub-iterations), "
                               "Poisson arrivals mean 50 ms" % (args.serve_requests, args.serve_requests - ndual, ndual),
                   "slots": args.serve_slots, "steps_per_chunk": args.serve_chunk,
                   "memory_budget": "80% of free device memory",
                   "modes": {"batched": "size-class groups, one launch per RK stage over the group's block table "
                                        "(body-tile entries first, stages chained by programmatic launch), group step "
                                        "in a CUDA graph, autotuned schedule",
                             "streams": "one stream and one step graph per case"}}
        bm = ibm.SERVE_BATCHED | ibm.SERVE_AUTOTUNE
        for name, mode in (("batched", bm), ("streams", 0)):
            serving[name] = {
                "poisson": run_serving(ibm, W, args.serve_requests, args.serve_slots, args.serve_chunk, False, mode),
                "burst": run_serving(ibm, W, args.serve_requests, args.serve_slots, args.serve_chunk, True, mode)}

    # end to end through the C ABI from pinned host memory
    state = case.state()
    host = torch.empty(state.shape, dtype=torch.float64, pin_memory=True)
    host.numpy()[...] = state
    forces = torch.empty(4, dtype=torch.float64, pin_memory=True)
    ke = max(3, min(args.steps, 50))
    barrier()
    t0 = time.perf_counter()
    for _ in range(ke):
        # upload (asynchronous: the pinned buffer stays unchanged), one step, forces back (the one host wait)
        case.set_state_from_ptr(host.data_ptr(), host.numel() * 8, False, wait=False)
        case.step(1)
        case.forces_into(forces.data_ptr())
    t_e2e = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e = {"value": whole_job_rate(cells * stages_per_step * ke, world, t_e2e) / 1e6, "unit": "Mcell-updates/s",
           "h2d_bytes_per_step": int(host.numel() * 8), "d2h_bytes_per_step": int(forces.numel() * 8),
           "steps": ke}

    # 3-D immersed-boundary pre-processing (Appendix A: a 1200-triangle sphere in a 40^3 lattice): classification,
    # tags, ordered lists, closest features and pseudo-normals, timed on the device
    geo3d = None
    if rank == 0 and not args.skip_geometry3d:
        from paper_1912_11908_gb300 import workloads as W
        sv, st_ = W.uv_sphere(21, 30, 0.35, (0.5, 0.5, 0.5))
        b3 = ibm.Body3D(sv, st_, stream=stream.cuda_stream)
        g3 = {}
        for n3 in (40, 128, 256):
            b3.classify((n3, n3, n3), (0.0,) * 3, (1.0,) * 3)  # warm-up (and buffer sizing)
            torch.cuda.synchronize()
            reps = 20 if n3 < 256 else 5
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                b3.classify((n3, n3, n3), (0.0,) * 3, (1.0,) * 3)
            e1.record(stream)
            e1.synchronize()
            g3["%d^3" % n3] = {"ms": e0.elapsed_time(e1) / reps, "listed_nodes": int(b3.counts().sum())}
        b3.close()
        geo3d = {"workload": "Appendix A: UV sphere of 1200 triangles, radius 0.35, in n^3 lattice nodes over the unit "
                             "cube", "kernels": "k3_classify_lines (x3), k3_tags, k3_scan, k3_scatter, k3_closest", "gpu": g3,
                 "paper_table_a1_context": "4.296e-2 s for 40^3 nodes on one Xeon E5-2670 core (the paper's "
                                           "pre-processing; other hardware, context only)"}

    # 3-D flow past Appendix A's sphere (FP64 SSP-RK3 steps on the case's stream)
    flow3d = None
    if rank == 0 and not args.skip_flow3d:
        flow3d = flow3d_block(ibm, stream, fma)

    accuracy = None
    if rank == 0 and not args.skip_accuracy:
        accuracy = accuracy_block(ibm, stream.cuda_stream)

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        cpu = cpu_baseline(args, cells)

    out = {
        "metric": "Mcell-updates/s per RK stage (FP32-bulk vs FP64)",
        "value": value,
        "unit": "Mcell-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_dev_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32_bulk" else "f64",
        "data": "synthetic (closed-form body, uniform free-stream start)",
        "config": {"workload": spec["name"], "grid": [spec["nx"], spec["ny"]], "active_cells": cells,
                   "precision": args.precision, "stages_per_step": stages_per_step,
                   "time_scheme": "dual time (BDF2, %d sub-iterations)" % spec["subiters"] if is_dual else "SSP-RK3",
                   "l2": "flushed between timed steps (512 MiB write outside the events)",
                   "parallelism": "replicas" if world > 1 else "single GPU", "cuda_graphs": True,
                   "autotuned_plain_variants": list(case.tuning()), "stage_launch": case.stage_launch()},
        "roofline": {"bound": rl_bound, "kernel": rl_kernel, "achieved": achieved_tf, "peak": rl_peak, "unit": "TFLOP/s",
                     "frac": achieved_tf / rl_peak, "peak_source": rl_src,
                     "flops_per_launch": flops_per_launch, "traffic": traffic, "avg_launch_ms": stage_avg_ms,
                     "timed_launches": stage_launches, "launch_timing": launch_timing, "measured_peaks": fma,
                     "hbm_view": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                                  "peak_source": peak_kind, "bytes_per_launch": bytes_per_launch}},
        "kernel_ms_per_step": {g: ms / nprof for g, (ms, n) in prof.items()},
        "accuracy": accuracy,
        "geometry3d": geo3d,
        "flow3d": flow3d,
        "fp64": fp64,
        "dual_time": dual,
        "moving_body": moving,
        "serving": serving,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(out))
    case.close()
    if dist:
        dist.destroy_process_group()


def flow3d_block(ibm, stream, fma, steps=10, warmup=3):
    """3-D steps of the 192 x 96 x 96 sphere case in FP32-bulk and in FP64, CUDA events on the case's stream (the
    working set, ~600 MB, is larger than L2); the achieved rate of the step's algorithmic flops against the
    measured FMA rate of the precision the fluxes run in."""
    import torch
    from paper_1912_11908_gb300 import workloads as W

    def run(precision, nsteps):
        spec = dict(W.sphere_m03_re100(), precision=precision)
        c = ibm.Case3D(spec, stream=stream.cuda_stream)
        cells = int((c.tags() != 1).sum())
        c.step(warmup)
        c.time()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n0 = c.launches()
        e0.record(stream)
        c.step(nsteps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / nsteps
        launches = (c.launches() - n0) // nsteps
        f = c.forces()
        t_end = float(c.time()[0])
        c.close()
        nint = spec["n"][0] * spec["n"][1] * spec["n"][2]
        tflops = FLOPS3D_PER_CELL_STAGE * nint * 3 / (ms * 1e-3) / 1e12
        key = "fp32" if precision == W.PREC_FP32_BULK else "fp64"
        peak = fma[key]["tflops"] if fma else None
        return spec, {"value": cells * 3 / (ms * 1e3), "unit": "Mcell-updates/s", "ms_per_step": ms,
                      "steps": nsteps, "kernels_per_step": int(launches), "active_cells": cells,
                      "roofline": {"bound": "alu", "unit": "TFLOP/s", "achieved": tflops, "peak": peak,
                                   "frac": tflops / peak if peak else None,
                                   "peak_source": "measured: %s FMA rate (ibm_fma_peak)" % key.upper(),
                                   "flops_per_cell_stage": FLOPS3D_PER_CELL_STAGE,
                                   "scope": "whole step (all kernels) over its device time"},
                      "cx_cy_cz": [float(v) for v in f[:3]], "t": t_end}

    spec, f32 = run(W.PREC_FP32_BULK, steps * 5)
    _, f64 = run(W.PREC_FP64, steps)
    out = {"workload": spec["name"], "time_scheme": "SSP-RK3", "grid": list(spec["n"]), "precision": "fp32_bulk"}
    out.update(f32)
    out["fp64"] = f64
    out["fp32_bulk_speedup"] = f32["value"] / f64["value"]
    return out


def accuracy_block(ibm, stream):
    """Error of each configuration's results in FP32-bulk form against the plain FP64 path on the GPU, at the
    configuration's own size (tests/test_gpu_accuracy.py holds that FP64 path to the FP64 oracle within 1e-10
    on the same configurations), and the wedge's oblique shock, in both precisions, against theta-beta-M."""
    import numpy as np

    from paper_1912_11908_gb300 import workloads as W
    from tests.flowmetrics import theta_beta_m, theta_from_beta, theta_from_ratio, wedge_shock

    def pair(spec):
        return (ibm.Case(dict(spec, precision=W.PREC_FP32_BULK), stream=stream),
                ibm.Case(dict(spec, precision=W.PREC_FP64), stream=stream))

    def compare(c32, c64, worst=0.0):
        f32, f64 = c32.forces(), c64.forces()
        cp32, _ = c32.surface()
        cp64, _ = c64.surface()
        ok = np.isfinite(cp32) & np.isfinite(cp64)
        d = {"dcd": abs(f32[0] - f64[0]), "dcl": abs(f32[1] - f64[1]),
             "max_dc_over_window": max(worst, abs(f32[0] - f64[0]), abs(f32[1] - f64[1])),
             "surface_cp_linf": float(np.abs(cp32 - cp64)[ok].max()), "surface_cp_range": float(np.ptp(cp64[ok])),
             "cd_fp64": f64[0], "cl_fp64": f64[1]}
        d["within_bar"] = bool(d["max_dc_over_window"] <= 1e-3)
        return d

    t0 = time.perf_counter()
    out = {"reference": "plain FP64 path on the GPU (matches the FP64 oracle within 1e-10 relative at these sizes "
                        "in tests/test_gpu_accuracy.py)", "bar": "|dCd|, |dCl| <= 1e-3; shock angle +-1 deg, "
                        "p2/p1 +-3% of theta-beta-M"}
    spec = W.wedge_m2_re1e4()
    c32, c64 = pair(spec)
    c32.step(2000)
    c64.step(2000)
    d = compare(c32, c64)
    d["steps"] = 2000
    beta_e, pr_e = theta_beta_m(2.0, math.radians(15.0))
    d["theta_beta_m"] = {"beta_deg": math.degrees(beta_e), "p2_p1": pr_e}
    # the impulsively started flow is still forming the shock at the configuration's 2000 steps (t = 1.2); the
    # steady shock is measured at t >= 4
    for when in ("after_2000_steps", "steady_t4"):
        for name, c in (("fp32_bulk", c32), ("fp64", c64)):
            if when == "steady_t4":
                while c.time()[0] < 4.0:
                    c.step(500)
            beta, ratio = wedge_shock(c.state(), c.tags(), dict(spec, precision=0))
            d["shock_%s_%s" % (name, when)] = {"t": c.time()[0], "beta_deg": beta, "p2_p1": ratio,
                                               "dbeta_deg": beta - math.degrees(beta_e),
                                               "dratio_rel": ratio / pr_e - 1.0,
                                               "effective_wedge_deg_from_beta": theta_from_beta(2.0, math.radians(beta)),
                                               "effective_wedge_deg_from_ratio": theta_from_ratio(2.0, ratio)}
    # theta-beta-M is inviscid: at Re 1e4 the laminar boundary layer's displacement slope (~1 deg at mid-chord)
    # thickens the wedge the stream sees; the bar brackets the effective wedge angle by 15 and 16.5 deg
    d["steady_shock_bar"] = "effective wedge angle (theta-beta-M inverted) between 15 and 16.5 deg"
    d["steady_shock_within_bar"] = all(15.0 <= d["shock_%s_steady_t4" % n][q] <= 16.5
                                       for n in ("fp32_bulk", "fp64")
                                       for q in ("effective_wedge_deg_from_beta", "effective_wedge_deg_from_ratio"))
    out[spec["name"]] = d
    spec = W.oscillating_cylinder_m02_re185()
    c32, c64 = pair(spec)
    worst = 0.0
    for _ in range(10):
        c32.step(100)
        c64.step(100)
        f32, f64 = c32.forces(), c64.forces()
        worst = max(worst, abs(f32[0] - f64[0]), abs(f32[1] - f64[1]))
    d = compare(c32, c64, worst)
    d["steps"] = 1000
    d["window"] = "Cd, Cl every 100 steps"
    out[spec["name"]] = d
    spec = W.naca0012_a5_m0001()
    c32, c64 = pair(spec)
    c32.step(2)
    c64.step(2)
    d = compare(c32, c64)
    d["physical_steps"] = 2
    d["subiters"] = spec["subiters"]
    out[spec["name"]] = d
    spec = W.cylinder_m02_re40()
    c32, c64 = pair(spec)
    c32.step(200)
    c64.step(200)
    d = compare(c32, c64)
    d["steps"] = 200
    out[spec["name"]] = d
    out["seconds"] = time.perf_counter() - t0
    return out


def run_serving(ibm, W, n, slots, chunk, burst, mode):
    """The seeded serving mix through the native request loop (ibm_server_*).

    Poisson mode submits each request when its arrival time has passed;
    burst mode submits all of them at once.  Latency (time to solution) runs
    from the arrival to the retirement of the request; throughput counts grid
    cells x stages x steps of all requests (dual time: 3 pseudo stages per
    sub-iteration) over the span from the first arrival to the last retirement.
    """
    reqs = W.serving_mix(n)
    srv = ibm.Server(max_active=slots, steps_per_chunk=chunk, mode=mode)
    ids, lag = {}, {}
    k = 0
    max_running = 0
    passes = 0
    t0 = time.perf_counter()
    while True:
        now = time.perf_counter() - t0
        while k < n and (burst or reqs[k]["arrival_s"] <= now):
            rid = srv.submit(reqs[k]["spec"], reqs[k]["nsteps"])
            ids[rid] = k
            lag[rid] = 0.0 if burst else max(0.0, (time.perf_counter() - t0) - reqs[k]["arrival_s"])
            k += 1
        na, npend = srv.progress()
        passes += 1
        max_running = max(max_running, na)
        if k == n and na == 0 and npend == 0:
            break
        if na == 0 and npend == 0:
            time.sleep(max(0.0, reqs[k]["arrival_s"] - (time.perf_counter() - t0)))
    span = time.perf_counter() - t0 - (0.0 if burst else reqs[0]["arrival_s"])
    stats = srv.stats()
    lat, work, failed = [], 0, 0
    for rid, kk in ids.items():
        r = srv.poll(rid)
        if r["state"] != ibm.REQ_DONE:
            failed += 1
            continue
        lat.append(r["finish_s"] - r["submit_s"] + lag[rid])
        sp = reqs[kk]["spec"]
        stages = 3 * sp["subiters"] if sp["time_scheme"] == W.TIME_DUAL else 3
        work += sp["nx"] * sp["ny"] * stages * r["steps_done"]
    srv.close()
    lat.sort()

    def pct(q):
        return lat[max(0, min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1))] * 1e3 if lat else None

    return {"requests": n, "failed": failed, "p50_ms": pct(0.50), "p99_ms": pct(0.99), "max_ms": pct(1.0),
            "mean_ms": statistics.fmean(lat) * 1e3 if lat else None, "span_s": span,
            "value": work / span / 1e6, "unit": "Mcell-updates/s (grid cells x stages)",
            "max_running": max_running, "loop_passes": passes, "loop_stats": stats}


def cpu_baseline(args, cells_gpu=None, sample_s=10.0, max_steps=400):
    """The FP64 oracle as it stands, on this host's cores, over a bounded number of steps."""
    import oracle
    spec = _spec(args.workload, "fp64")
    oracle.build()
    c = oracle.Case(spec)
    c.step(1)
    cells = int((c.tags() != 1).sum())
    n, t = 0, 0.0
    while t < sample_s and n < max_steps:
        t0 = time.perf_counter()
        c.step(1)
        t += time.perf_counter() - t0
        n += 1
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": cells * 3 * n / t / 1e6, "unit": "Mcell-updates/s", "cores": cores, "kind": "oracle",
            "sample": "%d RK3 steps of %s after 1 warm-up step (%.1f s)" % (n, spec["name"], t),
            "cpu_model": _cpu_model(), "nproc": os.cpu_count(),
            "single_core": _oracle_single_core(args.workload),
            "geometry3d_single_core": None if args.skip_geometry3d else _oracle_geometry3d_single_core(),
            "flow3d": None if args.skip_flow3d else _oracle_flow3d_step()}


def _oracle_flow3d_step():
    """One FP64 step of the oracle's 3-D sphere case (192 x 96 x 96) on this host's cores, after its
    classification."""
    import oracle
    from paper_1912_11908_gb300 import workloads as W
    spec = W.sphere_m03_re100()
    c = oracle.Case3D(spec)
    c.classify()
    t0 = time.perf_counter()
    c.step(1)
    t = time.perf_counter() - t0
    cells = int((c.tags() != 1).sum())
    return {"value": cells * 3 / t / 1e6, "unit": "Mcell-updates/s", "seconds_per_step": t,
            "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
            "sample": "1 SSP-RK3 step of %s" % spec["name"]}


def _oracle_geometry3d_single_core(n=40):
    """The oracle's 3-D pre-processing of Appendix A's sphere (1200 triangles) in n^3 lattice nodes on one host
    core (OMP_NUM_THREADS=1 in a child process): classification, tags, ordered lists, closest features and
    pseudo-normals of the listed nodes, as the device path computes them; None if it fails."""
    code = ("import sys, time; sys.path.insert(0, %r)\n"
            "import numpy as np, oracle\n"
            "from paper_1912_11908_gb300 import workloads as W\n"
            "oracle.build()\n"
            "v, t = W.uv_sphere(21, 30, 0.35, (0.5, 0.5, 0.5))\n"
            "ax = (np.arange(%d) + 0.5) / %d\n"
            "Z, Y, X = np.meshgrid(ax, ax, ax, indexing='ij')\n"
            "pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)\n"
            "t0 = time.perf_counter()\n"
            "solid = oracle.classify_points_3d(v, t, pts).reshape(%d, %d, %d)\n"
            "flat = oracle.tags_3d(solid).ravel()\n"
            "nodes = np.concatenate([np.nonzero(flat == k)[0] for k in (2, 3, 4, 5)])\n"
            "oracle.closest_3d(v, t, pts[nodes])\n"
            "print(time.perf_counter() - t0, len(nodes), len(t))\n") % (ROOT, n, n, n, n, n)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        sec, nodes, ntri = out.stdout.split()
        return {"workload": "Appendix A sphere, %s triangles, %d^3 lattice nodes" % (ntri, n), "s": float(sec),
                "listed_nodes": int(nodes), "cores": 1,
                "stages": "classification, tags, lists, closest features and pseudo-normals"}
    except Exception:
        return None


def _cpu_model():
    """The host CPU's model line from /proc/cpuinfo (x86 "model name"; Arm implementer / part), else the machine."""
    import platform
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
        for key in ("model name", "Model", "CPU part"):
            for line in info.splitlines():
                if line.startswith(key):
                    val = line.split(":", 1)[1].strip()
                    return "%s %s" % (platform.machine(), val) if key == "CPU part" else val
    except OSError:
        pass
    return platform.machine()


def _oracle_single_core(workload, sample_s=3.0, max_steps=100):
    """The oracle on one host core (OMP_NUM_THREADS=1 in a child process), a short sample; None if it fails."""
    code = ("import sys, time; sys.path.insert(0, %r)\n"
            "import oracle, bench\n"
            "spec = bench._spec(%r, 'fp64')\n"
            "oracle.build()\n"
            "c = oracle.Case(spec)\n"
            "c.step(1)\n"
            "cells = int((c.tags() != 1).sum())\n"
            "n, t = 0, 0.0\n"
            "while t < %r and n < %d:\n"
            "    t0 = time.perf_counter(); c.step(1); t += time.perf_counter() - t0; n += 1\n"
            "print(cells * 3 * n / t / 1e6, n, t)\n") % (ROOT, workload, sample_s, max_steps)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
        v, n, t = out.stdout.split()
        return {"value": float(v), "unit": "Mcell-updates/s", "cores": 1,
                "sample": "%s RK3 steps (%.1f s)" % (n, float(t))}
    except Exception:
        return None


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle timed on this host's cores, one full RK3 step per bench step."""
    if rank != 0:
        return
    import oracle
    spec = _spec(args.workload, "fp64")
    oracle.build()
    c = oracle.Case(spec)
    c.step(1)
    cells = int((c.tags() != 1).sum())
    c.step(args.warmup)
    t0 = time.perf_counter()
    c.step(args.steps)
    t = time.perf_counter() - t0
    value = cells * 3 * args.steps / t / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {
        "impl": "reference",
        "metric": "Mcell-updates/s per RK stage (FP32-bulk vs FP64)",
        "value": value, "unit": "Mcell-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (closed-form wedge, uniform free-stream start)",
        "config": {"workload": spec["name"], "grid": [spec["nx"], spec["ny"]], "active_cells": cells,
                   "precision": "fp64", "stages_per_step": 3, "time_scheme": "SSP-RK3"},
        "cpu_baseline": {"value": value, "unit": "Mcell-updates/s", "cores": cores, "kind": "oracle",
                         "sample": "%d full RK3 steps of %s" % (args.steps, spec["name"])},
        "e2e": {"value": value, "unit": "Mcell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="wedge_768x384", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32_bulk", choices=["fp32_bulk", "fp64"])
    ap.add_argument("--grid", default=None, help="override the workload grid, e.g. 3072x1536 (profiling)")
    ap.add_argument("--stage-launch", type=int, default=None, choices=[0, 1, 2],
                    help="pin the launch form of the FP32-bulk explicit stages (default: the autotuner's pick)")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-dual", action="store_true")
    ap.add_argument("--skip-moving", action="store_true")
    ap.add_argument("--skip-serving", action="store_true")
    ap.add_argument("--skip-accuracy", action="store_true")
    ap.add_argument("--skip-peaks", action="store_true", help="do not measure the FMA peaks (profiling runs)")
    ap.add_argument("--skip-geometry3d", action="store_true")
    ap.add_argument("--skip-flow3d", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=512)
    ap.add_argument("--serve-slots", type=int, default=32)
    ap.add_argument("--serve-chunk", type=int, default=10)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
