#!/usr/bin/env python
"""Benchmark of the contact-simulation substep: env-substeps/s on procedural M16
nut-on-bolt environments (1000 envs, 256^3 float32 bolt SDF shared by all envs, 10k
samples on each nut, 60 Hz frames of 8 substeps x 32 Gauss-Seidel sweeps).

One bench step = one frame (fw_step): 8 x (detection + reduction kernel, solve +
integration kernel).  Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fw|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Per-launch DRAM traffic (read + write bytes) of the substep kernels from a one-pass ncu
# capture of the default workload, keyed by the sha256 of the substep kernels' sources
# (SUBSTEP_SOURCES) it was taken on; reported only while they are unchanged (the capture's
# summary is kept under profiles/).
NCU_TRAFFIC = {
    # 1000 M16 nut-bolt envs, FP32, the bench's launch shapes fixed (solve 2 envs per warp x
    # 1 warp, query 256 threads, reduction 4 warps), launches in its per-kernel timing pass
    # over the timed frames, the query's cull off
    "0a232dc5237be478": {"map_kernel": 0.12e6, "query_kernel": 34.26e6, "reduce_kernel": 86.76e6,
                         "solve_kernel": 127.13e6},
}
# per-launch L2 traffic (lts__t_bytes.sum, one ncu pass) on the same workload, same keying
NCU_L2 = {
    "0a232dc5237be478": {"map_kernel": 0.74e6, "query_kernel": 603.9e6, "reduce_kernel": 307.2e6,
                         "solve_kernel": 3144.2e6},
}

FP32_LANES_PER_SM = 128
SOLVE_FLOPS_PER_CONTACT_SWEEP = 100   # normal row, joint friction rows and the 6-DoF velocity update of one body
SOLVE_FLOPS_PER_CONTACT_PREP = 300    # rows, effective masses, couplings, bias
QUERY_BYTES_PER_SAMPLE = 16           # float4 sample point
QUERY_BYTES_PER_CORNER = {False: 4, True: 2}   # 8 grid corners per query, float32 / float16
CANDIDATE_BYTES = 32                  # (x, phi), (n, sample) written by the query, read by the reduction
FACE_BYTES = 48                       # three float4 vertices of a face (per-triangle contact generation)
BRICK_ENTRY_BYTES = 4                 # brick-table entry read per lookup (narrow-band bricked SDF)
CONTACT_BYTES = 64                    # reduced contact (32 B) + its winner scratch line (32 B)


# the files that make up the substep kernels (map, query, reduction, solve); the traffic
# tables are keyed by the hash of these files (comments removed) and of their compile flags.
# The launch shapes the host code picks are part of the bench line (solve_shape,
# detect_shape), not of the key.
SUBSTEP_SOURCES = ("fw_detect.cu", "fw_solve.cu", "fw_device.cuh", "fw_internal.h")


def _code_only(text: str) -> str:
    """a source file without its comments and blank lines (comment edits leave the
    compiled kernels, and so their counters, unchanged)"""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(l.rstrip() for l in text.splitlines() if l.strip())


def _src_hash() -> str:
    from paper_2205_03532_b300.csrc import build as B
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2205_03532_b300", "csrc")
    for f in SUBSTEP_SOURCES:
        h.update(_code_only(open(os.path.join(d, f), encoding="utf-8").read()).encode())
        h.update(repr((B.ARCH, B.FLAGS, B.FILE_FLAGS.get(f, []))).encode())
    return h.hexdigest()[:16]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6400.0), d.get("sm_max_mhz", 2032.0), "measured"
    return 6400.0, 2032.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.device)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# workload -> (scene builder (n_envs, seed), default envs, name, SDF description, data description)
WORKLOADS = {
    "nut_bolt": ("nut_bolt_scene", 1000, "nut_bolt_m16", "256^3",
                 "synthetic (procedural ISO M16 nut/bolt meshes, seeded poses)"),
    "mixed": ("mixed_nut_bolt_scene", 4096, "mixed_nut_bolt_m8_m20", "128^3-256^3",
              "synthetic (procedural ISO M8-M20 nut/bolt meshes, sizes and poses seeded)"),
    "gears": ("gear_scene", 2048, "gear_train_z20_z30_z40", "256^3",
              "synthetic (procedural involute spur gears, seeded phases)"),
    "pile": ("pile_scene", 256, "nut_pile_7xM16", "128^3",
             "synthetic (procedural M16 nuts dropped on a plate, seeded poses)"),
}


def make_scene(workload: str, n_envs: int, seed: int):
    from paper_2205_03532_b300 import scenes as S
    return getattr(S, WORKLOADS[workload][0])(n_envs=n_envs, seed=seed)


def pair_sources(sc, per_triangle: bool) -> int:
    """Candidate sources of one substep over all envs: per pair, the samples (or faces) of
    its point body's asset."""
    n = 0
    for g in sc.groups:
        for a, _ in g.pairs:
            A = sc.assets[int(g.bodies["asset"][0, a])]
            n += len(g.bodies) * (len(A.tris) if per_triangle else len(A.samples))
    return n


def env_seed(seed: int, rank: int) -> int:
    """Scene seed of a rank: every rank simulates its own envs (weak scaling, no exchange)."""
    return seed + 1000 * rank


def job_rate(local_ms: float, local_units: int, ws: int, device=None):
    """Whole-job rate of a weak-scaled run.  Each rank processed local_units in a timed
    region of local_ms; the job's time is the longest rank's and its units are the sum over
    ranks.  Returns (units per second, job ms, job units); collective only when ws > 1."""
    job_ms, units = float(local_ms), int(local_units)
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([job_ms], dtype=torch.float64, device=device)
        u = torch.tensor([float(units)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        job_ms, units = float(t.item()), int(round(u.item()))
    return units / (job_ms * 1e-3), job_ms, units


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(n_envs: int, seed: int, frames: int = 2, workload: str = "nut_bolt"):
    """The FP64 oracle as it stands, on host cores, on a bounded sample of the workload:
    n_envs envs of it (0: one per core, the oracle parallelises over envs) for `frames`
    frames after one warm-up detection, then one frame of the same world on one core; the
    oracle's lazy SDF bake (set-up work on both sides) is excluded from both times."""
    from oracle import oracle as O
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    n_envs = n_envs if n_envs > 0 else cores
    sc = make_scene(workload, n_envs, seed)
    w = O.world_from_scene(sc, lazy_bake=True)
    w.collide()

    def timed(k):
        b0 = w.bake_seconds()
        t0 = time.perf_counter()
        for _ in range(k):
            w.step(sc.sim.n_substeps, sc.sim.n_iters)
        return time.perf_counter() - t0 - (w.bake_seconds() - b0)
    el = timed(frames)
    w.set_threads(1)
    el1 = timed(1)
    units = n_envs * sc.sim.n_substeps
    return (units * frames / el, units / el1, cores,
            f"{n_envs} envs x {frames} frame(s) of {sc.sim.n_substeps} substeps x {sc.sim.n_iters} sweeps on "
            f"{cores} threads, then 1 frame on 1 thread")


def run_reference(args):
    """--impl reference: the CPU oracle on this bench's workload, each step a bounded sample."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import oracle as O
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    n = args.ref_envs if args.ref_envs > 0 else cores   # one env per core: the oracle parallelises over envs
    wl = args.workload if args.workload in WORKLOADS else "nut_bolt"
    _, n_full, wl_name, sdf_desc, data_desc = WORKLOADS[wl]
    sc = make_scene(wl, n, args.seed)
    w = O.world_from_scene(sc, lazy_bake=True)
    w.collide()
    for _ in range(args.warmup):
        w.step(sc.sim.n_substeps, sc.sim.n_iters)
    b0 = w.bake_seconds()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        w.step(sc.sim.n_substeps, sc.sim.n_iters)
    el = time.perf_counter() - t0 - (w.bake_seconds() - b0)
    units = n * sc.sim.n_substeps * args.steps
    v = units / el
    out = {"impl": "reference", "metric": "env-substeps/s", "value": v, "unit": "env-substeps/s",
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": data_desc,
           "config": {"workload": wl_name, "n_envs": n, "sample_of_envs": n_full, "sdf": sdf_desc + " fp64 lazy",
                      "substeps": sc.sim.n_substeps, "iters": sc.sim.n_iters},
           "cpu_baseline": {"value": v, "unit": "env-substeps/s", "cores": cores, "kind": "oracle",
                            "sample": f"{n} envs per step, lazy SDF bake excluded"},
           "e2e": {"value": v, "unit": "env-substeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def single_pair_generate(sc, gen_cfg, fp16, dev, frames=5):
    """Per-triangle contact generation for ONE nut-bolt pair (the first env of the scene):
    the average query launch time over `frames` frames, after one warm-up frame.  This is
    the latency of generating one pair's contacts, the figure the paper gives for its own
    generator (Sec. III-A)."""
    import torch
    from paper_2205_03532_b300 import fw, scenes as S
    g = sc.groups[0]
    one = S.Scene(name=sc.name, assets=sc.assets, groups=[S.EnvGroup(bodies=g.bodies[:1].copy(), pairs=g.pairs)],
                  sim=sc.sim)
    w = fw.world_from_scene(one, fp16=fp16, device=dev, **gen_cfg)
    w.step(sc.sim.n_substeps, sc.sim.n_iters)
    w.sync()
    w.set_timing(True)
    for _ in range(frames):
        w.step(sc.sim.n_substeps, sc.sim.n_iters)
    tim = w.get_timings()
    w.set_timing(False)
    n_cand, n_cont = w.detect_stats()
    faces = len(sc.assets[int(g.bodies["asset"][0, 0])].tris)
    w.close()
    return {"faces": faces, "generate_ms": tim["query_ms"] / max(tim["detect_launches"], 1),
            "reduce_ms": tim["reduce_ms"] / max(tim["detect_launches"], 1),
            "candidates": n_cand, "contacts": n_cont}


def solve_chain_floor(sc, snap, gen_cfg, fp16, dev, sim, sm_max, cycles_bench):
    """One env of the workload alone (the first env's state at the start of the timed frames,
    its contacts detected there), one substep from that state twenty times: the solve
    kernel's cycles per row update for a single chain with the GPU otherwise idle."""
    from paper_2205_03532_b300 import fw, scenes as S
    g = sc.groups[0]
    b = g.bodies[:1].copy()
    nb = b.shape[1]
    state = [t[:nb].cpu().numpy() for t in snap]
    one = S.Scene(name=sc.name, assets=sc.assets, groups=[S.EnvGroup(bodies=b, pairs=g.pairs)], sim=sc.sim)
    w = fw.world_from_scene(one, fp16=fp16, device=dev, **gen_cfg)
    w.set_state(*state)
    w.collide()
    rows = len(w.get_contacts(0))
    w.set_timing(True)
    for _ in range(20):   # one substep per call (detection at the same state, then the solve)
        w.set_state(*state)
        w.step(1, sim.n_iters)
    tim = w.get_timings()
    w.set_timing(False)
    w.close()
    ms = tim["solve_ms"] / max(tim["solve_launches"], 1)
    cyc = ms * 1e-3 * sm_max * 1e6 / max(rows * sim.n_iters, 1)
    return {"rows": rows, "cycles_per_row_update_one_env": cyc, "frac_of_bench": cyc / cycles_bench,
            "note": "the same solve kernel on one env alone: the chain-latency floor of this formulation"}


def run_fw(args):
    import torch
    from paper_2205_03532_b300 import fw, scenes as S

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = local
    stream = torch.cuda.Stream(device=dev)
    t_setup = time.perf_counter()
    _, n_default, wl_name, sdf_desc, data_desc = WORKLOADS[args.workload]
    sc = make_scene(args.workload, args.envs if args.envs > 0 else n_default, env_seed(args.seed, rank))
    # the gear train's SDFs are stored in FP16 (FP32 interpolation and solve) unless --fp32
    fp16 = bool(args.fp16 or (args.workload == "gears" and not args.fp32))
    sim = sc.sim
    tri_mode = args.contact_gen == "triangles"
    gen_cfg = {"contact_gen": 1, "tri_iters": args.tri_iters} if tri_mode else {}
    if args.sdf_band > 0:
        gen_cfg["sdf_band"] = args.sdf_band
    if args.solver == "jacobi":
        gen_cfg["solver"] = 1
    if args.substeps > 0:
        sim.n_substeps = args.substeps
    if args.iters > 0:
        sim.n_iters = args.iters
    with torch.cuda.stream(stream):
        t_b = time.perf_counter()
        w = fw.world_from_scene(sc, fp16=fp16, stream=stream.cuda_stream, device=dev, **gen_cfg)
        bake_s = time.perf_counter() - t_b
    n_env, n_body, n_pair = w.counts()
    nodes = tests = 0
    for ai, a in enumerate(sc.assets):
        if a.sdf_res:
            d = w.get_sdf(ai, values=False)[2]
            nodes += int(d[0]) * int(d[1]) * int(d[2])
            tests += int(d[0]) * int(d[1]) * int(d[2]) * len(a.tris)
    bake_info = {"s": bake_s, "grid_nodes": nodes, "nodes_per_s": nodes / bake_s,
                 "brute_force_point_triangle_tests_per_s": tests / bake_s}
    storage = {"band_voxels": args.sdf_band, "lookup_bytes": 0, "bricks_stored": 0, "bricks_total": 0}
    for ai, a in enumerate(sc.assets):
        if a.sdf_res:
            nbytes, ns_b, nb_b = w.sdf_storage(ai)
            storage["lookup_bytes"] += nbytes
            storage["bricks_stored"] += ns_b
            storage["bricks_total"] += nb_b
    shape = [int(v) for v in args.solve_shape.split(",")]
    w.set_solve_shape(*shape)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 126 MB L2

    def one_step():
        w.step(sim.n_substeps, sim.n_iters)

    # warm-up frames, with the autotuner (untimed set-up: the fastest solve shape and the
    # shared-memory rows per env for the contacts then present) three frames before their
    # end, so that the timed frames start from the same state either way
    pre = max(0, args.warmup - 3)
    with torch.cuda.stream(stream):
        for _ in range(pre):
            one_step()
    tuned = None
    detect_tuned = None
    if shape == [0, 0] and not args.no_autotune:
        tuned = w.autotune_solve(sim.n_substeps, sim.n_iters, trials=6)
        detect_tuned = w.autotune_detect(trials=6)
    if args.query_cull != "auto":   # after the autotuner, which may have changed it
        w.set_query_cull(args.query_cull == "on")
    with torch.cuda.stream(stream):
        for _ in range(args.warmup - pre):
            one_step()
    torch.cuda.synchronize()
    w.sync()
    # the state the timed frames start from: the per-kernel timing pass and the end-to-end
    # pass replay the same frames from it (the contacts grow as the nut runs down the thread)
    snap = [torch.empty((n_body, k), dtype=torch.float32, device=dev) for k in (3, 4, 3, 3)]
    w.get_state(out=snap)
    torch.cuda.synchronize()
    # ---- timed region: K frames, each bracketed by events; L2 flushed between frames
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.zero_()
                evs[k][0].record(stream)
                one_step()
                evs[k][1].record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    w.sync()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    value, total_ms, units = job_rate(sum(step_ms), n_env * sim.n_substeps * args.steps, ws, device=dev)
    # ---- per-kernel durations (direct launches with events on the world stream), same frames
    with torch.cuda.stream(stream):
        w.set_state(*snap)
    w.set_timing(True)
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()
            one_step()
    tim = w.get_timings()
    w.set_timing(False)
    det_ms = tim["detect_ms"] / max(tim["detect_launches"], 1)
    qry_ms = tim["query_ms"] / max(tim["detect_launches"], 1)
    red_ms = tim["reduce_ms"] / max(tim["detect_launches"], 1)
    sol_ms = tim["solve_ms"] / max(tim["solve_launches"], 1)
    n_cand, n_cont = w.detect_stats()          # of the last substep
    c_mean = n_cont / max(n_env, 1)
    corner = QUERY_BYTES_PER_CORNER[fp16]
    queries = pair_sources(sc, tri_mode)
    if tri_mode:
        # one candidate source per face of the point body's mesh: its three vertices and
        # one SDF cell (the descent's further lookups stay in the cell's neighbourhood)
        q_bytes = queries * (FACE_BYTES + 8 * corner) + n_cand * CANDIDATE_BYTES
    else:
        q_bytes = queries * (QUERY_BYTES_PER_SAMPLE + 8 * corner) + n_cand * CANDIDATE_BYTES
    if args.sdf_band > 0:
        q_bytes += queries * BRICK_ENTRY_BYTES
    ns = queries / max(n_pair, 1)
    hbm, sm_max, peak_kind = _peaks()
    r_bytes = n_cand * CANDIDATE_BYTES + n_cont * CONTACT_BYTES
    sol_flops = n_cont * (SOLVE_FLOPS_PER_CONTACT_SWEEP * sim.n_iters + SOLVE_FLOPS_PER_CONTACT_PREP)
    alu_peak = 148 * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    src = _src_hash()
    # the table was taken on the default workload only (1000 M16 envs, FP32), with the
    # query's cull off (the autotuner's choice there; the cull runs other kernels)
    default_run = (args.workload == "nut_bolt" and not fp16 and sc.n_envs == 1000 and not tri_mode
                   and args.sdf_band == 0 and args.solver == "gs" and args.substeps == 0 and args.iters == 0
                   and not w.query_cull())
    traffic = NCU_TRAFFIC.get(src, {}) if default_run else {}
    l2_traffic = NCU_L2.get(src, {}) if default_run else {}
    l2_gbs = fw.measure_l2_read(dev)   # untimed: the L2 roofline's denominator on this device

    def l2_entry(name, ms):
        t = l2_traffic.get(name)
        a = None if t is None else t / (ms * 1e-3) / 1e9
        return {"achieved": a, "peak": l2_gbs, "unit": "GB/s", "frac": None if a is None else a / l2_gbs,
                "traffic": t, "peak_source": "measured L2 read bandwidth (fw_measure_l2_read, 48 MB, L1 bypassed)"}

    def hbm_entry(name, nbytes, ms):
        gbs = nbytes / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                "traffic": traffic.get(name), "avg_launch_ms": ms, "algorithmic_bytes": nbytes,
                "peak_source": f"{peak_kind} hbm_gbs", "l2": l2_entry(name, ms)}

    def l2_bound_entry(name, nbytes, ms):
        # a kernel whose working set (grid cells, samples) is shared by every env and stays
        # in the 126 MB L2: its algorithmic bytes are served by L2, so L2 bounds it; the HBM
        # figure is kept beside it
        gbs = nbytes / (ms * 1e-3) / 1e9
        return {"bound": "l2", "achieved": gbs, "peak": l2_gbs, "unit": "GB/s", "frac": gbs / l2_gbs,
                "traffic": traffic.get(name), "avg_launch_ms": ms, "algorithmic_bytes": nbytes,
                "peak_source": "measured L2 read bandwidth (fw_measure_l2_read, 48 MB, L1 bypassed)",
                "hbm": {"achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                        "peak_source": f"{peak_kind} hbm_gbs"},
                "l2": l2_entry(name, ms)}

    sol_tf = sol_flops / (sol_ms * 1e-3) / 1e12
    kernels = {
        "query_kernel": dict(l2_bound_entry("query_kernel", q_bytes, qry_ms),
                             **{("faces_per_s" if tri_mode else "queries_per_s"): queries / (qry_ms * 1e-3)}),
        "reduce_kernel": hbm_entry("reduce_kernel", r_bytes, red_ms),
        "solve_kernel": {"bound": "alu", "achieved": sol_tf, "peak": alu_peak, "unit": "TFLOP/s",
                         "frac": sol_tf / alu_peak, "traffic": traffic.get("solve_kernel"),
                         "avg_launch_ms": sol_ms, "algorithmic_flops": sol_flops,
                         "peak_source": "148 SMs x 128 FP32 lanes x 2 x max SM clock",
                         "cycles_per_row_update": sol_ms * 1e-3 * sm_max * 1e6 / max(c_mean * sim.n_iters, 1),
                         "l2": l2_entry("solve_kernel", sol_ms)},
    }
    dominant = max(kernels, key=lambda k: kernels[k]["avg_launch_ms"])
    roof = {k: v for k, v in kernels[dominant].items() if k in ("bound", "achieved", "peak", "unit", "frac", "traffic")}
    roof["kernel"] = dominant
    # deepest contact and patches per pair over a sample of envs at the end of the run
    sample_c = [w.get_contacts(e) for e in range(0, n_env, max(1, n_env // 64))]
    deepest = min([float(c["phi"].min(initial=np.inf)) for c in sample_c])
    patches = [len(np.unique(c["pair"].astype(np.int64) * 1024 + c["patch"])) for c in sample_c]
    patches_per_pair = float(np.mean(patches)) / max(n_pair / max(n_env, 1), 1e-9)
    single = None
    if tri_mode:
        single = single_pair_generate(sc, gen_cfg, fp16, dev)
    # The solve's latency floor: the same kernel on ONE env (one warp on an idle GPU, the
    # same contacts as the first env of the timed frames), cycles per row update.  The
    # 1000-env kernel can be no faster per env than its longest env's chain alone.
    if args.workload == "nut_bolt" and not tri_mode and args.solver == "gs":
        kernels["solve_kernel"]["latency_floor"] = solve_chain_floor(sc, snap, gen_cfg, fp16, dev, sim, sm_max,
                                                                     kernels["solve_kernel"]["cycles_per_row_update"])
    # ---- end to end through the public API with host buffers: state in, frame, state out
    pin = [torch.empty((n_body, k), dtype=torch.float32).pin_memory() for k in (3, 4, 3, 3)]
    torch.cuda.synchronize()
    for dst, src_ in zip(pin, snap):   # the same frames again, from the host
        dst.copy_(src_)
    e2e_ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        e2e_ev[0].record(stream)
        for k in range(args.steps):
            w.set_state(*pin)
            one_step()
            w.get_state(out=pin)
        e2e_ev[1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = e2e_ev[0].elapsed_time(e2e_ev[1])
    e2e_value = ws * n_env * sim.n_substeps * args.steps / (e2e_ms * 1e-3)
    state_bytes = n_body * (3 + 4 + 3 + 3) * 4
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, v1, cores, sample = cpu_baseline(args.cpu_envs, args.seed, workload=args.workload)
        cpu = {"value": v, "unit": "env-substeps/s", "cores": cores, "kind": "oracle", "sample": sample,
               "value_1core": v1}
    if rank == 0:
        out = {"metric": "env-substeps/s", "value": value, "unit": "env-substeps/s", "n_gpus": ws,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": data_desc,
               "config": {"workload": wl_name + ("_per_triangle" if tri_mode else ""),
                          "n_envs": n_env, "pairs_per_env": n_pair / max(n_env, 1),
                          ("faces_per_pair" if tri_mode else "samples_per_pair"): ns,
                          "contact_gen": args.contact_gen, "solver": args.solver,
                          **({"tri_iters": args.tri_iters} if tri_mode else {}),
                          "sdf": sdf_desc + (" fp16" if fp16 else " fp32")
                                 + (f" narrow-band bricks ({args.sdf_band:g} voxels)" if args.sdf_band > 0 else ""),
                          "sdf_storage": storage,
                          "substeps": sim.n_substeps,
                          "iters": sim.n_iters, "frame_dt": sim.dt, "l2": "flushed between steps (256 MB write)",
                          "parallelism": f"replicas x{ws}"},
               "roofline": roof, "kernels": kernels,
               "phase_ms_per_frame": {"query": qry_ms * sim.n_substeps, "reduce": red_ms * sim.n_substeps,
                                      "solve": sol_ms * sim.n_substeps},
               "contacts_per_env": c_mean, "deepest_contact_m": deepest, "candidates_per_pair": n_cand / max(n_pair, 1),
               "contact_statistics": {"contacts_per_pair": n_cont / max(n_pair, 1), "patches_per_pair": patches_per_pair,
                                      "paper_nut_bolt": {"contacts_per_pair": 195, "patches_per_pair": 53}},
               "solve_shape": list(w.solve_shape()), "autotuned": tuned is not None,
               "detect_shape": {"query_threads": w.detect_shape()[0], "reduce_warps": w.detect_shape()[1],
                                "query_cull": w.query_cull()},
               "graph_gap_ms_per_frame": total_ms / args.steps - (qry_ms + red_ms + sol_ms) * sim.n_substeps,
               "real_time_factor": (sim.dt / sim.n_substeps) / (total_ms / args.steps / sim.n_substeps * 1e-3) * n_env,
               "cpu_baseline": cpu, "clocks": clk.summary(),
               **({"single_pair_generate": single} if single else {}),
               "e2e": {"value": e2e_value, "unit": "env-substeps/s", "h2d_bytes_per_step": state_bytes,
                       "d2h_bytes_per_step": state_bytes},
               "gpu_launches": args.steps * w.launches_per_step(sim.n_substeps),
               "bake_s": bake_s, "bake": bake_info, "setup_s": time.perf_counter() - t_setup, "src": src}
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def run_pile_env(args):
    """The paper's pile scenes (--pile-body nut / torus / bowl): 1023 bodies dropped from a
    lattice into a round tray, ONE pile env (pairs found at every detection, colour-ordered
    Gauss-Seidel over the whole GPU).
    The pile first settles for --settle frames (4 substeps x 16 sweeps, untimed set-up);
    the warm-up and timed frames then run the paper's settings for that scene (nuts and
    toruses 1 substep x 16 position sweeps, bowls 2 x 50, each + 1 velocity sweep) unless
    --substeps / --iters say otherwise.
    One pile per GPU (replicas under torchrun)."""
    import torch
    from paper_2205_03532_b300 import fw, scenes as S
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = local
    stream = torch.cuda.Stream(device=dev)
    t_setup = time.perf_counter()
    n_nuts = args.envs if args.envs > 0 else 1023
    kind = args.pile_body
    # per body: samples, SDF resolution (the bowl's 2 mm wall needs finer voxels) and the
    # paper's substeps and position iterations for its pile (Table "performance statistics")
    samples, res, sub0, it0 = {"nut": (5000, 128, 1, 16), "torus": (3000, 128, 1, 16),
                               "bowl": (3000, 256, 2, 50)}[kind]
    sc = S.pile_env_scene(kind, n_nuts, seed=env_seed(args.seed, rank), mode="drop", n_samples=samples,
                          sdf_res=res)
    sub = args.substeps if args.substeps > 0 else sub0
    iters = args.iters if args.iters > 0 else it0
    with torch.cuda.stream(stream):
        w = fw.world_from_scene(sc, stream=stream.cuda_stream, device=dev)
        for _ in range(args.settle):
            w.step(4, 16)
    w.sync()
    # the detection autotuner on the settled pile (untimed set-up: query and reduction
    # shapes, and whether the sample-group cull pays)
    if not args.no_autotune:
        w.autotune_detect(trials=6)
    if args.query_cull != "auto":
        w.set_query_cull(args.query_cull == "on")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 126 MB L2
    n_env, n_body, _ = w.counts()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            w.step(sub, iters)
    w.sync()
    snap = [torch.empty((n_body, k), dtype=torch.float32, device=dev) for k in (3, 4, 3, 3)]
    w.get_state(out=snap)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.zero_()
                evs[k][0].record(stream)
                w.step(sub, iters)
                evs[k][1].record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    w.sync()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    # whole-job rate: frames of every rank's pile per second of the slowest rank
    value, total_ms, units = job_rate(sum(step_ms), args.steps, ws, device=dev)
    pairs, colours = w.pile_pairs(0)
    n_cand, n_cont = w.detect_stats()
    # ---- per-kernel durations (direct launches with events on the world stream), same frames
    with torch.cuda.stream(stream):
        w.set_state(*snap)
    w.set_timing(True)
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()
            w.step(sub, iters)
    tim = w.get_timings()
    w.set_timing(False)
    nd = max(tim["detect_launches"], 1)
    det_ms, red_ms = tim["query_ms"] / nd, tim["reduce_ms"] / nd
    sol_ms = tim["solve_ms"] / max(tim["solve_launches"], 1)
    hbm, sm_max, peak_kind = _peaks()
    l2_gbs = fw.measure_l2_read(dev)
    n_pairs = len(pairs)
    ns = len(sc.assets[0].samples)
    corner = QUERY_BYTES_PER_CORNER[False]
    q_bytes = n_pairs * ns * (QUERY_BYTES_PER_SAMPLE + 8 * corner) + n_cand * CANDIDATE_BYTES
    r_bytes = n_cand * CANDIDATE_BYTES + n_cont * CONTACT_BYTES
    sweeps = iters + sc.sim.n_vel_iters
    sol_flops = n_cont * (SOLVE_FLOPS_PER_CONTACT_SWEEP * sweeps + SOLVE_FLOPS_PER_CONTACT_PREP)
    sm_alu = FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12     # one SM: the pile solve is one block
    kernels = {
        "pile_detect (pair list, maps, query)": {
            "bound": "l2", "achieved": q_bytes / (det_ms * 1e-3) / 1e9, "peak": l2_gbs, "unit": "GB/s",
            "frac": q_bytes / (det_ms * 1e-3) / 1e9 / l2_gbs, "traffic": None, "avg_launch_ms": det_ms,
            "algorithmic_bytes": q_bytes, "queries_per_s": n_pairs * ns / (det_ms * 1e-3),
            "peak_source": "measured L2 read bandwidth (fw_measure_l2_read, 48 MB, L1 bypassed)"},
        "reduce_kernel": {
            "bound": "hbm", "achieved": r_bytes / (red_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
            "frac": r_bytes / (red_ms * 1e-3) / 1e9 / hbm, "traffic": None, "avg_launch_ms": red_ms,
            "algorithmic_bytes": r_bytes, "peak_source": f"{peak_kind} hbm_gbs"},
        "pile_solve_kernel": {
            "bound": "alu", "achieved": sol_flops / (sol_ms * 1e-3) / 1e12, "peak": sm_alu, "unit": "TFLOP/s",
            "frac": sol_flops / (sol_ms * 1e-3) / 1e12 / sm_alu, "traffic": None, "avg_launch_ms": sol_ms,
            "algorithmic_flops": sol_flops,
            "peak_source": "ONE SM (the pile's single block) x 128 FP32 lanes x 2 x max SM clock",
            "row_updates_per_s": n_cont * sweeps / (sol_ms * 1e-3)},
    }
    dominant = max(kernels, key=lambda k: kernels[k]["avg_launch_ms"])
    roof = {k: v for k, v in kernels[dominant].items() if k in ("bound", "achieved", "peak", "unit", "frac", "traffic")}
    roof["kernel"] = dominant
    # ---- end to end with host buffers: state in, frame, state out
    pin = [torch.empty((n_body, k), dtype=torch.float32).pin_memory() for k in (3, 4, 3, 3)]
    torch.cuda.synchronize()
    for dst, src_ in zip(pin, snap):
        dst.copy_(src_)
    e2e_ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    with torch.cuda.stream(stream):
        e2e_ev[0].record(stream)
        for k in range(args.steps):
            w.set_state(*pin)
            w.step(sub, iters)
            w.get_state(out=pin)
        e2e_ev[1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = e2e_ev[0].elapsed_time(e2e_ev[1])
    p_end = pin[0].numpy()
    state_bytes = n_body * (3 + 4 + 3 + 3) * 4
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import oracle as O
        cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        ow = O.world_from_scene(sc, lazy_bake=True)
        ow.collide()                                   # lazy bake of the cells it needs
        b0 = ow.bake_seconds()
        t0 = time.perf_counter()
        ow.step(sub, iters)
        el = time.perf_counter() - t0 - (ow.bake_seconds() - b0)
        cpu = {"value": 1.0 / el, "unit": "frames/s", "cores": cores, "kind": "oracle",
               "sample": f"1 frame of the {n_nuts}-{kind} pile from its initial lattice (before the fall: "
                         f"{sub} substep(s) x {iters} + {sc.sim.n_vel_iters} sweeps, every pair detected), "
                         f"lazy SDF bake excluded"}
    if rank == 0:
        frame_ms = total_ms / args.steps
        out = {"metric": f"{kind} pile frames/s", "value": value, "unit": "frames/s", "n_gpus": ws,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": frame_ms,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": f"synthetic (procedural {kind}s dropped from a seeded lattice into a tray)",
               "config": {"workload": f"{kind}_pile_env_{n_nuts}", "n_envs": 1, "bodies": n_body,
                          "settle_frames": args.settle, "substeps": sub, "iters": iters,
                          "vel_iters": sc.sim.n_vel_iters, "samples_per_body": ns, "sdf": f"{res}^3 fp32",
                          "frame_dt": sc.sim.dt, "l2": "flushed between steps (256 MB write)",
                          "parallelism": f"replicas x{ws}"},
               "roofline": roof, "kernels": kernels,
               "phase_ms_per_frame": {"detect": det_ms * sub, "reduce": red_ms * sub, "solve": sol_ms * sub},
               "detect_shape": {"query_threads": w.detect_shape()[0], "reduce_warps": w.detect_shape()[1],
                                "query_cull": w.query_cull()},
               "pairs": n_pairs, "pairs_with_contacts": int((colours >= 0).sum()),
               "colours": int(colours.max() + 1) if n_pairs else 0,
               "candidates": n_cand, "contacts": n_cont,
               "candidates_per_pair_with_contacts": n_cand / max(int((colours >= 0).sum()), 1),
               "contacts_per_pair_with_contacts": n_cont / max(int((colours >= 0).sum()), 1),
               "real_time_factor": sc.sim.dt / (frame_ms * 1e-3),
               "bodies_below_floor": int((p_end[:-1, 2] < -0.005).sum()),   # origin 5 mm under the floor
               "cpu_baseline": cpu, "clocks": clk.summary(),
               "e2e": {"value": ws * args.steps / (e2e_ms * 1e-3), "unit": "frames/s",
                       "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes},
               "gpu_launches": args.steps * w.launches_per_step(sub),
               "setup_s": time.perf_counter() - t_setup, "src": _src_hash()}
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def run_diff_peg(args):
    """Gradient throughput on the differentiable peg workload (256 envs, one frame of 32
    substeps x 8 sweeps): each step records the rollout from the same initial state and
    runs its adjoint for a squared-distance pose loss.  Reported separately from the
    headline (nut-bolt) line."""
    import torch
    from paper_2205_03532_b300 import fw, scenes as S
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    sc, tp, tq = S.diff_peg_scene(n_envs=args.envs if args.envs > 0 else 256, seed=env_seed(args.seed, rank))
    w = fw.world_from_scene(sc, device=local)
    n_env, nb, npair = w.counts()
    x0 = [torch.tensor(a, device="cuda") for a in w.get_state()]
    pegs = torch.arange(0, nb, 2, device="cuda")
    tpos = torch.tensor(tp, dtype=torch.float32, device="cuda")
    S_, K = sc.sim.n_substeps, sc.sim.n_iters

    def step():
        w.set_state(*x0)
        w.record_rollout(S_, K)
        out = [torch.empty((nb, k), device="cuda") for k in (3, 4, 3, 3)]
        w.get_state(out=out)
        w.sync()
        gp = torch.zeros(nb, 3, device="cuda")
        gp[pegs] = 2 * (out[0][pegs] - tpos)
        z3, z4 = torch.zeros(nb, 3, device="cuda"), torch.zeros(nb, 4, device="cuda")
        t0 = time.perf_counter()
        w.adjoint_rollout(gp, z4, z3, z3)
        return time.perf_counter() - t0

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    t_rec, t_adj = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        ta = step()
        t_rec.append(time.perf_counter() - t0 - ta)
        t_adj.append(ta)
    tot = sum(t_rec) + sum(t_adj)
    value, job_ms, units = job_rate(1e3 * tot, n_env * S_ * args.steps, ws, device=local)
    if rank == 0:
        print(json.dumps({"metric": "gradient env-substeps/s", "value": value, "unit": "env-substeps/s",
                          "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": job_ms / args.steps, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f32", "data": "synthetic (procedural peg in hole, seeded)",
                          "config": {"workload": "diff_peg", "n_envs": n_env, "substeps": S_, "iters": K},
                          "record_ms": 1e3 * sum(t_rec) / args.steps, "adjoint_ms": 1e3 * sum(t_adj) / args.steps,
                          "timing": "host wall clock around calls that synchronise"}), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="fw", choices=["fw", "reference"])
    ap.add_argument("--envs", type=int, default=0, help="envs (0: the workload's own count)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--fp16", action="store_true", help="store the SDFs in FP16 (FP32 interpolation and solve)")
    ap.add_argument("--fp32", action="store_true", help="gears: keep the SDFs in FP32 (its configuration stores FP16)")
    ap.add_argument("--solve-shape", default="0,0", help="envs per warp, warps per block (0,0: automatic)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-envs", type=int, default=0, help="envs of the oracle sample (0: one per core)")
    ap.add_argument("--ref-envs", type=int, default=0, help="envs of the reference arm's sample (0: one per core)")
    ap.add_argument("--workload", default="nut_bolt",
                    choices=["nut_bolt", "mixed", "gears", "pile", "pile1024", "diff_peg"],
                    help="nut_bolt: the headline substep benchmark (1000 M16 envs); mixed: 4096 envs of "
                         "M8-M20 pairs; gears: 2048 three-gear trains (FP16 SDFs); pile: 256 envs of 7 M16 "
                         "nuts dropped on a plate; pile1024: ONE env of 1023 M16 nuts dropped into a tray "
                         "(pairs found every detection; --envs sets the nut count); diff_peg: gradient "
                         "throughput of the differentiable peg")
    ap.add_argument("--settle", type=int, default=60, help="pile1024: untimed frames before the warm-up")
    ap.add_argument("--pile-body", default="nut", choices=["nut", "torus", "bowl"],
                    help="pile1024: the bodies of the pile (the paper's Nuts, Toruses and Bowls scenes)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default solve shape")
    ap.add_argument("--query-cull", choices=["auto", "on", "off"], default="auto",
                    help="the narrow phase's sample-group cull: the detection autotuner's choice (auto; on "
                         "without the autotuner), or forced on / off")
    ap.add_argument("--contact-gen", default="samples", choices=["samples", "triangles"],
                    help="samples: SDF query of the nut's surface samples; triangles: one contact per "
                         "face of the nut's mesh by local minimisation over the face")
    ap.add_argument("--tri-iters", type=int, default=16, help="descent steps per face (triangles)")
    ap.add_argument("--solver", default="gs", choices=["gs", "jacobi"],
                    help="gs: projected Gauss-Seidel; jacobi: weighted Jacobi (one movable body per env)")
    ap.add_argument("--substeps", type=int, default=0, help="substeps per frame (0: the workload's)")
    ap.add_argument("--iters", type=int, default=0, help="solver sweeps per substep (0: the workload's)")
    ap.add_argument("--sdf-band", type=float, default=0.0,
                    help="narrow-band bricked SDF storage, band half-width in voxels (0: dense)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "diff_peg":
        run_diff_peg(args)
    elif args.workload == "pile1024":
        run_pile_env(args)
    else:
        run_fw(args)


if __name__ == "__main__":
    main()
