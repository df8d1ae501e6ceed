#!/usr/bin/env python
"""Benchmark of the geodesic-distance path on the 168M-vertex mesh.

Default workload (one step = one geodesic solve): the seeded sinusoid
icosphere of level 12 (167,772,162 vertices, 335,544,320 faces, radial
displacement by 8 low-frequency sinusoids of amplitude 0.05) with one uniform
random source, edge form, t = 10 hbar^2, 4000 Gauss-Seidel sweeps, 10 ADMM
iterations: breadth-first sets and layout, diffusion, normalisation, ADMM,
integration.  FP32 sweeps and ADMM, FP64 integration.  The mesh is resident
(loaded once, its setup timed apart); inputs are far larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload c5|c2|c3|c4] [--level L] [--sweeps S]

The line also carries, measured in the same run: the 1025^2 grid (both forms,
2000 sweeps; its working set is L2-resident), the 10.5M-vertex mesh as one
query and as a batch of 64, and a short serving stream.  ``--workload c3|c4``
run the batched and serving configurations in full.

Multi-GPU: replicas only.  Every rank solves its own source (the queries are
independent), no collective touches the data path; value is the solves of all
ranks over the slowest rank's time (weak scaling).

``--impl reference`` times the FP64 CPU oracle (the reference arm, its
level-parallel build on all host cores) on a bounded sample of the same
workload: the same pipeline on the level-9 mesh of the same family, scaled
to the full mesh and sweep count.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "geodesic solves/s and HBM GB/s at <=1e-4 rel err vs oracle; serve p50/p99 latency"
UNIT = "solves/s"
ADMM = 10
C2_SWEEPS = 2000
C2_FORMS = ("face", "edge")
SAMPLE_LEVEL = 9          # the oracle's bounded sample: the level-9 mesh of the benchmark's family
SAMPLE_SWEEPS = 400       # Gauss-Seidel sweeps of the sample (scaled to the full count): about 10 s on 16 cores
E2E_MAX_STEPS = 3         # end-to-end steps (each copies the 1.3 GB distance field back to the host)


def _rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def rank_sources(rank: int, nv: int, base_sources, config: int = 5):
    """Replicas only: rank 0 solves the workload's source, every other rank a
    seeded source of its own (the queries are independent; nothing is
    exchanged between ranks on the data path)."""
    import meshgen
    if rank == 0:
        return base_sources
    return meshgen.random_sources(meshgen.rng_for(meshgen.config_seed(config) + 7 * rank), nv, 1, 1)


def max_over_ranks(x: float, dist, device=None) -> float:
    """The slowest rank's time (the job ends when the last replica ends)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, solves_per_step: int, steps: int, total_ms: float) -> float:
    """Solves of all ranks per second of the slowest rank (weak scaling)."""
    return world * solves_per_step * steps / (total_ms / 1000.0)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured (STREAM-style copy)"
    except Exception:
        return 6800.0, "fallback"


def host_info() -> dict:
    """Cores, CPU model and RAM of the host the oracle runs on."""
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    ram = None
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemTotal:"):
                    ram = round(int(ln.split()[1]) / 1024 / 1024, 1)
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "arch": platform.machine(), "ram_gib": ram}


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
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
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def gs_bytes(nv: int, ne: int, sweeps: int) -> int:
    """Algorithmic bytes of one diffusion-kernel launch by the rule 16 V + 16 E
    per sweep: per vertex a row pointer (4), the diagonal (4), u read (4) and
    u written (4); per directed edge (2E of them) a column index and a weight
    (8)."""
    return sweeps * (16 * nv + 16 * ne)


def gs_state_bytes(nv: int, sweeps: int) -> int:
    """The bytes this library moves beyond gs_bytes: its diffusion state is a
    4-byte mantissa and a 4-byte binary exponent per vertex (the heat
    solution spans far more than the FP32 range), read and written once per
    sweep, 8 bytes per vertex-sweep more than a 4-byte u."""
    return sweeps * 8 * nv


STAGES = ("bfs_layout", "diffusion", "normalize", "admm", "integrate")


def stage_bytes(nv: int, ne: int, nf: int, sweeps: int, iters: int, form: str, nlev: int) -> dict:
    """Algorithmic bytes of each stage of one FP32 solve: every array a stage
    must read or write, counted once (entries = 2 ne directed edges).
      breadth-first sets + layout: 88 per vertex (row pointers, queue, set,
        pairing, position, row length, scan, diagonal) + 52 per entry
        (offer and count reads of the column, the key atomic and read, and the
        layout's column, edge id, theta, position and the written entry)
      diffusion: see gs_bytes
      normalise: 66 per face (face, positions, state, gradient operator, h)
      face ADMM: 154 per face and iteration (g, lambda read and written, h, face
        edges, twins, area, edge vectors shared by the edge's two faces), less
        48 per face for the first iteration, which starts from g = h, lambda = 0
        and reads h in their place
      edge ADMM: 78 per face + 32 per edge to initialise, per iteration 69 per
        face (face pass: x, lambda, w, signs) + 40 per edge (edge pass: the
        edge's faces and slots, sum of targets, w, lambda, x written)
      integration: the increments, 40 (edge form: set index, pairing vertex
        and edge, one end of that edge, its x, increment, link and distance
        written) or 88 (face form: the same with the edge's two faces, the
        positions and g in place of x) per vertex, then 24 per vertex for
        each of ceil(log2 L) pointer-jumping rounds (distance and link read
        and written; the gathered elements of the same arrays count once)"""
    rows = 2 * ne
    adm = (max(iters, 1) * 154 * nf - 48 * nf) if form == "face" else (78 * nf + 32 * ne + iters * (69 * nf + 40 * ne))
    rounds = max(1, math.ceil(math.log2(max(nlev, 2))))
    return {"bfs_layout": 88 * nv + 52 * rows, "diffusion": gs_bytes(nv, ne, sweeps), "normalize": 66 * nf,
            "admm": adm, "integrate": (40 if form == "edge" else 88) * nv + 24 * nv * rounds}


def stage_roofline(stage_ms, nbytes, peak):
    """Achieved algorithmic GB/s of each stage against the HBM peak."""
    out = {}
    for i, k in enumerate(STAGES):
        ms = float(stage_ms[i])
        gbps = nbytes[k] / (ms / 1000.0) / 1e9 if ms > 0 else 0.0
        out[k] = {"bytes": int(nbytes[k]), "ms": round(ms, 4), "GBps": round(gbps, 1), "frac": round(gbps / peak, 3)}
    return out


def capture(name: str):
    """The committed ncu capture profiles/<name>.json of one diffusion launch
    (DRAM and L2 bytes), if it was taken on the current kernel source, else
    None."""
    path = os.path.join(ROOT, "profiles", f"{name}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        p = json.load(f)
    src = open(os.path.join(ROOT, "paper_1812_06060_gb300", "csrc", "gs.cu"), "rb").read()
    if p.get("gs_cu_sha256") != hashlib.sha256(src).hexdigest():
        return None
    return p


def scaled_traffic(cap, nv: int, sweeps: int):
    """DRAM bytes (read + write) of one diffusion launch on a mesh of nv
    vertices and `sweeps` sweeps, scaled from a capture on a smaller mesh of
    the same family by vertex-sweeps (the traffic of an HBM-resident launch
    grows in proportion), or None."""
    if cap is None or not cap.get("dram_bytes_per_launch") or not cap.get("vertex_sweeps"):
        return None
    return cap["dram_bytes_per_launch"] * (nv * sweeps) / cap["vertex_sweeps"]


def oracle_sample(md, src, m: float, sweeps_full: int, nv_full: int, sample_sweeps: int):
    """One bounded run of the FP64 oracle (the build selected by the caller)
    on the sample mesh: every stage once in the edge form, the Gauss-Seidel
    stage for ``sample_sweeps`` sweeps.  Scaled to the full workload: the
    sweeps by vertex-sweeps, the other stages by vertices (the per-vertex
    cost of a larger mesh is, if anything, higher: fewer cache hits).
    Returns (seconds per full solve, seconds spent)."""
    import oracle
    t0 = time.perf_counter()
    b = oracle.bfs(md, src)
    t1 = time.perf_counter()
    st = oracle.gs(md, b, oracle.diffusion_time(md, m), sample_sweeps)
    t2 = time.perf_counter()
    h = oracle.normalize(md, st)
    x = oracle.edge_admm(md, h, ADMM)[0]
    oracle.integrate_edge(md, b, x)
    t3 = time.perf_counter()
    scale_v = nv_full / md.nv
    est = (t1 - t0 + t3 - t2) * scale_v + (t2 - t1) * scale_v * sweeps_full / sample_sweeps
    return est, t3 - t0


def oracle_sample_setup(workload: str = "c5"):
    """The sample mesh, its oracle data and source: for the 168M-vertex line
    the level-9 member of its family; for the grid line the grid itself
    (the sample then bounds only the sweeps)."""
    import meshgen
    import oracle
    oracle.build()
    w = meshgen.workload_c2() if workload == "c2" else meshgen.workload_c5(SAMPLE_LEVEL)
    with oracle.parallel(True):
        md = oracle.mesh_data(w.mesh.V, w.mesh.F)
    return w, md


def cpu_baseline(steps: int, warmup: int, nv_full: int, sweeps_full: int, m: float, workload: str = "c5"):
    """The level-parallel oracle on all host cores on the bounded sample.
    Returns (solves/s scaled to the full workload, seconds per sample step,
    description, cores)."""
    import oracle
    w, md = oracle_sample_setup(workload)
    mesh_desc = (f"the jittered 1025^2 grid itself ({md.nv} V)" if workload == "c2" else
                 f"the sinusoid icosphere of level {SAMPLE_LEVEL} ({md.nv} V)")
    src = w.sources[0]
    with oracle.parallel(True):
        cores = oracle.threads()
        for _ in range(warmup):
            oracle_sample(md, src, m, sweeps_full, nv_full, SAMPLE_SWEEPS)
        est, spent = [], []
        for _ in range(steps):
            e, s = oracle_sample(md, src, m, sweeps_full, nv_full, SAMPLE_SWEEPS)
            est.append(e)
            spent.append(s)
    sec = statistics.mean(est)
    desc = (f"per step: the oracle's level-parallel build ({cores} threads) on {mesh_desc}, "
            f"edge form, m = {m}: sets, {SAMPLE_SWEEPS} sweeps, normalise, {ADMM} ADMM "
            f"iterations, integration; scaled to {nv_full} V and {sweeps_full} sweeps (sweeps by vertex-sweeps, "
            f"the rest by vertices); {statistics.mean(spent):.1f} s of CPU time per step")
    return 1.0 / sec, statistics.mean(spent), desc, cores


def line_spec(args):
    """(workload description, mesh, base sources, forms, sweeps, m, config
    number) of the bench line."""
    import meshgen
    if args.workload == "c2":
        w = meshgen.workload_c2()
        sweeps = args.sweeps or C2_SWEEPS
        desc = (f"jittered grid 1025x1025 ({w.mesh.nv} V, {w.mesh.nf} F), one uniform random source, {sweeps} "
                f"Gauss-Seidel sweeps, {ADMM} ADMM iterations, face + edge forms (2 solves per step)")
        return desc, w.mesh, w.sources[0], C2_FORMS, sweeps, w.m, 2
    w = meshgen.workload_c5(args.level)
    sweeps = args.sweeps or w.gs_edge
    desc = (f"sinusoid icosphere level {args.level} ({w.mesh.nv} V, {w.mesh.nf} F), one uniform random source, "
            f"edge form, m = {w.m}, {sweeps} Gauss-Seidel sweeps, {ADMM} ADMM iterations (1 solve per step)")
    return desc, w.mesh, w.sources[0], ("edge",), sweeps, w.m, 5


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = _rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1812_06060_gb300 import build as gbuild
    if rank == 0 or world == 1:
        gbuild.build()
    if dist:
        dist.barrier()
    import paper_1812_06060_gb300 as g
    g.load_library()

    t0 = time.perf_counter()
    desc, mesh, base_src, forms, sweeps, m, cfg = line_spec(args)
    generate_s = time.perf_counter() - t0
    src_np = np.asarray(rank_sources(rank, mesh.nv, base_src, cfg), np.int32)
    stream = torch.cuda.current_stream()
    ctx = g.Context(local, stream=stream)
    Vd, Fd = torch.from_numpy(mesh.V).cuda(), torch.from_numpy(mesh.F).cuda()
    torch.cuda.synchronize()
    ms0, ms1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms0.record(stream)
    M = g.Mesh(ctx, Vd, Fd)   # setup (a0): connectivity, geometry, operators, resident
    ms1.record(stream)
    torch.cuda.synchronize()
    setup_ms = ms0.elapsed_time(ms1)
    del Vd, Fd
    prm = {f: g.params(gs_sweeps=sweeps, admm_iters=ADMM, form=f, m=m) for f in forms}
    src = torch.from_numpy(src_np).cuda()
    out = {f: torch.empty(mesh.nv, dtype=torch.float64, device="cuda") for f in forms}
    big = mesh.nv * 64 > 4 * 129 * 2 ** 20      # working set far beyond L2: no flush needed
    flush = None if big else torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    # the mesh's first solve times its traversal cluster sizes (a 2-sweep solve)
    M.solve(src, out[forms[0]], g.params(gs_sweeps=2, admm_iters=ADMM, form=forms[0], m=m))

    def step(gs_ms, st):
        for f in forms:
            M.solve(src, out[f], prm[f])
            t = M.stage_times()
            gs_ms.append(t[5])
            st.append((f, t))

    for _ in range(args.warmup):
        step([], [])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    gs_ms, st_list = [], []
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    l0 = ctx.kernel_launches()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            if flush is not None:
                flush.zero_()
            evs[i][0].record(stream)
            step(gs_ms, st_list)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
    launches = ctx.kernel_launches() - l0
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), dist, "cuda")
    ms_per_step = total_ms / args.steps
    value = whole_job_value(world, len(forms), args.steps, total_ms)

    # end to end through the public API with host buffers: the source set is
    # copied from pinned host memory, the distances back into pinned memory
    src_host = torch.from_numpy(src_np).pin_memory()
    out_host = {f: torch.empty(mesh.nv, dtype=torch.float64).pin_memory() for f in forms}
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, E2E_MAX_STEPS))
    e2e_s = 0.0
    for i in range(e2e_steps):
        if flush is not None:
            flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for f in forms:
            M.solve(src_host, out_host[f], prm[f])
        e2e_s += time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist, "cuda")
    e2e_value = whole_job_value(world, len(forms), e2e_steps, 1000.0 * e2e_s)

    peak, peak_kind = measured_peaks()
    nlev = len(M.dump(g.GH_DUMP_LEVEL_OFF)) - 1
    ne, nf, nv = M.ne, mesh.nf, mesh.nv
    stages = {}
    for f, t in st_list[-len(forms):]:
        stages[f] = stage_roofline(t, stage_bytes(nv, ne, nf, sweeps, ADMM, f, nlev), peak)
    bytes_launch = gs_bytes(nv, ne, sweeps)
    gs_avg_ms = statistics.mean(gs_ms)
    achieved = bytes_launch / (gs_avg_ms / 1000.0) / 1e9
    with_state = (bytes_launch + gs_state_bytes(nv, sweeps)) / (gs_avg_ms / 1000.0) / 1e9
    result = None
    if rank == 0:
        if args.workload == "c2":
            cap = capture("k_gs_grid1025")
            traffic = cap.get("dram_bytes_per_full_launch") if cap else None
            roof = c2_roofline(cap, bytes_launch, gs_avg_ms, peak, peak_kind, achieved, with_state)
        else:
            cap = capture(f"k_gs_sinusoid_ico{args.level}")
            traffic = scaled_traffic(cap, nv, sweeps)
            roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": traffic, "kernel": "k_gs (Gauss-Seidel diffusion, persistent)",
                    "peak_kind": peak_kind, "bytes_rule": "16 V + 16 E per sweep",
                    "algorithmic_bytes_per_launch": bytes_launch, "avg_launch_ms": gs_avg_ms,
                    "with_state_bytes": {"bytes_per_launch": bytes_launch + gs_state_bytes(nv, sweeps),
                                         "GBps": with_state, "frac": with_state / peak,
                                         "rule": "24 V + 16 E per sweep: the 8-byte (mantissa, exponent) state"},
                    "traffic_source": (f"dram__bytes_read.sum + dram__bytes_write.sum of one launch on {cap['workload']}"
                                       f" (profiles/k_gs_sinusoid_ico{args.level}.json)"
                                       if cap else "no capture of the current kernel source"),
                    "dram_frac": (traffic / (gs_avg_ms / 1000.0) / 1e9 / peak) if traffic else None}
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "global_batch": len(forms) * world, "seq_len": None,
                       "parallelism": f"replicas{world}",
                       "l2": ("inputs larger than L2 (the mesh and a query hold far more than 129 MB)" if big else
                              "flushed (512 MiB write) before every step"),
                       "rel_err_bound_vs_oracle": 1e-4},
            "e2e": {"value": e2e_value, "unit": UNIT, "steps": e2e_steps,
                    "h2d_bytes_per_step": 4 * len(src_np) * len(forms),
                    "d2h_bytes_per_step": 8 * nv * len(forms)},
            "gpu_launches": int(launches),
            "roofline": roof,
            "mesh_generate_s": round(generate_s, 2),
            "mesh_setup_ms": round(setup_ms, 3),
            "device_bytes_held": ctx.memory(),
            "stage_ms_last_solve": dict(zip(list(STAGES) + ["k_gs"], [round(x, 4) for x in st_list[-1][1]])),
            "stage_roofline": {"peak_GBps": peak, "by_form": stages,
                               "note": "algorithmic bytes per stage (each array once) / CUDA-event stage time; "
                                       "the breadth-first stage is bound by its L dependent set steps, not HBM"},
            "clocks": clk.summary(),
        }
    if rank == 0 and world == 1 and not args.no_extras and args.workload == "c5":
        # the same mesh with t = hbar^2 (m = 1), same sweeps: one timed solve
        p1 = g.params(gs_sweeps=sweeps, admm_iters=ADMM, form=forms[0], m=1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        M.solve(src, out[forms[0]], p1)
        e1.record(stream)
        torch.cuda.synchronize()
        result["extra_m1"] = {"workload": desc.replace(f"m = {m}", "m = 1.0"), "solve_ms": e0.elapsed_time(e1),
                              "solves_per_s": 1000.0 / e0.elapsed_time(e1),
                              "stage_ms": dict(zip(list(STAGES) + ["k_gs"], [round(x, 4) for x in M.stage_times()]))}
    M.close()
    ctx.close()
    del out, src
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_extras and args.workload == "c5":
        import meshgen
        small = [m for m in meshgen.serving_meshes() if m.nv <= 263169]
        result["extra"] = {"c2": c2_summary(g, local, peak, peak_kind), "c3": c3_summary(g, local),
                           "c4": serve_summary(g, local, None, 240, 2.0, 4200),
                           "c4_small_meshes": serve_summary(g, local, small, 600, 4.0, 4300)}
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            v, spent, sdesc, cores = cpu_baseline(1, 0, nv, sweeps, m, args.workload)
            result["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                      "sample": sdesc, "host": host_info()}
        print(json.dumps(result), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def c2_roofline(cap, bytes_launch, gs_avg_ms, peak, peak_kind, achieved, with_state):
    """The grid's diffusion launch: its working set (padded operator about
    57 MB, state and diagonal 21 MB) fits in the 129 MB L2, so it is bound by
    L2 and the latency of its dependent steps, not by HBM."""
    out = {"bound": "l2", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "traffic": cap.get("dram_bytes_per_full_launch") if cap else None,
           "kernel": "k_gs (Gauss-Seidel diffusion, persistent)", "peak_kind": peak_kind + ", HBM: context only",
           "bytes_rule": "16 V + 16 E per sweep", "algorithmic_bytes_per_launch": bytes_launch,
           "avg_launch_ms": gs_avg_ms, "algorithmic_GBps_with_state": with_state}
    if cap:
        dram = cap.get("dram_bytes_per_full_launch")
        l2 = cap.get("lts_bytes")
        out.update({"dram_over_algorithmic": dram / bytes_launch if dram else None,
                    "l2_bytes_per_launch": l2, "l2_over_algorithmic": l2 / bytes_launch if l2 else None,
                    "l2_GBps": l2 / (gs_avg_ms / 1000.0) / 1e9 if l2 else None,
                    "l2_throughput_pct_of_peak": cap.get("lts_throughput_pct"),
                    "capture": "profiles/k_gs_grid1025.json"})
    return out


def c2_summary(g, device, peak, peak_kind, steps=3):
    """The 1025^2 grid, both forms, 2000 sweeps: solves/s with L2 flushed
    before every step, and the diffusion launch against L2."""
    import numpy as np
    import torch
    import meshgen
    w = meshgen.workload_c2()
    mesh = w.mesh
    stream = torch.cuda.current_stream()
    ctx = g.Context(device, stream=stream)
    M = g.Mesh(ctx, mesh.V, mesh.F)
    src = torch.from_numpy(np.asarray(w.sources[0], np.int32)).cuda()
    out = torch.empty(mesh.nv, dtype=torch.float64, device="cuda")
    prm = {f: g.params(gs_sweeps=C2_SWEEPS, admm_iters=ADMM, form=f) for f in C2_FORMS}
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    for f in C2_FORMS:
        M.solve(src, out, prm[f])
    gs_ms, total, st = [], 0.0, {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(steps):
        flush.zero_()
        e0.record(stream)
        for f in C2_FORMS:
            M.solve(src, out, prm[f])
            st[f] = M.stage_times()
            gs_ms.append(st[f][5])
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    nlev = len(M.dump(g.GH_DUMP_LEVEL_OFF)) - 1
    nb = gs_bytes(mesh.nv, M.ne, C2_SWEEPS)
    avg = statistics.mean(gs_ms)
    ach = nb / (avg / 1000.0) / 1e9
    ws = (nb + gs_state_bytes(mesh.nv, C2_SWEEPS)) / (avg / 1000.0) / 1e9
    res = {"workload": f"jittered grid 1025x1025 ({mesh.nv} V), one source, {C2_SWEEPS} sweeps, face + edge forms",
           "solves_per_s": len(C2_FORMS) * steps / (total / 1000.0), "steps": steps,
           "l2": "flushed (512 MiB write) before every step",
           "roofline": c2_roofline(capture("k_gs_grid1025"), nb, avg, peak, peak_kind, ach, ws),
           "stage_roofline": {"peak_GBps": peak, "note": "last step's stage times; algorithmic bytes",
                              "by_form": {f: stage_roofline(st[f], stage_bytes(mesh.nv, M.ne, mesh.nf, C2_SWEEPS,
                                                                                ADMM, f, nlev), peak)
                                          for f in C2_FORMS}}}
    M.close()
    ctx.close()
    return res


def c3_summary(g, device, form="edge"):
    """The 10.5M-vertex noisy icosphere: one query, then its 64 source sets
    as one batch."""
    import torch
    import meshgen
    w = meshgen.workload_c3()
    sweeps = w.gs_face if form == "face" else w.gs_edge
    ctx = g.Context(device)
    M = g.Mesh(ctx, w.mesh.V, w.mesh.F)
    prm = g.params(gs_sweeps=sweeps, form=form, m=w.m)
    one = torch.empty(w.mesh.nv, dtype=torch.float64, device="cuda")
    M.solve(w.sources[0], one, prm)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    M.solve(w.sources[1], one, prm)
    torch.cuda.synchronize()
    single_s = time.perf_counter() - t0
    K = len(w.sources)
    dout = torch.empty((K, w.mesh.nv), dtype=torch.float64, device="cuda")
    M.solve_batch(w.sources[:2], dout[:2], g.params(gs_sweeps=2, form=form, m=w.m))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    M.solve_batch(w.sources, dout, prm)
    torch.cuda.synchronize()
    batch_s = time.perf_counter() - t0
    res = {"workload": f"noisy icosphere level 10 ({w.mesh.nv} V), {form} form, {sweeps} sweeps, K = {K} source "
                       f"sets of 1..8 vertices", "single_solves_per_s": 1.0 / single_s,
           "batched_solves_per_s": K / batch_s, "speedup": (K / batch_s) * single_s,
           "batch_stage_ms": [round(x, 3) for x in M.stage_times()]}
    M.close()
    ctx.close()
    return res


def serve_stream(g, ctx, meshes, handles, n_req, rate, seed, form="edge"):
    """Poisson arrivals at `rate` requests/s, each on a uniform mesh with 1..16
    uniform sources; latency = submit to result on the host.  Returns
    (latencies in ms, wall seconds)."""
    import numpy as np
    import meshgen
    rng = meshgen.rng_for(seed)
    plan = []
    t = 0.0
    for _ in range(n_req):
        t += -np.log(1.0 - rng.random()) / rate
        k = int(rng.random() * len(meshes))
        plan.append((t, k, meshgen.random_sources(rng, meshes[k].nv, 1, 16)))
    prms = [g.params(gs_sweeps=meshgen.serving_sweeps(m), form=form) for m in meshes]
    sub_t = [0.0] * n_req
    done_t = [0.0] * n_req
    ids = [None] * n_req
    finished = [False] * n_req
    stop = threading.Event()

    def collector():
        outs = {}
        while not stop.is_set() or not all(finished):
            progressed = False
            for i in range(n_req):
                if ids[i] is None or finished[i]:
                    continue
                if ctx.poll(ids[i]):
                    k = plan[i][1]
                    out = outs.setdefault(k, np.empty(meshes[k].nv))
                    ctx.wait(ids[i], out)
                    done_t[i] = time.perf_counter()
                    finished[i] = True
                    progressed = True
            if not progressed:
                time.sleep(0.0002)

    th = threading.Thread(target=collector, daemon=True)
    th.start()
    t0 = time.perf_counter()
    for i, (ta, k, src) in enumerate(plan):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        sub_t[i] = time.perf_counter()
        ids[i] = ctx.submit(handles[k], src, prms[k])
    stop.set()
    th.join()
    wall = max(done_t) - t0
    lat = [1000.0 * (d - s) for s, d in zip(sub_t, done_t)]
    return lat, wall


def serve_summary(g, device, meshes, n_req, rate_factor, seed):
    """Single-stream capacity of the meshes (one query at a time, each mesh's
    own sweep count), then a Poisson stream at rate_factor times that
    capacity through the serving API.  meshes=None: the ten serving meshes."""
    import numpy as np
    import meshgen
    if meshes is None:
        meshes = meshgen.serving_meshes()
    cap_ctx = g.Context(device)
    times = []
    for m in meshes:
        M = g.Mesh(cap_ctx, m.V, m.F)
        out = np.empty(m.nv)
        prm = g.params(gs_sweeps=meshgen.serving_sweeps(m), form="edge")
        M.solve([0], out, prm)
        t0 = time.perf_counter()
        M.solve([1], out, prm)
        times.append(time.perf_counter() - t0)
        M.close()
    cap_ctx.close()
    capacity = 1.0 / float(np.mean(times))
    ctx = g.Context(device)
    handles = [g.Mesh(ctx, m.V, m.F) for m in meshes]
    lat, wall = serve_stream(g, ctx, meshes, handles, n_req, rate_factor * capacity, seed)
    for h in handles:
        h.close()
    ctx.close()
    return {"meshes": [f"{m.name} ({m.nv} V)" for m in meshes], "requests": n_req,
            "single_stream_capacity_solves_per_s": capacity, "offered_rate_per_s": rate_factor * capacity,
            "rate_factor": rate_factor, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "served_solves_per_s": n_req / wall,
            "served_over_single": (n_req / wall) / capacity, "form": "edge",
            "sweeps": "2x breadth-first depth bound per mesh",
            "single_query_ms": {m.name: round(1000 * t, 3) for m, t in zip(meshes, times)}}


def run_reference(args):
    """The reference arm: the oracle (level-parallel build, all host cores)
    on the bounded sample of the bench line's workload, each step one sample
    solve.  value is the sample scaled to the full workload; ms_per_step is
    the time a step actually took."""
    rank, world, _ = _rank()
    if rank != 0:
        return 0
    import meshgen
    if args.workload not in ("c5", "c2"):
        raise SystemExit("--impl reference times the default workload (c5) or the grid (c2)")
    if args.workload == "c2":
        w2 = meshgen.workload_c2()
        nv_full, sweeps, m = w2.mesh.nv, args.sweeps or C2_SWEEPS, 1.0
        desc = (f"jittered grid 1025x1025 ({nv_full} V), one source, {sweeps} sweeps, edge form (the oracle's "
                f"sample; the GPU line solves both forms)")
        del w2
    else:
        w5 = meshgen.workload_c5(args.level)
        nv_full = w5.mesh.nv
        sweeps, m = args.sweeps or w5.gs_edge, 10.0
        desc = (f"sinusoid icosphere level {args.level} ({nv_full} V, {w5.mesh.nf} F), one uniform random source, "
                f"edge form, m = {w5.m}, {sweeps} Gauss-Seidel sweeps, {ADMM} ADMM iterations (1 solve per step)")
        del w5
    t0 = time.perf_counter()
    v, spent, sdesc, cores = cpu_baseline(args.steps, args.warmup, nv_full, sweeps, m, args.workload)
    wall = time.perf_counter() - t0
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * spent,
           "extrapolated_ms_per_solve": 1000.0 / v, "wall_s": round(wall, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": desc, "global_batch": 1, "parallelism": "host"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sdesc,
                            "host": host_info()},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def run_workload(args):
    """The batched and serving configurations in full, one JSON line each
    (not the default bench):
    c3  noisy icosphere level 10 (10.5M V), 64 source sets of 1..8 vertices as
        K = 64 right-hand sides, edge form 700 sweeps (face form 1200 with
        --form face); batched solves/s against the single-query rate
    c4  serving stream over 10 meshes (grids 101..2000, noisy icospheres 5..9)
        at rates 0.25..4 x single-stream capacity: p50/p99 latency, solves/s"""
    import torch
    import meshgen
    from paper_1812_06060_gb300 import build as gbuild
    gbuild.build()
    import paper_1812_06060_gb300 as g
    g.load_library()
    dev = 0
    torch.cuda.set_device(dev)
    out = {"workload": args.workload, "data": "synthetic", "dtype": "f32"}
    if args.workload == "c3":
        out.update(c3_summary(g, dev, args.form))
    elif args.workload == "c4":
        res = []
        meshes = None
        rates = (0.25, 0.5, 1.0, 2.0, 4.0)
        if args.meshes == "small":
            # the latency-bound half of the stream: the meshes of at most 263k vertices
            meshes = [m for m in meshgen.serving_meshes() if m.nv <= 263169]
            rates = (0.5, 1.0, 2.0, 4.0, 8.0)
        for rf in rates:
            r = serve_summary(g, dev, meshes, args.requests, rf, meshgen.config_seed(4, 200) + int(rf * 100))
            res.append({k: r[k] for k in ("rate_factor", "offered_rate_per_s", "p50_ms", "p99_ms",
                                          "served_solves_per_s", "served_over_single",
                                          "single_stream_capacity_solves_per_s")})
        out.update({"config": ("10 meshes: jittered grids 101, 257, 513, 1025, 2000 and noisy icospheres 5..9; "
                               if meshes is None else
                               "the 6 meshes of at most 263k vertices: jittered grids 101, 257, 513 and noisy "
                               "icospheres 5..7; ") +
                              "1..16 uniform sources; edge form; sweeps 2x breadth-first depth bound",
                    "requests_per_rate": args.requests, "rates": res, "single_query_ms": r["single_query_ms"]})
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the grid, batch and serving measurements")
    ap.add_argument("--workload", default="c5", choices=["c5", "c2", "c3", "c4"],
                    help="c5: the benchmark line (168M-vertex mesh); c2: the 1025^2 grid as the line; "
                         "c3/c4: the batched and serving configurations")
    ap.add_argument("--level", type=int, default=12, help="icosphere level of the c5 family (12: the benchmark)")
    ap.add_argument("--form", default="edge", choices=["face", "edge"])
    ap.add_argument("--requests", type=int, default=2000, help="requests per rate (c4)")
    ap.add_argument("--meshes", default="all", choices=["all", "small"],
                    help="c4: all ten serving meshes, or the six of at most 263k vertices")
    ap.add_argument("--sweeps", type=int, default=0,
                    help="Gauss-Seidel sweeps per solve (a smaller case for profiling; default: the workload's)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("c3", "c4"):
        return run_workload(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
