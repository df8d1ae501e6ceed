#!/usr/bin/env python
"""Benchmark of the geodesic-distance path on the 1025^2 jittered grid.

Workload (one step): the seeded 1025 x 1025 jittered grid (1,050,625
vertices, 2,097,152 faces) with one uniform random source, solved once in the
face form and once in the edge form (2 geodesic solves per step): breadth-
first sets and layout, Gauss-Seidel diffusion (2000 sweeps), normalisation,
10 ADMM iterations, integration.  FP32 sweeps and ADMM, FP64 integration.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: replicas only.  Every rank solves its own source (the queries are
independent), no collective touches the data path; value is the solves of all
ranks over the slowest rank's time (weak scaling).

``--impl reference`` times the FP64 CPU oracle (the reference arm) on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

with open(os.path.join(ROOT, "BASELINE.json")) as _f:
    METRIC = json.load(_f)["metric"]
UNIT = "solves/s"
GRID_N = 1025
SWEEPS = 2000
ADMM = 10
FORMS = ("face", "edge")
WORKLOAD = (f"jittered grid {GRID_N}x{GRID_N} (1,050,625 V, 2,097,152 F), one uniform random source, "
            f"{SWEEPS} Gauss-Seidel sweeps, {ADMM} ADMM iterations, face + edge forms (2 solves per step)")
ORACLE_SAMPLE_SWEEPS = 40


def _rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


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
    """Algorithmic bytes of one diffusion-kernel launch (FP32): per vertex and
    sweep a row pointer (4), the diagonal (4), the state read once (8) and
    written once (8); per directed edge a column index and a weight (8)."""
    return sweeps * (24 * nv + 8 * 2 * ne)


def gs_traffic():
    """DRAM bytes per diffusion launch from the committed ncu capture, if it
    was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "k_gs_grid1025.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        p = json.load(f)
    src = open(os.path.join(ROOT, "paper_1812_06060_gb300", "csrc", "gs.cu"), "rb").read()
    if p.get("gs_cu_sha256") != hashlib.sha256(src).hexdigest():
        return None
    return p.get("dram_bytes_per_full_launch")


def oracle_sample(md, src, sweeps_full: int, sample_sweeps: int):
    """One bounded run of the FP64 oracle on the workload: every stage once per
    form, the Gauss-Seidel stage for ``sample_sweeps`` sweeps, scaled to the
    full sweep count.  Returns (seconds per solve, seconds of CPU work spent)."""
    import oracle
    per_solve = []
    spent = 0.0
    for form in FORMS:
        t0 = time.perf_counter()
        b = oracle.bfs(md, src)
        t1 = time.perf_counter()
        st = oracle.gs(md, b, oracle.diffusion_time(md), sample_sweeps)
        t2 = time.perf_counter()
        h = oracle.normalize(md, st)
        if form == "face":
            g = oracle.face_admm(md, h, ADMM)[0]
            oracle.integrate_face(md, b, g)
        else:
            x = oracle.edge_admm(md, h, ADMM)[0]
            oracle.integrate_edge(md, b, x)
        t3 = time.perf_counter()
        per_solve.append((t1 - t0) + (t2 - t1) * sweeps_full / sample_sweeps + (t3 - t2))
        spent += t3 - t0
    return sum(per_solve) / len(per_solve), spent


def run_reference(args):
    rank, world, _ = _rank()
    if rank != 0:
        return 0
    import meshgen
    import oracle
    oracle.build()
    w = meshgen.workload_c2(GRID_N)
    md = oracle.mesh_data(w.mesh.V, w.mesh.F)
    src = w.sources[0]
    for _ in range(args.warmup):
        oracle_sample(md, src, SWEEPS, ORACLE_SAMPLE_SWEEPS)
    per = []
    spent = 0.0
    for _ in range(args.steps):
        s, sp = oracle_sample(md, src, SWEEPS, ORACLE_SAMPLE_SWEEPS)
        per.append(s)
        spent += sp
    sec = statistics.mean(per)
    value = 1.0 / sec
    sample = (f"per step: each form once with {ORACLE_SAMPLE_SWEEPS} of {SWEEPS} Gauss-Seidel sweeps "
              f"(scaled linearly to {SWEEPS}), all other stages in full; {spent:.1f} s of CPU work timed")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 2000.0 * sec, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "global_batch": 2, "parallelism": "host"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = _rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import meshgen
    from paper_1812_06060_gb300 import build as gbuild
    if rank == 0 or world == 1:
        gbuild.build()
    if dist:
        dist.barrier()
    import paper_1812_06060_gb300 as g
    g.load_library()

    w = meshgen.workload_c2(GRID_N)
    mesh = w.mesh
    src_np = w.sources[0] if rank == 0 else meshgen.random_sources(meshgen.rng_for(meshgen.config_seed(2) + 7 * rank),
                                                                   mesh.nv, 1, 1)
    stream = torch.cuda.current_stream()
    ctx = g.Context(local, stream=stream)
    M = g.Mesh(ctx, torch.from_numpy(mesh.V).cuda(), torch.from_numpy(mesh.F).cuda())
    prm = {f: g.params(gs_sweeps=SWEEPS, admm_iters=ADMM, form=f) for f in FORMS}
    src = torch.from_numpy(np.asarray(src_np, np.int32)).cuda()
    out = {f: torch.empty(mesh.nv, dtype=torch.float64, device="cuda") for f in FORMS}
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")   # > L2: evicts it

    def step(gs_ms):
        for f in FORMS:
            M.solve(src, out[f], prm[f])
            gs_ms.append(M.stage_times()[5])

    for _ in range(args.warmup):
        step([])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    gs_ms = []
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    l0 = ctx.kernel_launches()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            evs[i][0].record(stream)
            step(gs_ms)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
    launches = ctx.kernel_launches() - l0
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    if dist:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * len(FORMS) * args.steps / (total_ms / 1000.0)

    # end to end through the public API with host buffers: the source set is
    # copied from pinned host memory, the distances back into pinned memory
    src_host = torch.from_numpy(np.asarray(src_np, np.int32)).pin_memory()
    out_host = {f: torch.empty(mesh.nv, dtype=torch.float64).pin_memory() for f in FORMS}
    torch.cuda.synchronize()
    e2e_s = 0.0
    for i in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for f in FORMS:
            M.solve(src_host, out_host[f], prm[f])
        e2e_s += time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = world * len(FORMS) * args.steps / e2e_s

    peak, peak_kind = measured_peaks()
    bytes_launch = gs_bytes(mesh.nv, M.ne, SWEEPS)
    gs_avg_ms = statistics.mean(gs_ms)
    achieved = bytes_launch / (gs_avg_ms / 1000.0) / 1e9
    result = None
    if rank == 0:
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "global_batch": len(FORMS) * world, "seq_len": None,
                       "parallelism": f"replicas{world}", "l2": "flushed (512 MiB write) before every step",
                       "rel_err_bound_vs_oracle": 1e-4},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * len(src_np) * len(FORMS),
                    "d2h_bytes_per_step": 8 * mesh.nv * len(FORMS)},
            "gpu_launches": int(launches),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": gs_traffic(),
                         "kernel": "k_gs (Gauss-Seidel diffusion, persistent)", "peak_kind": peak_kind,
                         "algorithmic_bytes_per_launch": bytes_launch, "avg_launch_ms": gs_avg_ms,
                         "note": "working set (75.6 MB) fits in the 129 MB L2; sweeps after the first are served "
                                 "from L2, so the HBM fraction can exceed 1"},
            "stage_ms_last_solve": dict(zip(["bfs_layout", "diffusion", "normalize", "admm", "integrate",
                                             "k_gs"], [round(x, 4) for x in M.stage_times()])),
            "clocks": clk.summary(),
        }
        if world == 1 and not args.no_cpu_baseline:
            import oracle
            oracle.build()
            md = oracle.mesh_data(mesh.V, mesh.F)
            sec, spent = oracle_sample(md, src_np, SWEEPS, ORACLE_SAMPLE_SWEEPS)
            result["cpu_baseline"] = {
                "value": 1.0 / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"each form once with {ORACLE_SAMPLE_SWEEPS} of {SWEEPS} sweeps scaled linearly, other "
                          f"stages in full ({spent:.1f} s of CPU work)"}
        print(json.dumps(result), flush=True)
    M.close()
    ctx.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    global SWEEPS, WORKLOAD
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweeps", type=int, default=SWEEPS,
                    help="Gauss-Seidel sweeps per solve (a smaller case for profiling; the benchmark is 2000)")
    args = ap.parse_args()
    if args.sweeps != SWEEPS:
        WORKLOAD = WORKLOAD.replace(f"{SWEEPS} Gauss-Seidel", f"{args.sweeps} Gauss-Seidel")
        SWEEPS = args.sweeps
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
