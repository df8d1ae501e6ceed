"""Expected distances at the benchmark's full sizes and sweep counts, from
the FP64 oracle alone (oracle/ and the seeded input generators; nothing from
the CUDA path).  The oracle takes minutes per case even in its level-parallel
build (bit-identical to the single-threaded one), so the values are stored: a
uniform seeded sample of vertices with their oracle distance and set index.

    python tests/golden/make_fullsize_golden.py c2-face|c2-edge|c3-edge|c3-face|c4-<k>[-face]|c4-all

c4-<k> is serving mesh k (0..9: jittered grids 101, 257, 513, 1025, 2000 and
noisy icospheres 5..9) with its seeded request of 1..16 sources and its
serving sweep count, edge form unless -face is given; c4-all writes the ten
edge-form cases and the face form of meshes 2 and 6.

Writes tests/golden/fullsize_<case>.json."""
import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import meshgen  # noqa: E402
import oracle  # noqa: E402

SAMPLES = 5000
SAMPLES_SERVING = 2000
C4_ALL = [f"c4-{k}" for k in range(10)] + ["c4-2-face", "c4-6-face"]


def case(name):
    """(description, mesh, sources, form, sweeps, m, samples)"""
    if name.startswith("c2-"):
        w = meshgen.workload_c2()
        form = name[3:]
        return ("jittered grid 1025x1025 (the benchmark mesh), its source", w.mesh, w.sources[0], form, 2000, 1.0,
                SAMPLES)
    if name in ("c3-edge", "c3-face"):
        w = meshgen.workload_c3()
        form = name[3:]
        return ("noisy icosphere level 10 (10.5M V), the batched configuration's second source set",
                w.mesh, w.sources[1], form, w.gs_face if form == "face" else w.gs_edge, w.m, SAMPLES)
    if name.startswith("c4-"):
        parts = name.split("-")
        k = int(parts[1])
        form = parts[2] if len(parts) > 2 else "edge"
        mesh = meshgen.serving_meshes()[k]
        return (f"serving mesh {k}: {mesh.name} ({mesh.nv} V), its seeded request", mesh,
                meshgen.serving_request(k, mesh), form, meshgen.serving_sweeps(mesh), 1.0, SAMPLES_SERVING)
    raise SystemExit(f"unknown case {name}")


def write(name):
    desc, mesh, src, form, sweeps, m, samples = case(name)
    t0 = time.time()
    with oracle.parallel(True):
        md = oracle.mesh_data(mesh.V, mesh.F)
        ref = oracle.solve(md, src, form, sweeps=sweeps, m=m)
        threads = oracle.threads()
    rng = meshgen.rng_for(4242)
    idx = np.unique((rng.random(samples) * md.nv).astype(np.int64))
    out = {"case": name, "mesh": desc, "nv": int(md.nv), "sources": [int(s) for s in np.atleast_1d(src)],
           "form": form, "sweeps": int(sweeps), "m": m, "admm_iters": oracle.ADMM_ITERS, "mu": oracle.MU,
           "hbar": float(md.hbar), "oracle_seconds": round(time.time() - t0, 1),
           "oracle_threads": threads, "host": platform.machine(),
           "index": [int(i) for i in idx], "d": [float(ref["d"][i]) for i in idx],
           "level": [int(ref["bfs"].level[i]) for i in idx]}
    with open(os.path.join(HERE, f"fullsize_{name}.json"), "w") as f:
        json.dump(out, f)
    print(name, "done in", out["oracle_seconds"], "s", flush=True)


def main():
    names = C4_ALL if sys.argv[1] == "c4-all" else sys.argv[1:]
    for name in names:
        write(name)


if __name__ == "__main__":
    main()
