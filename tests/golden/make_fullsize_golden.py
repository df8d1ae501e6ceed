"""Expected distances at the benchmark's full sizes and sweep counts, from
the FP64 oracle alone (oracle/ and the seeded input generators; nothing from
the CUDA path).  The oracle takes minutes to an hour per case, so the values
are stored: a uniform seeded sample of vertices with their oracle distance.

    python tests/golden/make_fullsize_golden.py c2-face|c2-edge|c3-edge

writes tests/golden/fullsize_<case>.json."""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import meshgen  # noqa: E402
import oracle  # noqa: E402

SAMPLES = 5000


def case(name):
    if name.startswith("c2-"):
        w = meshgen.workload_c2()
        form = name[3:]
        return "jittered grid 1025x1025 (the benchmark mesh), its source", w.mesh, w.sources[0], form, 2000, 1.0
    if name == "c3-edge":
        w = meshgen.workload_c3()
        return ("noisy icosphere level 10 (10.5M V), the batched configuration's second source set",
                w.mesh, w.sources[1], "edge", w.gs_edge, w.m)
    raise SystemExit(f"unknown case {name}")


def main():
    name = sys.argv[1]
    desc, mesh, src, form, sweeps, m = case(name)
    t0 = time.time()
    md = oracle.mesh_data(mesh.V, mesh.F)
    ref = oracle.solve(md, src, form, sweeps=sweeps, m=m)
    rng = meshgen.rng_for(4242)
    idx = np.unique((rng.random(SAMPLES) * md.nv).astype(np.int64))
    out = {"case": name, "mesh": desc, "nv": int(md.nv), "sources": [int(s) for s in np.atleast_1d(src)],
           "form": form, "sweeps": int(sweeps), "m": m, "admm_iters": oracle.ADMM_ITERS, "mu": oracle.MU,
           "hbar": float(md.hbar), "oracle_seconds": round(time.time() - t0, 1),
           "index": [int(i) for i in idx], "d": [float(ref["d"][i]) for i in idx],
           "level": [int(ref["bfs"].level[i]) for i in idx]}
    with open(os.path.join(HERE, f"fullsize_{name}.json"), "w") as f:
        json.dump(out, f)
    print(name, "done in", out["oracle_seconds"], "s")


if __name__ == "__main__":
    main()
