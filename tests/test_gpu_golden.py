"""The FP32 path at the benchmark's full sizes and sweep counts against
distances the FP64 oracle computed for the same seeded inputs
(tests/golden/fullsize_*.json, written by make_fullsize_golden.py, which
calls only the oracle and the input generators): the contract, relative
error <= 1e-4 against max(|d*|, hbar), on a uniform sample of vertices, and
the sampled vertices' breadth-first set indices bit-exact."""
import json
import os

import numpy as np
import pytest

import meshgen

pytestmark = pytest.mark.gpu

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
# the stored serving cases (tests/golden/make_fullsize_golden.py c4-all)
C4_ALL = [f"c4-{k}" for k in range(10)] + ["c4-2-face", "c4-6-face"]


@pytest.fixture(scope="module")
def gh():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_06060_gb300 import build
    build.build()
    import paper_1812_06060_gb300 as g
    g.load_library()
    return g


def _golden(name):
    path = os.path.join(HERE, f"fullsize_{name}.json")
    if not os.path.exists(path):
        pytest.skip(f"{path} not generated")
    with open(path) as f:
        return json.load(f)


def _mesh(name):
    if name.startswith("c2-"):
        return meshgen.workload_c2().mesh
    return meshgen.workload_c3().mesh


def _rel_err(d, gd):
    idx = np.asarray(gd["index"])
    ref = np.asarray(gd["d"])
    keep = ~np.isin(idx, gd["sources"])
    return np.abs(d[idx][keep] - ref[keep]) / np.maximum(np.abs(ref[keep]), gd["hbar"]), keep


def _log(line):
    path = os.environ.get("GEOHEAT_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(line + "\n")


@pytest.mark.parametrize("name", ["c2-face", "c2-edge", "c3-edge", "c3-face"])
def test_fp32_contract_at_full_size(gh, name):
    gd = _golden(name)
    mesh = _mesh(name)
    assert mesh.nv == gd["nv"]
    ctx = gh.Context(0)
    M = gh.Mesh(ctx, mesh.V, mesh.F)
    try:
        d = np.empty(mesh.nv)
        M.solve(np.asarray(gd["sources"], np.int32), d,
                gh.params(gs_sweeps=gd["sweeps"], form=gd["form"], m=gd["m"], admm_iters=gd["admm_iters"],
                          mu=gd["mu"]))
        idx = np.asarray(gd["index"])
        assert np.array_equal(M.dump(gh.GH_DUMP_LEVEL)[idx], np.asarray(gd["level"]))
        err, keep = _rel_err(d, gd)
        _log(f"golden {name} nv={gd['nv']} sweeps={gd['sweeps']} fp32: d max {err.max():.2e} "
             f"p99 {np.percentile(err, 99):.2e} over {keep.sum()} sampled vertices")
        assert err.max() <= 1e-4
    finally:
        M.close()
        ctx.close()


def test_serving_meshes_against_oracle(gh):
    """One seeded request per serving mesh (the ten meshes of the serving
    stream, edge form, and the face form on two of them), all submitted at
    once through the serving API so that they share batches and overlap on
    the device; each result against the oracle's stored distances."""
    import meshgen as mg
    golds = [_golden(n) for n in C4_ALL]
    meshes = mg.serving_meshes()
    ctx = gh.Context(0)
    ctx.serve_config(workers=2, max_batch=8)
    handles = [gh.Mesh(ctx, m.V, m.F) for m in meshes]
    try:
        ids = []
        for name, gd in zip(C4_ALL, golds):
            k = int(name.split("-")[1])
            assert meshes[k].nv == gd["nv"]
            prm = gh.params(gs_sweeps=gd["sweeps"], form=gd["form"], m=gd["m"], admm_iters=gd["admm_iters"],
                            mu=gd["mu"])
            ids.append((k, ctx.submit(handles[k], np.asarray(gd["sources"], np.int32), prm)))
        for (k, rid), name, gd in zip(ids, C4_ALL, golds):
            d = np.empty(meshes[k].nv)
            ctx.wait(rid, d)
            err, keep = _rel_err(d, gd)
            _log(f"golden {name} ({gd['mesh']}) served, sweeps={gd['sweeps']} {gd['form']} fp32: "
                 f"d max {err.max():.2e} over {keep.sum()} sampled vertices")
            assert err.max() <= 1e-4, name
    finally:
        for h in handles:
            h.close()
        ctx.close()
