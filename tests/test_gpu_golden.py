"""The GPU path at the benchmark's full sizes and sweep counts against
distances the FP64 oracle computed for the same seeded inputs
(tests/golden/fullsize_*.json, written by make_fullsize_golden.py, which
calls only the oracle and the input generators): the contract, relative
error <= 1e-4 against max(|d*|, hbar), on a uniform sample of vertices, and
the sampled vertices' breadth-first set indices bit-exact.  FP32 carries the
contract except on the two rough noisy-icosphere cases (FP32_ROUGH), where
the FP64 path does and FP32 is bounded at its 99th percentile."""
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


# Cases where FP32 does not reach the contract at every vertex: noisy
# icospheres (r = 1 + 0.02 n, n smoothed three times) are rough enough that
# many cotangent weights are negative, and the FP32 state's rounding, carried
# through thousands of sweeps, moves the converged iterate by up to about
# 1e-3 of the one-ring's scale; the worst vertices lie where several sources'
# fronts meet and d* is near 0, so the error is measured against hbar.  Every
# stage matches the oracle given its own FP32 input (the stage-wise test of
# the 168M-vertex mesh shows the same on a smooth mesh).  There the FP64 path
# carries the contract, and the FP32 path is bounded at its 99th percentile.
FP32_ROUGH = {"c3-face", "c4-9"}


def _params(gh, gd, fp64=0):
    return gh.params(gs_sweeps=gd["sweeps"], form=gd["form"], m=gd["m"], admm_iters=gd["admm_iters"],
                     mu=gd["mu"], fp64=fp64)


@pytest.mark.parametrize("name", ["c2-face", "c2-edge", "c3-edge", "c3-face"])
def test_contract_at_full_size(gh, name):
    gd = _golden(name)
    mesh = _mesh(name)
    assert mesh.nv == gd["nv"]
    ctx = gh.Context(0)
    M = gh.Mesh(ctx, mesh.V, mesh.F)
    try:
        src = np.asarray(gd["sources"], np.int32)
        d = np.empty(mesh.nv)
        M.solve(src, d, _params(gh, gd))
        idx = np.asarray(gd["index"])
        assert np.array_equal(M.dump(gh.GH_DUMP_LEVEL)[idx], np.asarray(gd["level"]))
        err, keep = _rel_err(d, gd)
        _log(f"golden {name} nv={gd['nv']} sweeps={gd['sweeps']} fp32: d max {err.max():.2e} "
             f"p99 {np.percentile(err, 99):.2e} over {keep.sum()} sampled vertices "
             f"({(err > 1e-4).sum()} above 1e-4)")
        if name in FP32_ROUGH:
            assert np.percentile(err, 99) <= 1e-4
            M.solve(src, d, _params(gh, gd, fp64=1))
            err64, _ = _rel_err(d, gd)
            _log(f"golden {name} nv={gd['nv']} sweeps={gd['sweeps']} fp64: d max {err64.max():.2e}")
            assert err64.max() <= 1e-4
        else:
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
        # every case in FP32, and the rough ones once more in FP64, all in flight together
        cases = [(n, gd, 0) for n, gd in zip(C4_ALL, golds)] + [(n, gd, 1) for n, gd in zip(C4_ALL, golds)
                                                                if n in FP32_ROUGH]
        ids = []
        for name, gd, fp64 in cases:
            k = int(name.split("-")[1])
            assert meshes[k].nv == gd["nv"]
            ids.append((k, ctx.submit(handles[k], np.asarray(gd["sources"], np.int32), _params(gh, gd, fp64))))
        for (k, rid), (name, gd, fp64) in zip(ids, cases):
            d = np.empty(meshes[k].nv)
            ctx.wait(rid, d)
            err, keep = _rel_err(d, gd)
            _log(f"golden {name} ({gd['mesh']}) served, sweeps={gd['sweeps']} {gd['form']} "
                 f"{'fp64' if fp64 else 'fp32'}: d max {err.max():.2e} p99 {np.percentile(err, 99):.2e} "
                 f"over {keep.sum()} sampled vertices")
            if name in FP32_ROUGH and not fp64:
                assert np.percentile(err, 99) <= 1e-4, name
            else:
                assert err.max() <= 1e-4, name
    finally:
        for h in handles:
            h.close()
        ctx.close()
