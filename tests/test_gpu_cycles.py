"""Cycle constraints of a closed surface (Sec. 5.1) on the GPU against the
FP64 oracle: the tree-cotree cycles' entries bit-exact (alone and after the
multi-source path constraints), distances within the contract, the
constraints satisfied, and the meshes that get none (genus 0, a boundary,
two pieces)."""
import numpy as np
import pytest

import meshgen
import oracle

pytestmark = pytest.mark.gpu

D_TOL = {False: 1e-4, True: 1e-9}


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


@pytest.fixture(scope="module")
def ctx(gh):
    c = gh.Context(0)
    yield c
    c.close()


def _d_err(d, dref, sources, hbar):
    mask = np.isfinite(dref)
    mask[np.asarray(sources)] = False
    return np.max(np.abs(d[mask] - dref[mask]) / np.maximum(np.abs(dref[mask]), hbar))


def _constraint_values(pc, var, form):
    out = []
    for j in range(len(pc.off) - 1):
        a, b = pc.off[j], pc.off[j + 1]
        if form == "edge":
            out.append(np.sum(pc.coef[a:b, 0] * var[pc.var[a:b]]))
        else:
            out.append(np.sum(np.einsum("ij,ij->i", pc.coef[a:b], var[pc.var[a:b]])))
    return np.asarray(out)


def _log(line):
    import os
    path = os.environ.get("GEOHEAT_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(line + "\n")


@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("form", ["edge", "face"])
@pytest.mark.parametrize("src,paths", [([5], False), ([5, 140, 200], True)], ids=["cycles", "paths+cycles"])
def test_torus_cycles_match_oracle(gh, ctx, form, fp64, src, paths):
    mesh = meshgen.torus(24, 12, seed=3)
    md = oracle.mesh_data(mesh.V, mesh.F)
    M = gh.Mesh(ctx, mesh.V, mesh.F)
    try:
        d = np.empty(md.nv)
        M.solve(np.asarray(src, np.int32), d, gh.params(gs_sweeps=150, form=form, fp64=fp64, path_constraints=paths,
                                                       cycle_constraints=True))
        ref = oracle.solve(md, src, form, sweeps=150, path_constraints_on=paths, cycle_constraints_on=True)
        pc = ref["pc"]
        assert len(pc.off) - 1 == (len(src) - 1 if paths else 0) + 2
        assert np.array_equal(M.dump(gh.GH_DUMP_PC_OFF), pc.off)
        assert np.array_equal(M.dump(gh.GH_DUMP_PC_VAR), pc.var)
        assert np.array_equal(M.dump(gh.GH_DUMP_PC_COEF), pc.coef.ravel())
        derr = _d_err(d, ref["d"], src, md.hbar)
        var = M.dump(gh.GH_DUMP_X) if form == "edge" else M.dump(gh.GH_DUMP_G).reshape(-1, 3)
        cv = np.abs(_constraint_values(pc, var, form)).max()
        scale = np.abs(var).max() * np.abs(pc.coef).max() * len(pc.var)
        _log(f"cycle constraints torus24x12 form={form} fp64={fp64} paths={paths}: d {derr:.2e} "
             f"constraint {cv / scale:.2e}")
        assert derr <= D_TOL[fp64]
        assert cv <= (1e-13 if fp64 else 1e-6) * scale
    finally:
        M.close()


def test_meshes_without_cycles(gh, ctx):
    a = meshgen.torus(12, 8, seed=1)
    two = meshgen.Mesh(V=np.vstack([a.V, a.V + [5.0, 0.0, 0.0]]), F=np.vstack([a.F, a.F + a.V.shape[0]]))
    for mesh in (meshgen.noisy_icosphere(3, 2), meshgen.jittered_grid(17, 3), two):
        M = gh.Mesh(ctx, mesh.V, mesh.F)
        for form in ("edge", "face"):
            x, y = np.empty(mesh.nv), np.empty(mesh.nv)
            M.solve([3], x, gh.params(gs_sweeps=60, form=form))
            M.solve([3], y, gh.params(gs_sweeps=60, form=form, cycle_constraints=True))
            assert M.dump(gh.GH_DUMP_PC_OFF).size == 0
            assert np.array_equal(x, y, equal_nan=True)
        M.close()


def test_larger_torus_both_forms(gh, ctx):
    mesh = meshgen.torus(160, 64, seed=9)
    md = oracle.mesh_data(mesh.V, mesh.F)
    M = gh.Mesh(ctx, mesh.V, mesh.F)
    for form in ("edge", "face"):
        d = np.empty(md.nv)
        M.solve([100], d, gh.params(gs_sweeps=300, form=form, fp64=True, cycle_constraints=True))
        ref = oracle.solve(md, [100], form, sweeps=300, cycle_constraints_on=True)
        assert np.array_equal(M.dump(gh.GH_DUMP_PC_VAR), ref["pc"].var)
        assert np.array_equal(M.dump(gh.GH_DUMP_PC_COEF), ref["pc"].coef.ravel())
        assert _d_err(d, ref["d"], [100], md.hbar) <= D_TOL[True]
    M.close()
