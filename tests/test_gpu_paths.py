"""Multi-source path constraints (Sec. 5.2) on the GPU against the FP64
oracle: the path entries (variables and coefficients) bit-exact, distances
within the contract (1e-4 relative in FP32, 1e-9 in FP64), the constrained
variables satisfying the constraints, batches and served requests equal to
solo solves, and the special cases (one source, an unreachable source, too
many sources)."""
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


CASES = [
    ("grid33", lambda: meshgen.jittered_grid(33, 7), [1, 12, 30, 600, 1000], 300),
    ("ico4", lambda: meshgen.noisy_icosphere(4, 3), [0, 400, 1100, 2000, 2500, 77], 200),
]


@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("form", ["edge", "face"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_path_constraints_match_oracle(gh, ctx, case, form, fp64):
    name, make, src, sweeps = case
    mesh = make()
    md = oracle.mesh_data(mesh.V, mesh.F)
    M = gh.Mesh(ctx, mesh.V, mesh.F)
    try:
        d = np.empty(md.nv)
        M.solve(np.asarray(src, np.int32), d, gh.params(gs_sweeps=sweeps, form=form, fp64=fp64,
                                                       path_constraints=True))
        ref = oracle.solve(md, src, form, sweeps=sweeps, path_constraints_on=True)
        pc = ref["pc"]
        # the path entries: integer work, bit-exact
        assert np.array_equal(M.dump(gh.GH_DUMP_PC_OFF), pc.off)
        assert np.array_equal(M.dump(gh.GH_DUMP_PC_VAR), pc.var)
        assert np.array_equal(M.dump(gh.GH_DUMP_PC_COEF), pc.coef.ravel())
        # the breadth-first products of the solve itself are those of all sources
        assert np.array_equal(M.dump(gh.GH_DUMP_ORDER), ref["bfs"].order)
        derr = _d_err(d, ref["d"], src, md.hbar)
        var = M.dump(gh.GH_DUMP_X) if form == "edge" else M.dump(gh.GH_DUMP_G).reshape(-1, 3)
        cv = np.abs(_constraint_values(pc, var, form)).max()
        scale = np.abs(var).max() * np.abs(pc.coef).max() * len(pc.var)
        plain = oracle.solve(md, src, form, sweeps=sweeps)
        moved = np.abs(ref["d"] - plain["d"])[np.isfinite(plain["d"])].max()
        _log(f"path constraints {name} form={form} fp64={fp64}: d {derr:.2e} constraint {cv / scale:.2e} "
             f"(oracle's change from the plain solve {moved:.2e})")
        assert moved > 1e-6                       # the constraints act on this case
        assert derr <= D_TOL[fp64]
        assert cv <= (1e-13 if fp64 else 1e-6) * scale
    finally:
        M.close()


def test_single_source_is_unchanged(gh, ctx):
    mesh = meshgen.noisy_icosphere(4, 3)
    M = gh.Mesh(ctx, mesh.V, mesh.F)
    a, b = np.empty(mesh.nv), np.empty(mesh.nv)
    M.solve([17], a, gh.params(gs_sweeps=100, form="edge"))
    M.solve([17], b, gh.params(gs_sweeps=100, form="edge", path_constraints=True))
    assert np.array_equal(a, b)
    assert M.dump(gh.GH_DUMP_PC_OFF).size == 0
    M.close()


def test_unreachable_source_gets_an_empty_path(gh, ctx):
    a = meshgen.jittered_grid(9, 1)
    V = np.vstack([a.V, a.V + [10.0, 0.0, 0.0]])
    F = np.vstack([a.F, a.F + a.V.shape[0]])
    md = oracle.mesh_data(V, F)
    src = [0, 40, a.V.shape[0] + 3]
    M = gh.Mesh(ctx, V, F)
    for form in ("edge", "face"):
        d = np.empty(md.nv)
        M.solve(src, d, gh.params(gs_sweeps=60, form=form, fp64=True, path_constraints=True))
        ref = oracle.solve(md, src, form, sweeps=60, path_constraints_on=True)
        assert np.array_equal(M.dump(gh.GH_DUMP_PC_OFF), ref["pc"].off)
        assert ref["pc"].off[2] == ref["pc"].off[1]
        assert _d_err(d, ref["d"], src, md.hbar) <= D_TOL[True]
    M.close()


def test_long_paths_several_chunks(gh, ctx):
    """More than 1024 entries (the setup kernel's block) and sources on the
    boundary: paths along boundary and interior edges."""
    mesh = meshgen.jittered_grid(257, 4)
    md = oracle.mesh_data(mesh.V, mesh.F)
    n = 257
    src = [0, n - 1, n * (n - 1), n * n - 1, n * (n // 2) + n // 2, 5 * n + 100, 100 * n + 7]
    M = gh.Mesh(ctx, mesh.V, mesh.F)
    for form in ("edge", "face"):
        d = np.empty(md.nv)
        M.solve(src, d, gh.params(gs_sweeps=300, form=form, fp64=True, path_constraints=True))
        ref = oracle.solve(md, src, form, sweeps=300, path_constraints_on=True)
        assert ref["pc"].off[-1] > 1024
        assert np.array_equal(M.dump(gh.GH_DUMP_PC_VAR), ref["pc"].var)
        assert _d_err(d, ref["d"], src, md.hbar) <= D_TOL[True]
    M.close()


def test_early_stop_and_diagnostics_with_constraints(gh, ctx):
    mesh = meshgen.noisy_icosphere(4, 5)
    md = oracle.mesh_data(mesh.V, mesh.F)
    src = [3, 900, 1800]
    M = gh.Mesh(ctx, mesh.V, mesh.F)
    for form, eps in (("edge", (1e-3, 1e-3)), ("face", (2e-3, 5e-2))):
        d = np.empty(md.nv)
        M.solve(src, d, gh.params(gs_sweeps=200, form=form, fp64=True, diagnostics=True, admm_iters=40, eps=eps,
                                  path_constraints=True))
        ref = oracle.solve(md, src, form, sweeps=200, admm_iters=40, eps=eps, path_constraints_on=True)
        iters = int(M.dump(gh.GH_DUMP_ITERS)[0])
        assert iters == len(ref["res"])
        res = M.dump(gh.GH_DUMP_RESID).reshape(-1, 2)[:iters]
        assert np.allclose(res, ref["res"][:, :2], rtol=1e-8, atol=1e-14)
        assert _d_err(d, ref["d"], src, md.hbar) <= D_TOL[True]
    M.close()


def test_batch_and_serving_equal_solo(gh, ctx):
    mesh = meshgen.noisy_icosphere(4, 8)
    rng = meshgen.rng_for(15)
    sets = [meshgen.random_sources(rng, mesh.nv, 1, 8) for _ in range(5)]
    M = gh.Mesh(ctx, mesh.V, mesh.F)
    prm = gh.params(gs_sweeps=120, form="edge", path_constraints=True)
    out = np.empty((len(sets), mesh.nv))
    M.solve_batch(sets, out, prm)
    solo = []
    for q, s in enumerate(sets):
        one = np.empty(mesh.nv)
        M.solve(s, one, prm)
        assert np.array_equal(one, out[q])
        solo.append(one)
    plain = gh.params(gs_sweeps=120, form="edge")
    rids = [(ctx.submit(M, s, prm if q % 2 == 0 else plain), q) for q, s in enumerate(sets)]
    for rid, q in rids:
        d = ctx.wait(rid, np.empty(mesh.nv))
        if q % 2 == 0:
            assert np.array_equal(d, solo[q])
        else:
            ref = np.empty(mesh.nv)
            M.solve(sets[q], ref, plain)
            assert np.array_equal(d, ref)
    M.close()


def test_too_many_sources_rejected(gh, ctx):
    mesh = meshgen.noisy_icosphere(3, 1)
    M = gh.Mesh(ctx, mesh.V, mesh.F)
    d = np.empty(mesh.nv)
    with pytest.raises(gh.GeoheatError):
        M.solve(np.arange(33, dtype=np.int32), d, gh.params(gs_sweeps=20, path_constraints=True))
    M.solve(np.arange(32, dtype=np.int32), d, gh.params(gs_sweeps=20, path_constraints=True))
    M.close()
