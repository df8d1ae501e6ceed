"""The diffusion stopped on the heat residual E1 (eq. HeatSolutionError) on
the GPU: rounds of gs_check sweeps continue one iteration (state and
distances bit-identical to an uninterrupted run), the stop lands on the same
check as the FP64 oracle's, each query of a batch stops on its own, and bad
parameters are refused."""
import math

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


@pytest.fixture(scope="module")
def grid():
    m = meshgen.jittered_grid(65, 6)
    return m, oracle.mesh_data(m.V, m.F)


def _d_err(d, dref, sources, hbar):
    mask = np.isfinite(dref)
    mask[np.asarray(sources)] = False
    return np.max(np.abs(d[mask] - dref[mask]) / np.maximum(np.abs(dref[mask]), hbar))


def _log(line):
    import os
    path = os.environ.get("GEOHEAT_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(line + "\n")


@pytest.mark.parametrize("fp64", [False, True])
def test_rounds_continue_one_iteration(gh, ctx, grid, fp64):
    mesh, md = grid
    src = [70, 3000]
    M = gh.Mesh(ctx, mesh.V, mesh.F)
    try:
        a, b = np.empty(md.nv), np.empty(md.nv)
        M.solve(src, a, gh.params(gs_sweeps=300, fp64=fp64))
        ua = (M.dump(gh.GH_DUMP_U_MANT), M.dump(gh.GH_DUMP_U_EXP))
        assert M.dump(gh.GH_DUMP_GS_SWEEPS)[0] == 300
        # never within the tolerance: rounds of 70, 70, 70, 70 and 20 sweeps
        M.solve(src, b, gh.params(gs_sweeps=300, fp64=fp64, gs_tol=1e-300, gs_check=70))
        assert M.dump(gh.GH_DUMP_GS_SWEEPS)[0] == 300
        assert np.array_equal(M.dump(gh.GH_DUMP_U_MANT), ua[0])
        assert np.array_equal(M.dump(gh.GH_DUMP_U_EXP), ua[1])
        assert np.array_equal(a, b)
    finally:
        M.close()


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("form", ["edge", "face"])
def test_stop_matches_oracle(gh, ctx, grid, form, fp64):
    mesh, md = grid
    src = [70, 3000]
    check = 5
    b = oracle.bfs(md, src)
    t = oracle.diffusion_time(md)
    _, _, e1 = oracle.gs_until(md, b, t, 60, 0.0, check)
    # a tolerance half way (geometrically) between the E1 of the third and
    # fourth checks, both far above the FP32 state's own residual
    assert e1[2] > 1.5 * e1[3] and e1[3] > 1e-4
    tol = math.sqrt(e1[2] * e1[3])
    ref = oracle.solve(md, src, form, sweeps=400, gs_tol=tol, gs_check=check)
    assert ref["gs_sweeps"] == 4 * check
    M = gh.Mesh(ctx, mesh.V, mesh.F)
    try:
        d = np.empty(md.nv)
        M.solve(src, d, gh.params(gs_sweeps=400, form=form, fp64=fp64, gs_tol=tol, gs_check=check, diagnostics=True))
        assert M.dump(gh.GH_DUMP_GS_SWEEPS)[0] == 4 * check
        assert M.dump(gh.GH_DUMP_E1)[0] == pytest.approx(e1[3], rel=1e-3 if not fp64 else 1e-9)
        derr = _d_err(d, ref["d"], src, md.hbar)
        _log(f"GS stop on E1 grid65 form={form} fp64={fp64}: {4 * check} sweeps (oracle {ref['gs_sweeps']}), d {derr:.2e}")
        assert derr <= D_TOL[fp64]
    finally:
        M.close()


def test_batch_queries_stop_on_their_own(gh, ctx, grid):
    mesh, md = grid
    sets = [[70], [2100, 2110, 2120], [4224]]   # stop after 24, 27 and 27 sweeps
    prm = gh.params(gs_sweeps=500, gs_tol=4.5e-4, gs_check=3)
    M = gh.Mesh(ctx, mesh.V, mesh.F)
    try:
        out = np.empty((len(sets), md.nv))
        M.solve_batch(sets, out, prm)
        got = [int(M.dump(gh.GH_DUMP_GS_SWEEPS, q)[0]) for q in range(len(sets))]
        for q, s in enumerate(sets):
            one = np.empty(md.nv)
            M.solve(s, one, prm)
            assert M.dump(gh.GH_DUMP_GS_SWEEPS)[0] == got[q]
            assert np.array_equal(one, out[q])
            ref = oracle.solve(md, s, "edge", sweeps=500, gs_tol=4.5e-4, gs_check=3)
            assert got[q] == ref["gs_sweeps"]
        _log(f"GS stop on E1 batch grid65: sweeps per query {got}")
        assert len(set(got)) > 1
    finally:
        M.close()


def test_bad_parameters_are_refused(gh, ctx, grid):
    mesh, md = grid
    M = gh.Mesh(ctx, mesh.V, mesh.F)
    try:
        d = np.empty(md.nv)
        for kw in ({"gs_tol": -1.0}, {"gs_tol": float("nan")}, {"gs_tol": 1e-3, "gs_check": 0}):
            with pytest.raises(gh.GeoheatError):
                M.solve([5], d, gh.params(gs_sweeps=50, **kw))
        M.solve([5], d, gh.params(gs_sweeps=50, gs_check=0))   # gs_check is unused without gs_tol
        assert M.dump(gh.GH_DUMP_GS_SWEEPS)[0] == 50
    finally:
        M.close()
