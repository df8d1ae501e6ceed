"""The level-parallel oracle (the same C source built with OpenMP) is
bit-identical to the single-threaded one.

Every parallel loop of the oracle updates locations no other iteration of
the loop reads: the vertices of one breadth-first set in a sweep are a
Jacobi step (eq. HeatDiffusionUpdate: a set's new values come from the
state before the set), the faces and edges of one ADMM block update are
independent (Sec. 3.2, Sec. 4.1), and the vertices of one set in the
integration read only the previous set's distances (eq. IntegrationStep).
Sums whose value depends on their order (vertex areas, the mean edge length,
the residual norms) stay sequential.  So the two builds must agree bit for
bit, on meshes whose sets are wide enough to be split among threads."""
import numpy as np
import pytest

import meshgen
import oracle


def _both(fn):
    with oracle.parallel(False):
        a = fn()
    with oracle.parallel(True):
        b = fn()
    return a, b


def _same(a, b, what):
    a, b = np.asarray(a), np.asarray(b)
    assert a.dtype == b.dtype and a.shape == b.shape, what
    assert np.array_equal(a.view(np.uint8), b.view(np.uint8)), what


def test_parallel_build_uses_threads():
    with oracle.parallel(False):
        assert oracle.threads() == 1
    with oracle.parallel(True):
        n = oracle.threads()
    import os
    if (os.cpu_count() or 1) > 1 and "OMP_NUM_THREADS" not in os.environ:
        assert n > 1


def _mesh_fields(md):
    return [md.edges, md.face_edge, md.face_sign, md.edge_face, md.edge_slot, md.rowptr, md.col, md.col_edge,
            md.Af, md.Av, md.cot, md.theta, np.array([md.hbar])]


@pytest.mark.parametrize("case", ["noisy_ico6", "strip", "grid"])
def test_parallel_solve_is_bit_identical(case):
    if case == "noisy_ico6":
        mesh, src, sweeps = meshgen.noisy_icosphere(6, 11), [5, 1700, 30001], 40
    elif case == "strip":
        mesh, src, sweeps = meshgen.strip_grid(3000, 6), [0, 700, 1400, 2100, 2999], 30
    else:
        mesh, src, sweeps = meshgen.jittered_grid(257, 3), [257 * 128 + 128], 60
    mda, mdb = _both(lambda: oracle.mesh_data(mesh.V, mesh.F))
    for x, y in zip(_mesh_fields(mda), _mesh_fields(mdb)):
        _same(x, y, "mesh data")
    for form in ("face", "edge"):
        with oracle.parallel(False):
            ra = oracle.solve(mda, src, form, sweeps=sweeps, eps=(1e-9, 1e-9), path_constraints_on=True)
        with oracle.parallel(True):
            rb = oracle.solve(mdb, src, form, sweeps=sweeps, eps=(1e-9, 1e-9), path_constraints_on=True)
        for f in ("level", "parent", "order", "level_off"):
            _same(getattr(ra["bfs"], f), getattr(rb["bfs"], f), f)
        _same(ra["u"][0], rb["u"][0], "u mantissa")
        _same(ra["u"][1], rb["u"][1], "u exponent")
        _same(ra["h"], rb["h"], "h")
        _same(ra["res"], rb["res"], "residuals")
        _same(ra["g" if form == "face" else "x"], rb["g" if form == "face" else "x"], "g or x")
        _same(ra["d"], rb["d"], "d")


def test_parallel_stopped_diffusion_is_bit_identical():
    mesh = meshgen.jittered_grid(129, 5)
    src = [64 * 129 + 3]
    mda, mdb = _both(lambda: oracle.mesh_data(mesh.V, mesh.F))
    with oracle.parallel(False):
        ra = oracle.solve(mda, src, "edge", sweeps=400, gs_tol=1e-6, gs_check=10)
    with oracle.parallel(True):
        rb = oracle.solve(mdb, src, "edge", sweeps=400, gs_tol=1e-6, gs_check=10)
    assert ra["gs_sweeps"] == rb["gs_sweeps"]
    _same(ra["d"], rb["d"], "d")


def test_parallel_build_rejects_bad_meshes():
    mesh = meshgen.jittered_grid(9, 1)
    bad = mesh.F.copy()
    bad[3, 1] = mesh.nv + 5
    for on in (False, True):
        with oracle.parallel(on):
            with pytest.raises(oracle.OracleError):
                oracle.mesh_data(mesh.V, bad)
            # two faces through one edge in the same direction: not oriented
            F2 = np.vstack([mesh.F, mesh.F[:1]])
            with pytest.raises(oracle.OracleError):
                oracle.mesh_data(mesh.V, F2)
