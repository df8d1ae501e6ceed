"""Oracle connectivity and geometry (Sec. 3, Sec. 3.1, Sec. 4.1) against
closed forms, the paper's Fig. 5 example and invariants."""
import json
import math
import os

import numpy as np
import pytest

import meshgen
import oracle


def test_fig5_signs(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "fig5_edge_signs.json")))
    F = np.array(g["faces"], np.int32)
    V = np.array([[0, 0, 0], [1, 0, 0], [0.5, 0.8, 0], [0.5, -0.8, 0]], float)
    md0 = oracle.mesh_data(V, F)
    name_of = {}
    for name, (a, b) in g["edge_vertices"].items():
        e = [i for i, (x, y) in enumerate(md0.edges) if {x, y} == {a, b}]
        name_of[e[0]] = name
    flip = np.zeros(md0.ne, np.uint8)
    for e, name in name_of.items():
        if name in g["flipped"]:
            flip[e] = 1
    md = oracle.mesh_data(V, F, flip)
    for cond in g["conditions"]:
        f = cond["face"]
        got = {name_of[int(md.face_edge[f, k])]: int(md.face_sign[f, k]) for k in range(3)}
        assert got == cond["signs"]


def test_icosahedron_closed_form():
    V, F = meshgen.icosahedron()
    md = oracle.mesh_data(V, F)
    a = 1.0 / math.sin(2 * math.pi / 5)          # edge of the unit-circumradius icosahedron
    Af = math.sqrt(3) / 4 * a * a
    assert np.allclose(md.Af, Af, rtol=1e-14)
    assert np.allclose(md.theta, 1 / math.sqrt(3), rtol=1e-14)   # 1/2 (cot 60 + cot 60)
    assert np.allclose(md.Av, 5 * Af / 3, rtol=1e-14)
    assert math.isclose(md.hbar, a, rel_tol=1e-14)


def test_regular_grid_closed_form():
    N = 9
    h = 1.0 / (N - 1)
    m = meshgen.jittered_grid(N, None)
    md = oracle.mesh_data(m.V, m.F)
    deg = np.diff(md.rowptr)
    ev = m.V[md.edges[:, 1]] - m.V[md.edges[:, 0]]
    axis = (np.abs(ev[:, 0]) < 1e-12) | (np.abs(ev[:, 1]) < 1e-12)
    boundary = md.edge_face[:, 1] < 0
    # right isosceles triangles: cot 45 = 1 opposite a leg, cot 90 = 0 opposite the hypotenuse
    assert np.allclose(md.theta[axis & ~boundary], 1.0, atol=1e-14)
    assert np.allclose(md.theta[axis & boundary], 0.5, atol=1e-14)
    assert np.allclose(md.theta[~axis], 0.0, atol=1e-14)
    interior = np.array([0 < m.V[v, 0] < 1 and 0 < m.V[v, 1] < 1 for v in range(m.nv)])
    assert set(deg[interior]) == {4, 8}
    assert np.allclose(md.Av[interior & (deg == 8)], 8 * (h * h / 2) / 3, rtol=1e-13)
    assert np.allclose(md.Av[interior & (deg == 4)], 4 * (h * h / 2) / 3, rtol=1e-13)
    assert math.isclose(md.hbar, (2 * N * (N - 1) * h + (N - 1) ** 2 * h * math.sqrt(2)) / (3 * N * N - 4 * N + 1),
                        rel_tol=1e-13)


def test_linear_precision_planar():
    """sum_w theta_vw (p_w - p_v) = 0 at interior vertices of a planar mesh."""
    m = meshgen.jittered_grid(17, 3)
    md = oracle.mesh_data(m.V, m.F)
    interior = (m.V[:, 0] > 0) & (m.V[:, 0] < 1) & (m.V[:, 1] > 0) & (m.V[:, 1] < 1)
    for v in np.nonzero(interior)[0]:
        r = slice(md.rowptr[v], md.rowptr[v + 1])
        s = (md.theta[md.col_edge[r]][:, None] * (m.V[md.col[r]] - m.V[v])).sum(0)
        assert np.abs(s).max() < 1e-13


def test_quadratic_reproduction_planar():
    """For f = x^2 + y^2 (Laplacian 4) the cotangent Laplacian gives
    sum_w theta_vw (f_w - f_v) = sum over the one-ring faces of
    (their area contribution), i.e. 4 A_v on a regular equilateral patch:
    pins the 1/2 in theta against the 1/3 in A_v."""
    h = 0.1
    ring = [(h * math.cos(k * math.pi / 3), h * math.sin(k * math.pi / 3), 0.0) for k in range(6)]
    V = np.array([(0.0, 0.0, 0.0)] + ring)
    F = np.array([(0, 1 + k, 1 + (k + 1) % 6) for k in range(6)], np.int32)
    md = oracle.mesh_data(V, F)
    f = V[:, 0] ** 2 + V[:, 1] ** 2
    r = slice(md.rowptr[0], md.rowptr[1])
    lap = np.sum(md.theta[md.col_edge[r]] * (f[md.col[r]] - f[0]))
    assert math.isclose(md.Av[0], math.sqrt(3) / 2 * h * h, rel_tol=1e-14)
    assert math.isclose(lap, 4 * md.Av[0], rel_tol=1e-13)


def test_sphere_areas_and_symmetry():
    m = meshgen.noisy_icosphere(3, 5)
    md = oracle.mesh_data(m.V, m.F)
    assert math.isclose(md.Av.sum(), md.Af.sum(), rel_tol=1e-13)
    # CSR is symmetric and rows ascending
    for v in range(md.nv):
        row = md.col[md.rowptr[v]:md.rowptr[v + 1]]
        assert np.all(np.diff(row) > 0)
        for w in row:
            rw = md.col[md.rowptr[w]:md.rowptr[w + 1]]
            assert v in rw
    # each edge of a closed mesh has two faces with opposite signs
    assert (md.edge_face >= 0).all()
    s0 = md.face_sign[md.edge_face[:, 0], md.edge_slot[:, 0]]
    s1 = md.face_sign[md.edge_face[:, 1], md.edge_slot[:, 1]]
    assert np.all(s0 == -s1)
    # local edge k is opposite corner k
    for f in range(0, md.nf, 37):
        for k in range(3):
            e = md.face_edge[f, k]
            assert m.F[f, k] not in md.edges[e]


def test_nonmanifold_rejected():
    V = np.zeros((5, 3))
    V[:, 0] = [0, 1, 0, 0, 1]
    V[:, 1] = [0, 0, 1, -1, 1]
    F = np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4]], np.int32)     # edge {0,1} in three faces
    with pytest.raises(oracle.OracleError):
        oracle.mesh_data(V, F)
    F2 = np.array([[0, 1, 2], [0, 1, 3]], np.int32)               # same direction twice
    with pytest.raises(oracle.OracleError):
        oracle.mesh_data(V, F2)
    with pytest.raises(oracle.OracleError):
        oracle.mesh_data(V, np.array([[0, 1, 7]], np.int32))


def test_diffusion_time_and_parameters(golden_dir):
    p = json.load(open(os.path.join(golden_dir, "paper_parameters.json")))
    assert oracle.MU == p["mu"] and oracle.ADMM_ITERS == p["admm_iters"]
    m = meshgen.icosphere(4)
    md = oracle.mesh_data(m.V, m.F)
    assert math.isclose(oracle.diffusion_time(md, 1.0), md.hbar ** 2)
    assert math.isclose(oracle.diffusion_time(md, 10.0), 10 * md.hbar ** 2)
