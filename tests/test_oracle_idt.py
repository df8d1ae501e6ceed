"""Oracle intrinsic Delaunay triangulation and the edge form on it (Sec. 5.3),
pinned against what geometry fixes: on a planar mesh the iDT is the Delaunay
triangulation of the points (scipy), its lengths are the Euclidean ones, its
geometry from lengths is the geometry from positions, and the intrinsic solve
is the ordinary solve on that triangulation; on a curved mesh every edge ends
Delaunay, the surface area is kept, and a second pass flips nothing."""
import numpy as np
import pytest
from scipy.spatial import Delaunay

import meshgen
import oracle
from oracle import idt


@pytest.fixture(scope="module")
def planar():
    m = meshgen.jittered_grid(17, 5)
    V = m.V.copy()
    V[:, 0] *= 3.0          # stretched: many diagonals are not Delaunay
    Fi, L, flips = idt.intrinsic_delaunay(V, m.F)
    return m, V, Fi, L, flips


def _lengths(V, F):
    return np.array([[np.linalg.norm(V[b] - V[c]), np.linalg.norm(V[c] - V[a]), np.linalg.norm(V[a] - V[b])]
                     for a, b, c in F])


def test_planar_idt_is_the_delaunay_triangulation(planar):
    m, V, Fi, L, flips = planar
    assert flips > 50
    tri = Delaunay(V[:, :2])
    assert set(tuple(sorted(t)) for t in Fi.tolist()) == set(tuple(sorted(t)) for t in tri.simplices.tolist())
    assert np.allclose(L, _lengths(V, Fi), rtol=1e-13, atol=0)


def test_geometry_from_lengths_equals_geometry_from_positions(planar):
    m, V, Fi, L, _ = planar
    mi = idt.mesh_data_intrinsic(Fi, L, len(V))
    me = oracle.mesh_data(V, Fi)
    for name in ("Af", "Av", "theta", "cot"):
        a, b = getattr(mi, name), getattr(me, name)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), name
    assert mi.hbar == pytest.approx(me.hbar, rel=1e-14)
    assert np.array_equal(mi.edges, me.edges) and np.array_equal(mi.col, me.col)


def test_intrinsic_solve_is_the_solve_on_the_triangulation(planar):
    """normalisation and targets in each face's own frame give what the
    positions give: h turns with the frame, h . e does not"""
    m, V, Fi, L, _ = planar
    mi = idt.mesh_data_intrinsic(Fi, L, len(V))
    me = oracle.mesh_data(V, Fi)
    src = [40, 200]
    ri = idt.solve_intrinsic(mi, src, sweeps=150)
    re = oracle.solve(me, src, "edge", sweeps=150)
    assert np.abs(ri["z"] - re["z"]).max() <= 1e-12 * np.abs(re["z"]).max()
    assert np.abs(ri["x"] - re["x"]).max() <= 1e-12 * np.abs(re["x"]).max()
    fin = np.isfinite(re["d"])
    assert np.abs(ri["d"][fin] - re["d"][fin]).max() <= 1e-12 * np.abs(re["d"][fin]).max()
    assert np.allclose(np.linalg.norm(ri["h"], axis=1), np.linalg.norm(re["h"], axis=1), atol=1e-12)


def test_curved_mesh_ends_delaunay_area_kept_second_pass_idle():
    m = meshgen.noisy_icosphere(3, 2)
    m.V[:, 0] *= 3.0        # an ellipsoid: stretched triangles, many edges not Delaunay
    Fi, L, flips = idt.intrinsic_delaunay(m.V, m.F)
    assert flips > 0
    mi = idt.mesh_data_intrinsic(Fi, L, m.nv)
    me = oracle.mesh_data(m.V, m.F)
    assert mi.Af.sum() == pytest.approx(me.Af.sum(), rel=1e-12)
    assert mi.nv - mi.ne + mi.nf == me.nv - me.ne + me.nf
    interior = mi.edge_face[:, 1] >= 0
    ef, es = mi.edge_face[interior], mi.edge_slot[interior]
    s = mi.cot[ef[:, 0], es[:, 0]] + mi.cot[ef[:, 1], es[:, 1]]
    assert s.min() >= -idt.IDT_TOL
    F2, L2, flips2 = idt.intrinsic_delaunay(None, Fi, L)
    assert flips2 == 0 and np.array_equal(F2, Fi)


def test_intrinsic_face_form_is_the_face_form_on_the_triangulation(planar):
    """on a planar mesh the frames only rotate g: the face-form distances of
    the intrinsic formulation are those of the ordinary one"""
    m, V, Fi, L, _ = planar
    mi = idt.mesh_data_intrinsic(Fi, L, len(V))
    me = oracle.mesh_data(V, Fi)
    src = [40, 200]
    ri = idt.solve_intrinsic(mi, src, sweeps=150, form="face")
    re = oracle.solve(me, src, "face", sweeps=150)
    fin = np.isfinite(re["d"])
    assert np.abs(ri["d"][fin] - re["d"][fin]).max() <= 1e-12 * np.abs(re["d"][fin]).max()
    assert np.allclose(np.linalg.norm(ri["g"], axis=1), np.linalg.norm(re["g"], axis=1), rtol=0, atol=1e-12)
    assert np.allclose(ri["res"], re["res"], rtol=1e-10, atol=1e-14)


def test_intrinsic_face_form_on_an_ellipsoid_ends_close_to_the_edge_form():
    m = meshgen.noisy_icosphere(3, 2)
    m.V[:, 0] *= 3.0
    Fi, L, _ = idt.intrinsic_delaunay(m.V, m.F)
    mi = idt.mesh_data_intrinsic(Fi, L, m.nv)
    rf = idt.solve_intrinsic(mi, [0], sweeps=200, form="face", admm_iters=200)
    re = idt.solve_intrinsic(mi, [0], sweeps=200, form="edge", admm_iters=200)
    fin = np.isfinite(re["d"]) & (re["d"] > 0)
    assert np.max(np.abs(rf["d"][fin] - re["d"][fin]) / re["d"][fin]) < 0.05
