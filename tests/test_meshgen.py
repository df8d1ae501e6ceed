"""Seeded synthetic inputs: closed-form counts and invariants."""
import numpy as np
import pytest

import meshgen
import oracle


def _edges(F):
    e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    return np.unique(np.sort(e, axis=1), axis=0)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4])
def test_icosphere_counts_and_orientation(n):
    m = meshgen.icosphere(n)
    N = 1 << n
    E = _edges(m.F)
    assert m.nv == 10 * N * N + 2
    assert m.nf == 20 * N * N
    assert len(E) == 30 * N * N
    assert m.nv - len(E) + m.nf == 2                      # Euler characteristic of a sphere
    assert np.allclose(np.linalg.norm(m.V, axis=1), 1.0, atol=1e-15)
    nrm = np.cross(m.V[m.F[:, 1]] - m.V[m.F[:, 0]], m.V[m.F[:, 2]] - m.V[m.F[:, 0]])
    assert (np.einsum("ij,ij->i", nrm, m.V[m.F].mean(1)) > 0).all()   # outward, counter-clockwise
    # every directed halfedge appears once: consistently oriented closed manifold
    he = np.concatenate([m.F[:, [0, 1]], m.F[:, [1, 2]], m.F[:, [2, 0]]])
    assert len(np.unique(he, axis=0)) == 3 * m.nf


@pytest.mark.parametrize("N", [2, 3, 8, 33])
def test_grid_counts(N):
    m = meshgen.jittered_grid(N, 1)
    assert m.nv == N * N and m.nf == 2 * (N - 1) ** 2
    E = _edges(m.F)
    assert len(E) == 3 * N * N - 4 * N + 1
    assert m.nv - len(E) + m.nf == 1                      # a disk
    nrm = np.cross(m.V[m.F[:, 1]] - m.V[m.F[:, 0]], m.V[m.F[:, 2]] - m.V[m.F[:, 0]])
    assert (nrm[:, 2] > 0).all()
    h = 1.0 / (N - 1)
    reg = meshgen.jittered_grid(N, None)
    d = m.V - reg.V
    assert np.abs(d).max() <= 0.2 * h + 1e-15
    border = (reg.V[:, 0] == 0) | (reg.V[:, 0] == 1) | (reg.V[:, 1] == 0) | (reg.V[:, 1] == 1)
    assert np.all(d[border] == 0)


def test_seeded_determinism():
    a = meshgen.noisy_icosphere(3, 11)
    b = meshgen.noisy_icosphere(3, 11)
    c = meshgen.noisy_icosphere(3, 12)
    assert np.array_equal(a.V, b.V) and not np.array_equal(a.V, c.V)
    r = np.linalg.norm(a.V, axis=1)
    assert 0.9 < r.min() and r.max() < 1.1


def test_box_muller_moments():
    z = meshgen.normal(meshgen.rng_for(5), 200001)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_sources():
    rng = meshgen.rng_for(3)
    for _ in range(50):
        s = meshgen.random_sources(rng, 100, 1, 8)
        assert 1 <= len(s) <= 8 and np.all(np.diff(s) > 0) and s.min() >= 0 and s.max() < 100


def test_workload_c1_shape():
    w = meshgen.workload_c1()
    assert w.mesh.nv == 2562 and w.mesh.nf == 5120 and list(w.sources[0]) == [0]


def test_torus_is_closed_oriented_genus_one():
    m = meshgen.torus(16, 10, seed=2)
    md = oracle.mesh_data(m.V, m.F)          # rejects inconsistent orientation
    assert md.nv == 160 and md.nf == 320 and md.ne == 480
    assert (md.edge_face[:, 1] >= 0).all()
    assert md.nv - md.ne + md.nf == 0
    # outward normals: the face normal points away from the core circle
    p = md.P[m.F].mean(1)
    n = np.cross(md.P[m.F[:, 1]] - md.P[m.F[:, 0]], md.P[m.F[:, 2]] - md.P[m.F[:, 0]])
    core = p.copy()
    core[:, 2] = 0
    core *= (1.0 / np.linalg.norm(core, axis=1))[:, None]
    assert np.all(np.einsum("ij,ij->i", n, p - core) > 0)


def test_jittered_delaunay_is_an_oriented_disk_with_varied_degrees():
    m = meshgen.jittered_delaunay(60, 5)
    md = oracle.mesh_data(m.V, m.F)          # rejects inconsistent orientation
    assert md.nv - md.ne + md.nf == 1        # a disk
    P = m.V[m.F]
    area = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])[:, 2]
    assert np.all(area > 0) and 0.5 * area.sum() == pytest.approx(1.0, rel=1e-12)   # tiles the square
    deg = np.diff(md.rowptr)
    assert deg.min() <= 3 and deg.max() >= 9
    assert np.array_equal(m.F, meshgen.jittered_delaunay(60, 5).F)   # seeded


def test_mixed_density_strip_rows():
    m = meshgen.mixed_density_strip(40, 5)
    md = oracle.mesh_data(m.V, m.F)          # rejects inconsistent orientation
    assert md.nv == 40 * 3 + 118 * 2 and md.nv - md.ne + md.nf == 1
    P = m.V[m.F]
    area = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])[:, 2]
    assert np.all(area > 0) and 0.5 * area.sum() == pytest.approx(39.0 * 4, rel=1e-12)
    deg = np.diff(md.rowptr)
    assert np.all(deg[40 + 118 + 1:2 * 40 + 118 - 1] == 10)   # the interior of the middle sparse row
