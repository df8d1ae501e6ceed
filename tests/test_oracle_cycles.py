"""Oracle cycle constraints of a closed surface of genus g (Sec. 5.1,
eq. TopologyConstraint, eq. EdgeTopologyConstraint), pinned against what
topology fixes: 2g cycles (Euler characteristic), closed simple loops checked
against the face list, the winding of the torus' two angle fields around
them (the cycles generate the homology: the winding matrix is unimodular), the
constraints themselves, and the KKT minimiser with path and cycle
constraints together."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

import meshgen
import oracle


@pytest.fixture(scope="module")
def torus():
    m = meshgen.torus(24, 12, seed=3)
    return m, oracle.mesh_data(m.V, m.F)


def _edge_table(F):
    t = {}
    for f, tri in enumerate(np.asarray(F)):
        for k in range(3):
            a, b = int(tri[(k + 1) % 3]), int(tri[(k + 2) % 3])
            t.setdefault((min(a, b), max(a, b)), []).append(f)
    return t


@pytest.mark.parametrize("form", ["edge", "face"])
def test_cycle_count_is_twice_the_genus(torus, form):
    m, md = torus
    genus = (2 - (md.nv - md.ne + md.nf)) // 2
    assert genus == 1
    assert len(oracle.cycle_constraints(md, form).off) - 1 == 2 * genus
    ico = meshgen.icosphere(3)
    assert len(oracle.cycle_constraints(oracle.mesh_data(ico.V, ico.F), form).off) == 1
    grid = meshgen.jittered_grid(9, 1)   # boundary: none by the reading
    assert len(oracle.cycle_constraints(oracle.mesh_data(grid.V, grid.F), form).off) == 1


def test_edge_cycles_are_closed_simple_loops(torus):
    m, md = torus
    et = _edge_table(m.F)
    cc = oracle.cycle_constraints(md, "edge")
    for steps in cc.paths:
        assert steps[0][0] == steps[-1][1]
        for (p, q), (p2, _) in zip(steps, steps[1:]):
            assert q == p2
        keys = [(min(p, q), max(p, q)) for p, q in steps]
        assert all(k in et for k in keys)
        assert len(set(keys)) == len(keys)
        nodes = [p for p, _ in steps]
        assert len(set(nodes)) == len(nodes)


def test_face_loops_are_closed_dual_loops(torus):
    m, md = torus
    F = np.asarray(m.F)
    cc = oracle.cycle_constraints(md, "face")
    for j, loop in enumerate(cc.paths):
        assert loop[0] == loop[-1]
        assert len(set(loop[:-1])) == len(loop) - 1
        for f, g in zip(loop[:-1], loop[1:]):
            assert len(set(F[f]) & set(F[g])) == 2
        seg = cc.coef[cc.off[j]:cc.off[j + 1]]
        assert np.abs(seg.sum(0)).max() < 1e-14          # the polyline closes
        assert list(cc.var[cc.off[j]:cc.off[j + 1]]) == loop[:-1]


def _angles(V):
    a = np.arctan2(V[:, 1], V[:, 0])
    b = np.arctan2(V[:, 2], np.hypot(V[:, 0], V[:, 1]) - 1.0)
    return a, b


def _wrap(d):
    return (d + np.pi) % (2 * np.pi) - np.pi


@pytest.mark.parametrize("form", ["edge", "face"])
def test_cycles_wind_around_the_torus(torus, form):
    """The two angle fields are locally gradients but not globally: their
    sums around the cycles are 2 pi times integer windings, and the 2 x 2
    winding matrix has determinant +-1."""
    m, md = torus
    cc = oracle.cycle_constraints(md, form)
    W = np.zeros((2, 2))
    for r, ang in enumerate(_angles(md.P)):
        if form == "edge":
            x = _wrap(ang[md.edges[:, 1]] - ang[md.edges[:, 0]])
            vals = [np.sum(cc.coef[cc.off[j]:cc.off[j + 1], 0] * x[cc.var[cc.off[j]:cc.off[j + 1]]])
                    for j in range(2)]
        else:
            # gradient of the angle, unwrapped inside each face, as a linear function on the face
            g = np.zeros((md.nf, 3))
            for f, tri in enumerate(np.asarray(m.F)):
                p = md.P[tri]
                u = ang[tri[0]] + _wrap(ang[tri] - ang[tri[0]])
                e1, e2 = p[1] - p[0], p[2] - p[0]
                G = np.array([e1, e2])
                g[f] = np.linalg.lstsq(G, np.array([u[1] - u[0], u[2] - u[0]]), rcond=None)[0]
            vals = [np.sum(np.einsum("ij,ij->i", cc.coef[cc.off[j]:cc.off[j + 1]], g[cc.var[cc.off[j]:cc.off[j + 1]]]))
                    for j in range(2)]
        W[r] = np.asarray(vals) / (2 * np.pi)
    assert np.allclose(W, np.round(W), atol=1e-9)
    assert abs(round(np.linalg.det(np.round(W)))) == 1


@pytest.mark.parametrize("form", ["edge", "face"])
def test_cycle_constraints_hold_and_are_the_kkt_minimiser(torus, form):
    m, md = torus
    src = [5, 140]
    r = oracle.solve(md, src, form, sweeps=150)
    pc = oracle.join_constraints(oracle.path_constraints(md, src, form), oracle.cycle_constraints(md, form))
    assert len(pc.off) - 1 == 3
    mu = oracle.MU
    dim = 1 if form == "edge" else 3
    nvar = md.ne if form == "edge" else md.nf
    S = np.zeros((len(pc.off) - 1, nvar * dim))
    for j in range(len(pc.off) - 1):
        for i in range(pc.off[j], pc.off[j + 1]):
            S[j, dim * pc.var[i]:dim * pc.var[i] + dim] += pc.coef[i]
    if form == "edge":
        vh = oracle.edge_admm(md, r["h"], 1)[0]
        vc = oracle.edge_admm(md, r["h"], 1, pc=pc)[0]
        v10 = oracle.edge_admm(md, r["h"], 10, pc=pc)[0]
        Dv = (md.edge_face >= 0).sum(1) * (1.0 + mu)
    else:
        vh = oracle.face_admm(md, r["h"], 1)[0].ravel()
        vc = oracle.face_admm(md, r["h"], 1, pc=pc)[0].ravel()
        v10 = oracle.face_admm(md, r["h"], 10, pc=pc)[0].ravel()
        interior = (md.edge_face[md.face_edge, 1] >= 0).sum(1)
        Dv = np.repeat(md.Af * (2.0 + mu * interior), 3)
    K = sp.bmat([[sp.diags(Dv), sp.csr_matrix(S.T)], [sp.csr_matrix(S), None]]).tocsc()
    sol = sla.spsolve(K, np.concatenate([Dv * vh, np.zeros(S.shape[0])]))[:len(vh)]
    assert np.abs(vc - vh).max() > 1e-6
    assert np.abs(vc - sol).max() <= 1e-12 * max(1.0, np.abs(vh).max())
    assert np.abs(S @ v10).max() <= 1e-12 * np.abs(v10).max() * np.abs(S).sum(1).max()


@pytest.mark.parametrize("form", ["edge", "face"])
def test_disconnected_closed_mesh_gets_none(form):
    a = meshgen.torus(12, 8, seed=1)
    V = np.vstack([a.V, a.V + [5.0, 0.0, 0.0]])
    F = np.vstack([a.F, a.F + a.V.shape[0]])
    md = oracle.mesh_data(V, F)
    assert len(oracle.cycle_constraints(md, form).off) == 1
