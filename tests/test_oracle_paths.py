"""Oracle multi-source path constraints (Sec. 5.2, eq. MultiSourceConstraint,
eq. MultiSourceConstraintEdgeBased), pinned against what the paper and the
mathematics fix: the paths against brute-force hop distances, the projected
ADMM block against a dense KKT solve of the constrained subproblem built here
from the paths, the constraints themselves, and the special cases."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg
import scipy.sparse.linalg as sla

import meshgen
import oracle


def _grid(N=17, seed=7):
    m = meshgen.jittered_grid(N, seed)
    return m, oracle.mesh_data(m.V, m.F)


def _edge_table(F):
    """edge (a, b), a < b -> sorted list of adjacent faces, from the face list"""
    t = {}
    for f, tri in enumerate(np.asarray(F)):
        for k in range(3):
            a, b = int(tri[(k + 1) % 3]), int(tri[(k + 2) % 3])
            t.setdefault((min(a, b), max(a, b)), []).append(f)
    return t


def test_source_paths_are_fewest_edge_paths():
    m, md = _grid(17)
    src = [200, 3, 150, 288]
    paths = oracle.source_paths(md, src)
    s = sorted(src)
    et = _edge_table(m.F)
    nv = md.nv
    rows = [a for (a, b) in et] + [b for (a, b) in et]
    cols = [b for (a, b) in et] + [a for (a, b) in et]
    A = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(nv, nv))
    hops = csg.shortest_path(A, unweighted=True, indices=[s[0]])[0]
    assert len(paths) == len(s) - 1
    for sj, steps in zip(s[1:], paths):
        assert len(steps) == hops[sj]
        assert steps[0][0] == s[0] and steps[-1][1] == sj
        for (p, v), (p2, _) in zip(steps, steps[1:]):
            assert v == p2
        for p, v in steps:
            assert (min(p, v), max(p, v)) in et


def test_source_paths_unreachable_source_gets_empty_path():
    a = meshgen.jittered_grid(5, 1)
    V = np.vstack([a.V, a.V + [10.0, 0.0, 0.0]])
    F = np.vstack([a.F, a.F + a.V.shape[0]])
    md = oracle.mesh_data(V, F)
    paths = oracle.source_paths(md, [0, 7, a.V.shape[0] + 3])
    assert len(paths[0]) > 0 and paths[1] == []


def test_single_source_has_no_constraints():
    _, md = _grid(13)
    for form in ("edge", "face"):
        a = oracle.solve(md, [40], form, sweeps=60)
        b = oracle.solve(md, [40], form, sweeps=60, path_constraints_on=True)
        assert np.array_equal(a["d"], b["d"])


def _constraint_values(pc, var, form):
    out = []
    for j in range(len(pc.off) - 1):
        a, b = pc.off[j], pc.off[j + 1]
        if form == "edge":
            out.append(np.sum(pc.coef[a:b, 0] * var[pc.var[a:b]]))
        else:
            out.append(np.sum(np.einsum("ij,ij->i", pc.coef[a:b], var[pc.var[a:b]])))
    return np.asarray(out)


@pytest.mark.parametrize("form", ["edge", "face"])
def test_constraints_hold_after_every_iteration_count(form):
    _, md = _grid(17)
    src = [20, 160, 250]
    r = oracle.solve(md, src, form, sweeps=100)
    pc = oracle.path_constraints(md, src, form)
    for iters in (1, 3, 10):
        if form == "edge":
            v = oracle.edge_admm(md, r["h"], iters, pc=pc)[0]
            scale = np.abs(v).max()
        else:
            v = oracle.face_admm(md, r["h"], iters, pc=pc)[0]
            scale = np.abs(v).max() * np.abs(pc.coef).max()
        assert np.abs(_constraint_values(pc, v, form)).max() <= 1e-13 * scale * len(pc.var)


def _S_from_paths(md, m, paths, form):
    """constraint matrix built from the path steps and the face list alone"""
    et = _edge_table(m.F)
    edge_id = {tuple(e): i for i, e in enumerate(md.edges.tolist())}
    nvar = md.ne if form == "edge" else 3 * md.nf
    S = np.zeros((len(paths), nvar))
    for j, steps in enumerate(paths):
        for p, v in steps:
            a, b = min(p, v), max(p, v)
            if form == "edge":
                # x_e is the difference head - tail of the (min, max) halfedge
                S[j, edge_id[(a, b)]] += 1.0 if p == a else -1.0
            else:
                f = min(et[(a, b)])
                S[j, 3 * f:3 * f + 3] += md.P[v] - md.P[p]
    return S


@pytest.mark.parametrize("form", ["edge", "face"])
def test_projection_is_the_constrained_minimiser(form):
    """One ADMM iteration with the constraints equals the minimiser of that
    iteration's X (or G) subproblem under them: a quadratic with Hessian
    D_e = |H_e| (1 + mu) (edge) or A_f (2 + mu n_f) (face) around the
    unconstrained update, solved here as a dense KKT system."""
    m, md = _grid(17)
    src = [1, 12, 30, 170, 260, 100]   # 1 and 12 on the boundary row: paths along boundary edges too
    r = oracle.solve(md, src, form, sweeps=100)
    pc = oracle.path_constraints(md, src, form)
    S = _S_from_paths(md, m, pc.paths, form)
    if form == "edge":
        on_path = np.abs(S).sum(0) > 0
        nface = (md.edge_face >= 0).sum(1)
        assert set(nface[on_path]) == {1, 2}       # the weights D_e differ along the paths
    mu = oracle.MU
    if form == "edge":
        vh = oracle.edge_admm(md, r["h"], 1)[0]
        vc = oracle.edge_admm(md, r["h"], 1, pc=pc)[0]
        Dv = (md.edge_face >= 0).sum(1) * (1.0 + mu)
    else:
        vh = oracle.face_admm(md, r["h"], 1)[0].ravel()
        vc = oracle.face_admm(md, r["h"], 1, pc=pc)[0].ravel()
        interior = (md.edge_face[md.face_edge, 1] >= 0).sum(1)
        Dv = np.repeat(md.Af * (2.0 + mu * interior), 3)
    k = S.shape[0]
    K = sp.bmat([[sp.diags(Dv), sp.csr_matrix(S.T)], [sp.csr_matrix(S), None]]).tocsc()
    sol = sla.spsolve(K, np.concatenate([Dv * vh, np.zeros(k)]))[:len(vh)]
    assert np.abs(vc - vh).max() > 1e-6            # the constraints do act
    assert np.abs(vc - sol).max() <= 1e-12 * max(1.0, np.abs(vh).max())


@pytest.mark.parametrize("form", ["edge", "face"])
def test_dependent_constraint_is_dropped(form):
    """A repeated constraint has a zero pivot and is dropped: the result is
    the one of the constraint alone."""
    _, md = _grid(13)
    src = [10, 120]
    r = oracle.solve(md, src, form, sweeps=60)
    pc = oracle.path_constraints(md, src, form)
    n = pc.off[1]
    twice = oracle.PathConstraints(np.array([0, n, 2 * n], np.int32), np.concatenate([pc.var, pc.var]),
                                   np.concatenate([pc.coef, pc.coef]), pc.paths * 2)
    f = oracle.edge_admm if form == "edge" else oracle.face_admm
    a = f(md, r["h"], 5, pc=pc)[0]
    b = f(md, r["h"], 5, pc=twice)[0]
    assert np.allclose(a, b, rtol=0, atol=1e-14 * np.abs(a).max())


def test_edge_constraints_follow_the_orientation_choice():
    """Flipping orientation halfedges negates their x and the constraint
    signs with them: the distances do not change (Sec. 4.1)."""
    m = meshgen.noisy_icosphere(3, 2)
    md = oracle.mesh_data(m.V, m.F)
    flip = (meshgen.rng_for(9).random(md.ne) < 0.5).astype(np.uint8)
    mdf = oracle.mesh_data(m.V, m.F, flip)
    src = [5, 300, 600]
    o = oracle.solve(md, src, "edge", sweeps=60, path_constraints_on=True)
    of = oracle.solve(mdf, src, "edge", sweeps=60, path_constraints_on=True)
    sgn = np.where(flip == 1, -1.0, 1.0)
    assert np.allclose(of["x"], sgn * o["x"], rtol=0, atol=1e-14)
    assert np.allclose(of["d"], o["d"], rtol=0, atol=1e-13)
