"""Oracle breadth-first sets and pairing (eq. VertexSets, Sec. 3.3, Sec. 5.2)
against brute force and a naive queue."""
from collections import deque

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

import meshgen
import oracle


def _naive_fifo(md, sources):
    """Textbook FIFO traversal written independently of the oracle."""
    nbrs = [sorted(set(md.col[md.rowptr[v]:md.rowptr[v + 1]].tolist())) for v in range(md.nv)]
    level = [-1] * md.nv
    parent = [-1] * md.nv
    q = deque()
    order = []
    for s in sorted(set(int(s) for s in sources)):
        level[s] = 0
        q.append(s)
    while q:
        v = q.popleft()
        order.append(v)
        for w in nbrs[v]:
            if level[w] < 0:
                level[w] = level[v] + 1
                parent[w] = v
                q.append(w)
    return np.array(level), np.array(parent), np.array(order)


@pytest.mark.parametrize("mesh,sources", [
    (meshgen.jittered_grid(23, 1), [0]),
    (meshgen.jittered_grid(23, 1), [250, 17, 250, 400]),
    (meshgen.noisy_icosphere(3, 2), [5]),
    (meshgen.noisy_icosphere(3, 2), [641, 0, 300]),
])
def test_bfs_matches_brute_force_and_fifo(mesh, sources):
    md = oracle.mesh_data(mesh.V, mesh.F)
    b = oracle.bfs(md, sources)
    rows = np.repeat(np.arange(md.nv), np.diff(md.rowptr))
    G = sp.csr_matrix((np.ones(len(md.col)), (rows, md.col)), shape=(md.nv, md.nv))
    hop = shortest_path(G, unweighted=True, indices=sorted(set(sources))).min(axis=0)
    assert np.array_equal(b.level, hop.astype(np.int32))
    lv, par, order = _naive_fifo(md, sources)
    assert np.array_equal(b.level, lv) and np.array_equal(b.parent, par) and np.array_equal(b.order, order)
    # level sets are contiguous in the order and D_0 is the sorted source set
    assert np.array_equal(b.order[b.level_off[0]:b.level_off[1]], np.unique(sources))
    for i in range(b.nlev):
        assert np.all(b.level[b.order[b.level_off[i]:b.level_off[i + 1]]] == i)
    # the pairing vertex is adjacent and one set closer
    for v in range(md.nv):
        if b.level[v] > 0:
            p = b.parent[v]
            assert b.level[p] == b.level[v] - 1
            assert v in md.col[md.rowptr[p]:md.rowptr[p + 1]]


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_icosphere_depth(n):
    """From an icosahedron vertex the deepest set of an n-times subdivided
    icosphere is 3 * 2^n edges away (the antipodal vertex)."""
    m = meshgen.icosphere(n)
    md = oracle.mesh_data(m.V, m.F)
    b = oracle.bfs(md, [0])
    assert b.nlev == 3 * (1 << n) + 1
    assert list(b.order[b.level_off[-2]:b.level_off[-1]]) == [int(np.argmin(m.V @ m.V[0]))]


def test_unreachable_and_errors():
    g = meshgen.jittered_grid(5, None)
    V = np.concatenate([g.V, g.V + [2.0, 0, 0]])
    F = np.concatenate([g.F, g.F + g.nv]).astype(np.int32)
    md = oracle.mesh_data(V, F)
    b = oracle.bfs(md, [3])
    assert np.all(b.level[g.nv:] == -1) and np.all(b.level[:g.nv] >= 0)
    assert len(b.order) == g.nv
    with pytest.raises(oracle.OracleError):
        oracle.bfs(md, [])
    with pytest.raises(oracle.OracleError):
        oracle.bfs(md, [md.nv])
    with pytest.raises(oracle.OracleError):
        oracle.bfs(md, [-1])
