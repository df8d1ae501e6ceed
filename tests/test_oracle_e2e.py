"""Algorithm 1 end to end in the oracle against closed-form and graph
distances (accuracy bands, not parity)."""
import heapq

import numpy as np
import pytest

import meshgen
import oracle


def _eps(d, ref, sources):
    mask = np.ones(len(d), bool)
    mask[np.asarray(sources)] = False
    return np.mean(np.abs(d[mask] - ref[mask]) / np.abs(ref[mask]))


def _dijkstra(md, sources):
    dist = np.full(md.nv, np.inf)
    pq = []
    for s in sources:
        dist[s] = 0.0
        pq.append((0.0, int(s)))
    heapq.heapify(pq)
    while pq:
        dv, v = heapq.heappop(pq)
        if dv > dist[v]:
            continue
        for w in md.col[md.rowptr[v]:md.rowptr[v + 1]]:
            nd = dv + np.linalg.norm(md.P[w] - md.P[v])
            if nd < dist[w]:
                dist[w] = nd
                heapq.heappush(pq, (nd, int(w)))
    return dist


@pytest.mark.parametrize("form", ["face", "edge"])
def test_icosphere_level4_vs_great_circle(form):
    """Unit icosphere, source vertex 0, t = hbar^2, 200 sweeps, 10 ADMM
    iterations: the paper reports mean relative errors of 0.3-1.5 percent
    on its models (Table 1); here the reference is R arccos(p.p0)."""
    w = meshgen.workload_c1()
    md = oracle.mesh_data(w.mesh.V, w.mesh.F)
    o = oracle.solve(md, [0], form, sweeps=200)
    p = w.mesh.V / np.linalg.norm(w.mesh.V, axis=1, keepdims=True)
    ref = np.arccos(np.clip(p @ p[0], -1, 1))
    assert _eps(o["d"], ref, [0]) < 0.015
    assert np.abs(o["d"] - ref).max() < 0.05


@pytest.mark.parametrize("form", ["face", "edge"])
def test_flat_grid_vs_euclidean(form):
    m = meshgen.jittered_grid(65, 12)
    md = oracle.mesh_data(m.V, m.F)
    src = [2000]
    b = oracle.bfs(md, src)
    o = oracle.solve(md, src, form, sweeps=4 * b.nlev)
    ref = np.linalg.norm(m.V - m.V[src[0]], axis=1)
    assert _eps(o["d"], ref, src) < 0.03


@pytest.mark.parametrize("form", ["face", "edge"])
def test_graph_distance_bounds_multi_source(form):
    """chord (1 - delta) - hbar <= d <= Dijkstra on edges (1 + delta) + hbar,
    d = 0 on every source (Sec. 5.2)."""
    m = meshgen.noisy_icosphere(3, 21)
    md = oracle.mesh_data(m.V, m.F)
    src = [4, 321, 600]
    o = oracle.solve(md, src, form, sweeps=200)
    d = o["d"]
    assert np.all(d[src] == 0)
    dj = _dijkstra(md, src)
    chord = np.min(np.linalg.norm(m.V[:, None, :] - m.V[src][None, :, :], axis=2), axis=1)
    delta = 0.05
    assert np.all(d <= dj * (1 + delta) + md.hbar)
    assert np.all(d >= chord * (1 - delta) - md.hbar)
