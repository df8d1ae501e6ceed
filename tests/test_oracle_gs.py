"""Oracle Gauss-Seidel heat diffusion (eq. heat, eq. HeatDiffusionUpdate)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import meshgen
import oracle
import oracle.hm as hm


def _state_to_float(st):
    return np.ldexp(st[0], st[1].clip(-1100, 1100))


def test_icosahedron_symmetry_reduction():
    """The icosahedron's five-fold symmetry about vertex 0 keeps every set
    D_0..D_3 at one common value, so a sweep reduces to four scalars.  In
    D_1 each vertex sees 1 neighbour in D_0, 2 in D_1, 2 in D_2; in D_2, 2 in
    D_1, 2 in D_2, 1 in D_3.  Same-set neighbours carry the previous sweep's
    value (simultaneous update within a set)."""
    V, F = meshgen.icosahedron()
    md = oracle.mesh_data(V, F)
    b = oracle.bfs(md, [0])
    assert list(np.diff(b.level_off)) == [1, 5, 5, 1]
    t = 0.37
    a, th = md.Av[0], md.theta[0]
    D, c = a + 5 * t * th, t * th
    prev = [0.0, 0.0, 0.0, 0.0]
    st = None
    for sweep in range(1, 6):
        st = oracle.gs(md, b, t, 1, st)
        a0 = (1 + 5 * c * prev[1]) / D
        a1 = c * (a0 + 2 * prev[1] + 2 * prev[2]) / D
        a2 = c * (2 * a1 + 2 * prev[2] + prev[3]) / D
        a3 = c * (5 * a2) / D
        prev = [a0, a1, a2, a3]
        u = _state_to_float(st)
        for i in range(4):
            vs = b.order[b.level_off[i]:b.level_off[i + 1]]
            assert np.allclose(u[vs], prev[i], rtol=1e-14, atol=0)


@pytest.mark.parametrize("mesh,src", [(meshgen.icosphere(2), [0]), (meshgen.jittered_grid(15, 2), [37]),
                                      (meshgen.noisy_icosphere(2, 9), [3, 100])])
def test_converges_to_direct_solve(mesh, src):
    md = oracle.mesh_data(mesh.V, mesh.F)
    b = oracle.bfs(md, src)
    t = oracle.diffusion_time(md)
    st = oracle.gs(md, b, t, 20 * b.nlev + 200)
    ustar = hm.heat_direct(md, src, t)
    assert np.allclose(_state_to_float(st), ustar, rtol=1e-11, atol=0)
    assert oracle.heat_residual(md, b, t, st) < 1e-13


def test_extended_exponent_equals_plain():
    """Carrying the binary exponent separately changes no bit while plain
    double arithmetic stays in its normal range."""
    m = meshgen.jittered_grid(21, 5)
    md = oracle.mesh_data(m.V, m.F)
    b = oracle.bfs(md, [200])
    t = oracle.diffusion_time(md, 3.0)
    for sweeps in (1, 2, 7, 40):
        st = oracle.gs(md, b, t, sweeps)
        u = oracle.gs_plain(md, b, t, sweeps)
        assert np.abs(u[u != 0]).min() > 1e-290
        assert np.array_equal(np.ldexp(st[0], st[1]), u)


def test_sweep_split_is_bit_identical():
    m = meshgen.noisy_icosphere(3, 4)
    md = oracle.mesh_data(m.V, m.F)
    b = oracle.bfs(md, [7, 99])
    t = oracle.diffusion_time(md)
    full = oracle.gs(md, b, t, 30)
    part = oracle.gs(md, b, t, 19, oracle.gs(md, b, t, 11))
    assert np.array_equal(full[0], part[0]) and np.array_equal(full[1], part[1])


def test_energy_norm_decreases_on_m_matrix():
    """With all theta >= 0 the simultaneous update of one set cannot raise
    the energy norm of the error, so sweeps are monotone in it."""
    m = meshgen.jittered_grid(13, None)
    md = oracle.mesh_data(m.V, m.F)
    assert md.theta.min() >= 0
    b = oracle.bfs(md, [40])
    t = oracle.diffusion_time(md)
    K = sp.diags(md.Av) + t * hm.cotan_stiffness(md)
    ustar = hm.heat_direct(md, [40], t)
    st, last = None, np.inf
    for _ in range(60):
        st = oracle.gs(md, b, t, 1, st)
        e = _state_to_float(st) - ustar
        en = math.sqrt(e @ (K @ e))
        assert en <= last * (1 + 1e-12)
        last = en


def test_far_field_beyond_double_range():
    """On a long strip the solution falls below the smallest double; the
    separate exponent keeps every vertex positive and, once converged, each
    row of (A - t L_c) u = u_0 holds relative to the row's largest term."""
    n = 1600
    xs = np.arange(n, dtype=float)
    V = np.concatenate([np.stack([xs, np.zeros(n), np.zeros(n)], 1), np.stack([xs, np.ones(n), np.zeros(n)], 1)])
    F = []
    for i in range(n - 1):
        a, b_, c, d = i, i + 1, n + i, n + i + 1
        F += [(a, b_, d), (a, d, c)]
    F = np.array(F, np.int32)
    md = oracle.mesh_data(V, F)
    b = oracle.bfs(md, [0])
    t = oracle.diffusion_time(md)
    st = oracle.gs(md, b, t, 4 * b.nlev)
    assert np.all(st[0][b.order] > 0)
    assert st[1].min() < -1100                      # far below the double range
    plain = oracle.gs_plain(md, b, t, 4 * b.nlev)
    assert np.sum(plain == 0) > 0                   # plain arithmetic underflowed
    for v in range(0, md.nv, 7):
        r = slice(md.rowptr[v], md.rowptr[v + 1])
        nb = md.col[r]
        th = md.theta[md.col_edge[r]]
        emax = max(st[1][v], st[1][nb].max())
        uv = np.ldexp(st[0][v], st[1][v] - emax)
        un = np.ldexp(st[0][nb], st[1][nb] - emax)
        u0 = np.ldexp(1.0, -emax) if b.level[v] == 0 else 0.0
        terms = np.concatenate([[md.Av[v] * uv, t * th.sum() * uv], t * th * un])
        res = md.Av[v] * uv + t * np.sum(th * (uv - un)) - u0
        assert abs(res) <= 1e-12 * np.abs(terms).max()
