"""Oracle Gauss-Seidel diffusion stopped on the heat residual E1 (eq.
HeatSolutionError), pinned against what the definitions fix: E1 of u = 0 is
|u_0| = sqrt(#sources), E1 of the direct solution vanishes, resuming the
iteration from its state equals running it uninterrupted (bit for bit), and
the stop lands on the first check whose E1 (from a fresh run of that many
sweeps) is within the tolerance."""
import math

import numpy as np
import pytest

import meshgen
import oracle
import oracle.hm as hm


@pytest.fixture(scope="module")
def grid():
    m = meshgen.jittered_grid(33, 4)
    md = oracle.mesh_data(m.V, m.F)
    src = [40, 700]
    b = oracle.bfs(md, src)
    return md, src, b, oracle.diffusion_time(md)


def test_residual_closed_forms(grid):
    md, src, b, t = grid
    zero = (np.zeros(md.nv), np.full(md.nv, oracle.ZERO_EXP, np.int32))
    assert oracle.heat_residual(md, b, t, zero) == pytest.approx(math.sqrt(len(src)), rel=1e-15)
    ustar = hm.heat_direct(md, src, t)
    m_, e_ = np.frexp(ustar)
    assert oracle.heat_residual(md, b, t, (m_, e_.astype(np.int32))) < 1e-13


def test_resuming_equals_one_run(grid):
    md, src, b, t = grid
    whole = oracle.gs(md, b, t, 70)
    parts = oracle.gs(md, b, t, 30)
    parts = oracle.gs(md, b, t, 25, parts)
    parts = oracle.gs(md, b, t, 15, parts)
    assert np.array_equal(whole[0], parts[0]) and np.array_equal(whole[1], parts[1])


@pytest.mark.parametrize("check", [20, 45])
def test_stop_is_the_first_check_within_tolerance(grid, check):
    md, src, b, t = grid
    counts = list(range(check, 400, check)) + [400]
    e1 = [oracle.heat_residual(md, b, t, oracle.gs(md, b, t, c)) for c in counts]
    assert e1[-1] < e1[0] * 1e-3   # the iteration converges
    tol = math.sqrt(e1[2] * e1[3])  # between the third and fourth checks
    first = next(c for c, e in zip(counts, e1) if e <= tol)
    st, done, hist = oracle.gs_until(md, b, t, 400, tol, check)
    assert done == first == counts[3]
    assert hist == e1[:4]
    assert np.array_equal(st[0], oracle.gs(md, b, t, done)[0])
    # never within the tolerance: every check runs and the sweeps end at the cap
    st, done, hist = oracle.gs_until(md, b, t, 400, 0.0, check)
    assert done == 400 and len(hist) == len(counts) and hist == e1


def test_solve_with_the_stop(grid):
    md, src, b, t = grid
    loose = oracle.solve(md, src, "edge", sweeps=400, gs_tol=1e-3, gs_check=25)
    assert loose["gs_sweeps"] < 400
    assert oracle.heat_residual(md, loose["bfs"], loose["t"], loose["u"]) <= 1e-3
    tight = oracle.solve(md, src, "edge", sweeps=400, gs_tol=1e-300, gs_check=25)
    fixed = oracle.solve(md, src, "edge", sweeps=400)
    assert tight["gs_sweeps"] == fixed["gs_sweeps"] == 400
    assert np.array_equal(tight["d"], fixed["d"])
