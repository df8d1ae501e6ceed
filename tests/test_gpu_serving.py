"""Serving (gh_submit / gh_poll / gh_wait): continuous batching over several
meshes, forms and sweep counts in one batch; every served result equals the
same request solved alone, and admission by memory keeps working under a
tight budget."""
import threading
import time

import numpy as np
import pytest

import meshgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gh():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_06060_gb300 import build
    build.build()
    import paper_1812_06060_gb300 as g
    g.load_library()
    return g


def _meshes():
    return [meshgen.noisy_icosphere(4, 41), meshgen.jittered_grid(65, 42), meshgen.icosphere(3)]


def test_served_results_equal_solo_results(gh):
    ctx = gh.Context(0)
    ctx.serve_config(workers=2, max_batch=8)
    meshes = _meshes()
    M = [gh.Mesh(ctx, m.V, m.F) for m in meshes]
    rng = meshgen.rng_for(77)
    reqs = []
    for _ in range(36):
        k = int(rng.random() * len(M))
        src = meshgen.random_sources(rng, meshes[k].nv, 1, 16)
        form = "face" if rng.random() < 0.5 else "edge"
        sweeps = 100 if rng.random() < 0.5 else 150
        reqs.append((k, src, (form, sweeps)))
    prms = {(f, n): gh.params(gs_sweeps=n, form=f) for f in ("face", "edge") for n in (100, 150)}
    ids = [None] * len(reqs)

    def submitter(part):
        for i in part:
            k, src, form = reqs[i]
            ids[i] = ctx.submit(M[k], src, prms[form])
            time.sleep(0.002 * (i % 3))   # staggered arrivals while others run

    th = [threading.Thread(target=submitter, args=(range(j, len(reqs), 3),)) for j in range(3)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    served = []
    for i, (k, src, form) in enumerate(reqs):
        out = np.empty(meshes[k].nv)
        ctx.wait(ids[i], out)
        served.append(out)
    for i, (k, src, form) in enumerate(reqs):
        solo = np.empty(meshes[k].nv)
        M[k].solve(src, solo, prms[form])
        assert np.array_equal(served[i], solo), f"request {i} differs from its solo solve"
    # and one of them against the oracle
    k, src, (form, sweeps) = reqs[0]
    md = oracle.mesh_data(meshes[k].V, meshes[k].F)
    ref = oracle.solve(md, src, form, sweeps=sweeps)
    mask = np.ones(md.nv, bool)
    mask[src] = False
    err = np.max(np.abs(served[0][mask] - ref["d"][mask]) / np.maximum(np.abs(ref["d"][mask]), md.hbar))
    assert err < 1e-4
    for m in M:
        m.close()
    ctx.close()


def test_admission_under_tight_budget(gh):
    mesh = meshgen.jittered_grid(129, 5)
    prm = gh.params(gs_sweeps=100, form="edge")
    rng = meshgen.rng_for(3)
    srcs = [meshgen.random_sources(rng, mesh.nv, 1, 4) for _ in range(10)]
    # reference solves in an unbudgeted context
    free_ctx = gh.Context(0)
    Mf = gh.Mesh(free_ctx, mesh.V, mesh.F)
    mesh_bytes = free_ctx.memory()
    solo = []
    for s_ in srcs:
        out = np.empty(mesh.nv)
        Mf.solve(s_, out, prm)
        solo.append(out)
    Mf.close()
    free_ctx.close()
    # room for the mesh and about one query workspace per worker: the
    # workers admit one request at a time instead of batches of 16
    budget = int(mesh_bytes * 4)
    ctx = gh.Context(0, hbm_budget=budget)
    ctx.serve_config(workers=2, max_batch=16)
    M = gh.Mesh(ctx, mesh.V, mesh.F)
    ids = [ctx.submit(M, s_, prm) for s_ in srcs]
    for ref, rid in zip(solo, ids):
        out = np.empty(mesh.nv)
        ctx.wait(rid, out)
        assert np.array_equal(out, ref)
    assert ctx.memory() <= budget
    M.close()
    ctx.close()


def test_serving_errors(gh):
    ctx = gh.Context(0)
    m = meshgen.icosphere(2)
    M = gh.Mesh(ctx, m.V, m.F)
    prm = gh.params(gs_sweeps=50)
    with pytest.raises(gh.GeoheatError) as e:
        ctx.submit(M, [m.nv + 5], prm)
    assert e.value.status == gh.GH_EINVAL
    with pytest.raises(gh.GeoheatError) as e:
        ctx.wait(987654, np.empty(m.nv))
    assert e.value.status == gh.GH_ENOTFOUND
    rid = ctx.submit(M, [0], prm)
    out = np.empty(m.nv)
    ctx.wait(rid, out)
    assert out[0] == 0.0 and np.all(np.isfinite(out))
    with pytest.raises(gh.GeoheatError) as e:
        ctx.poll(rid)   # forgotten after gh_wait
    assert e.value.status == gh.GH_ENOTFOUND
    with pytest.raises(gh.GeoheatError) as e:
        ctx.serve_config(3, 4)   # serving already started
    assert e.value.status == gh.GH_EBUSY
    M.close()
    ctx.close()


def test_admission_waits_for_memory_across_meshes(gh):
    """Two workers, three meshes and a budget with room for the meshes and
    less than two query workspaces: a request whose workspace does not fit
    waits until memory comes back (idle workspaces of other meshes are
    released), and every request is served, bit-equal to its solo solve."""
    meshes = [meshgen.jittered_grid(129, 61), meshgen.noisy_icosphere(5, 62), meshgen.jittered_grid(121, 63)]
    prm = gh.params(gs_sweeps=120, form="edge")
    rng = meshgen.rng_for(64)
    reqs = [(k % 3, meshgen.random_sources(rng, meshes[k % 3].nv, 1, 6)) for k in range(18)]
    free_ctx = gh.Context(0)
    mesh_bytes, ws_max, solo = 0, 0, []
    Ms = []
    for m in meshes:
        before = free_ctx.memory()
        Ms.append(gh.Mesh(free_ctx, m.V, m.F))
        mesh_bytes += free_ctx.memory() - before
    for k, M in enumerate(Ms):
        before = free_ctx.memory()
        out = np.empty(meshes[k].nv)
        M.solve([1], out, prm)
        ws_max = max(ws_max, free_ctx.memory() - before)
    for k, s_ in reqs:
        out = np.empty(meshes[k].nv)
        Ms[k].solve(s_, out, prm)
        solo.append(out)
    for M in Ms:
        M.close()
    free_ctx.close()
    budget = int(mesh_bytes + 1.5 * ws_max)
    ctx = gh.Context(0, hbm_budget=budget)
    ctx.serve_config(workers=2, max_batch=8)
    M = [gh.Mesh(ctx, m.V, m.F) for m in meshes]
    ids = [ctx.submit(M[k], s_, prm) for k, s_ in reqs]
    for (k, _), ref, rid in zip(reqs, solo, ids):
        out = np.empty(meshes[k].nv)
        ctx.wait(rid, out)   # raises on any status but GH_OK
        assert np.array_equal(out, ref)
    assert ctx.memory() <= budget
    for m in M:
        m.close()
    ctx.close()


def test_request_that_can_never_fit_fails(gh):
    """With room for the mesh but not for one query workspace, a served
    request returns GH_ENOMEM (it would never fit) instead of waiting."""
    mesh = meshgen.jittered_grid(129, 65)
    probe = gh.Context(0)
    Mp = gh.Mesh(probe, mesh.V, mesh.F)
    mesh_bytes = probe.memory()
    Mp.close()
    probe.close()
    # the mesh's setup needs about a sixth more than it keeps; a query
    # workspace needs more than half the mesh again
    ctx = gh.Context(0, hbm_budget=int(mesh_bytes * 1.3))
    M = gh.Mesh(ctx, mesh.V, mesh.F)
    rid = ctx.submit(M, [3], gh.params(gs_sweeps=50, form="edge"))
    with pytest.raises(gh.GeoheatError) as e:
        ctx.wait(rid, np.empty(mesh.nv), timeout_us=30_000_000)
    assert e.value.status == gh.GH_ENOMEM
    M.close()
    ctx.close()
