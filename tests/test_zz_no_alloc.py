"""gh_mean_edge_length_noalloc: the allocation-free variant of the mesh
setup's mean-edge-length reduction, for callers that cannot allocate device
memory (inside stream capture, under an application-owned allocator, on
latency-critical paths).  Checked through the C-ABI against the mean edge
length gh_mesh_load reports, on two calls in a row (the fixed scratch array
keeps the previous call's partial sums).  This file is collected last."""
import math

import numpy as np
import pytest

import meshgen

pytestmark = pytest.mark.gpu

REL_TOL = 1e-12   # the tolerance the setup parity tests use for mean edge length


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


def test_noalloc_matches_mesh_load_twice(gh):
    import torch
    ctx = gh.Context(0)
    try:
        for mesh in (meshgen.noisy_icosphere(4, 3), meshgen.jittered_grid(301, 9)):
            M = gh.Mesh(ctx, mesh.V, mesh.F)
            edges = torch.from_numpy(M.dump(gh.GH_DUMP_EDGES).reshape(-1, 2)).cuda()
            V = torch.from_numpy(mesh.V).cuda()
            for _ in range(2):
                out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
                gh.mean_edge_length_noalloc(V, edges, out)
                torch.cuda.synchronize()
                got = float(out.item())
                assert math.isclose(got, M.hbar, rel_tol=REL_TOL), (got, M.hbar)
            M.close()
    finally:
        ctx.close()


def test_noalloc_rejects_bad_sizes_and_host_pointers(gh):
    import torch
    V = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    edges = torch.zeros((2, 2), dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    lib = gh.lib()
    import ctypes as C
    too_many = 8192 * 65536 + 1
    rc = lib.gh_mean_edge_length_noalloc(C.c_void_p(V.data_ptr()), C.c_void_p(edges.data_ptr()), too_many,
                                         C.c_void_p(out.data_ptr()), None)
    assert rc == gh.GH_EINVAL and "exceeds" in lib.gh_last_error().decode()
    host_out = np.zeros(1)
    rc = lib.gh_mean_edge_length_noalloc(C.c_void_p(V.data_ptr()), C.c_void_p(edges.data_ptr()), 2,
                                         host_out.ctypes.data_as(C.c_void_p), None)
    assert rc == gh.GH_EINVAL
    rc = lib.gh_mean_edge_length_noalloc(C.c_void_p(V.data_ptr()), C.c_void_p(edges.data_ptr()), 0,
                                         C.c_void_p(out.data_ptr()), None)
    assert rc == gh.GH_EINVAL
