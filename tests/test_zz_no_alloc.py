"""gh_mean_edge_length_noalloc: the allocation-free variant of the mesh
setup's mean-edge-length reduction, for callers that cannot have a library
allocate device memory (an application whose own allocator owns the device
memory, a latency-critical loop where cudaMalloc may wait for the device to
go idle).  Checked through the C-ABI against the mean edge length
gh_mesh_load reports (the same fixed-order sum: bit for bit) and against the
oracle's, on two calls in a row (the fixed scratch array keeps the previous
call's partial sums), and for leaving the device's free memory unchanged.
This file is collected last."""
import ctypes as C

import numpy as np
import pytest

import meshgen
import oracle

pytestmark = pytest.mark.gpu

REL_TOL = 1e-12   # the tolerance the setup parity tests use for mean edge length against the oracle


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


def _free_bytes():
    import torch
    return torch.cuda.mem_get_info()[0]


def test_noalloc_matches_mesh_load_twice(gh):
    import torch
    ctx = gh.Context(0)
    try:
        for mesh in (meshgen.noisy_icosphere(4, 3), meshgen.jittered_grid(301, 9)):
            md = oracle.mesh_data(mesh.V, mesh.F)
            M = gh.Mesh(ctx, mesh.V, mesh.F)
            edges = torch.from_numpy(M.dump(gh.GH_DUMP_EDGES).reshape(-1, 2)).cuda()
            V = torch.from_numpy(mesh.V).cuda()
            outs = [torch.full((1,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
            gh.mean_edge_length_noalloc(V, edges, outs[0])   # the first call on the device does the set-up
            torch.cuda.synchronize()
            free0 = _free_bytes()
            for out in outs:
                out.fill_(float("nan"))
                gh.mean_edge_length_noalloc(V, edges, out)
                torch.cuda.synchronize()
                got = float(out.item())
                assert np.float64(got).tobytes() == np.float64(M.hbar).tobytes(), (got, M.hbar)
                assert abs(got - md.hbar) <= REL_TOL * md.hbar, (got, md.hbar)
            torch.cuda.synchronize()
            assert _free_bytes() == free0   # the device's free memory is unchanged by the calls
            M.close()
    finally:
        ctx.close()


def test_noalloc_rejects_bad_sizes_and_foreign_pointers(gh):
    import torch
    V = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    edges = torch.zeros((2, 2), dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    lib = gh.lib()
    too_many = 8192 * 65536 + 1
    rc = lib.gh_mean_edge_length_noalloc(C.c_void_p(V.data_ptr()), C.c_void_p(edges.data_ptr()), too_many,
                                         C.c_void_p(out.data_ptr()), None)
    assert rc == gh.GH_EINVAL and "exceeds" in lib.gh_last_error().decode()
    host_out = np.zeros(1)
    rc = lib.gh_mean_edge_length_noalloc(C.c_void_p(V.data_ptr()), C.c_void_p(edges.data_ptr()), 2,
                                         host_out.ctypes.data_as(C.c_void_p), None)
    assert rc == gh.GH_EINVAL and "current device" in lib.gh_last_error().decode()
    rc = lib.gh_mean_edge_length_noalloc(C.c_void_p(V.data_ptr()), C.c_void_p(edges.data_ptr()), 0,
                                         C.c_void_p(out.data_ptr()), None)
    assert rc == gh.GH_EINVAL
    if torch.cuda.device_count() > 1:
        # memory of another device is refused while device 0 is current
        other = torch.zeros(1, dtype=torch.float64, device="cuda:1")
        torch.cuda.set_device(0)
        rc = lib.gh_mean_edge_length_noalloc(C.c_void_p(V.data_ptr()), C.c_void_p(edges.data_ptr()), 2,
                                             C.c_void_p(other.data_ptr()), None)
        assert rc == gh.GH_EINVAL
