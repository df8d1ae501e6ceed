"""The C-ABI used from plain C (tests/c_api/solve_mesh.c): it compiles against
include/geoheat.h and links against libgeoheat.so alone (CPU); on a GPU its
distances equal the Python binding's bit for bit and meet the contract
against the oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import meshgen
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_1812_06060_gb300 import build
    lib = build.build()
    out = tmp_path_factory.mktemp("c_api") / "solve_mesh"
    libdir = os.path.dirname(lib)
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c_api", "solve_mesh.c"), "-o", str(out), "-L", libdir,
                           "-lgeoheat", f"-Wl,-rpath,{libdir}"])
    return str(out)


def test_c_program_compiles_and_links(exe):
    assert os.access(exe, os.X_OK)


def _write_input(path, mesh, src):
    with open(path, "wb") as f:
        np.array([mesh.nv, mesh.nf], np.int64).tofile(f)
        np.ascontiguousarray(mesh.V, np.float64).tofile(f)
        np.ascontiguousarray(mesh.F, np.int32).tofile(f)
        np.array([len(src)], np.int32).tofile(f)
        np.asarray(src, np.int32).tofile(f)


@pytest.mark.gpu
@pytest.mark.parametrize("form", ["face", "edge"])
def test_c_program_solves(exe, tmp_path, form):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mesh = meshgen.noisy_icosphere(4, 6)
    src = [3, 999]
    _write_input(tmp_path / "in.bin", mesh, src)
    r = subprocess.run([exe, str(tmp_path / "in.bin"), str(tmp_path / "out.bin"), "200",
                        "1" if form == "edge" else "0", "0"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    d = np.fromfile(tmp_path / "out.bin", np.float64)
    import paper_1812_06060_gb300 as g
    g.load_library()
    ctx = g.Context(0)
    M = g.Mesh(ctx, mesh.V, mesh.F)
    dp = np.empty(mesh.nv)
    M.solve(src, dp, g.params(gs_sweeps=200, form=form))
    M.close()
    ctx.close()
    assert np.array_equal(d, dp)
    md = oracle.mesh_data(mesh.V, mesh.F)
    ref = oracle.solve(md, src, form, sweeps=200)
    mask = np.isfinite(ref["d"])
    mask[src] = False
    assert np.max(np.abs(d[mask] - ref["d"][mask]) / np.maximum(np.abs(ref["d"][mask]), md.hbar)) <= 1e-4
