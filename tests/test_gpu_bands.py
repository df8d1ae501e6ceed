"""The order of the pipelined sweeps (gs_band): the diffusion's pairs (sweep
k, set i) depend only on (k, i-1), (k-1, i) and (k-1, i+1) (eq.
HeatDiffusionUpdate in breadth-first order), so running the sweeps in bands
of any size gives the same state and distances, bit for bit, as the plain
wavefront (one band of all sweeps) -- both forms, FP32 and FP64, batches,
and the rounds of the residual stop."""
import numpy as np
import pytest

import meshgen

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


@pytest.fixture(scope="module")
def ctx(gh):
    c = gh.Context(0)
    yield c
    c.close()


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint64)


CASES = [("sinusoid_ico8", lambda: meshgen.sinusoid_icosphere(8, 3), 300),
         ("grid301", lambda: meshgen.jittered_grid(301, 9), 400),
         ("mixed_strip", lambda: meshgen.mixed_density_strip(600, 40), 250)]


@pytest.mark.parametrize("name,make,sweeps", CASES, ids=[c[0] for c in CASES])
def test_bands_give_the_plain_wavefront_bit_for_bit(gh, ctx, name, make, sweeps):
    mesh = make()
    M = gh.Mesh(ctx, mesh.V, mesh.F)
    src = meshgen.random_sources(meshgen.rng_for(100), mesh.nv, 1, 4)
    for form in ("edge", "face"):
        for fp64 in (False, True):
            ref = np.empty(mesh.nv)
            M.solve(src, ref, gh.params(gs_sweeps=sweeps, form=form, fp64=fp64, gs_band=sweeps))
            um, ue = M.dump(gh.GH_DUMP_U_MANT), M.dump(gh.GH_DUMP_U_EXP)
            for band in (0, 1, 3, 17, sweeps - 1):
                d = np.empty(mesh.nv)
                M.solve(src, d, gh.params(gs_sweeps=sweeps, form=form, fp64=fp64, gs_band=band))
                assert np.array_equal(_bits(d), _bits(ref)), (form, fp64, band)
                assert np.array_equal(_bits(M.dump(gh.GH_DUMP_U_MANT)), _bits(um)), (form, fp64, band)
                assert np.array_equal(M.dump(gh.GH_DUMP_U_EXP), ue), (form, fp64, band)
    M.close()


def test_bands_in_a_batch_and_in_residual_rounds(gh, ctx):
    mesh = meshgen.noisy_icosphere(6, 4)
    M = gh.Mesh(ctx, mesh.V, mesh.F)
    sets = [meshgen.random_sources(meshgen.rng_for(200 + k), mesh.nv, 1, 8) for k in range(5)]
    ref = np.empty((len(sets), mesh.nv))
    M.solve_batch(sets, ref, gh.params(gs_sweeps=200, gs_band=200))
    got = np.empty_like(ref)
    M.solve_batch(sets, got, gh.params(gs_sweeps=200, gs_band=7))
    assert np.array_equal(_bits(got), _bits(ref))
    # the residual stop runs the sweeps in rounds of gs_check; bands apply inside each round
    a, b = np.empty(mesh.nv), np.empty(mesh.nv)
    M.solve(sets[0], a, gh.params(gs_sweeps=300, gs_tol=1e-300, gs_check=70))
    M.solve(sets[0], b, gh.params(gs_sweeps=300, gs_tol=1e-300, gs_check=70, gs_band=9))
    assert np.array_equal(_bits(a), _bits(b))
    assert M.dump(gh.GH_DUMP_GS_SWEEPS)[0] == 300
    M.close()
