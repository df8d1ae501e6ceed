"""Failure detection on the GPU without a fault: the diffusion kernel's
dependency waits are bounded; a limit too short for any wait to be met makes
every CTA give up, the solve returns GH_ETIMEOUT, and the same context then
solves normally.  Host-side failures (bad meshes, bad sources) are injected in
test_gpu_parity.py::test_errors."""
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


def test_bounded_wait_times_out_and_context_recovers(gh):
    ctx = gh.Context(0)
    m = meshgen.jittered_grid(129, 13)
    M = gh.Mesh(ctx, m.V, m.F)
    prm = gh.params(gs_sweeps=200, form="edge")
    ref = np.empty(m.nv)
    M.solve([100], ref, prm)
    ctx.set_wait_limit(1)   # 1 us: no dependency wait can be met
    with pytest.raises(gh.GeoheatError) as e:
        M.solve([100], np.empty(m.nv), prm)
    assert e.value.status == gh.GH_ETIMEOUT
    ctx.set_wait_limit(0)   # back to the default
    again = np.empty(m.nv)
    M.solve([100], again, prm)
    assert np.array_equal(again, ref)
    M.close()
    ctx.close()
