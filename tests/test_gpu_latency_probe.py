"""Latencies behind the floor of the breadth-first traversal (one thread-block
cluster walks the sets one after another): a dependent L2 round trip (one
thread chasing a cycle through a 32 MB buffer held in L2) and one cluster
barrier (arrive + wait) for clusters of 8 and 16 CTAs of 1024 threads, as the
traversal launches them.  Each set of the traversal costs at least two cluster
barriers and three dependent L2 round trips; the measured values go to the
file GEOHEAT_PARITY_LOG names, and the test checks that they are plausible."""
import ctypes as C
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = str(tmp_path_factory.mktemp("probe") / "liblatency.so")
    nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared", "-Xcompiler",
                           "-fPIC", os.path.join(HERE, "gpu_probes", "latency.cu"), "-o", out])
    L = C.CDLL(out)
    L.probe_l2_round_trip_ns.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_double)]
    L.probe_cluster_barrier_ns.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double)]
    return L


def _log(line):
    path = os.environ.get("GEOHEAT_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(line + "\n")


def test_traversal_latency_floor(probe):
    l2 = C.c_double()
    assert probe.probe_l2_round_trip_ns(8 << 20, 20000, C.byref(l2)) == 0
    bar = {}
    for cl in (8, 16):
        x = C.c_double()
        assert probe.probe_cluster_barrier_ns(cl, 1024, 20000, C.byref(x)) == 0
        bar[cl] = x.value
    per_set = {cl: 2 * bar[cl] + 3 * l2.value for cl in bar}
    _log(f"latency probe: L2 round trip {l2.value:.0f} ns; cluster barrier {bar[8]:.0f} ns (8 CTAs), "
         f"{bar[16]:.0f} ns (16 CTAs); traversal floor per set (2 barriers + 3 round trips) "
         f"{per_set[8]:.0f} / {per_set[16]:.0f} ns")
    assert 50 < l2.value < 5000
    assert all(10 < b < 20000 for b in bar.values())
