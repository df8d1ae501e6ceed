"""The replica dispatcher (paper_1812_06060_gb300/replicas.py) with CPU
processes standing in for devices: one submit queue, one worker process per
"device", queries sharded by source set with no exchange between replicas;
a solve error is returned for its query only; a replica that dies is
detected on the host and its queries go to the live replicas.  The stand-in
solver returns a deterministic field of the query (no GPU, no oracle): the
test checks routing, not arithmetic."""
import os

import numpy as np
import pytest

from paper_1812_06060_gb300.replicas import ReplicaDispatcher, ReplicaError


class FakeWorker:
    """Stands in for one GPU: holds its meshes, 'solves' by a closed form of
    the source set, tags the result with its device."""

    def __init__(self, device):
        self.device = device
        self.meshes = {}

    def add_mesh(self, key, V, F):
        self.meshes[key] = V.shape[0]

    def solve(self, key, sources, params):
        if params.get("fail"):
            raise ValueError("planted failure")
        if params.get("die") and self.device == params["die"]:
            os._exit(3)   # the process ends with the query in flight
        nv = self.meshes[key]
        out = np.arange(nv, dtype=np.float64) + float(sum(sources)) * params.get("scale", 1.0)
        out[0] = self.device
        return out


def _expect(nv, sources, scale=1.0):
    return np.arange(nv, dtype=np.float64) + float(sum(sources)) * scale


@pytest.fixture
def pool():
    d = ReplicaDispatcher([0, 1], worker_factory=FakeWorker, start_timeout=120)
    yield d
    d.close()


def test_queries_shard_over_replicas(pool):
    V = np.zeros((50, 3))
    F = np.zeros((10, 3), np.int32)
    pool.add_mesh("m", V, F)
    tickets = [(pool.submit("m", [i, i + 1], {"scale": 2.0}), [i, i + 1]) for i in range(24)]
    used = set()
    for t, src in tickets:
        out = pool.result(t, timeout=60)
        used.add(int(out[0]))
        assert np.array_equal(out[1:], _expect(50, src, 2.0)[1:])
    assert used == {0, 1}   # both replicas took queries


def test_error_is_returned_for_its_query_only(pool):
    pool.add_mesh("m", np.zeros((8, 3)), np.zeros((2, 3), np.int32))
    good = pool.submit("m", [1], {})
    bad = pool.submit("m", [2], {"fail": True})
    assert np.array_equal(pool.result(good, timeout=60)[1:], _expect(8, [1])[1:])
    with pytest.raises(ReplicaError, match="planted failure"):
        pool.result(bad, timeout=60)


def test_dead_replica_queries_go_to_the_live_one(pool):
    pool.add_mesh("m", np.zeros((8, 3)), np.zeros((2, 3), np.int32))
    # replica 1 exits on its first query; the query is given to replica 0
    tickets = [pool.submit("m", [k], {"die": 1}) for k in range(6)]
    for k, t in enumerate(tickets):
        out = pool.result(t, timeout=60)
        assert out[0] == 0.0 and np.array_equal(out[1:], _expect(8, [k])[1:])
    assert pool.live == [0]
