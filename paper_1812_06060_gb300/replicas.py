"""Replicas on several GPUs: one submit queue feeding one worker process per
device.

Queries (a mesh, a source set, parameters) are independent, so work on
several GPUs shards by query: every worker holds its own context and its own
copy of every registered mesh's operators, solves the queries it is given
with the C-ABI (gh_solve), and sends the distances back to the host.  Nothing
is exchanged between replicas on the data path: there is no collective.  A
mesh cannot be split across GPUs without a halo exchange at every one of the
L + 2(N - 1) wavefront steps of the diffusion, and the largest benchmark mesh
fits one GPU.

Dispatch: a query goes to the replica with the fewest outstanding queries
(ties to the lowest rank).  A replica whose process dies is detected on the
host (its process has exited); its outstanding queries go back to the queue
and are given to the live replicas (a query is idempotent).  An exception
inside a solve is returned for that query only.

Workers are started with the ``spawn`` method (a CUDA context does not
survive fork).  ``worker_factory`` builds the per-process solver; the default
one uses the CUDA library on the worker's device.
"""
from __future__ import annotations

import multiprocessing as mp
import queue as _queue
import threading
import time

import numpy as np


class CudaWorker:
    """The solver of one replica: a context on its device and a copy of every
    mesh (gh_ctx_create, gh_mesh_load, gh_solve)."""

    def __init__(self, device: int):
        import paper_1812_06060_gb300 as g
        g.load_library()
        self.g = g
        self.ctx = g.Context(device)
        self.meshes = {}

    def add_mesh(self, key, V, F):
        self.meshes[key] = self.g.Mesh(self.ctx, V, F)

    def solve(self, key, sources, params: dict) -> np.ndarray:
        M = self.meshes[key]
        out = np.empty(M.nv)
        M.solve(np.asarray(sources, np.int32), out, self.g.params(**params))
        return out

    def close(self):
        for M in self.meshes.values():
            M.close()
        self.ctx.close()


def _worker_main(rank, device, factory, inq, outq):
    try:
        w = factory(device)
    except Exception as ex:  # the replica cannot start: report and leave
        outq.put(("dead", rank, None, f"{type(ex).__name__}: {ex}"))
        return
    outq.put(("ready", rank, None, None))
    while True:
        msg = inq.get()
        kind = msg[0]
        if kind == "stop":
            break
        if kind == "mesh":
            _, key, V, F = msg
            try:
                w.add_mesh(key, V, F)
                outq.put(("mesh", rank, key, None))
            except Exception as ex:
                outq.put(("mesh", rank, key, f"{type(ex).__name__}: {ex}"))
            continue
        _, ticket, key, src, params = msg
        try:
            outq.put(("done", rank, ticket, w.solve(key, src, params)))
        except Exception as ex:
            outq.put(("error", rank, ticket, f"{type(ex).__name__}: {ex}"))
    try:
        w.close()
    except Exception:
        pass


class ReplicaError(RuntimeError):
    pass


class ReplicaDispatcher:
    """Queries over replicas on ``devices`` (one worker process each)."""

    def __init__(self, devices, worker_factory=CudaWorker, start_timeout: float = 300.0):
        ctx = mp.get_context("spawn")
        self._outq = ctx.Queue()
        self._inq = []
        self._procs = []
        self._lock = threading.Lock()
        self._outstanding = {}     # rank -> {ticket: query}
        self._results = {}         # ticket -> ("done", array) | ("error", message)
        self._cv = threading.Condition(self._lock)
        self._next = 0
        self._meshes = {}
        self._dead = set()
        self._pending = []         # queries waiting for a live replica
        for r, dev in enumerate(devices):
            q = ctx.Queue()
            p = ctx.Process(target=_worker_main, args=(r, dev, worker_factory, q, self._outq), daemon=True)
            p.start()
            self._inq.append(q)
            self._procs.append(p)
            self._outstanding[r] = {}
        ready, t0 = set(), time.monotonic()
        while len(ready) + len(self._dead) < len(devices):
            try:
                kind, rank, _, err = self._outq.get(timeout=1.0)
            except _queue.Empty:
                self._check_dead()
                if time.monotonic() - t0 > start_timeout:
                    raise ReplicaError("replicas did not start in time")
                continue
            if kind == "ready":
                ready.add(rank)
            elif kind == "dead":
                self._dead.add(rank)
        if not ready:
            raise ReplicaError("no replica started")
        self._stop = False
        self._th = threading.Thread(target=self._collect, daemon=True)
        self._th.start()

    @property
    def live(self):
        return [r for r in range(len(self._procs)) if r not in self._dead]

    def add_mesh(self, key, V, F, timeout: float = 600.0):
        """Every live replica loads its own copy of the mesh."""
        with self._lock:
            self._meshes[key] = (np.ascontiguousarray(V, np.float64), np.ascontiguousarray(F, np.int32))
            self._results[("mesh", key)] = set()
            for r in self.live:
                self._inq[r].put(("mesh", key, *self._meshes[key]))
            t0 = time.monotonic()
            while not set(self.live) <= self._results[("mesh", key)]:
                if not self._cv.wait(timeout=1.0) and time.monotonic() - t0 > timeout:
                    raise ReplicaError(f"mesh {key!r} not loaded by every replica in time")

    def submit(self, key, sources, params: dict | None = None) -> int:
        """Queue one query; returns its ticket."""
        with self._lock:
            t = self._next
            self._next += 1
            self._dispatch((t, key, [int(s) for s in np.atleast_1d(sources)], dict(params or {})))
            return t

    def _dispatch(self, query):
        live = self.live
        if not live:
            self._results[query[0]] = ("error", "no live replica")
            self._cv.notify_all()
            return
        r = min(live, key=lambda k: (len(self._outstanding[k]), k))
        self._outstanding[r][query[0]] = query
        self._inq[r].put(("solve", *query))

    def _check_dead(self):
        for r, p in enumerate(self._procs):
            if r not in self._dead and not p.is_alive():
                self._dead.add(r)
                lost = list(self._outstanding.get(r, {}).values())
                self._outstanding[r] = {}
                for q in lost:   # back to the live replicas
                    self._dispatch(q)

    def _collect(self):
        while not self._stop:
            try:
                kind, rank, ticket, payload = self._outq.get(timeout=0.2)
            except _queue.Empty:
                with self._lock:
                    self._check_dead()
                    self._cv.notify_all()
                continue
            except (EOFError, OSError):
                break
            with self._lock:
                if kind == "mesh":
                    if payload is None:
                        self._results[("mesh", ticket)].add(rank)
                elif kind in ("done", "error"):
                    if self._outstanding[rank].pop(ticket, None) is not None or ticket not in self._results:
                        self._results[ticket] = (kind, payload)
                elif kind == "dead":
                    self._dead.add(rank)
                self._check_dead()
                self._cv.notify_all()

    def result(self, ticket: int, timeout: float | None = None) -> np.ndarray:
        """The distances of a query (blocks); raises ReplicaError if its solve failed."""
        t0 = time.monotonic()
        with self._lock:
            while ticket not in self._results:
                left = None if timeout is None else timeout - (time.monotonic() - t0)
                if left is not None and left <= 0:
                    raise TimeoutError(f"query {ticket} not finished")
                self._cv.wait(timeout=0.5 if left is None else min(0.5, left))
            kind, payload = self._results.pop(ticket)
        if kind == "error":
            raise ReplicaError(payload)
        return payload

    def close(self):
        self._stop = True
        for r, q in enumerate(self._inq):
            if r not in self._dead:
                try:
                    q.put(("stop",))
                except Exception:
                    pass
        for p in self._procs:
            p.join(timeout=30)
            if p.is_alive():
                p.terminate()
        self._th.join(timeout=5)
