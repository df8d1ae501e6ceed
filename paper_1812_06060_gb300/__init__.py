"""Python binding of the geoheat C-ABI (include/geoheat.h).

Geodesic distance on triangle meshes by the parallel heat method of
arXiv 1812.06060 (breadth-first Gauss-Seidel diffusion, face-wise gradient
normalisation, face- or edge-based ADMM, breadth-first integration), run by
hand-written CUDA kernels for sm_103a in ``libgeoheat.so``.

This module only marshals arguments: every step of the path runs in the
library's kernels.  PyTorch supplies device memory and the stream.  There is
no CPU fallback: importing the binding fails loudly when the library is
missing (build it with ``python -m paper_1812_06060_gb300.build``).

The functions ``gh_*`` carry the C names; ``Context`` and ``Mesh`` wrap them.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgeoheat.so")

GH_OK, GH_EINVAL, GH_ENOMEM, GH_EDEVICE, GH_ETIMEOUT, GH_EBUSY, GH_ENOTFOUND, GH_ENONMANIFOLD = range(8)
GH_FORM_FACE, GH_FORM_EDGE = 0, 1
(GH_DUMP_LEVEL, GH_DUMP_PARENT, GH_DUMP_ORDER, GH_DUMP_LEVEL_OFF, GH_DUMP_U_MANT, GH_DUMP_U_EXP, GH_DUMP_H,
 GH_DUMP_G, GH_DUMP_X, GH_DUMP_D, GH_DUMP_EDGES, GH_DUMP_FACE_EDGE, GH_DUMP_FACE_SIGN, GH_DUMP_THETA, GH_DUMP_AV,
 GH_DUMP_AF, GH_DUMP_ROWPTR, GH_DUMP_COL, GH_DUMP_RESID, GH_DUMP_E1, GH_DUMP_T, GH_DUMP_ITERS, GH_DUMP_PC_OFF,
 GH_DUMP_PC_VAR, GH_DUMP_PC_COEF, GH_DUMP_FACES, GH_DUMP_ELEN, GH_DUMP_GS_SWEEPS) = range(28)

STATUS_NAMES = {0: "GH_OK", 1: "GH_EINVAL", 2: "GH_ENOMEM", 3: "GH_EDEVICE", 4: "GH_ETIMEOUT", 5: "GH_EBUSY",
                6: "GH_ENOTFOUND", 7: "GH_ENONMANIFOLD"}

# symbols declared in include/geoheat.h
EXPORTS = ["gh_params_default", "gh_version", "gh_ctx_create", "gh_ctx_destroy", "gh_ctx_set_stream", "gh_ctx_set_wait_limit", "gh_ctx_memory",
           "gh_ctx_stats",
           "gh_mesh_load", "gh_mesh_info", "gh_mesh_tuning", "gh_mesh_set_tuning", "gh_mesh_intrinsic_delaunay", "gh_mesh_free", "gh_solve", "gh_solve_batch", "gh_debug_size",
           "gh_debug_dump", "gh_stage_times", "gh_mean_edge_length_noalloc", "gh_serve_config", "gh_submit", "gh_poll",
           "gh_wait", "gh_last_error"]


class GhParams(C.Structure):
    _fields_ = [("m", C.c_double), ("t", C.c_double), ("gs_sweeps", C.c_int32), ("admm_iters", C.c_int32),
                ("mu", C.c_double), ("form", C.c_int32), ("fp64", C.c_int32), ("diagnostics", C.c_int32),
                ("early_stop", C.c_int32), ("eps1", C.c_double), ("eps2", C.c_double),
                ("path_constraints", C.c_int32), ("cycle_constraints", C.c_int32), ("gs_tol", C.c_double),
                ("gs_check", C.c_int32), ("gs_band", C.c_int32)]


class GeoheatError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libgeoheat.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"geoheat CUDA library not built: {path} is missing "
                          f"(run: python -m paper_1812_06060_gb300.build)")
    L = C.CDLL(path)
    P, I32, I64, D, S = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_int
    L.gh_params_default.restype = None
    L.gh_params_default.argtypes = [C.POINTER(GhParams)]
    L.gh_version.restype = C.c_char_p
    L.gh_last_error.restype = C.c_char_p
    L.gh_ctx_create.restype = S
    L.gh_ctx_create.argtypes = [C.c_int, C.c_size_t, C.POINTER(P)]
    L.gh_ctx_destroy.restype = S
    L.gh_ctx_destroy.argtypes = [P]
    L.gh_ctx_set_stream.restype = S
    L.gh_ctx_set_stream.argtypes = [P, P]
    L.gh_ctx_set_wait_limit.restype = S
    L.gh_ctx_set_wait_limit.argtypes = [P, I64]
    L.gh_ctx_memory.restype = S
    L.gh_ctx_memory.argtypes = [P, C.POINTER(C.c_size_t)]
    L.gh_ctx_stats.restype = S
    L.gh_ctx_stats.argtypes = [P, C.POINTER(C.c_uint64)]
    L.gh_mesh_load.restype = S
    L.gh_mesh_load.argtypes = [P, P, I64, P, I64, C.POINTER(P)]
    L.gh_mesh_info.restype = S
    L.gh_mesh_info.argtypes = [P, C.POINTER(I64), C.POINTER(I64), C.POINTER(I64), C.POINTER(D)]
    L.gh_mesh_tuning.restype = S
    L.gh_mesh_tuning.argtypes = [P, C.POINTER(I32)]
    L.gh_mesh_set_tuning.restype = S
    L.gh_mesh_set_tuning.argtypes = [P, I32, I32]
    L.gh_mesh_intrinsic_delaunay.restype = S
    L.gh_mesh_intrinsic_delaunay.argtypes = [P, C.POINTER(I64)]
    L.gh_mesh_free.restype = S
    L.gh_mesh_free.argtypes = [P]
    L.gh_solve.restype = S
    L.gh_solve.argtypes = [P, P, I32, C.POINTER(GhParams), P]
    L.gh_solve_batch.restype = S
    L.gh_solve_batch.argtypes = [P, P, P, I32, C.POINTER(GhParams), P]
    L.gh_debug_size.restype = S
    L.gh_debug_size.argtypes = [P, I32, I32, C.POINTER(I64), C.POINTER(I32)]
    L.gh_debug_dump.restype = S
    L.gh_debug_dump.argtypes = [P, I32, I32, P]
    L.gh_stage_times.restype = S
    L.gh_stage_times.argtypes = [P, C.POINTER(D)]
    L.gh_serve_config.restype = S
    L.gh_serve_config.argtypes = [P, I32, I32]
    L.gh_submit.restype = S
    L.gh_submit.argtypes = [P, P, P, I32, C.POINTER(GhParams), C.POINTER(C.c_uint64)]
    L.gh_poll.restype = S
    L.gh_poll.argtypes = [P, C.c_uint64, C.POINTER(C.c_int)]
    L.gh_wait.restype = S
    L.gh_wait.argtypes = [P, C.c_uint64, P, I64]
    L.gh_mean_edge_length_noalloc.restype = S
    L.gh_mean_edge_length_noalloc.argtypes = [P, P, I64, P, P]
    _lib = L
    return L


def lib():
    return load_library()


def _check(rc: int):
    if rc != GH_OK:
        raise GeoheatError(rc, lib().gh_last_error().decode())


def params(m=1.0, t=0.0, gs_sweeps=200, admm_iters=10, mu=100.0, form="edge", fp64=False, diagnostics=False,
           eps=None, path_constraints=False, cycle_constraints=False, gs_tol=0.0, gs_check=100, gs_band=0):
    """Solver parameters; eps = (eps1, eps2) turns on early termination of the
    ADMM; path_constraints adds the multi-source path constraints,
    cycle_constraints the cycle constraints of a closed mesh of genus >= 1;
    gs_tol > 0 ends the diffusion once the heat residual E1 is within it
    (checked every gs_check sweeps, at most gs_sweeps); gs_band sets the
    sweeps per band of the pipelined diffusion (0: chosen from the layout;
    the result is the same for every value)."""
    p = GhParams()
    lib().gh_params_default(C.byref(p))
    p.m, p.t, p.gs_sweeps, p.admm_iters, p.mu = m, t, gs_sweeps, admm_iters, mu
    p.form = {"face": GH_FORM_FACE, "edge": GH_FORM_EDGE}[form] if isinstance(form, str) else int(form)
    p.fp64, p.diagnostics = int(bool(fp64)), int(bool(diagnostics))
    if eps is not None:
        p.early_stop, p.eps1, p.eps2 = 1, float(eps[0]), float(eps[1])
    p.path_constraints = int(bool(path_constraints))
    p.cycle_constraints = int(bool(cycle_constraints))
    p.gs_tol, p.gs_check = float(gs_tol), int(gs_check)
    p.gs_band = int(gs_band)
    return p


def _addr(x):
    """Data pointer of a torch tensor or a numpy array (no copy)."""
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    return x.ctypes.data_as(C.c_void_p)


class Context:
    """A geoheat context on one CUDA device, bound to a torch stream."""

    def __init__(self, device: int = 0, hbm_budget: int = 0, stream=None):
        h = C.c_void_p()
        _check(lib().gh_ctx_create(device, hbm_budget, C.byref(h)))
        self.handle = h
        self.device = device
        self.meshes = []
        if stream is not None:
            self.set_stream(stream)

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t (int) or None."""
        raw = getattr(stream, "cuda_stream", stream)
        _check(lib().gh_ctx_set_stream(self.handle, C.c_void_p(raw or 0)))

    def set_wait_limit(self, microseconds: int):
        """Limit of the diffusion kernel's dependency waits (<= 0: 2 s)."""
        _check(lib().gh_ctx_set_wait_limit(self.handle, microseconds))

    def memory(self) -> int:
        n = C.c_size_t()
        _check(lib().gh_ctx_memory(self.handle, C.byref(n)))
        return n.value

    def serve_config(self, workers: int = 2, max_batch: int = 32):
        _check(lib().gh_serve_config(self.handle, workers, max_batch))

    def submit(self, mesh: "Mesh", sources, prm: GhParams) -> int:
        """Queue one source set (gh_submit); returns the request id."""
        src = np.ascontiguousarray(np.atleast_1d(sources), dtype=np.int32)
        rid = C.c_uint64()
        _check(lib().gh_submit(self.handle, mesh.handle, _addr(src), int(src.shape[0]), C.byref(prm), C.byref(rid)))
        return rid.value

    def poll(self, rid: int) -> bool:
        done = C.c_int()
        _check(lib().gh_poll(self.handle, rid, C.byref(done)))
        return bool(done.value)

    def wait(self, rid: int, out, timeout_us: int = -1):
        """Wait for a request and copy its distances into ``out`` (gh_wait)."""
        _check(lib().gh_wait(self.handle, rid, _addr(out), timeout_us))
        return out

    def kernel_launches(self) -> int:
        n = C.c_uint64()
        _check(lib().gh_ctx_stats(self.handle, C.byref(n)))
        return n.value

    def close(self):
        if self.handle:
            for m in self.meshes:
                m.handle = None          # freed with the context
            lib().gh_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    """A mesh resident on the device (gh_mesh_load)."""

    def __init__(self, ctx: Context, V, F):
        self.ctx = ctx
        if isinstance(V, np.ndarray):
            V = np.ascontiguousarray(V, dtype=np.float64)
            F = np.ascontiguousarray(F, dtype=np.int32)
        else:
            V = V.contiguous()
            F = F.contiguous()
            assert V.dtype.__repr__() == "torch.float64" and F.dtype.__repr__() == "torch.int32"
        h = C.c_void_p()
        _check(lib().gh_mesh_load(ctx.handle, _addr(V), V.shape[0], _addr(F), F.shape[0], C.byref(h)))
        self.handle = h
        ctx.meshes.append(self)
        nv, ne, nf, hb = C.c_int64(), C.c_int64(), C.c_int64(), C.c_double()
        _check(lib().gh_mesh_info(h, C.byref(nv), C.byref(ne), C.byref(nf), C.byref(hb)))
        self.nv, self.ne, self.nf, self.hbar = nv.value, ne.value, nf.value, hb.value

    def solve(self, sources, out, prm: GhParams):
        """One source set -> distances into ``out`` (float64 [nv], host numpy or
        device torch tensor)."""
        src = np.ascontiguousarray(np.atleast_1d(sources), dtype=np.int32) if not hasattr(sources, "data_ptr") else sources
        _check(lib().gh_solve(self.handle, _addr(src), int(src.shape[0]), C.byref(prm), _addr(out)))
        return out

    def solve_batch(self, source_sets, out, prm: GhParams):
        """K source sets -> distances into ``out`` (float64 [K, nv])."""
        off = np.zeros(len(source_sets) + 1, np.int32)
        off[1:] = np.cumsum([len(s) for s in source_sets])
        src = np.ascontiguousarray(np.concatenate([np.asarray(s, np.int32) for s in source_sets]), dtype=np.int32)
        _check(lib().gh_solve_batch(self.handle, _addr(off), _addr(src), len(source_sets), C.byref(prm), _addr(out)))
        return out

    def intrinsic_delaunay(self) -> int:
        """Replace the triangulation by its intrinsic Delaunay triangulation
        (gh_mesh_intrinsic_delaunay); returns the number of flips."""
        n = C.c_int64()
        _check(lib().gh_mesh_intrinsic_delaunay(self.handle, C.byref(n)))
        return n.value

    def tuning(self) -> tuple:
        """Breadth-first cluster sizes in use (single query, batch); 0 = not tuned yet."""
        out = (C.c_int32 * 2)()
        _check(lib().gh_mesh_tuning(self.handle, out))
        return int(out[0]), int(out[1])

    def set_tuning(self, kind: int, bfs_cluster: int):
        """Force the breadth-first cluster size (8 or 16) for kind 0 (single) or 1 (batch); 0 tunes again."""
        _check(lib().gh_mesh_set_tuning(self.handle, kind, bfs_cluster))

    def dump(self, what: int, query: int = 0) -> np.ndarray:
        n, eb = C.c_int64(), C.c_int32()
        _check(lib().gh_debug_size(self.handle, query, what, C.byref(n), C.byref(eb)))
        arr = np.empty(n.value, np.float64 if eb.value == 8 else np.int32)
        if n.value:
            _check(lib().gh_debug_dump(self.handle, query, what, arr.ctypes.data_as(C.c_void_p)))
        return arr

    def stage_times(self) -> np.ndarray:
        a = (C.c_double * 6)()
        _check(lib().gh_stage_times(self.handle, a))
        return np.array(a[:])

    def close(self):
        if self.handle:
            lib().gh_mesh_free(self.handle)
            self.handle = None
            self.ctx.meshes.remove(self)


def gh_version() -> str:
    return lib().gh_version().decode()


def mean_edge_length_noalloc(V, edges, out, stream=None):
    """gh_mean_edge_length_noalloc: V (float64 [nv,3]), edges (int32 [ne,2]) and
    out (float64 [1]) are device tensors; nothing is allocated on the device."""
    raw = getattr(stream, "cuda_stream", stream)
    _check(lib().gh_mean_edge_length_noalloc(_addr(V), _addr(edges), int(edges.shape[0]), _addr(out),
                                             C.c_void_p(raw or 0)))
    return out
