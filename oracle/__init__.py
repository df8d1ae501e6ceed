"""FP64 CPU oracle of the parallel heat method (arXiv 1812.06060).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users.  The product path never
imports this package.  The arithmetic lives in ``geoheat_oracle.c`` (plain,
single-threaded C, one function per step of the paper); this module compiles
it with gcc, loads it with ctypes and chains the steps of Algorithm 1.

Parity status of each function (pins in tests/test_oracle_*.py):
  connectivity, geometry, bfs, gs, normalize, face_admm, edge_admm,
  integrate_face, integrate_edge, source_paths, path_constraints and the
  path-constrained ADMM, cycle_constraints; idt.py (the intrinsic Delaunay
  triangulation and the edge form on it): pinned.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "geoheat_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libgeoheat_oracle.so")
_LIB_OMP = os.path.join(_HERE, "_build", "libgeoheat_oracle_omp.so")
_lock = threading.Lock()
_libs = {}
_parallel = False

MU = 100.0          # penalty parameter, Sec. 3.2 and Sec. 4.1
ADMM_ITERS = 10     # I_max, Sec. 6
ZERO_EXP = -(1 << 28)


def _compile(target: str, extra: list, force: bool) -> str:
    if force or not os.path.exists(target) or os.path.getmtime(target) < os.path.getmtime(_SRC):
        tmp = target + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", *extra, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, target)
    return target


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE double: no fast-math, no FMA
    contraction) into oracle/_build: the single-threaded library and, from
    the same source with -fopenmp, the level-parallel one."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    _compile(_LIB, [], force)
    _compile(_LIB_OMP, ["-fopenmp"], force)
    return _LIB


def lib():
    """The library the oracle functions call: the single-threaded one, or the
    level-parallel one after set_parallel(True).  Both give bit-identical
    results (tests/test_oracle_parallel.py)."""
    key = bool(_parallel)
    with _lock:
        if key not in _libs:
            build()
            L = C.CDLL(_LIB_OMP if key else _LIB)
            _declare(L)
            _libs[key] = L
        return _libs[key]


def set_parallel(on: bool) -> None:
    """Select the level-parallel build (OpenMP on all the host's cores, or
    OMP_NUM_THREADS of them) or the single-threaded one."""
    global _parallel
    _parallel = bool(on)


class parallel:
    """Context manager: the level-parallel build inside the block."""

    def __init__(self, on: bool = True):
        self.on = on

    def __enter__(self):
        self.prev = _parallel
        set_parallel(self.on)
        return self

    def __exit__(self, *exc):
        set_parallel(self.prev)


def threads() -> int:
    """Threads the selected build's parallel loops use (1 single-threaded)."""
    return int(lib().orc_threads())


P = C.c_void_p
I64 = C.c_int64
I32 = C.c_int32
D = C.c_double


def _declare(L):
    L.orc_threads.restype = C.c_int
    L.orc_threads.argtypes = []
    L.orc_edges.restype = I64
    L.orc_edges.argtypes = [I64, I64, P, P]
    L.orc_connectivity.restype = C.c_int
    L.orc_connectivity.argtypes = [I64, I64, P, I64, P, P, P, P, P, P, P, P, P]
    L.orc_geometry.restype = C.c_int
    L.orc_geometry.argtypes = [I64, P, I64, P, I64, P, P, P, P, P, P, P, P]
    L.orc_bfs.restype = C.c_int
    L.orc_bfs.argtypes = [I64, P, P, I64, P, P, P, P, P]
    L.orc_gs.restype = C.c_int
    L.orc_gs.argtypes = [I64, P, P, P, P, P, D, P, P, I32, I32, P, P]
    L.orc_gs_plain.restype = C.c_int
    L.orc_gs_plain.argtypes = [I64, P, P, P, P, P, D, P, P, I32, I32, P]
    L.orc_heat_residual.restype = D
    L.orc_heat_residual.argtypes = [I64, P, P, P, P, P, D, P, P, P]
    L.orc_normalize.restype = C.c_int
    L.orc_normalize.argtypes = [I64, P, I64, P, P, P, P]
    L.orc_face_admm.restype = C.c_int
    L.orc_face_admm.argtypes = [I64, P, I64, I64, P, P, P, P, P, P, I32, D, D, D, I32, I32, P, P, P, P, P, P, P, P,
                                P]
    L.orc_edge_admm.restype = C.c_int
    L.orc_edge_admm.argtypes = [I64, P, I64, P, I64, P, P, P, P, P, P, P, I32, D, D, D, I32, I32, P, P, P, P, P, P,
                                P, P, P, P]
    L.orc_integrate_face.restype = C.c_int
    L.orc_integrate_face.argtypes = [I64, P, P, P, P, P, P, P, P, P, I32, P, P, P]
    L.orc_integrate_edge.restype = C.c_int
    L.orc_integrate_edge.argtypes = [I64, P, P, P, P, P, P, P, I32, P, P, P]


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc < 0:
        raise OracleError(f"{what} failed with code {rc}")
    return rc


@dataclass
class MeshData:
    """Connectivity and geometry of one mesh (Sec. 3, Sec. 3.1, Sec. 4.1)."""
    P: np.ndarray
    F: np.ndarray
    edges: np.ndarray
    flip: np.ndarray | None
    face_edge: np.ndarray
    face_sign: np.ndarray
    edge_face: np.ndarray
    edge_slot: np.ndarray
    rowptr: np.ndarray
    col: np.ndarray
    col_edge: np.ndarray
    Af: np.ndarray
    Av: np.ndarray
    cot: np.ndarray
    theta: np.ndarray
    hbar: float
    elen: np.ndarray | None = None     # intrinsic meshes: edge lengths
    frame: np.ndarray | None = None    # intrinsic meshes: [nf,3,2] corner coordinates in each face's frame

    @property
    def nv(self):
        return self.P.shape[0]

    @property
    def nf(self):
        return self.F.shape[0]

    @property
    def ne(self):
        return self.edges.shape[0]


def mesh_data(V, F, flip=None) -> MeshData:
    """Connectivity (orc_edges, orc_connectivity) and geometry (orc_geometry)."""
    L = lib()
    P_ = np.ascontiguousarray(V, dtype=np.float64)
    F_ = np.ascontiguousarray(F, dtype=np.int32)
    nv, nf = P_.shape[0], F_.shape[0]
    edges = np.empty((3 * nf, 2), np.int32)
    ne = _check(L.orc_edges(nv, nf, _p(F_), _p(edges)), "orc_edges")
    edges = np.ascontiguousarray(edges[:ne])
    if flip is not None:
        flip = np.ascontiguousarray(flip, dtype=np.uint8)
        assert flip.shape == (ne,)
    face_edge = np.empty((nf, 3), np.int32)
    face_sign = np.empty((nf, 3), np.int8)
    edge_face = np.empty((ne, 2), np.int32)
    edge_slot = np.empty((ne, 2), np.int32)
    rowptr = np.empty(nv + 1, np.int32)
    col = np.empty(2 * ne, np.int32)
    col_edge = np.empty(2 * ne, np.int32)
    _check(L.orc_connectivity(nv, nf, _p(F_), ne, _p(edges), _p(flip), _p(face_edge), _p(face_sign),
                              _p(edge_face), _p(edge_slot), _p(rowptr), _p(col), _p(col_edge)),
           "orc_connectivity")
    Af = np.empty(nf)
    Av = np.empty(nv)
    cot = np.empty((nf, 3))
    theta = np.empty(ne)
    hbar = C.c_double(0.0)
    _check(L.orc_geometry(nv, _p(P_), nf, _p(F_), ne, _p(edges), _p(edge_face), _p(edge_slot), _p(Af),
                          _p(Av), _p(cot), _p(theta), C.byref(hbar)), "orc_geometry")
    return MeshData(P_, F_, edges, flip, face_edge, face_sign, edge_face, edge_slot, rowptr, col, col_edge,
                    Af, Av, cot, theta, hbar.value)


@dataclass
class BFS:
    level: np.ndarray
    parent: np.ndarray
    order: np.ndarray
    level_off: np.ndarray
    nlev: int


def bfs(md: MeshData, sources) -> BFS:
    """Breadth-first vertex sets and pairing (eq. VertexSets, Sec. 3.3)."""
    src = np.ascontiguousarray(np.atleast_1d(sources), dtype=np.int32)
    nv = md.nv
    level = np.empty(nv, np.int32)
    parent = np.empty(nv, np.int32)
    order = np.full(nv, -1, np.int32)
    level_off = np.empty(nv + 1, np.int32)
    nlev = _check(lib().orc_bfs(nv, _p(md.rowptr), _p(md.col), src.size, _p(src), _p(level), _p(parent),
                                _p(order), _p(level_off)), "orc_bfs")
    nreach = int(level_off[nlev])
    return BFS(level, parent, order[:nreach].copy(), level_off[:nlev + 1].copy(), nlev)


def gs(md: MeshData, b: BFS, t: float, sweeps: int, state=None):
    """Gauss-Seidel heat diffusion (eq. HeatDiffusionUpdate).  Returns the
    state (um, ue) with u = um * 2^ue; ``state`` resumes from a previous one
    (default u = 0)."""
    if state is None:
        um = np.zeros(md.nv)
        ue = np.full(md.nv, ZERO_EXP, np.int32)
    else:
        um, ue = state[0].copy(), state[1].copy()
    _check(lib().orc_gs(md.nv, _p(md.rowptr), _p(md.col), _p(md.col_edge), _p(md.theta), _p(md.Av), t,
                        _p(b.order), _p(b.level_off), b.nlev, sweeps, _p(um), _p(ue)), "orc_gs")
    return um, ue


def gs_plain(md: MeshData, b: BFS, t: float, sweeps: int, u=None):
    u = np.zeros(md.nv) if u is None else np.ascontiguousarray(u, dtype=np.float64).copy()
    _check(lib().orc_gs_plain(md.nv, _p(md.rowptr), _p(md.col), _p(md.col_edge), _p(md.theta), _p(md.Av), t,
                              _p(b.order), _p(b.level_off), b.nlev, sweeps, _p(u)), "orc_gs_plain")
    return u


def heat_residual(md: MeshData, b: BFS, t: float, state) -> float:
    um, ue = state
    return lib().orc_heat_residual(md.nv, _p(md.rowptr), _p(md.col), _p(md.col_edge), _p(md.theta), _p(md.Av),
                                   t, _p(b.level), _p(um), _p(ue))


def gs_until(md: MeshData, b: BFS, t: float, max_sweeps: int, tol: float, check: int):
    """Gauss-Seidel diffusion stopped on the heat residual E1 (eq.
    HeatSolutionError): E1 is evaluated after every ``check`` sweeps (and
    after the last), and the sweeps end at the first evaluation with
    E1 <= tol, or after max_sweeps.  Each round resumes the same iteration
    (the state is the whole iterate).  Returns (state, sweeps run, the E1
    of every evaluation)."""
    st, done, hist = None, 0, []
    while done < max_sweeps:
        k = min(check, max_sweeps - done)
        st = gs(md, b, t, k, st)
        done += k
        hist.append(heat_residual(md, b, t, st))
        if hist[-1] <= tol:
            break
    return st, done, hist


def normalize(md: MeshData, state) -> np.ndarray:
    """h = -grad u / |grad u| per face (eq. HeatDiffusionNormalization)."""
    um, ue = state
    um = np.ascontiguousarray(um, dtype=np.float64)
    ue = np.ascontiguousarray(ue, dtype=np.int32)
    h = np.empty((md.nf, 3))
    _check(lib().orc_normalize(md.nv, _p(md.P), md.nf, _p(md.F), _p(um), _p(ue), _p(h)), "orc_normalize")
    return h


def face_admm(md: MeshData, h, iters=ADMM_ITERS, mu=MU, eps=None, pc=None, eslot=None):
    """Face-based ADMM (Sec. 3.2).  Returns g [nf,3], y [nf,3,3],
    lambda [nf,3,3] (NaN on boundary slots) and residuals [iterations run, 3]
    (|r_primal|, |r_dual|, |M|_F).  eps = (eps1, eps2) stops once both
    residuals are within |M|_F * eps (Sec. 3.2); None runs all iters.
    pc = path_constraints(md, sources, "face") adds the multi-source
    constraints of Sec. 5.2.  eslot [nf,3,3]: an intrinsic triangulation's
    slot edge vectors in each face's own frame (Sec. 5.3)."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    npc, off, var, coef = _pc_args(pc, 3)
    es = None if eslot is None else np.ascontiguousarray(eslot, dtype=np.float64)
    g = np.empty((md.nf, 3))
    y = np.empty((md.nf, 3, 3))
    lam = np.empty((md.nf, 3, 3))
    res = np.empty((max(iters, 1), 3))
    done = C.c_int32(0)
    e1, e2 = eps if eps is not None else (0.0, 0.0)
    _check(lib().orc_face_admm(md.nv, _p(md.P), md.nf, md.ne, _p(md.edges), _p(md.face_edge), _p(md.edge_face),
                               _p(md.edge_slot), _p(md.Af), _p(h), iters, mu, e1, e2, int(eps is not None), npc,
                               _p(off), _p(var), _p(coef), _p(es), _p(g), _p(y), _p(lam), _p(res), C.byref(done)),
           "orc_face_admm")
    return g, y, lam, res[:done.value]


def edge_admm(md: MeshData, h, iters=ADMM_ITERS, mu=MU, eps=None, pc=None, z_in=None):
    """Edge-based ADMM (Sec. 4.1).  Returns x [ne], w [nf,3], lambda [nf,3],
    z [nf,3] and residuals [iterations run, 2].  eps = (eps1, eps2) stops
    once both residuals are within |Z|_F * eps (the targets' norm standing
    in for Sec. 3.2's |M|_F); None runs all iters.  pc =
    path_constraints(md, sources, "edge") adds the multi-source constraints
    of Sec. 5.2.  z_in [nf,3] gives the target differences instead of h . e
    (an intrinsic triangulation, Sec. 5.3)."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    npc, off, var, coef = _pc_args(pc, 1)
    zi = None if z_in is None else np.ascontiguousarray(z_in, dtype=np.float64)
    x = np.empty(md.ne)
    w = np.empty((md.nf, 3))
    lam = np.empty((md.nf, 3))
    z = np.empty((md.nf, 3))
    res = np.empty((max(iters, 1), 2))
    done = C.c_int32(0)
    e1, e2 = eps if eps is not None else (0.0, 0.0)
    _check(lib().orc_edge_admm(md.nv, _p(md.P), md.nf, _p(md.F), md.ne, _p(md.edges), _p(md.flip),
                               _p(md.face_edge), _p(md.face_sign), _p(md.edge_face), _p(md.edge_slot), _p(h),
                               iters, mu, e1, e2, int(eps is not None), npc, _p(off), _p(var), _p(coef),
                               None if zi is None else _p(zi), _p(x), _p(w), _p(lam), _p(z), _p(res),
                               C.byref(done)), "orc_edge_admm")
    return x, w, lam, z, res[:done.value]


@dataclass
class PathConstraints:
    """One linear constraint per path (Sec. 5.2): entries [off[j], off[j+1])
    of constraint j, each a variable (edge id, or face id) and a coefficient
    (the sign, or the 3-vector of the path's edge)."""
    off: np.ndarray
    var: np.ndarray
    coef: np.ndarray
    paths: list


def source_paths(md: MeshData, sources) -> list:
    """Paths along edges from the first source to each other source
    (Sec. 5.2).  READING: the paper asks for shortest paths along edges; here
    a path has the fewest edges, the one a breadth-first traversal from the
    first (lowest-index) source alone gives by following each vertex's FIFO
    pairing vertex (eq. VertexSets, Sec. 3.3).  Any path between two sources
    gives a valid constraint (the exact distance is 0 at both ends), so the
    choice only selects which one is imposed.  Each path is a list of steps
    (p, v) in the direction first source -> other source; a source that the
    first cannot reach gets an empty path."""
    src = sorted(set(int(s) for s in np.atleast_1d(sources)))
    if len(src) < 2:
        return []
    b = bfs(md, [src[0]])
    paths = []
    for sj in src[1:]:
        steps = []
        v = sj
        if b.level[v] >= 0:
            while b.level[v] > 0:
                p = int(b.parent[v])
                steps.append((p, v))
                v = p
            steps.reverse()
        paths.append(steps)
    return paths


def _edge_id(md: MeshData, a: int, b: int) -> int:
    for j in range(md.rowptr[a], md.rowptr[a + 1]):
        if md.col[j] == b:
            return int(md.col_edge[j])
    raise ValueError(f"{a} and {b} are not adjacent")


def path_constraints(md: MeshData, sources, form: str) -> PathConstraints:
    """The constraints of the paths of ``source_paths``:
    edge form (eq. MultiSourceConstraintEdgeBased): sum s_e x_e = 0, s_e = +1
      where the path runs from tail to head of the edge's orientation
      halfedge, -1 against it;
    face form (eq. MultiSourceConstraint): sum e_j . g_f = 0, e_j the vector
      of the path's edge in the path's direction and f the edge's adjacent
      face of lowest index (READING: the paper leaves the choice among the
      adjacent faces open)."""
    paths = source_paths(md, sources)
    off = [0]
    var, coef = [], []
    for steps in paths:
        for p, v in steps:
            e = _edge_id(md, p, v)
            if form == "edge":
                a, b = int(md.edges[e, 0]), int(md.edges[e, 1])
                tail = b if (md.flip is not None and md.flip[e]) else a
                var.append(e)
                coef.append([1.0 if p == tail else -1.0])
            elif form == "face":
                var.append(int(md.edge_face[e, 0]))
                coef.append(list(md.P[v] - md.P[p]))
            else:
                raise ValueError(form)
        off.append(len(var))
    dim = 1 if form == "edge" else 3
    return PathConstraints(np.asarray(off, np.int32), np.asarray(var, np.int32),
                           np.asarray(coef, np.float64).reshape(-1, dim), paths)


def _bfs_graph(rowptr, col, sources):
    """orc_bfs on any graph in CSR form (rows ascending): set index and FIFO
    pairing node of every node."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    col = np.ascontiguousarray(col if len(col) else np.zeros(1), dtype=np.int32)
    n = len(rowptr) - 1
    src = np.ascontiguousarray(np.atleast_1d(sources), dtype=np.int32)
    level = np.empty(n, np.int32)
    parent = np.empty(n, np.int32)
    order = np.full(n, -1, np.int32)
    level_off = np.empty(n + 1, np.int32)
    _check(lib().orc_bfs(n, _p(rowptr), _p(col), src.size, _p(src), _p(level), _p(parent), _p(order),
                         _p(level_off)), "orc_bfs")
    return level, parent


def _csr(rows):
    """rows: list of lists of (node, edge) -> rowptr, col, col_edge, each row
    sorted by node"""
    rowptr = [0]
    col, cedge = [], []
    for r in rows:
        for nb, e in sorted(r):
            col.append(nb)
            cedge.append(e)
        rowptr.append(len(col))
    return np.asarray(rowptr, np.int32), np.asarray(col, np.int32), np.asarray(cedge, np.int32)


def _tree_edges(rowptr, col_edge, col, level, parent):
    """edge crossed from each node to its pairing node"""
    pe = np.full(len(level), -1, np.int64)
    for v in range(len(level)):
        if level[v] > 0:
            for j in range(rowptr[v], rowptr[v + 1]):
                if col[j] == parent[v]:
                    pe[v] = col_edge[j]
                    break
    return pe


def _lca_walk(a, b, level, parent):
    """the tree paths a -> lca and b -> lca (node lists, lca last)"""
    pa, pb = [a], [b]
    while level[pa[-1]] > level[pb[-1]]:
        pa.append(int(parent[pa[-1]]))
    while level[pb[-1]] > level[pa[-1]]:
        pb.append(int(parent[pb[-1]]))
    while pa[-1] != pb[-1]:
        pa.append(int(parent[pa[-1]]))
        pb.append(int(parent[pb[-1]]))
    return pa, pb


def cycle_constraints(md: MeshData, form: str) -> PathConstraints:
    """Integrability on a cycle basis (Sec. 5.1, eq. TopologyConstraint,
    eq. EdgeTopologyConstraint) from a tree-cotree decomposition.

    READING: the paper treats surfaces of genus g (2g non-contractible
    cycles) and says nothing of boundaries; only a connected closed mesh
    gets cycle constraints here (a mesh with boundary edges, or whose trees
    below do not reach every vertex and face, gets none).  The trees are breadth-first trees with FIFO
    pairing (eq. VertexSets), rooted at vertex 0 and face 0, rows in
    ascending order:
    edge form: T = the primal tree; C = the dual tree over the edges not in
      T; each edge in neither closes the cycle e, then T from its higher
      end to the common ancestor and back down to its lower end, oriented
      lower end -> higher end first; coefficient +1 where the cycle runs
      along the edge's orientation halfedge, -1 against it;
    face form: T* = the dual tree (faces across edges); C = the primal tree
      over the edges not crossed by T*; each edge in neither closes a loop of
      faces: its lower face, its higher face, then T* up to the common
      ancestor and back down; for every face of the loop the coefficient is
      the segment between the midpoints of the edge it is entered through
      and the edge it is left through.
    Cycles come in ascending order of their closing edge."""
    nv, nf, ne = md.nv, md.nf, md.ne
    empty = PathConstraints(np.zeros(1, np.int32), np.zeros(0, np.int32),
                            np.zeros((0, 1 if form == "edge" else 3)), [])
    if (md.edge_face[:, 1] < 0).any() or nf == 0:
        return empty
    efaces = md.edge_face
    dual_all = [[] for _ in range(nf)]
    for e in range(ne):
        f1, f2 = int(efaces[e, 0]), int(efaces[e, 1])
        dual_all[f1].append((f2, e))
        dual_all[f2].append((f1, e))
    off, var, coef, cycles = [0], [], [], []
    if form == "edge":
        plev, ppar = _bfs_graph(md.rowptr, md.col, [0])
        pedge = _tree_edges(md.rowptr, md.col_edge, md.col, plev, ppar)
        tree = np.zeros(ne, bool)
        tree[pedge[pedge >= 0]] = True
        drp, dcol, dce = _csr([[x for x in r if not tree[x[1]]] for r in dual_all])
        dlev, dpar = _bfs_graph(drp, dcol, [0])
        if (plev < 0).any() or (dlev < 0).any():
            return empty
        dedge = _tree_edges(drp, dce, dcol, dlev, dpar)
        dual = np.zeros(ne, bool)
        dual[dedge[dedge >= 0]] = True
        for e in np.flatnonzero(~tree & ~dual):
            a, b = int(md.edges[e, 0]), int(md.edges[e, 1])
            pa, pb = _lca_walk(a, b, plev, ppar)
            nodes = [a] + pb + pa[::-1][1:]          # a -> b -> ... -> lca -> ... -> a
            steps = list(zip(nodes[:-1], nodes[1:]))
            for p, q in steps:
                ee = _edge_id(md, p, q)
                x, y = int(md.edges[ee, 0]), int(md.edges[ee, 1])
                tail = y if (md.flip is not None and md.flip[ee]) else x
                var.append(ee)
                coef.append([1.0 if p == tail else -1.0])
            off.append(len(var))
            cycles.append(steps)
    elif form == "face":
        drp, dcol, dce = _csr(dual_all)
        dlev, dpar = _bfs_graph(drp, dcol, [0])
        dedge = _tree_edges(drp, dce, dcol, dlev, dpar)
        dual = np.zeros(ne, bool)
        dual[dedge[dedge >= 0]] = True
        keep = ~dual[md.col_edge]
        rows = [[(int(md.col[j]), int(md.col_edge[j])) for j in range(md.rowptr[v], md.rowptr[v + 1]) if keep[j]]
                for v in range(nv)]
        crp, ccol, cce = _csr(rows)
        clev, cpar = _bfs_graph(crp, ccol, [0])
        if (dlev < 0).any() or (clev < 0).any():
            return empty
        cedge = _tree_edges(crp, cce, ccol, clev, cpar)
        cot = np.zeros(ne, bool)
        cot[cedge[cedge >= 0]] = True
        mid = 0.5 * (md.P[md.edges[:, 0]] + md.P[md.edges[:, 1]])

        def crossing(f, g):
            for nb, e in dual_all[f]:
                if nb == g:
                    return e
            raise ValueError("faces not adjacent")

        for e in np.flatnonzero(~dual & ~cot):
            f1, f2 = int(efaces[e, 0]), int(efaces[e, 1])
            pa, pb = _lca_walk(f1, f2, dlev, dpar)
            loop = [f1] + pb + pa[::-1][1:]         # f1 -> f2 -> ... -> lca -> ... -> f1
            cross = [crossing(x, y) for x, y in zip(loop[:-1], loop[1:])]
            m = len(cross)
            for i in range(m):                        # face loop[i] entered via cross[i-1], left via cross[i]
                var.append(loop[i])
                coef.append(list(mid[cross[i]] - mid[cross[i - 1]]))
            off.append(len(var))
            cycles.append(loop)
    else:
        raise ValueError(form)
    dim = 1 if form == "edge" else 3
    return PathConstraints(np.asarray(off, np.int32), np.asarray(var, np.int32),
                           np.asarray(coef, np.float64).reshape(-1, dim), cycles)


def join_constraints(*pcs) -> PathConstraints:
    """One constraint list from several, in the given order."""
    pcs = [p for p in pcs if p is not None]
    off = [0]
    var, coef, paths = [], [], []
    for p in pcs:
        base = off[-1]
        off.extend(base + int(x) for x in p.off[1:])
        var.append(p.var)
        coef.append(p.coef)
        paths.extend(p.paths)
    dim = pcs[0].coef.shape[1] if pcs else 1
    return PathConstraints(np.asarray(off, np.int32),
                           np.concatenate(var).astype(np.int32) if var else np.zeros(0, np.int32),
                           np.concatenate(coef) if coef else np.zeros((0, dim)), paths)


def _pc_args(pc, dim):
    if pc is None or len(pc.off) < 2:
        z = np.zeros(1, np.int32)
        return 0, z, z, np.zeros(dim)
    if pc.coef.shape[1] != dim:
        raise ValueError("path constraints of the other form")
    coef = np.ascontiguousarray(pc.coef, dtype=np.float64)
    if coef.size == 0:
        coef = np.zeros(dim)
    var = pc.var if pc.var.size else np.zeros(1, np.int32)
    return len(pc.off) - 1, np.ascontiguousarray(pc.off), np.ascontiguousarray(var), coef


def integrate_face(md: MeshData, b: BFS, g, parent=None, eslot=None) -> np.ndarray:
    """Breadth-first integration of face gradients (eq. IntegrationStep);
    eslot as for face_admm on an intrinsic triangulation."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    es = None if eslot is None else np.ascontiguousarray(eslot, dtype=np.float64)
    par = np.ascontiguousarray(b.parent if parent is None else parent, dtype=np.int32)
    d = np.empty(md.nv)
    _check(lib().orc_integrate_face(md.nv, _p(md.P), _p(md.rowptr), _p(md.col), _p(md.col_edge),
                                    _p(md.edge_face), _p(md.edge_slot), _p(es), _p(b.order), _p(b.level_off),
                                    b.nlev, _p(par), _p(g), _p(d)), "orc_integrate_face")
    return d


def integrate_edge(md: MeshData, b: BFS, x, parent=None) -> np.ndarray:
    """Breadth-first integration of edge differences (Sec. 4)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    par = np.ascontiguousarray(b.parent if parent is None else parent, dtype=np.int32)
    d = np.empty(md.nv)
    _check(lib().orc_integrate_edge(md.nv, _p(md.edges), _p(md.flip), _p(md.rowptr), _p(md.col),
                                    _p(md.col_edge), _p(b.order), _p(b.level_off), b.nlev, _p(par), _p(x),
                                    _p(d)), "orc_integrate_edge")
    return d


def diffusion_time(md: MeshData, m: float = 1.0) -> float:
    """t = m * hbar^2 (eq. DiffusionTime)."""
    return m * md.hbar * md.hbar


def solve(md: MeshData, sources, form: str = "edge", sweeps: int = 200, m: float = 1.0, t: float | None = None,
          admm_iters: int = ADMM_ITERS, mu: float = MU, eps=None, path_constraints_on: bool = False,
          cycle_constraints_on: bool = False, gs_tol: float = 0.0, gs_check: int = 100) -> dict:
    """Algorithm 1 end to end: Diffusion -> normalise -> Integrable ->
    Recovery, in the face form (Sec. 3) or the edge form (Sec. 4).  Returns
    every intermediate.  eps = (eps1, eps2) ends the ADMM early on its
    residuals (Sec. 3.2); the iterations run are len(out["res"]).
    path_constraints_on adds the multi-source constraints (Sec. 5.2),
    cycle_constraints_on the cycle constraints of a closed mesh of genus
    g >= 1 (Sec. 5.1), after the path constraints.  gs_tol > 0 stops the
    diffusion on E1 (gs_until, at most ``sweeps``); out["gs_sweeps"] is the
    number of sweeps run."""
    t = diffusion_time(md, m) if t is None else t
    b = bfs(md, sources)
    if gs_tol > 0:
        st, nsw, _ = gs_until(md, b, t, sweeps, gs_tol, gs_check)
    else:
        st, nsw = gs(md, b, t, sweeps), sweeps
    h = normalize(md, st)
    out = {"t": t, "bfs": b, "u": st, "h": h, "gs_sweeps": nsw}
    parts = []
    if path_constraints_on:
        parts.append(path_constraints(md, sources, form))
    if cycle_constraints_on:
        parts.append(cycle_constraints(md, form))
    pc = join_constraints(*parts) if parts else None
    if pc is not None:
        out["pc"] = pc
    if form == "face":
        g, y, lam, res = face_admm(md, h, admm_iters, mu, eps, pc)
        out.update(g=g, res=res, d=integrate_face(md, b, g))
    elif form == "edge":
        x, w, lam, z, res = edge_admm(md, h, admm_iters, mu, eps, pc)
        out.update(x=x, z=z, res=res, d=integrate_edge(md, b, x))
    else:
        raise ValueError(form)
    return out


def u_float(state) -> np.ndarray:
    """u = m * 2^e as plain doubles (underflows to 0 far from the sources)."""
    um, ue = state
    return np.ldexp(um, np.clip(ue, -2000, 2000))
