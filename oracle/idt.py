"""Oracle of the intrinsic Delaunay triangulation and the edge-form path on it
(Sec. 5.3).  TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``.

An intrinsic triangulation is the face list plus the length of every edge
(Sec. 5.3).  The intrinsic Delaunay triangulation (iDT) comes from the
edge-flipping algorithm the paper cites: an interior edge whose two opposite
angles sum to more than pi (cot a + cot b < 0) is flipped, the new edge's
length found by unfolding the two triangles into the plane, until no such
edge is left.

READINGS:
- the tie tolerance: an edge is flipped when cot a + cot b < -1e-12;
- a flip that would join two vertices already joined by an edge (or a vertex
  to itself) is skipped: the face and edge structures here hold one edge per
  vertex pair;
- the flips run in first-in first-out order from the interior edges in
  ascending (min, max) order, re-queueing the four outer edges of each flip
  (the iDT is unique for vertices in general position, so the order does not
  change the result there);
- on the iDT the diffusion uses cotangents and vertex areas from the
  lengths; normalisation and the edge form's target differences use each
  face's own frame (corner 0 at the origin, corner 1 on the +x axis, corner 2
  above it);
- the face form on the iDT (Sec. 5.3 leaves its derivation to the reader):
  g, y and lambda live in each face's frame, and the compatibility condition
  of an edge compares each face's projection on its own unit vector of the
  edge, e_1 . g_1 = e_2 . g_2, so the Y-update becomes
  y_1 = q_1 + A2/(A1+A2) e_1 p, y_2 = q_2 - A1/(A1+A2) e_2 p with
  p = e_2 . q_2 - e_1 . q_1 (the 3D update when e_1 = e_2); the integration
  takes p_j - p_k in each face's frame.
"""
from __future__ import annotations

import math
from collections import deque

import numpy as np

from . import (ADMM_ITERS, MU, MeshData, _check, _p, bfs, diffusion_time, edge_admm, face_admm, gs,
               integrate_edge, integrate_face, lib)

IDT_TOL = 1e-12


def heron(a: float, b: float, c: float) -> float:
    """Triangle area from its side lengths, in the cancellation-free
    arrangement of Kahan (sides sorted a >= b >= c)."""
    a, b, c = sorted((a, b, c), reverse=True)
    q = (a + (b + c)) * (c - (a - b)) * (c + (a - b)) * (a + (b - c))
    return 0.25 * math.sqrt(max(q, 0.0))


def corner_cot(l_opp: float, l1: float, l2: float, area: float) -> float:
    """cot of the angle between sides l1, l2 (opposite side l_opp):
    (l1^2 + l2^2 - l_opp^2) / (4 area)"""
    return (l1 * l1 + l2 * l2 - l_opp * l_opp) / (4.0 * area)


def _slot_of(face, v):
    for k in range(3):
        if face[k] == v:
            return k
    raise ValueError("vertex not in face")


def intrinsic_delaunay(V, F, L=None):
    """iDT of the mesh (V, F), or of the intrinsic triangulation (F, L) when
    the lengths L[f,k] of the edge opposite corner k are given: returns the
    new face list [nf,3], its lengths and the number of flips."""
    Fl = [list(map(int, f)) for f in np.asarray(F)]
    if L is None:
        V = np.asarray(V, np.float64)
        L = []
        for a, b, c in Fl:
            L.append([float(np.linalg.norm(V[b] - V[c])), float(np.linalg.norm(V[c] - V[a])),
                      float(np.linalg.norm(V[a] - V[b]))])
    else:
        L = [list(map(float, l)) for l in np.asarray(L)]
    emap = {}

    def add_face(f):
        for k in range(3):
            x, y = Fl[f][(k + 1) % 3], Fl[f][(k + 2) % 3]
            emap.setdefault((min(x, y), max(x, y)), []).append((f, k))

    def drop_face(f):
        for k in range(3):
            x, y = Fl[f][(k + 1) % 3], Fl[f][(k + 2) % 3]
            key = (min(x, y), max(x, y))
            emap[key] = [s for s in emap[key] if s[0] != f]
            if not emap[key]:
                del emap[key]

    for f in range(len(Fl)):
        add_face(f)
    queue = deque(sorted(k for k, s in emap.items() if len(s) == 2))
    queued = set(queue)
    flips = 0
    while queue:
        key = queue.popleft()
        queued.discard(key)
        s = emap.get(key)
        if s is None or len(s) != 2:
            continue
        (f1, k1), (f2, k2) = s
        A1 = heron(*L[f1])
        A2 = heron(*L[f2])
        c1 = corner_cot(L[f1][k1], L[f1][(k1 + 1) % 3], L[f1][(k1 + 2) % 3], A1)
        c2 = corner_cot(L[f2][k2], L[f2][(k2 + 1) % 3], L[f2][(k2 + 2) % 3], A2)
        if not (c1 + c2 < -IDT_TOL):
            continue
        c, d = Fl[f1][k1], Fl[f2][k2]
        x, y = Fl[f1][(k1 + 1) % 3], Fl[f1][(k1 + 2) % 3]      # f1 runs x -> y -> c
        if c == d or (min(c, d), max(c, d)) in emap:
            continue
        lxy = L[f1][k1]
        lxc = L[f1][_slot_of(Fl[f1], y)]
        lyc = L[f1][_slot_of(Fl[f1], x)]
        lxd = L[f2][_slot_of(Fl[f2], y)]
        lyd = L[f2][_slot_of(Fl[f2], x)]
        # unfold: x at the origin, y on the +x axis, c above, d below
        xc = (lxy * lxy + lxc * lxc - lyc * lyc) / (2.0 * lxy)
        yc = math.sqrt(max(lxc * lxc - xc * xc, 0.0))
        xd = (lxy * lxy + lxd * lxd - lyd * lyd) / (2.0 * lxy)
        yd = -math.sqrt(max(lxd * lxd - xd * xd, 0.0))
        lcd = math.hypot(xc - xd, yc - yd)
        drop_face(f1)
        drop_face(f2)
        Fl[f1] = [c, x, d]
        L[f1] = [lxd, lcd, lxc]
        Fl[f2] = [d, y, c]
        L[f2] = [lyc, lcd, lyd]
        add_face(f1)
        add_face(f2)
        flips += 1
        for u, v in ((x, d), (c, x), (y, c), (d, y)):
            k2_ = (min(u, v), max(u, v))
            if len(emap.get(k2_, ())) == 2 and k2_ not in queued:
                queue.append(k2_)
                queued.add(k2_)
    return np.asarray(Fl, np.int32), np.asarray(L, np.float64), flips


def face_frames(L):
    """corner coordinates of every face in its own frame: corner 0 at the
    origin, corner 1 on the +x axis, corner 2 above it"""
    L = np.asarray(L, np.float64)
    Q = np.zeros((len(L), 3, 2))
    for f, (l0, l1, l2) in enumerate(L):
        x2 = (l2 * l2 + l1 * l1 - l0 * l0) / (2.0 * l2)
        Q[f, 1] = (l2, 0.0)
        Q[f, 2] = (x2, math.sqrt(max(l1 * l1 - x2 * x2, 0.0)))
    return Q


def mesh_data_intrinsic(F, L, nv: int) -> MeshData:
    """Connectivity of the face list (orc_edges, orc_connectivity) and the
    geometry from the lengths: face areas (Heron), corner cotangents, cotan
    weights theta = 1/2 sum cot, vertex areas (a third of every adjacent
    face, as orc_geometry), the mean edge length, each face's frame."""
    Lib = lib()
    F_ = np.ascontiguousarray(F, dtype=np.int32)
    L = np.asarray(L, np.float64)
    nf = F_.shape[0]
    edges = np.empty((3 * nf, 2), np.int32)
    ne = _check(Lib.orc_edges(nv, nf, _p(F_), _p(edges)), "orc_edges")
    edges = np.ascontiguousarray(edges[:ne])
    face_edge = np.empty((nf, 3), np.int32)
    face_sign = np.empty((nf, 3), np.int8)
    edge_face = np.empty((ne, 2), np.int32)
    edge_slot = np.empty((ne, 2), np.int32)
    rowptr = np.empty(nv + 1, np.int32)
    col = np.empty(2 * ne, np.int32)
    col_edge = np.empty(2 * ne, np.int32)
    _check(Lib.orc_connectivity(nv, nf, _p(F_), ne, _p(edges), None, _p(face_edge), _p(face_sign),
                                _p(edge_face), _p(edge_slot), _p(rowptr), _p(col), _p(col_edge)),
           "orc_connectivity")
    Af = np.array([heron(*l) for l in L])
    cot = np.zeros((nf, 3))
    Av = np.zeros(nv)
    for f in range(nf):
        for k in range(3):
            cot[f, k] = corner_cot(L[f, k], L[f, (k + 1) % 3], L[f, (k + 2) % 3], Af[f])
            Av[F_[f, k]] += Af[f] / 3.0
    theta = np.zeros(ne)
    elen = np.zeros(ne)
    for e in range(ne):
        for j in range(2):
            f = edge_face[e, j]
            if f >= 0:
                theta[e] += 0.5 * cot[f, edge_slot[e, j]]
                elen[e] = L[f, edge_slot[e, j]]
    hbar = float(elen.sum() / ne)
    return MeshData(np.zeros((nv, 3)), F_, edges, None, face_edge, face_sign, edge_face, edge_slot, rowptr, col,
                    col_edge, Af, Av, cot, theta, hbar, elen, face_frames(L))


def normalize_intrinsic(md: MeshData, state) -> np.ndarray:
    """h = -grad u / |grad u| per face (eq. HeatDiffusionNormalization) in
    the face's frame: grad u = sum_i u_i (N x e_i) / (2 A), N = +z, e_i the
    edge opposite corner i from corner i+1 to corner i+2; returned as
    [nf,3] with a zero third component."""
    um, ue = state
    h = np.zeros((md.nf, 3))
    for f in range(md.nf):
        vs = md.F[f]
        ms = [um[v] for v in vs]
        es = [int(ue[v]) for v in vs]
        nz = [e for m_, e in zip(ms, es) if m_ != 0.0]
        if not nz:
            continue
        eref = max(nz)
        q = md.frame[f]
        g = np.zeros(2)
        for i in range(3):
            e = q[(i + 2) % 3] - q[(i + 1) % 3]
            g += math.ldexp(ms[i], es[i] - eref) * np.array([-e[1], e[0]])
        g /= 2.0 * md.Af[f]
        n = math.hypot(g[0], g[1])
        if n > 0.0:
            h[f, :2] = -g / n
    return h


def slot_vectors(md: MeshData) -> np.ndarray:
    """[nf,3,3]: the edge opposite corner k in face f's frame, from its lower
    to its higher vertex (third component 0)"""
    S = np.zeros((md.nf, 3, 3))
    for f in range(md.nf):
        q = md.frame[f]
        vs = md.F[f]
        for k in range(3):
            i, j = (k + 1) % 3, (k + 2) % 3
            tail, head = (i, j) if vs[i] < vs[j] else (j, i)
            S[f, k, :2] = q[head] - q[tail]
    return S


def edge_targets_intrinsic(md: MeshData, h) -> np.ndarray:
    """z[f,k] = h_f . (q_head - q_tail) in the face's frame, for the edge
    opposite corner k oriented from its lower to its higher vertex
    (eq. TargetDifference)."""
    z = np.zeros((md.nf, 3))
    for f in range(md.nf):
        q = md.frame[f]
        vs = md.F[f]
        for k in range(3):
            i, j = (k + 1) % 3, (k + 2) % 3
            tail, head = (i, j) if vs[i] < vs[j] else (j, i)
            z[f, k] = float(np.dot(h[f, :2], q[head] - q[tail]))
    return z


def solve_intrinsic(md: MeshData, sources, sweeps: int = 200, m: float = 1.0, t: float | None = None,
                    admm_iters: int = ADMM_ITERS, mu: float = MU, form: str = "edge") -> dict:
    """Algorithm 1 on an intrinsic triangulation (Sec. 5.3), edge or face form."""
    t = diffusion_time(md, m) if t is None else t
    b = bfs(md, sources)
    st = gs(md, b, t, sweeps)
    h = normalize_intrinsic(md, st)
    out = {"t": t, "bfs": b, "u": st, "h": h}
    if form == "edge":
        z = edge_targets_intrinsic(md, h)
        x, w, lam, z2, res = edge_admm(md, h, admm_iters, mu, z_in=z)
        out.update(z=z2, x=x, res=res, d=integrate_edge(md, b, x))
    elif form == "face":
        S = slot_vectors(md)
        g, y, lam, res = face_admm(md, h, admm_iters, mu, eslot=S)
        out.update(g=g, res=res, d=integrate_face(md, b, g, eslot=S))
    else:
        raise ValueError(form)
    return out


def quality(V_or_none, F, L) -> float:
    """Triangulation quality tau (eq. TriangulationQuality): the mean over
    faces of 2 sqrt(3) inradius / longest edge."""
    L = np.asarray(L, np.float64)
    tot = 0.0
    for l in L:
        A = heron(*l)
        r = 2.0 * A / float(np.sum(l))
        tot += 2.0 * math.sqrt(3.0) * r / float(np.max(l))
    return tot / len(L)
