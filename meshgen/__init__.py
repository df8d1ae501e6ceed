"""Seeded synthetic triangle meshes and source sets.

This module only produces inputs: vertex positions, faces and source vertex
sets.  It holds none of the heat method's arithmetic and is shared, as an
input generator, by the CPU oracle and by the GPU library's tests and bench.

The paper measures on scanned models (Table 1, Sec. 6.1) that are not
available here; these generators stand in for them with the same kind of
input: closed or open 2-manifold triangle meshes with about 2V faces, and one
or several source vertices.

Random numbers come from numpy's PCG64 bit generator.  Uniform doubles are
``Generator.random`` (53-bit); normal deviates are made here by the
Box-Muller transform from two uniforms so that the sequence does not depend on
numpy's choice of normal sampler.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 20181206


def config_seed(config: int, mesh_index: int = 0) -> int:
    """Seed of mesh ``mesh_index`` of workload ``config`` (1-based config)."""
    return BASE_SEED + 1000 * config + mesh_index


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def normal(rng: np.random.Generator, n: int) -> np.ndarray:
    """n standard normal deviates by the Box-Muller transform."""
    m = (n + 1) // 2
    u1 = rng.random(m)
    u2 = rng.random(m)
    u1 = 1.0 - u1  # (0, 1]: log is finite
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2.0 * math.pi * u2), r * np.sin(2.0 * math.pi * u2)])
    return z[:n]


# --------------------------------------------------------------------------
# Icosahedron and icospheres
# --------------------------------------------------------------------------

def icosahedron() -> tuple[np.ndarray, np.ndarray]:
    """Unit icosahedron: 12 vertices (golden-ratio construction), 20 faces
    oriented counter-clockwise seen from outside."""
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    raw = np.array([
        (-1, phi, 0), (1, phi, 0), (-1, -phi, 0), (1, -phi, 0),
        (0, -1, phi), (0, 1, phi), (0, -1, -phi), (0, 1, -phi),
        (phi, 0, -1), (phi, 0, 1), (-phi, 0, -1), (-phi, 0, 1),
    ], dtype=np.float64)
    faces = []
    for a in range(12):
        for b in range(a + 1, 12):
            if abs(np.sum((raw[a] - raw[b]) ** 2) - 4.0) > 1e-9:
                continue
            for c in range(b + 1, 12):
                if (abs(np.sum((raw[a] - raw[c]) ** 2) - 4.0) > 1e-9
                        or abs(np.sum((raw[b] - raw[c]) ** 2) - 4.0) > 1e-9):
                    continue
                n = np.cross(raw[b] - raw[a], raw[c] - raw[a])
                if np.dot(n, raw[a] + raw[b] + raw[c]) > 0:
                    faces.append((a, b, c))
                else:
                    faces.append((a, c, b))
    V = raw / np.linalg.norm(raw, axis=1, keepdims=True)
    F = np.array(faces, dtype=np.int32)
    assert F.shape == (20, 3)
    return V, F


def _normalize_rows(x: np.ndarray) -> np.ndarray:
    with np.errstate(invalid="ignore", divide="ignore"):
        return x / np.sqrt(np.sum(x * x, axis=-1, keepdims=True))


def _refine_face_grid(A: np.ndarray, B: np.ndarray, C: np.ndarray, n: int) -> np.ndarray:
    """Positions P[i, j] (i + j <= 2^n) of one icosahedron face after n rounds
    of 1-to-4 midpoint subdivision, each new midpoint projected to the unit
    sphere.  P[i, 0] runs A->B, P[0, j] runs A->C.  A point on a shared
    icosahedron edge only depends on that edge's end points, so both faces
    that share the edge compute bit-identical positions."""
    P = np.zeros((2, 2, 3))
    P[0, 0], P[1, 0], P[0, 1] = A, B, C
    for _ in range(n):
        M = P.shape[0] - 1
        Q = np.zeros((2 * M + 1, 2 * M + 1, 3))
        Q[0::2, 0::2] = P
        Q[1::2, 0::2] = _normalize_rows(P[:-1, :] + P[1:, :])          # odd i, even j
        Q[0::2, 1::2] = _normalize_rows(P[:, :-1] + P[:, 1:])          # even i, odd j
        Q[1::2, 1::2] = _normalize_rows(P[:-1, 1:] + P[1:, :-1])       # odd i, odd j
        P = Q
    return P


@dataclass
class Mesh:
    V: np.ndarray            # float64 [nv, 3]
    F: np.ndarray            # int32 [nf, 3], counter-clockwise seen from outside
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nv(self) -> int:
        return int(self.V.shape[0])

    @property
    def nf(self) -> int:
        return int(self.F.shape[0])


def icosphere(level: int) -> Mesh:
    """Unit icosphere after ``level`` rounds of midpoint subdivision with
    projection (V = 10*4^n + 2, E = 30*4^n, F = 20*4^n).

    Vertex numbering: the 12 icosahedron vertices first, then the interior
    points of the 30 icosahedron edges (edges sorted by (min, max), points
    from the min end), then the interior points of each icosahedron face in
    row-major (i, j) order.  Vertex 0 is an icosahedron vertex."""
    V0, F0 = icosahedron()
    N = 1 << level
    nv = 10 * N * N + 2
    edges = sorted({(min(a, b), max(a, b)) for f in F0 for a, b in ((f[0], f[1]), (f[1], f[2]), (f[2], f[0]))})
    eidx = {e: k for k, e in enumerate(edges)}
    assert len(edges) == 30
    ne_int = N - 1
    n_face_int = (N - 1) * (N - 2) // 2
    face_base = 12 + 30 * ne_int
    V = np.zeros((nv, 3))
    V[:12] = V0
    ii, jj = np.meshgrid(np.arange(N + 1), np.arange(N + 1), indexing="ij")
    valid = ii + jj <= N
    faces_out = []
    # row-major numbering of interior points (i >= 1, j >= 1, i + j <= N - 1)
    interior = (ii >= 1) & (jj >= 1) & (ii + jj <= N - 1)
    int_rank = np.cumsum(interior.ravel()).reshape(ii.shape) - 1

    def edge_ids(a, b, t):
        """global ids of points at parameter t (0..N) from a towards b."""
        t = np.asarray(t)
        lo, hi = min(a, b), max(a, b)
        s = t if a == lo else N - t
        out = 12 + eidx[(lo, hi)] * ne_int + (s - 1)
        out = np.where(s == 0, lo, out)
        out = np.where(s == N, hi, out)
        return out

    for f, (a, b, c) in enumerate(F0):
        P = _refine_face_grid(V0[a], V0[b], V0[c], level)
        gid = np.full((N + 1, N + 1), -1, dtype=np.int64)
        gid[interior] = face_base + f * n_face_int + int_rank[interior]
        gid[:, 0] = edge_ids(a, b, np.arange(N + 1))           # A->B
        gid[0, :] = edge_ids(a, c, np.arange(N + 1))           # A->C
        hyp_j = np.arange(N + 1)
        gid[N - hyp_j, hyp_j] = edge_ids(b, c, hyp_j)          # B->C
        V[gid[valid]] = P[valid]
        # up triangles (i,j),(i+1,j),(i,j+1); down (i+1,j),(i+1,j+1),(i,j+1)
        up = ii + jj <= N - 1
        iu, ju = ii[up], jj[up]
        faces_out.append(np.stack([gid[iu, ju], gid[iu + 1, ju], gid[iu, ju + 1]], axis=1))
        dn = ii + jj <= N - 2
        idn, jdn = ii[dn], jj[dn]
        faces_out.append(np.stack([gid[idn + 1, jdn], gid[idn + 1, jdn + 1], gid[idn, jdn + 1]], axis=1))
    F = np.concatenate(faces_out).astype(np.int32)
    assert F.shape[0] == 20 * N * N
    return Mesh(V=V, F=F, name=f"icosphere{level}", meta={"level": level})


def vertex_adjacency(nv: int, F: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """CSR one-ring of each vertex (neighbours in ascending order); used only
    to smooth the synthetic noise field."""
    import scipy.sparse as sp
    F = F.astype(np.int64)
    a = np.concatenate([F[:, 0], F[:, 1], F[:, 2], F[:, 1], F[:, 2], F[:, 0]])
    b = np.concatenate([F[:, 1], F[:, 2], F[:, 0], F[:, 0], F[:, 1], F[:, 2]])
    A = sp.csr_matrix((np.ones(a.size, np.int8), (a, b)), shape=(nv, nv))
    A.sum_duplicates()
    A.sort_indices()
    return A.indptr.astype(np.int64), A.indices.astype(np.int64)


def noisy_icosphere(level: int, seed: int, amplitude: float = 0.02, smooth_rounds: int = 3) -> Mesh:
    """Icosphere with radial noise r = 1 + amplitude * n, where n is a
    per-vertex standard normal field averaged ``smooth_rounds`` times over
    each vertex's closed one-ring (the vertex and its neighbours)."""
    import scipy.sparse as sp
    m = icosphere(level)
    rng = rng_for(seed)
    n = normal(rng, m.nv)
    rowptr, col = vertex_adjacency(m.nv, m.F)
    deg = np.diff(rowptr)
    # closed one-ring sum as a sparse matrix (adjacency + identity)
    A = sp.csr_matrix((np.ones(col.size), col, rowptr), shape=(m.nv, m.nv)) + sp.identity(m.nv, format="csr")
    for _ in range(smooth_rounds):
        n = (A @ n) / (deg + 1.0)
    r = 1.0 + amplitude * n
    m.V = m.V * r[:, None]
    m.name = f"noisy_icosphere{level}"
    m.meta.update({"seed": seed, "amplitude": amplitude, "smooth_rounds": smooth_rounds})
    return m


def sinusoid_icosphere(level: int, seed: int, terms: int = 8, amplitude: float = 0.05) -> Mesh:
    """Icosphere displaced radially by r = 1 + sum_j amplitude *
    sin(f_j (a_j . p) + phi_j) with a_j a uniform unit vector, f_j uniform in
    {1, 2, 3, 4} and phi_j uniform in [0, 2 pi)."""
    m = icosphere(level)
    rng = rng_for(seed)
    r = np.ones(m.nv)
    for _ in range(terms):
        a = normal(rng, 3)
        a /= np.linalg.norm(a)
        f = 1 + int(rng.random() * 4.0)
        ph = 2.0 * math.pi * rng.random()
        r += amplitude * np.sin(f * (m.V @ a) + ph)
    m.V = m.V * r[:, None]
    m.name = f"sinusoid_icosphere{level}"
    m.meta.update({"seed": seed, "terms": terms, "amplitude": amplitude})
    return m


# --------------------------------------------------------------------------
# Flat grids
# --------------------------------------------------------------------------

def jittered_grid(N: int, seed: int | None, jitter: float = 0.2) -> Mesh:
    """N x N vertex grid on [0, 1]^2 (h = 1 / (N - 1), z = 0), vertex
    (i, j) = index i*N + j at (x, y) = (j h, i h).  Cell (i, j) is split along
    the diagonal (i, j)-(i+1, j+1) when i + j is even and along
    (i, j+1)-(i+1, j) otherwise (alternating diagonals).  Interior vertices
    move by independent uniform offsets in [-jitter h, jitter h) in x and y;
    boundary vertices stay put.  ``seed=None`` gives the regular grid."""
    h = 1.0 / (N - 1)
    i, j = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    V = np.zeros((N * N, 3))
    V[:, 0] = (j * h).ravel()
    V[:, 1] = (i * h).ravel()
    if seed is not None and jitter > 0:
        rng = rng_for(seed)
        d = (rng.random((N * N, 2)) * 2.0 - 1.0) * (jitter * h)
        inner = ((i > 0) & (i < N - 1) & (j > 0) & (j < N - 1)).ravel()
        V[inner, 0] += d[inner, 0]
        V[inner, 1] += d[inner, 1]
    ci, cj = np.meshgrid(np.arange(N - 1), np.arange(N - 1), indexing="ij")
    ci, cj = ci.ravel(), cj.ravel()
    v00 = ci * N + cj
    v01 = v00 + 1
    v10 = v00 + N
    v11 = v10 + 1
    even = (ci + cj) % 2 == 0
    t1 = np.where(even[:, None], np.stack([v00, v01, v11], 1), np.stack([v00, v01, v10], 1))
    t2 = np.where(even[:, None], np.stack([v00, v11, v10], 1), np.stack([v01, v11, v10], 1))
    F = np.stack([t1, t2], axis=1).reshape(-1, 3).astype(np.int32)
    return Mesh(V=V, F=F, name=f"grid{N}", meta={"N": N, "seed": seed, "jitter": jitter})


def torus(nu: int, nw: int, seed: int | None = None, R: float = 1.0, r: float = 0.4, jitter: float = 0.2) -> Mesh:
    """Closed torus of genus 1: vertex (i, j) = index i*nw + j at major angle
    a = 2 pi i / nu and minor angle b = 2 pi j / nw, p = ((R + r cos b) cos a,
    (R + r cos b) sin a, r sin b).  Each cell (i, j)-(i+1, j+1) (indices
    wrapping around) is split along one of its diagonals by the parity of
    i + j, faces counter-clockwise seen from outside.  With a seed both
    angles move by independent uniform offsets in [-jitter, jitter) of a
    step."""
    i, j = np.meshgrid(np.arange(nu), np.arange(nw), indexing="ij")
    a = 2.0 * np.pi * i.ravel() / nu
    b = 2.0 * np.pi * j.ravel() / nw
    if seed is not None and jitter > 0:
        rng = rng_for(seed)
        d = (rng.random((nu * nw, 2)) * 2.0 - 1.0) * jitter
        a = a + d[:, 0] * (2.0 * np.pi / nu)
        b = b + d[:, 1] * (2.0 * np.pi / nw)
    V = np.stack([(R + r * np.cos(b)) * np.cos(a), (R + r * np.cos(b)) * np.sin(a), r * np.sin(b)], axis=1)
    ci, cj = np.meshgrid(np.arange(nu), np.arange(nw), indexing="ij")
    ci, cj = ci.ravel(), cj.ravel()
    v00 = ci * nw + cj
    v10 = ((ci + 1) % nu) * nw + cj
    v01 = ci * nw + (cj + 1) % nw
    v11 = ((ci + 1) % nu) * nw + (cj + 1) % nw
    even = (ci + cj) % 2 == 0
    t1 = np.where(even[:, None], np.stack([v00, v10, v11], 1), np.stack([v00, v10, v01], 1))
    t2 = np.where(even[:, None], np.stack([v00, v11, v01], 1), np.stack([v10, v11, v01], 1))
    F = np.stack([t1, t2], axis=1).reshape(-1, 3).astype(np.int32)
    return Mesh(V=V, F=F, name=f"torus{nu}x{nw}", meta={"nu": nu, "nw": nw, "seed": seed})


def strip_grid(nx: int, ny: int) -> Mesh:
    """Regular ny x nx vertex grid with unit spacing (vertex (i, j) = index
    i*nx + j at (x, y) = (j, i)), cells split by the same alternating
    diagonals as ``jittered_grid``.  With the first row as sources every
    breadth-first set is a row of about nx vertices: a long, shallow
    front for exercising wide sets."""
    i, j = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    V = np.zeros((nx * ny, 3))
    V[:, 0] = j.ravel().astype(np.float64)
    V[:, 1] = i.ravel().astype(np.float64)
    ci, cj = np.meshgrid(np.arange(ny - 1), np.arange(nx - 1), indexing="ij")
    ci, cj = ci.ravel(), cj.ravel()
    v00 = ci * nx + cj
    v01 = v00 + 1
    v10 = v00 + nx
    v11 = v10 + 1
    even = (ci + cj) % 2 == 0
    t1 = np.where(even[:, None], np.stack([v00, v01, v11], 1), np.stack([v00, v01, v10], 1))
    t2 = np.where(even[:, None], np.stack([v00, v11, v10], 1), np.stack([v01, v11, v10], 1))
    F = np.stack([t1, t2], axis=1).reshape(-1, 3).astype(np.int32)
    return Mesh(V=V, F=F, name=f"strip{nx}x{ny}", meta={"nx": nx, "ny": ny})


def mixed_density_strip(nx: int, ny: int, dense: int = 3) -> Mesh:
    """Strip of ny rows (y = row index, z = 0): even rows hold nx vertices
    at unit spacing, odd rows dense * (nx - 1) + 1 vertices at spacing
    1 / dense; consecutive rows are zipped into triangles from left to right
    (the next triangle takes the lower row's next vertex while it lies no
    further right than the upper row's next).  Interior sparse-row vertices
    have 10 neighbours with dense = 3, so with the first row as sources whole
    breadth-first sets consist of long rows."""
    xs_rows, base = [], 0
    V = []
    for r in range(ny):
        xs = np.arange(nx, dtype=np.float64) if r % 2 == 0 else np.arange(dense * (nx - 1) + 1) / dense
        xs_rows.append((xs, base))
        V.append(np.stack([xs, np.full(xs.size, float(r)), np.zeros(xs.size)], axis=1))
        base += xs.size
    F = []
    for r in range(ny - 1):
        (xb, b0), (xt, t0) = xs_rows[r], xs_rows[r + 1]
        i = j = 0
        while i < xb.size - 1 or j < xt.size - 1:
            if j == xt.size - 1 or (i < xb.size - 1 and xb[i + 1] <= xt[j + 1]):
                F.append((b0 + i, b0 + i + 1, t0 + j))
                i += 1
            else:
                F.append((b0 + i, t0 + j + 1, t0 + j))
                j += 1
    return Mesh(V=np.concatenate(V), F=np.asarray(F, dtype=np.int32), name=f"mixedstrip{nx}x{ny}",
                meta={"nx": nx, "ny": ny, "dense": dense})


def jittered_delaunay(N: int, seed: int, jitter: float = 0.45) -> Mesh:
    """Delaunay triangulation (scipy.spatial) of an N x N lattice on the unit
    square (spacing h = 1 / (N - 1)), z = 0, faces turned counter-clockwise.
    Inner points move by independent uniform offsets in [-jitter h, jitter h)
    in x and y; boundary points stay put.  Unlike the fixed diagonals of
    ``jittered_grid`` the connectivity follows the points: vertex degrees
    vary from 3 to 10 around a mean of 6 (with jitter 0.45 no angle is below
    about 4 degrees)."""
    from scipy.spatial import Delaunay
    rng = rng_for(seed)
    h = 1.0 / (N - 1)
    i, j = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    P = np.stack([(j * h).ravel(), (i * h).ravel()], axis=1)
    inner = ((i > 0) & (i < N - 1) & (j > 0) & (j < N - 1)).ravel()
    P[inner] += (rng.random((int(inner.sum()), 2)) * 2.0 - 1.0) * (jitter * h)
    F = Delaunay(P).simplices.astype(np.int32)
    a, b, c = P[F[:, 0]], P[F[:, 1]], P[F[:, 2]]
    cw = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0]) < 0
    F[cw] = F[cw][:, [0, 2, 1]]
    V = np.zeros((N * N, 3))
    V[:, :2] = P
    return Mesh(V=V, F=np.ascontiguousarray(F), name=f"delaunay{N}", meta={"N": N, "seed": seed, "jitter": jitter})


# --------------------------------------------------------------------------
# Source sets
# --------------------------------------------------------------------------

def random_sources(rng: np.random.Generator, nv: int, kmin: int, kmax: int) -> np.ndarray:
    """A sorted set of uniformly many (kmin..kmax) distinct uniform vertices."""
    k = kmin + int(rng.random() * (kmax - kmin + 1))
    out: list[int] = []
    while len(out) < k:
        v = int(rng.random() * nv)
        if v not in out:
            out.append(v)
    return np.array(sorted(out), dtype=np.int32)


# --------------------------------------------------------------------------
# The five workloads
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    mesh: Mesh
    sources: list            # list of int32 arrays, one per query
    m: float                 # diffusion time factor, t = m * hbar^2
    gs_face: int
    gs_edge: int
    admm_iters: int = 10
    forms: tuple = ("face", "edge")


def workload_c1() -> Workload:
    """Unit icosphere level 4, source vertex 0, t = hbar^2; 200 sweeps."""
    return Workload("ico4", icosphere(4), [np.array([0], np.int32)], m=1.0, gs_face=200, gs_edge=200)


def workload_c2(N: int = 1025) -> Workload:
    """Jittered 1025^2 grid with one uniform random source; sweep counts of
    Table 1's 1M-vertex row (300 face form, 200 edge form)."""
    seed = config_seed(2)
    mesh = jittered_grid(N, seed)
    rng = rng_for(seed + 500)
    src = random_sources(rng, mesh.nv, 1, 1)
    return Workload(f"grid{N}", mesh, [src], m=1.0, gs_face=300, gs_edge=200)


def workload_c3(level: int = 10, K: int = 64) -> Workload:
    """Noisy icosphere level 10, K source sets of 1..8 vertices; sweep counts
    of Table 1's 9.9M-vertex row (1200 face form, 700 edge form)."""
    seed = config_seed(3)
    mesh = noisy_icosphere(level, seed)
    rng = rng_for(seed + 500)
    srcs = [random_sources(rng, mesh.nv, 1, 8) for _ in range(K)]
    return Workload(f"noisy_ico{level}", mesh, srcs, m=1.0, gs_face=1200, gs_edge=700)


def workload_c5(level: int = 12) -> Workload:
    """Sinusoid-displaced icosphere level 12, one uniform source, edge form,
    m = 10 and 4000 sweeps (Table 1's edge row for the largest models)."""
    seed = config_seed(5)
    mesh = sinusoid_icosphere(level, seed)
    rng = rng_for(seed + 500)
    src = random_sources(rng, mesh.nv, 1, 1)
    return Workload(f"sinusoid_ico{level}", mesh, [src], m=10.0, gs_face=2000, gs_edge=4000, forms=("edge",))


def serving_sweeps(mesh: Mesh) -> int:
    """Sweep count of a serving mesh: about twice its breadth-first depth, the
    count at which breadth-first Gauss-Seidel has converged (grid side N:
    depth <= N; icosphere level n: depth <= 3 * 2^n)."""
    if "N" in mesh.meta:
        return 2 * int(mesh.meta["N"])
    return 6 * (1 << int(mesh.meta["level"]))


def serving_request(k: int, mesh: Mesh) -> np.ndarray:
    """The seeded request (1..16 uniform sources) whose oracle distances are
    stored for serving mesh k."""
    return random_sources(rng_for(config_seed(4, 300 + k)), mesh.nv, 1, 16)


def serving_meshes() -> list[Mesh]:
    """The ten meshes of the serving stream: jittered grids of side 101, 257,
    513, 1025, 2000 and noisy icospheres of level 5..9."""
    out = [jittered_grid(n, config_seed(4, k)) for k, n in enumerate((101, 257, 513, 1025, 2000))]
    out += [noisy_icosphere(lv, config_seed(4, 5 + k)) for k, lv in enumerate((5, 6, 7, 8, 9))]
    return out
