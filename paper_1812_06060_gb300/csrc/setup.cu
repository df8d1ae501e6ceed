// Per-mesh setup on the device (the "initialization of data structures" of
// Sec. 6.4): one-ring CSR, edge ids, orientation signs (Sec. 4.1), vertex and
// face areas and cotangent weights (Sec. 3.1), gradient operators
// (eq. HeatDiffusionNormalization), mean edge length (eq. DiffusionTime).
// Geometry is computed in FP64; per-face operators used by the FP32 stages
// are stored rounded to FP32.
#include "internal.cuh"

namespace gh {

namespace {

__global__ void k_check_faces(const int32_t *__restrict__ F, int64_t nf, int64_t nv, int *err) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int a = F[3 * f], b = F[3 * f + 1], c = F[3 * f + 2];
    bool bad = a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv || a == b || b == c || a == c;
    if (bad) atomicCAS(err, DEV_OK, DEV_EINVAL);
}

// every face adds, to the row of each corner, the two other corners
__global__ void k_count_dup(const int32_t *__restrict__ F, int64_t nf, int32_t *cnt) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    for (int k = 0; k < 3; ++k) atomicAdd(&cnt[F[3 * f + k]], 2);
}

__global__ void k_fill_dup(const int32_t *__restrict__ F, int64_t nf, const int32_t *__restrict__ dptr,
                           int32_t *fill, int32_t *dcol) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    for (int k = 0; k < 3; ++k) {
        int v = F[3 * f + k];
        int at = dptr[v] + atomicAdd(&fill[v], 2);
        dcol[at] = F[3 * f + (k + 1) % 3];
        dcol[at + 1] = F[3 * f + (k + 2) % 3];
    }
}

// sort each duplicated row, count distinct neighbours (deg) and those above
// the row's vertex (up); a neighbour listed more than twice means an edge in
// more than two faces
__global__ void k_sort_rows(const int32_t *__restrict__ dptr, int32_t *dcol, int64_t nv, int32_t *deg, int32_t *up,
                            int *err) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    int b = dptr[v], e = dptr[v + 1];
    for (int i = b + 1; i < e; ++i) {
        int x = dcol[i], j = i - 1;
        while (j >= b && dcol[j] > x) { dcol[j + 1] = dcol[j]; --j; }
        dcol[j + 1] = x;
    }
    int nd = 0, nu = 0, run = 0;
    for (int i = b; i < e; ++i) {
        if (i == b || dcol[i] != dcol[i - 1]) {
            ++nd;
            if (dcol[i] > v) ++nu;
            run = 1;
        } else if (++run > 2) {
            atomicCAS(err, DEV_OK, DEV_ENONMANIFOLD);
        }
    }
    deg[v] = nd;
    up[v] = nu;
}

__global__ void k_compact_rows(const int32_t *__restrict__ dptr, const int32_t *__restrict__ dcol, int64_t nv,
                               const int32_t *__restrict__ rowptr, int32_t *col) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    int o = rowptr[v];
    for (int i = dptr[v]; i < dptr[v + 1]; ++i)
        if (i == dptr[v] || dcol[i] != dcol[i - 1]) col[o++] = dcol[i];
}

__device__ __forceinline__ int find_in_row(const int32_t *__restrict__ col, int b, int e, int x) {
    while (b < e) {
        int m = (b + e) >> 1;
        int c = col[m];
        if (c == x) return m;
        if (c < x) b = m + 1; else e = m;
    }
    return -1;
}

// edge id of (v, w), v < w: eoff[v] + rank of w among the row's entries above v
__global__ void k_edges(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col, int64_t nv,
                        const int32_t *__restrict__ up, const int32_t *__restrict__ eoff, int32_t *col_edge,
                        int32_t *edges) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    int b = rowptr[v], e = rowptr[v + 1];
    int first_up = e - up[v];
    for (int j = b; j < e; ++j) {
        int w = col[j];
        int id;
        if (w > v) {
            id = eoff[v] + (j - first_up);
            edges[2 * id] = (int)v;
            edges[2 * id + 1] = w;
        } else {
            int jw = find_in_row(col, rowptr[w], rowptr[w + 1], (int)v);
            if (jw < 0) { col_edge[j] = 0; continue; }  // rows are symmetric by construction
            id = eoff[w] + (jw - (rowptr[w + 1] - up[w]));
        }
        col_edge[j] = id;
    }
}

// local edge k of face (a, b, c) is opposite corner k; the loop halfedge is
// F[k+1] -> F[k+2]; the orientation halfedge runs min -> max, so the sign is
// +1 when the loop runs upwards
__global__ void k_face_edges(const int32_t *__restrict__ F, int64_t nf, const int32_t *__restrict__ rowptr,
                             const int32_t *__restrict__ col, const int32_t *__restrict__ col_edge,
                             int32_t *face_edge, int8_t *face_sign, int32_t *ecnt, int32_t *etmp, int *err) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    for (int k = 0; k < 3; ++k) {
        int a = F[3 * f + (k + 1) % 3], b = F[3 * f + (k + 2) % 3];
        int j = find_in_row(col, rowptr[a], rowptr[a + 1], b);
        if (j < 0) { atomicCAS(err, DEV_OK, DEV_ENONMANIFOLD); return; }  // rows are symmetric by construction
        int e = col_edge[j];
        face_edge[3 * f + k] = e;
        face_sign[3 * f + k] = (a < b) ? 1 : -1;
        int s = atomicAdd(&ecnt[e], 1);
        if (s < 2) etmp[2 * e + s] = (int)(f << 2) | k;
        else atomicCAS(err, DEV_OK, DEV_ENONMANIFOLD);
    }
}

__global__ void k_edge_faces(const int32_t *__restrict__ ecnt, const int32_t *__restrict__ etmp, int64_t ne,
                             const int8_t *__restrict__ face_sign, int32_t *edge_face, int32_t *edge_slot,
                             int32_t *twin, int *err) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    int n = ecnt[e];
    if (n < 1 || n > 2) { atomicCAS(err, DEV_OK, DEV_ENONMANIFOLD); return; }
    int x = etmp[2 * e], y = (n == 2) ? etmp[2 * e + 1] : -1;
    if (n == 2 && (y >> 2) < (x >> 2)) { int t = x; x = y; y = t; }
    edge_face[2 * e] = x >> 2;
    edge_slot[2 * e] = x & 3;
    edge_face[2 * e + 1] = (n == 2) ? (y >> 2) : -1;
    edge_slot[2 * e + 1] = (n == 2) ? (y & 3) : -1;
    if (n == 2) {
        // face_sign and twin are indexed by 3f + k
        int ix = 3 * (x >> 2) + (x & 3), iy = 3 * (y >> 2) + (y & 3);
        if (face_sign[ix] == face_sign[iy]) atomicCAS(err, DEV_OK, DEV_ENONMANIFOLD);
        twin[ix] = y;
        twin[iy] = x;
    } else {
        twin[3 * (x >> 2) + (x & 3)] = -1;
    }
}

__device__ __forceinline__ void ld3(const double *P, int v, double *o) {
    o[0] = P[3 * v]; o[1] = P[3 * v + 1]; o[2] = P[3 * v + 2];
}

// per face, FP64: area, cot of each corner, gradient of each corner's hat
// function (N x e_k)/(2A) with e_k the edge opposite corner k (counter-clockwise)
__global__ void k_face_geom(const double *__restrict__ P, const int32_t *__restrict__ F, int64_t nf, double *Af,
                            float *Aff, double *cot, float *gradop) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    double p[3][3];
    for (int k = 0; k < 3; ++k) ld3(P, F[3 * f + k], p[k]);
    double u[3], w[3], n[3];
    for (int i = 0; i < 3; ++i) { u[i] = p[1][i] - p[0][i]; w[i] = p[2][i] - p[0][i]; }
    n[0] = u[1] * w[2] - u[2] * w[1];
    n[1] = u[2] * w[0] - u[0] * w[2];
    n[2] = u[0] * w[1] - u[1] * w[0];
    double twoA = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    Af[f] = 0.5 * twoA;
    Aff[f] = (float)(0.5 * twoA);
    double N[3] = {n[0] / twoA, n[1] / twoA, n[2] / twoA};
    for (int k = 0; k < 3; ++k) {
        const double *a = p[k], *b = p[(k + 1) % 3], *c = p[(k + 2) % 3];
        double x[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        double y[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        double cr[3] = {x[1] * y[2] - x[2] * y[1], x[2] * y[0] - x[0] * y[2], x[0] * y[1] - x[1] * y[0]};
        cot[3 * f + k] = (x[0] * y[0] + x[1] * y[1] + x[2] * y[2]) /
                         sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        double e[3] = {c[0] - b[0], c[1] - b[1], c[2] - b[2]};
        double g[3] = {N[1] * e[2] - N[2] * e[1], N[2] * e[0] - N[0] * e[2], N[0] * e[1] - N[1] * e[0]};
        for (int i = 0; i < 3; ++i) gradop[9 * f + 3 * k + i] = (float)(g[i] / twoA);
    }
}

// per edge: theta_e = 1/2 sum cot(opposite corner), the orientation-halfedge
// vector (max - min) and its length
__global__ void k_edge_geom(const double *__restrict__ P, const int32_t *__restrict__ edges, int64_t ne,
                            const int32_t *__restrict__ edge_face, const int32_t *__restrict__ edge_slot,
                            const double *__restrict__ cot, double *theta, float *ev, double *elen) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    double th = 0.0;
    for (int j = 0; j < 2; ++j) {
        int f = edge_face[2 * e + j];
        if (f >= 0) th += 0.5 * cot[3 * f + edge_slot[2 * e + j]];
    }
    theta[e] = th;
    double a[3], b[3];
    ld3(P, edges[2 * e], a);
    ld3(P, edges[2 * e + 1], b);
    double d[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    ev[3 * e] = (float)d[0];
    ev[3 * e + 1] = (float)d[1];
    ev[3 * e + 2] = (float)d[2];
    elen[e] = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
}

// per face of an intrinsic triangulation, from the lengths L[3f+k] of the
// edge opposite corner k: area, corner cotangents (l1^2 + l2^2 - l_opp^2)/(4A),
// and in the face's own frame (corner 0 at the origin, corner 1 on the +x
// axis, corner 2 above) the hat-function gradients (N x e_k)/(2A), N = +z,
// and the slot edge vectors oriented from the lower to the higher vertex
__global__ void k_face_geom_len(const int32_t *__restrict__ F, const double *__restrict__ L, int64_t nf, double *Af,
                                float *Aff, double *cot, float *gradop, double *gradop64, double *evf64,
                                float *evf32) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const double l[3] = {L[3 * f], L[3 * f + 1], L[3 * f + 2]};
    const double A = heron_d(l[0], l[1], l[2]);
    Af[f] = A;
    Aff[f] = (float)A;
    const double x2 = (l[2] * l[2] + l[1] * l[1] - l[0] * l[0]) / (2.0 * l[2]);
    const double y2s = l[1] * l[1] - x2 * x2;
    const double q[3][2] = {{0.0, 0.0}, {l[2], 0.0}, {x2, sqrt(y2s > 0.0 ? y2s : 0.0)}};
    for (int k = 0; k < 3; ++k) {
        const int i = (k + 1) % 3, j = (k + 2) % 3;
        cot[3 * f + k] = (l[i] * l[i] + l[j] * l[j] - l[k] * l[k]) / (4.0 * A);
        const double e[2] = {q[j][0] - q[i][0], q[j][1] - q[i][1]};
        const double g[2] = {-e[1] / (2.0 * A), e[0] / (2.0 * A)};
        gradop64[9 * f + 3 * k] = g[0];
        gradop64[9 * f + 3 * k + 1] = g[1];
        gradop64[9 * f + 3 * k + 2] = 0.0;
        gradop[9 * f + 3 * k] = (float)g[0];
        gradop[9 * f + 3 * k + 1] = (float)g[1];
        gradop[9 * f + 3 * k + 2] = 0.0f;
        const bool fwd = F[3 * f + i] < F[3 * f + j];
        const int t = fwd ? i : j, h = fwd ? j : i;
        const double v[2] = {q[h][0] - q[t][0], q[h][1] - q[t][1]};
        evf64[9 * f + 3 * k] = v[0];
        evf64[9 * f + 3 * k + 1] = v[1];
        evf64[9 * f + 3 * k + 2] = 0.0;
        evf32[9 * f + 3 * k] = (float)v[0];
        evf32[9 * f + 3 * k + 1] = (float)v[1];
        evf32[9 * f + 3 * k + 2] = 0.0f;
    }
}

// per edge of an intrinsic triangulation: theta_e = 1/2 sum cot(opposite
// corner), the length (from its first face) and no ambient edge vector
__global__ void k_edge_geom_len(int64_t ne, const int32_t *__restrict__ edge_face, const int32_t *__restrict__ edge_slot,
                                const double *__restrict__ cot, const double *__restrict__ L, double *theta, float *ev,
                                double *elen) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    double th = 0.0;
    for (int j = 0; j < 2; ++j) {
        int f = edge_face[2 * e + j];
        if (f >= 0) th += 0.5 * cot[3 * f + edge_slot[2 * e + j]];
    }
    theta[e] = th;
    elen[e] = L[3 * edge_face[2 * e] + edge_slot[2 * e]];
    ev[3 * e] = ev[3 * e + 1] = ev[3 * e + 2] = 0.0f;
}

// A_v = 1/3 of the incident face area.  Every face at v has exactly two edges
// at v, so A_v = 1/6 sum over v's edges of the areas of their faces: a
// deterministic gather.
__global__ void k_vertex_area(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col_edge, int64_t nv,
                              const int32_t *__restrict__ edge_face, const double *__restrict__ Af, double *Av) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    double s = 0.0;
    for (int j = rowptr[v]; j < rowptr[v + 1]; ++j) {
        int e = col_edge[j];
        for (int k = 0; k < 2; ++k) {
            int f = edge_face[2 * e + k];
            if (f >= 0) s += Af[f];
        }
    }
    Av[v] = s / 6.0;
}

// deterministic sum: each block reduces a fixed chunk in a fixed tree order
constexpr int RB = 256;
__global__ void k_sum_partial(const double *__restrict__ x, int64_t n, int64_t per_block, double *part) {
    __shared__ double s[RB];
    int64_t b0 = (int64_t)blockIdx.x * per_block;
    int64_t b1 = min(n, b0 + per_block);
    double acc = 0.0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += RB) acc += x[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = RB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

}  // namespace

// mean of x[0..n) with a fixed summation order
static gh_status det_mean(Ctx *c, const double *x, int64_t n, double *out) {
    cudaStream_t st = c->stream;
    const int64_t per_block = 65536;
    int64_t nb = (n + per_block - 1) / per_block;
    DBuf part;
    gh_status s;
    if ((s = dalloc(c, part, sizeof(double) * (nb + 1))) != GH_OK) return s;
    k_sum_partial<<<(unsigned)nb, RB, 0, st>>>(x, n, per_block, ptr<double>(part)); ++c->launches;
    k_sum_partial<<<1, RB, 0, st>>>(ptr<double>(part), nb, nb, ptr<double>(part) + nb); ++c->launches;
    double total = 0.0;
    GH_CUDA(cudaMemcpyAsync(&total, ptr<double>(part) + nb, sizeof(double), cudaMemcpyDeviceToHost, st));
    GH_CUDA(cudaStreamSynchronize(st));
    dfree(c, part);
    *out = total / (double)n;
    return GH_OK;
}

gh_status build_mesh(Ctx *c, DevMesh &m, const double *V_dev, const int32_t *F_dev) {
    cudaStream_t st = c->stream;
    const int T = 256;
    int64_t nv = m.nv, nf = m.nf;
    int *err = dev_status(c);
    GH_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    gh_status s;
    if ((s = dalloc(c, m.P, sizeof(double) * 3 * nv)) != GH_OK) return s;
    if ((s = dalloc(c, m.F, sizeof(int32_t) * 3 * nf)) != GH_OK) return s;
    GH_CUDA(cudaMemcpyAsync(m.P.p, V_dev, sizeof(double) * 3 * nv, cudaMemcpyDefault, st));
    GH_CUDA(cudaMemcpyAsync(m.F.p, F_dev, sizeof(int32_t) * 3 * nf, cudaMemcpyDefault, st));
    k_check_faces<<<blocks_for(nf, T), T, 0, st>>>(ptr<int32_t>(m.F), nf, nv, err); ++c->launches;
    if ((s = check_status(c, "face indices")) != GH_OK) return s;
    if ((s = build_connectivity(c, m)) != GH_OK) return s;
    return build_geometry_positions(c, m);
}

gh_status build_connectivity(Ctx *c, DevMesh &m) {
    cudaStream_t st = c->stream;
    const int T = 256;
    int64_t nv = m.nv, nf = m.nf;
    int *err = dev_status(c);
    GH_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    gh_status s;
    const int32_t *F = ptr<int32_t>(m.F);

    // duplicated rows -> sorted distinct rows
    DBuf cnt, dptr, fill, dcol, deg, up, eoff;
    auto cleanup = [&]() { dfree(c, cnt); dfree(c, dptr); dfree(c, fill); dfree(c, dcol); dfree(c, deg);
                           dfree(c, up); dfree(c, eoff); };
    if ((s = dalloc(c, cnt, sizeof(int32_t) * nv)) != GH_OK) { cleanup(); return s; }
    if ((s = dalloc(c, dptr, sizeof(int32_t) * (nv + 1))) != GH_OK) { cleanup(); return s; }
    if ((s = dalloc(c, fill, sizeof(int32_t) * nv)) != GH_OK) { cleanup(); return s; }
    if ((s = dalloc(c, dcol, sizeof(int32_t) * 6 * nf)) != GH_OK) { cleanup(); return s; }
    if ((s = dalloc(c, deg, sizeof(int32_t) * nv)) != GH_OK) { cleanup(); return s; }
    if ((s = dalloc(c, up, sizeof(int32_t) * (nv + 1))) != GH_OK) { cleanup(); return s; }
    if ((s = dalloc(c, eoff, sizeof(int32_t) * (nv + 1))) != GH_OK) { cleanup(); return s; }
    GH_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * nv, st));
    GH_CUDA(cudaMemsetAsync(fill.p, 0, sizeof(int32_t) * nv, st));
    k_count_dup<<<blocks_for(nf, T), T, 0, st>>>(F, nf, ptr<int32_t>(cnt)); ++c->launches;
    if ((s = exclusive_scan_u32_dev(c, ptr<int32_t>(cnt), ptr<int32_t>(dptr), nv)) != GH_OK) { cleanup(); return s; }
    k_fill_dup<<<blocks_for(nf, T), T, 0, st>>>(F, nf, ptr<int32_t>(dptr), ptr<int32_t>(fill), ptr<int32_t>(dcol)); ++c->launches;
    k_sort_rows<<<blocks_for(nv, T), T, 0, st>>>(ptr<int32_t>(dptr), ptr<int32_t>(dcol), nv, ptr<int32_t>(deg),
                                                ptr<int32_t>(up), err); ++c->launches;
    if ((s = check_status(c, "one-ring rows")) != GH_OK) { cleanup(); return s; }
    if ((s = dalloc(c, m.rowptr, sizeof(int32_t) * (nv + 1))) != GH_OK) { cleanup(); return s; }
    int32_t nnz = 0, ne32 = 0;
    if ((s = exclusive_scan_i32(c, ptr<int32_t>(deg), ptr<int32_t>(m.rowptr), nv, &nnz)) != GH_OK) { cleanup(); return s; }
    if ((s = exclusive_scan_i32(c, ptr<int32_t>(up), ptr<int32_t>(eoff), nv, &ne32)) != GH_OK) { cleanup(); return s; }
    m.ne = ne32;
    int64_t ne = m.ne;
    if (nnz != 2 * ne32) { cleanup(); set_error("internal: one-ring is not symmetric"); return GH_ENONMANIFOLD; }
    if ((s = dalloc(c, m.col, sizeof(int32_t) * nnz)) != GH_OK) { cleanup(); return s; }
    if ((s = dalloc(c, m.col_edge, sizeof(int32_t) * nnz)) != GH_OK) { cleanup(); return s; }
    if ((s = dalloc(c, m.edges, sizeof(int32_t) * 2 * ne)) != GH_OK) { cleanup(); return s; }
    k_compact_rows<<<blocks_for(nv, T), T, 0, st>>>(ptr<int32_t>(dptr), ptr<int32_t>(dcol), nv,
                                                   ptr<int32_t>(m.rowptr), ptr<int32_t>(m.col)); ++c->launches;
    k_edges<<<blocks_for(nv, T), T, 0, st>>>(ptr<int32_t>(m.rowptr), ptr<int32_t>(m.col), nv, ptr<int32_t>(up),
                                            ptr<int32_t>(eoff), ptr<int32_t>(m.col_edge), ptr<int32_t>(m.edges)); ++c->launches;
    cleanup();

    // faces <-> edges
    DBuf ecnt, etmp;
    auto cleanup2 = [&]() { dfree(c, ecnt); dfree(c, etmp); };
    if ((s = dalloc(c, m.face_edge, sizeof(int32_t) * 3 * nf)) != GH_OK) return s;
    if ((s = dalloc(c, m.face_sign, sizeof(int8_t) * 3 * nf)) != GH_OK) return s;
    if ((s = dalloc(c, m.edge_face, sizeof(int32_t) * 2 * ne)) != GH_OK) return s;
    if ((s = dalloc(c, m.edge_slot, sizeof(int32_t) * 2 * ne)) != GH_OK) return s;
    if ((s = dalloc(c, m.twin, sizeof(int32_t) * 3 * nf)) != GH_OK) return s;
    if ((s = dalloc(c, ecnt, sizeof(int32_t) * ne)) != GH_OK) { cleanup2(); return s; }
    if ((s = dalloc(c, etmp, sizeof(int32_t) * 2 * ne)) != GH_OK) { cleanup2(); return s; }
    GH_CUDA(cudaMemsetAsync(ecnt.p, 0, sizeof(int32_t) * ne, st));
    k_face_edges<<<blocks_for(nf, T), T, 0, st>>>(F, nf, ptr<int32_t>(m.rowptr), ptr<int32_t>(m.col),
                                                 ptr<int32_t>(m.col_edge), ptr<int32_t>(m.face_edge),
                                                 ptr<int8_t>(m.face_sign), ptr<int32_t>(ecnt), ptr<int32_t>(etmp), err); ++c->launches;
    k_edge_faces<<<blocks_for(ne, T), T, 0, st>>>(ptr<int32_t>(ecnt), ptr<int32_t>(etmp), ne, ptr<int8_t>(m.face_sign),
                                                 ptr<int32_t>(m.edge_face), ptr<int32_t>(m.edge_slot),
                                                 ptr<int32_t>(m.twin), err); ++c->launches;
    cleanup2();
    return check_status(c, "edge-face incidence");
}

gh_status build_geometry_positions(Ctx *c, DevMesh &m) {
    cudaStream_t st = c->stream;
    const int T = 256;
    const int64_t nv = m.nv, nf = m.nf, ne = m.ne;
    const int32_t *F = ptr<int32_t>(m.F);
    gh_status s;
    // geometry, FP64
    DBuf cot;
    auto cleanup3 = [&]() { dfree(c, cot); };
    if ((s = dalloc(c, m.Af, sizeof(double) * nf)) != GH_OK) return s;
    if ((s = dalloc(c, m.Aff, sizeof(float) * nf)) != GH_OK) return s;
    if ((s = dalloc(c, m.Av, sizeof(double) * nv)) != GH_OK) return s;
    if ((s = dalloc(c, m.theta, sizeof(double) * ne)) != GH_OK) return s;
    if ((s = dalloc(c, m.ev, sizeof(float) * 3 * ne)) != GH_OK) return s;
    if ((s = dalloc(c, m.gradop, sizeof(float) * 9 * nf)) != GH_OK) return s;
    if ((s = dalloc(c, cot, sizeof(double) * 3 * nf)) != GH_OK) { cleanup3(); return s; }
    if ((s = dalloc(c, m.elen, sizeof(double) * ne)) != GH_OK) { cleanup3(); return s; }
    k_face_geom<<<blocks_for(nf, T), T, 0, st>>>(ptr<double>(m.P), F, nf, ptr<double>(m.Af), ptr<float>(m.Aff),
                                                ptr<double>(cot), ptr<float>(m.gradop)); ++c->launches;
    k_edge_geom<<<blocks_for(ne, T), T, 0, st>>>(ptr<double>(m.P), ptr<int32_t>(m.edges), ne, ptr<int32_t>(m.edge_face),
                                                ptr<int32_t>(m.edge_slot), ptr<double>(cot), ptr<double>(m.theta),
                                                ptr<float>(m.ev), ptr<double>(m.elen)); ++c->launches;
    k_vertex_area<<<blocks_for(nv, T), T, 0, st>>>(ptr<int32_t>(m.rowptr), ptr<int32_t>(m.col_edge), nv,
                                                  ptr<int32_t>(m.edge_face), ptr<double>(m.Af), ptr<double>(m.Av)); ++c->launches;
    // mean edge length: fixed chunks, fixed tree order, then one block
    cleanup3();
    if ((s = det_mean(c, ptr<double>(m.elen), ne, &m.hbar)) != GH_OK) return s;
    return check_status(c, "geometry");
}

}  // namespace gh

namespace gh {

gh_status build_geometry_lengths(Ctx *c, DevMesh &m, const double *L) {
    cudaStream_t st = c->stream;
    const int T = 256;
    const int64_t nv = m.nv, nf = m.nf, ne = m.ne;
    gh_status s;
    DBuf cot;
    if ((s = dalloc(c, m.Af, sizeof(double) * nf)) != GH_OK) return s;
    if ((s = dalloc(c, m.Aff, sizeof(float) * nf)) != GH_OK) return s;
    if ((s = dalloc(c, m.Av, sizeof(double) * nv)) != GH_OK) return s;
    if ((s = dalloc(c, m.theta, sizeof(double) * ne)) != GH_OK) return s;
    if ((s = dalloc(c, m.ev, sizeof(float) * 3 * ne)) != GH_OK) return s;
    if ((s = dalloc(c, m.gradop, sizeof(float) * 9 * nf)) != GH_OK) return s;
    if ((s = dalloc(c, m.gradop64, sizeof(double) * 9 * nf)) != GH_OK) return s;
    if ((s = dalloc(c, m.evf64, sizeof(double) * 9 * nf)) != GH_OK) return s;
    if ((s = dalloc(c, m.evf32, sizeof(float) * 9 * nf)) != GH_OK) return s;
    if ((s = dalloc(c, m.elen, sizeof(double) * ne)) != GH_OK) return s;
    if ((s = dalloc(c, cot, sizeof(double) * 3 * nf)) != GH_OK) return s;
    k_face_geom_len<<<blocks_for(nf, T), T, 0, st>>>(ptr<int32_t>(m.F), L, nf, ptr<double>(m.Af), ptr<float>(m.Aff),
                                                    ptr<double>(cot), ptr<float>(m.gradop), ptr<double>(m.gradop64),
                                                    ptr<double>(m.evf64), ptr<float>(m.evf32)); ++c->launches;
    k_edge_geom_len<<<blocks_for(ne, T), T, 0, st>>>(ne, ptr<int32_t>(m.edge_face), ptr<int32_t>(m.edge_slot),
                                                    ptr<double>(cot), L, ptr<double>(m.theta), ptr<float>(m.ev),
                                                    ptr<double>(m.elen)); ++c->launches;
    k_vertex_area<<<blocks_for(nv, T), T, 0, st>>>(ptr<int32_t>(m.rowptr), ptr<int32_t>(m.col_edge), nv,
                                                  ptr<int32_t>(m.edge_face), ptr<double>(m.Af), ptr<double>(m.Av)); ++c->launches;
    dfree(c, cot);
    if ((s = det_mean(c, ptr<double>(m.elen), ne, &m.hbar)) != GH_OK) return s;
    return check_status(c, "intrinsic geometry");
}

}  // namespace gh
