// Intrinsic Delaunay triangulation (Sec. 5.3) by parallel edge flips.
//
// The triangulation is the face list F plus the lengths L[3f+k] of the edge
// opposite corner k.  An interior edge whose opposite angles sum to more than
// pi (cot a + cot b < -1e-12) is flipped: faces (c, x, y) and (d, y, x)
// become (c, x, d) and (d, y, c), the new length |c - d| taken from the pair
// unfolded into the plane.  A flip that would join two vertices already
// joined (or a vertex to itself) is left out: the structures here hold one
// edge per vertex pair.  Rounds: the connectivity of the current faces; the
// flippable non-Delaunay edges; each face's lowest such edge; every edge that
// is the lowest of both its faces flips, so no face takes part in two flips
// of one round and the lowest one of the mesh always flips.  The rounds end
// when nothing flips.  For vertices in general position the result is the
// unique intrinsic Delaunay triangulation, whatever the order of the flips.
#include <climits>

#include "internal.cuh"

namespace gh {

namespace {

constexpr double kIdtTol = 1e-12;
constexpr int kMaxRounds = 1 << 20;

__global__ void k_slot_len(const double *__restrict__ P, const int32_t *__restrict__ F, int64_t nf, double *L) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    for (int k = 0; k < 3; ++k) {
        const double *a = P + 3 * F[3 * f + (k + 1) % 3], *b = P + 3 * F[3 * f + (k + 2) % 3];
        const double d[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        L[3 * f + k] = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    }
}

__device__ inline double corner_cot(const double *l, int k) {
    const int i = (k + 1) % 3, j = (k + 2) % 3;
    return (l[i] * l[i] + l[j] * l[j] - l[k] * l[k]) / (4.0 * heron_d(l[0], l[1], l[2]));
}

__device__ inline bool adjacent(const int32_t *rowptr, const int32_t *col, int a, int b) {
    int lo = rowptr[a], hi = rowptr[a + 1] - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1, v = col[mid];
        if (v == b) return true;
        if (v < b) lo = mid + 1; else hi = mid - 1;
    }
    return false;
}

// edges to flip: interior, cot a + cot b < -tol, and the new edge is new
__global__ void k_idt_mark(int64_t ne, const int32_t *__restrict__ edge_face, const int32_t *__restrict__ edge_slot,
                           const int32_t *__restrict__ F, const double *__restrict__ L,
                           const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col, int32_t *nd) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const int f1 = edge_face[2 * e], f2 = edge_face[2 * e + 1];
    int flip = 0;
    if (f2 >= 0) {
        const int k1 = edge_slot[2 * e], k2 = edge_slot[2 * e + 1];
        const double s = corner_cot(L + 3 * f1, k1) + corner_cot(L + 3 * f2, k2);
        if (s < -kIdtTol) {
            const int c = F[3 * f1 + k1], d = F[3 * f2 + k2];
            flip = (c != d) && !adjacent(rowptr, col, c, d);
        }
    }
    nd[e] = flip;
}

__global__ void k_idt_win(int64_t nf, const int32_t *__restrict__ face_edge, const int32_t *__restrict__ nd,
                          int32_t *win) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int w = INT_MAX;
    for (int k = 0; k < 3; ++k) {
        const int e = face_edge[3 * f + k];
        if (nd[e] && e < w) w = e;
    }
    win[f] = w;
}

__global__ void k_idt_flip(int64_t ne, const int32_t *__restrict__ edge_face, const int32_t *__restrict__ edge_slot,
                           const int32_t *__restrict__ nd, const int32_t *__restrict__ win, int32_t *F, double *L,
                           int32_t *count) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne || !nd[e]) return;
    const int f1 = edge_face[2 * e], f2 = edge_face[2 * e + 1];
    if (win[f1] != (int)e || win[f2] != (int)e) return;
    const int k1 = edge_slot[2 * e], k2 = edge_slot[2 * e + 1];
    // f1 = (c, x, y) runs x -> y, so f2 = (d, y, x)
    const int c = F[3 * f1 + k1], x = F[3 * f1 + (k1 + 1) % 3], y = F[3 * f1 + (k1 + 2) % 3];
    const int d = F[3 * f2 + k2];
    const double lxy = L[3 * f1 + k1];
    const double lxc = L[3 * f1 + (k1 + 2) % 3], lyc = L[3 * f1 + (k1 + 1) % 3];
    const double lxd = L[3 * f2 + (k2 + 1) % 3], lyd = L[3 * f2 + (k2 + 2) % 3];
    // unfolded: x at the origin, y on the +x axis, c above, d below
    const double xc = (lxy * lxy + lxc * lxc - lyc * lyc) / (2.0 * lxy);
    const double yc2 = lxc * lxc - xc * xc;
    const double xd = (lxy * lxy + lxd * lxd - lyd * lyd) / (2.0 * lxy);
    const double yd2 = lxd * lxd - xd * xd;
    const double yc = sqrt(yc2 > 0.0 ? yc2 : 0.0), yd = -sqrt(yd2 > 0.0 ? yd2 : 0.0);
    const double lcd = hypot(xc - xd, yc - yd);
    F[3 * f1] = c; F[3 * f1 + 1] = x; F[3 * f1 + 2] = d;
    L[3 * f1] = lxd; L[3 * f1 + 1] = lcd; L[3 * f1 + 2] = lxc;
    F[3 * f2] = d; F[3 * f2 + 1] = y; F[3 * f2 + 2] = c;
    L[3 * f2] = lyc; L[3 * f2 + 1] = lcd; L[3 * f2 + 2] = lyd;
    atomicAdd(count, 1);
}

}  // namespace

gh_status mesh_intrinsic_delaunay(Ctx *c, DevMesh &m, int64_t *flips) {
    cudaStream_t st = c->stream;
    const int T = 256;
    const int64_t nf = m.nf, ne = m.ne;
    DBuf L, nd, win, cnt;
    auto cleanup = [&]() { dfree(c, L); dfree(c, nd); dfree(c, win); dfree(c, cnt); };
    gh_status s;
#define TRY(x) if ((s = (x)) != GH_OK) { cleanup(); return s; }
    TRY(dalloc(c, L, sizeof(double) * 3 * nf));
    TRY(dalloc(c, nd, sizeof(int32_t) * ne));
    TRY(dalloc(c, win, sizeof(int32_t) * nf));
    TRY(dalloc(c, cnt, sizeof(int32_t)));
    if (m.intrinsic) {
        set_error("the mesh is already an intrinsic Delaunay triangulation");
        cleanup();
        return GH_EINVAL;
    }
    k_slot_len<<<blocks_for(nf, T), T, 0, st>>>(ptr<double>(m.P), ptr<int32_t>(m.F), nf, ptr<double>(L)); ++c->launches;
    int64_t total = 0;
    int round = 0;
    for (; round < kMaxRounds; ++round) {
        if (round > 0) TRY(build_connectivity(c, m));
        k_idt_mark<<<blocks_for(ne, T), T, 0, st>>>(ne, ptr<int32_t>(m.edge_face), ptr<int32_t>(m.edge_slot),
                                                    ptr<int32_t>(m.F), ptr<double>(L), ptr<int32_t>(m.rowptr),
                                                    ptr<int32_t>(m.col), ptr<int32_t>(nd)); ++c->launches;
        k_idt_win<<<blocks_for(nf, T), T, 0, st>>>(nf, ptr<int32_t>(m.face_edge), ptr<int32_t>(nd), ptr<int32_t>(win)); ++c->launches;
        GH_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t), st));
        k_idt_flip<<<blocks_for(ne, T), T, 0, st>>>(ne, ptr<int32_t>(m.edge_face), ptr<int32_t>(m.edge_slot),
                                                    ptr<int32_t>(nd), ptr<int32_t>(win), ptr<int32_t>(m.F),
                                                    ptr<double>(L), ptr<int32_t>(cnt)); ++c->launches;
        int32_t n = 0;
        GH_CUDA(cudaMemcpyAsync(&n, cnt.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        GH_CUDA(cudaStreamSynchronize(st));
        if (n == 0) break;
        total += n;
    }
    if (round == kMaxRounds) {
        set_error("intrinsic Delaunay flips did not end");
        cleanup();
        return GH_EDEVICE;
    }
    // the connectivity built at the start of the last round is that of the final faces
    TRY(build_geometry_lengths(c, m, ptr<double>(L)));
    {
        std::lock_guard<std::mutex> lk(*m.rec_mu);
        dfree(c, m.face_rec32);
        dfree(c, m.face_rec64);
        m.bfs_cluster[0] = m.bfs_cluster[1] = 0;
    }
    {
        std::lock_guard<std::mutex> lk(*m.cyc_mu);
        for (int i = 0; i < 2; ++i) {
            m.ncyc[i] = -1;
            dfree(c, m.cyc_var[i]);
            dfree(c, m.cyc_coef[i]);
        }
    }
    m.intrinsic = 1;
    cleanup();
    if (flips) *flips = total;
    return GH_OK;
#undef TRY
}

}  // namespace gh
