// Cycle constraints of a connected closed surface of genus g (Sec. 5.1,
// eq. TopologyConstraint, eq. EdgeTopologyConstraint): a basis of 2g
// non-contractible cycles from a tree-cotree decomposition, built once per
// mesh and form.
//
// Trees are breadth-first trees with FIFO pairing (the traversal kernel of
// bfs.cu on the graph at hand), rooted at vertex 0 and face 0, every row in
// ascending order.
//   Edge form: T = the primal tree; C = the dual tree (faces across the
//   edges not in T); each edge in neither closes a cycle of edges: its lower
//   end -> its higher end, then T up to the common ancestor and back down.
//   Entry coefficients are +1 where the cycle runs along the edge's
//   orientation halfedge (lower -> higher vertex), -1 against it.
//   Face form: T* = the dual tree (faces across all edges); C = the primal
//   tree over the edges T* does not cross; each edge in neither closes a
//   loop of faces: its lower face, its higher face, T* up to the common
//   ancestor and back down.  A face of the loop gets the segment between the
//   midpoints of the edge it is entered through and the edge it is left
//   through.
// Cycles come in ascending order of their closing edge.  Only a connected
// closed mesh gets cycles: with a boundary edge, or trees that miss a vertex
// or a face, the basis is empty.
#include <algorithm>

#include "internal.cuh"

namespace gh {

namespace {

__global__ void k_count_open(int64_t ne, const int32_t *__restrict__ edge_face, int32_t *out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < ne && edge_face[2 * e + 1] < 0) atomicAdd(out, 1);
}

// mark[pedge[v]] = 1 for every non-root node of a breadth-first tree
__global__ void k_mark_tree(int64_t n, const int32_t *__restrict__ level, const int32_t *__restrict__ pedge,
                            int32_t *mark) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n && level[v] > 0) mark[pedge[v]] = 1;
}

// dual graph: row f lists (face across edge k, that edge) for the edges of f
// that are not excluded (excl null: none is), sorted by face then edge
__global__ void k_dual_len(int64_t nf, const int32_t *__restrict__ face_edge, const int32_t *__restrict__ excl,
                           int32_t *len) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int n = 0;
    for (int k = 0; k < 3; ++k) n += !(excl && excl[face_edge[3 * f + k]]);
    len[f] = n;
}
__global__ void k_dual_fill(int64_t nf, const int32_t *__restrict__ face_edge, const int32_t *__restrict__ twin,
                            const int32_t *__restrict__ excl, const int32_t *__restrict__ rowptr, int32_t *col,
                            int32_t *cedge) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int nb[3], ed[3], n = 0;
    for (int k = 0; k < 3; ++k) {
        const int e = face_edge[3 * f + k];
        if (excl && excl[e]) continue;
        nb[n] = twin[3 * f + k] >> 2;
        ed[n] = e;
        ++n;
    }
    for (int i = 1; i < n; ++i)   // insertion sort by (face, edge)
        for (int j = i; j > 0 && (nb[j] < nb[j - 1] || (nb[j] == nb[j - 1] && ed[j] < ed[j - 1])); --j) {
            int t = nb[j]; nb[j] = nb[j - 1]; nb[j - 1] = t;
            t = ed[j]; ed[j] = ed[j - 1]; ed[j - 1] = t;
        }
    const int b = rowptr[f];
    for (int i = 0; i < n; ++i) {
        col[b + i] = nb[i];
        cedge[b + i] = ed[i];
    }
}

// primal rows without the excluded edges (the ascending order is kept)
__global__ void k_prim_len(int64_t nv, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col_edge,
                           const int32_t *__restrict__ excl, int32_t *len) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    int n = 0;
    for (int j = rowptr[v]; j < rowptr[v + 1]; ++j) n += !excl[col_edge[j]];
    len[v] = n;
}
__global__ void k_prim_fill(int64_t nv, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                            const int32_t *__restrict__ col_edge, const int32_t *__restrict__ excl,
                            const int32_t *__restrict__ orow, int32_t *ocol, int32_t *ocedge) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    int o = orow[v];
    for (int j = rowptr[v]; j < rowptr[v + 1]; ++j)
        if (!excl[col_edge[j]]) {
            ocol[o] = col[j];
            ocedge[o] = col_edge[j];
            ++o;
        }
}

// generators: edges in neither tree
__global__ void k_gen_flag(int64_t ne, const int32_t *__restrict__ m1, const int32_t *__restrict__ m2, int32_t *flag) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < ne) flag[e] = !m1[e] && !m2[e];
}
__global__ void k_gen_list(int64_t ne, const int32_t *__restrict__ flag, const int32_t *__restrict__ pos, int32_t *gens) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < ne && flag[e]) gens[pos[e]] = (int32_t)e;
}

__device__ int cyc_lca(int a, int b, const int32_t *level, const int32_t *parent) {
    while (level[a] > level[b]) a = parent[a];
    while (level[b] > level[a]) b = parent[b];
    while (a != b) {
        a = parent[a];
        b = parent[b];
    }
    return a;
}

// steps of the cycle of generator g: 1 + (level[b] - level[lca]) + (level[a] - level[lca])
__global__ void k_cyc_len(int G, const int32_t *__restrict__ gens, const int32_t *__restrict__ ends,
                          const int32_t *__restrict__ level, const int32_t *__restrict__ parent, int32_t *len) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const int e = gens[g], a = ends[2 * e], b = ends[2 * e + 1];
    const int l = cyc_lca(a, b, level, parent);
    len[g] = 1 + (level[b] - level[l]) + (level[a] - level[l]);
}

// the closed node sequence a, b, ..., lca, ..., a (m + 1 nodes at off[g] + g)
// and the m crossings between consecutive nodes (at off[g])
__global__ void k_cyc_walk(int G, const int32_t *__restrict__ gens, const int32_t *__restrict__ ends,
                           const int32_t *__restrict__ level, const int32_t *__restrict__ parent,
                           const int32_t *__restrict__ pedge, const int32_t *__restrict__ off, int32_t *node,
                           int32_t *cross) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const int e = gens[g], a = ends[2 * e], b = ends[2 * e + 1];
    const int l = cyc_lca(a, b, level, parent);
    const int m = off[g + 1] - off[g];
    int32_t *nd = node + off[g] + g, *cr = cross + off[g];
    nd[0] = a;
    cr[0] = e;
    nd[1] = b;
    int i = 1;
    for (int x = b; x != l; x = parent[x], ++i) {   // b up to the common ancestor
        cr[i] = pedge[x];
        nd[i + 1] = parent[x];
    }
    int t = 0;
    for (int y = a; y != l; y = parent[y], ++t) {   // and down to a, written from the end
        cr[m - 1 - t] = pedge[y];
        nd[m - t] = y;
        nd[m - 1 - t] = parent[y];
    }
}

// entries: edge form (crossing edge, +-1 along its orientation halfedge);
// face form (face, midpoint of its exit edge - midpoint of its entry edge)
__global__ void k_cyc_coef(int G, const int32_t *__restrict__ off, const int32_t *__restrict__ node,
                           const int32_t *__restrict__ cross, int form, const int32_t *__restrict__ edges,
                           const double *__restrict__ P, int32_t *var, double *coef) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const int m = off[g + 1] - off[g];
    const int32_t *nd = node + off[g] + g, *cr = cross + off[g];
    for (int i = 0; i < m; ++i) {
        const int o = off[g] + i;
        if (form == GH_FORM_EDGE) {
            const int ce = cr[i];
            var[o] = ce;
            coef[o] = (nd[i] == edges[2 * ce]) ? 1.0 : -1.0;
        } else {
            const int cn = cr[i], cp = cr[(i + m - 1) % m];
            var[o] = nd[i];
            for (int c = 0; c < 3; ++c) {
                const double mn = 0.5 * (P[3 * edges[2 * cn] + c] + P[3 * edges[2 * cn + 1] + c]);
                const double mp = 0.5 * (P[3 * edges[2 * cp] + c] + P[3 * edges[2 * cp + 1] + c]);
                coef[3 * o + c] = mn - mp;
            }
        }
    }
}

gh_status alloc_bfs_ws(Ctx *c, QueryWs &w, int64_t n) {
    gh_status s;
    DBuf *b4[] = {&w.level, &w.parent, &w.pedge, &w.order, &w.pos, &w.n0};
    for (DBuf *b : b4)
        if ((s = dalloc(c, *b, sizeof(int32_t) * (n + 1))) != GH_OK) return s;
    if ((s = dalloc(c, w.key, sizeof(unsigned long long) * n)) != GH_OK) return s;
    if ((s = dalloc(c, w.lvl_off, sizeof(int32_t) * (n + 2))) != GH_OK) return s;
    return dalloc(c, w.meta, 16);
}

}  // namespace

gh_status mesh_cycles(Ctx *c, DevMesh &m, int form) {
    const int fi = (form == GH_FORM_EDGE) ? 1 : 0;
    std::lock_guard<std::mutex> lk(*m.cyc_mu);
    if (m.ncyc[fi] >= 0) return GH_OK;
    cudaStream_t st = c->stream;
    const int64_t nv = m.nv, nf = m.nf, ne = m.ne, nmax = std::max(nv, nf);
    const unsigned T = 256;
    DBuf open1, markA, markB, len, row, col, cedge, flag, pos, gens, glen, goff, node, cross;
    QueryWs W1, W2;
    auto cleanup = [&]() {
        DBuf *all[] = {&open1, &markA, &markB, &len, &row, &col, &cedge, &flag, &pos, &gens, &glen, &goff, &node,
                       &cross};
        for (DBuf *b : all) dfree(c, *b);
        free_ws(c, &W1);
        free_ws(c, &W2);
    };
    auto none = [&]() {
        m.ncyc[fi] = 0;
        m.cyc_ent[fi] = 0;
        m.cyc_off_h[fi].assign(1, 0);
        cleanup();
        return GH_OK;
    };
    gh_status s;
#define TRY(x) if ((s = (x)) != GH_OK) { cleanup(); return s; }
    TRY(dalloc(c, open1, sizeof(int32_t)));
    GH_CUDA(cudaMemsetAsync(open1.p, 0, sizeof(int32_t), st));
    k_count_open<<<blocks_for(ne, T), T, 0, st>>>(ne, ptr<int32_t>(m.edge_face), ptr<int32_t>(open1)); ++c->launches;
    int32_t nopen = 0;
    GH_CUDA(cudaMemcpyAsync(&nopen, open1.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    GH_CUDA(cudaStreamSynchronize(st));
    if (nopen > 0 || nf == 0) return none();
    TRY(dalloc(c, markA, sizeof(int32_t) * ne));
    TRY(dalloc(c, markB, sizeof(int32_t) * ne));
    TRY(dalloc(c, len, sizeof(int32_t) * (nmax + 1)));
    TRY(dalloc(c, row, sizeof(int32_t) * (nmax + 1)));
    TRY(dalloc(c, col, sizeof(int32_t) * 2 * ne));
    TRY(dalloc(c, cedge, sizeof(int32_t) * 2 * ne));
    TRY(alloc_bfs_ws(c, W1, nv));
    TRY(alloc_bfs_ws(c, W2, nf));
    GH_CUDA(cudaMemsetAsync(markA.p, 0, sizeof(int32_t) * ne, st));
    GH_CUDA(cudaMemsetAsync(markB.p, 0, sizeof(int32_t) * ne, st));
    std::vector<std::vector<int32_t>> root = {{0}};
    int32_t tot = 0;
    DevMesh g;   // the graph of the second traversal: rows, columns, crossing edges
    g.rowptr = row;
    g.col = col;
    g.col_edge = cedge;
    QueryWs *tree = nullptr;   // the traversal whose tree carries the cycles
    const int32_t *ends = nullptr;
    if (form == GH_FORM_EDGE) {
        std::vector<DevMesh *> mq = {&m};
        std::vector<QueryWs *> wq = {&W1};
        TRY(run_bfs_fixed(c, mq, wq, root, 8));
        if (W1.nreach != nv) return none();
        k_mark_tree<<<blocks_for(nv, T), T, 0, st>>>(nv, ptr<int32_t>(W1.level), ptr<int32_t>(W1.pedge), ptr<int32_t>(markA)); ++c->launches;
        k_dual_len<<<blocks_for(nf, T), T, 0, st>>>(nf, ptr<int32_t>(m.face_edge), ptr<int32_t>(markA), ptr<int32_t>(len)); ++c->launches;
        TRY(exclusive_scan_i32(c, ptr<int32_t>(len), ptr<int32_t>(row), nf, &tot));
        k_dual_fill<<<blocks_for(nf, T), T, 0, st>>>(nf, ptr<int32_t>(m.face_edge), ptr<int32_t>(m.twin), ptr<int32_t>(markA),
                                                     ptr<int32_t>(row), ptr<int32_t>(col), ptr<int32_t>(cedge)); ++c->launches;
        g.nv = nf;
        std::vector<DevMesh *> gq = {&g};
        std::vector<QueryWs *> w2 = {&W2};
        TRY(run_bfs_fixed(c, gq, w2, root, 8));
        if (W2.nreach != nf) return none();
        k_mark_tree<<<blocks_for(nf, T), T, 0, st>>>(nf, ptr<int32_t>(W2.level), ptr<int32_t>(W2.pedge), ptr<int32_t>(markB)); ++c->launches;
        tree = &W1;
        ends = ptr<int32_t>(m.edges);
    } else {
        k_dual_len<<<blocks_for(nf, T), T, 0, st>>>(nf, ptr<int32_t>(m.face_edge), nullptr, ptr<int32_t>(len)); ++c->launches;
        TRY(exclusive_scan_i32(c, ptr<int32_t>(len), ptr<int32_t>(row), nf, &tot));
        k_dual_fill<<<blocks_for(nf, T), T, 0, st>>>(nf, ptr<int32_t>(m.face_edge), ptr<int32_t>(m.twin), nullptr,
                                                     ptr<int32_t>(row), ptr<int32_t>(col), ptr<int32_t>(cedge)); ++c->launches;
        g.nv = nf;
        {
            std::vector<DevMesh *> gq = {&g};
            std::vector<QueryWs *> w2 = {&W2};
            TRY(run_bfs_fixed(c, gq, w2, root, 8));
        }
        if (W2.nreach != nf) return none();
        k_mark_tree<<<blocks_for(nf, T), T, 0, st>>>(nf, ptr<int32_t>(W2.level), ptr<int32_t>(W2.pedge), ptr<int32_t>(markA)); ++c->launches;
        // the primal cotree over the edges the dual tree does not cross
        k_prim_len<<<blocks_for(nv, T), T, 0, st>>>(nv, ptr<int32_t>(m.rowptr), ptr<int32_t>(m.col_edge), ptr<int32_t>(markA),
                                                    ptr<int32_t>(len)); ++c->launches;
        TRY(exclusive_scan_i32(c, ptr<int32_t>(len), ptr<int32_t>(row), nv, &tot));
        k_prim_fill<<<blocks_for(nv, T), T, 0, st>>>(nv, ptr<int32_t>(m.rowptr), ptr<int32_t>(m.col), ptr<int32_t>(m.col_edge),
                                                     ptr<int32_t>(markA), ptr<int32_t>(row), ptr<int32_t>(col),
                                                     ptr<int32_t>(cedge)); ++c->launches;
        g.nv = nv;
        {
            std::vector<DevMesh *> gq = {&g};
            std::vector<QueryWs *> w1 = {&W1};
            TRY(run_bfs_fixed(c, gq, w1, root, 8));
        }
        if (W1.nreach != nv) return none();
        k_mark_tree<<<blocks_for(nv, T), T, 0, st>>>(nv, ptr<int32_t>(W1.level), ptr<int32_t>(W1.pedge), ptr<int32_t>(markB)); ++c->launches;
        tree = &W2;
        ends = ptr<int32_t>(m.edge_face);
    }
    // generators in ascending edge order
    TRY(dalloc(c, flag, sizeof(int32_t) * ne));
    TRY(dalloc(c, pos, sizeof(int32_t) * (ne + 1)));
    k_gen_flag<<<blocks_for(ne, T), T, 0, st>>>(ne, ptr<int32_t>(markA), ptr<int32_t>(markB), ptr<int32_t>(flag)); ++c->launches;
    int32_t G = 0;
    TRY(exclusive_scan_i32(c, ptr<int32_t>(flag), ptr<int32_t>(pos), ne, &G));
    if (G == 0) return none();
    TRY(dalloc(c, gens, sizeof(int32_t) * G));
    TRY(dalloc(c, glen, sizeof(int32_t) * G));
    TRY(dalloc(c, goff, sizeof(int32_t) * (G + 1)));
    k_gen_list<<<blocks_for(ne, T), T, 0, st>>>(ne, ptr<int32_t>(flag), ptr<int32_t>(pos), ptr<int32_t>(gens)); ++c->launches;
    k_cyc_len<<<blocks_for(G, 32), 32, 0, st>>>(G, ptr<int32_t>(gens), ends, ptr<int32_t>(tree->level),
                                                ptr<int32_t>(tree->parent), ptr<int32_t>(glen)); ++c->launches;
    std::vector<int32_t> lens(G), off(G + 1, 0);
    GH_CUDA(cudaMemcpyAsync(lens.data(), glen.p, sizeof(int32_t) * G, cudaMemcpyDeviceToHost, st));
    GH_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < G; ++i) off[i + 1] = off[i] + lens[i];
    const int dim = (form == GH_FORM_EDGE) ? 1 : 3;
    const int64_t nent = off[G];
    TRY(dalloc(c, node, sizeof(int32_t) * (nent + G)));
    TRY(dalloc(c, cross, sizeof(int32_t) * nent));
    TRY(dalloc(c, m.cyc_var[fi], sizeof(int32_t) * nent));
    TRY(dalloc(c, m.cyc_coef[fi], sizeof(double) * nent * dim));
    GH_CUDA(cudaMemcpyAsync(goff.p, off.data(), sizeof(int32_t) * (G + 1), cudaMemcpyHostToDevice, st));
    k_cyc_walk<<<blocks_for(G, 32), 32, 0, st>>>(G, ptr<int32_t>(gens), ends, ptr<int32_t>(tree->level),
                                                 ptr<int32_t>(tree->parent), ptr<int32_t>(tree->pedge),
                                                 ptr<int32_t>(goff), ptr<int32_t>(node), ptr<int32_t>(cross)); ++c->launches;
    k_cyc_coef<<<blocks_for(G, 32), 32, 0, st>>>(G, ptr<int32_t>(goff), ptr<int32_t>(node), ptr<int32_t>(cross), form,
                                                 ptr<int32_t>(m.edges), ptr<double>(m.P), ptr<int32_t>(m.cyc_var[fi]),
                                                 ptr<double>(m.cyc_coef[fi])); ++c->launches;
    GH_CUDA(cudaGetLastError());
    GH_CUDA(cudaStreamSynchronize(st));   // off must outlive its transfer
    m.ncyc[fi] = G;
    m.cyc_ent[fi] = (int)nent;
    m.cyc_off_h[fi] = off;
    cleanup();
    return GH_OK;
#undef TRY
}

}  // namespace gh
