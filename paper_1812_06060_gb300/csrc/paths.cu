// Multi-source path constraints (Sec. 5.2, eq. MultiSourceConstraint,
// eq. MultiSourceConstraintEdgeBased) and, appended after them, the cycle
// constraints of a closed mesh (Sec. 5.1, built once per mesh in cycles.cu):
// the per-solve setup.
//
// Paths run from the first (lowest-index) source to each other source.  A
// path has the fewest edges: the one a breadth-first traversal from the first
// source alone gives by following each vertex's FIFO pairing vertex (any
// path between two sources gives a valid constraint, since the exact distance
// is 0 at both ends).  Constraint j is sum_i c_i . v_{var_i} = 0 over its
// path's edges: in the edge form v = x and c = +1 where the path runs from
// the edge's lower vertex to its higher one (the orientation halfedge), -1
// against it; in the face form v = g on the edge's adjacent face of lowest
// index and c = the edge's vector in the path's direction.
//
// The constraints join the ADMM block they act on.  That block's subproblem
// is separable, 1/2 sum_v D_v |v - vhat_v|^2 around its unconstrained update
// (D_e = |H_e| (1 + mu) for x, D_f = A_f (2 + mu n_f) for g), and its
// minimiser under C v = 0 is v = vhat - D^-1 C^T nu with
// (C D^-1 C^T) nu = C vhat.  This file builds, per solve, the entries, the
// distinct constrained variables with their summed coefficients and 1/D, and
// the Cholesky factor of the Gram matrix (FP64; a pivot at most 1e-12 of its
// diagonal entry drops its constraint, which then depends on the others).
// The per-iteration projection is in stages.cu.
#include "admm.cuh"
#include "internal.cuh"

namespace gh {

namespace {

constexpr int PT = 1024;   // threads of the single-CTA setup kernel

struct PcBuild {
    int npc, dim, nent, form;
    const int32_t *off;
    int32_t *var;
    double *coef;
    int32_t *entu, *uvar, *meta, *drop, *map;
    double *ucoef, *dinv, *L;
};

// levels of the sources in the traversal from the first source
__global__ void k_pc_levels(const int32_t *__restrict__ src, int ns, const int32_t *__restrict__ level,
                            int32_t *out) {
    const int i = threadIdx.x;
    if (i < ns) out[i] = level[src[i]];
}

// One thread per path j: walks from source j + 1 back to the first source
// through the pairing vertices (off[j+1] - off[j] steps, the source's set
// index) and writes the entries in the path's direction.
__global__ void k_pc_paths(const int32_t *__restrict__ src, int npc, const int32_t *__restrict__ off,
                           const int32_t *__restrict__ parent, const int32_t *__restrict__ pedge,
                           const int32_t *__restrict__ edges, const int32_t *__restrict__ edge_face,
                           const double *__restrict__ P, int form, int32_t *var, double *coef) {
    const int j = threadIdx.x;
    if (j >= npc) return;
    int v = src[j + 1];
    for (int i = off[j + 1] - 1; i >= off[j]; --i) {
        const int p = parent[v], e = pedge[v];
        if (form == GH_FORM_EDGE) {
            var[i] = e;
            coef[i] = (p == edges[2 * e]) ? 1.0 : -1.0;
        } else {
            var[i] = edge_face[2 * e];
            for (int c = 0; c < 3; ++c) coef[3 * i + c] = P[3 * v + c] - P[3 * p + c];
        }
        v = p;
    }
}

__device__ int pc_scan(int v, int &excl) {
    __shared__ int ws[PT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = ws[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;
    }
    __syncthreads();
    excl = (wid ? ws[wid - 1] : 0) + x - v;
    const int total = ws[PT / 32 - 1];
    __syncthreads();
    return total;
}

// The distinct constrained variables, their coefficient rows and 1/D, the
// Gram matrix and its Cholesky factor; leaves map[v] = the distinct index of
// each constrained variable (map starts at -1 everywhere).  One CTA.
__global__ void __launch_bounds__(PT, 1) k_pc_setup(PcBuild b, double mu, const int32_t *__restrict__ edge_face,
                                                 const int32_t *__restrict__ twin, const double *__restrict__ Af) {
    __shared__ double sG[kMaxPc * kMaxPc], sL[kMaxPc * kMaxPc];
    const int tid = threadIdx.x, npc = b.npc, dim = b.dim, nent = b.nent;
    // the owner of a variable: its entry of highest index
    for (int i = tid; i < nent; i += PT) atomicMax(&b.map[b.var[i]], i);
    __syncthreads();
    // distinct indices in the order of the owners
    int nu = 0;
    for (int i0 = 0; i0 < nent; i0 += PT) {
        const int i = i0 + tid;
        const int own = (i < nent && __ldcg(&b.map[b.var[i]]) == i) ? 1 : 0;
        int excl;
        const int tot = pc_scan(own, excl);
        if (own) {
            b.entu[i] = nu + excl;
            b.uvar[nu + excl] = b.var[i];
        }
        nu += tot;
    }
    __syncthreads();
    for (int i = tid; i < nent; i += PT) {
        const int o = __ldcg(&b.map[b.var[i]]);
        if (o != i) b.entu[i] = __ldcg(&b.entu[o]);
    }
    __syncthreads();
    // coefficient rows: a path or cycle has at most one entry per edge and
    // at most two per face (a simple path uses at most two edges of a
    // triangle; a loop of faces visits a face once), so these sums from zero
    // do not depend on the order of the additions
    for (int j = 0; j < npc; ++j)
        for (int i = b.off[j] + tid; i < b.off[j + 1]; i += PT)
            for (int c = 0; c < dim; ++c)
                atomicAdd(&b.ucoef[((size_t)b.entu[i] * npc + j) * dim + c], b.coef[(size_t)i * dim + c]);
    for (int u = tid; u < nu; u += PT) {
        const int v = b.uvar[u];
        double D;
        if (b.form == GH_FORM_EDGE) {
            D = ((edge_face[2 * v] >= 0) + (edge_face[2 * v + 1] >= 0)) * (1.0 + mu);
        } else {
            int n = 0;
            for (int k = 0; k < 3; ++k) n += twin[3 * v + k] >= 0;
            D = Af[v] * (2.0 + mu * n);
        }
        b.dinv[u] = 1.0 / D;
    }
    __syncthreads();
    // each constrained variable's map entry becomes its distinct index
    for (int i = tid; i < nent; i += PT)
        if (__ldcg(&b.map[b.var[i]]) == i) b.map[b.var[i]] = __ldcg(&b.entu[i]);
    // Gram matrix G_jk = sum_u (c_uj . c_uk) / D_u, one warp per pair j <= k
    const int warp = tid >> 5, lane = tid & 31;
    for (int pr = warp; pr < npc * npc; pr += PT / 32) {
        const int j = pr / npc, k = pr % npc;
        if (k < j) continue;
        double acc = 0.0;
        for (int u = lane; u < nu; u += 32) {
            double s = 0.0;
            for (int c = 0; c < dim; ++c)
                s += __ldcg(&b.ucoef[((size_t)u * npc + j) * dim + c]) * __ldcg(&b.ucoef[((size_t)u * npc + k) * dim + c]);
            acc += s * __ldcg(&b.dinv[u]);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            sG[j * npc + k] = acc;
            sG[k * npc + j] = acc;
        }
    }
    for (int i = tid; i < npc * npc; i += PT) sL[i] = 0.0;
    __syncthreads();
    if (tid == 0) {
        b.meta[0] = nu;
        for (int j = 0; j < npc; ++j) {
            double d = sG[j * npc + j];
            for (int m = 0; m < j; ++m) d -= sL[j * npc + m] * sL[j * npc + m];
            if (!(d > 1e-12 * sG[j * npc + j])) {   // row j of L stays 0
                b.drop[j] = 1;
                continue;
            }
            b.drop[j] = 0;
            const double ljj = sqrt(d);
            sL[j * npc + j] = ljj;
            for (int k = j + 1; k < npc; ++k) {
                double s = sG[k * npc + j];
                for (int m = 0; m < j; ++m) s -= sL[k * npc + m] * sL[j * npc + m];
                sL[k * npc + j] = s / ljj;
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < npc * npc; i += PT) b.L[i] = sL[i];
}

}  // namespace

gh_status build_path_constraints(Ctx *c, std::vector<Item> &items) {
    cudaStream_t st = c->stream;
    gh_status s;
    // what every item asks for: its source paths and its mesh's cycles
    std::vector<int> npath(items.size(), 0), ncyc(items.size(), 0);
    std::vector<DevMesh *> mq;
    std::vector<QueryWs *> wq;
    std::vector<std::vector<int32_t>> sq;
    std::vector<size_t> need;
    for (size_t k = 0; k < items.size(); ++k) {
        Item &x = items[k];
        x.w->pc_n = 0;
        x.w->pc_ent = 0;
        if (x.p->path_constraints && x.src->size() >= 2) npath[k] = (int)x.src->size() - 1;
        if (x.p->cycle_constraints) {
            if ((s = mesh_cycles(c, *x.m, x.p->form)) != GH_OK) return s;
            ncyc[k] = x.m->ncyc[x.p->form == GH_FORM_EDGE ? 1 : 0];
        }
        if (npath[k] + ncyc[k] == 0) continue;
        if (npath[k] + ncyc[k] > kMaxPc) {
            set_error("at most " + std::to_string(kMaxPc) + " path and cycle constraints per query (" +
                      std::to_string(npath[k]) + " + " + std::to_string(ncyc[k]) + " asked for)");
            return GH_EINVAL;
        }
        need.push_back(k);
        if (npath[k]) {
            mq.push_back(x.m);
            wq.push_back(x.w);
            sq.push_back({(*x.src)[0]});
        }
    }
    if (need.empty()) return GH_OK;
    // the traversal from each path query's first source (into the query's
    // own traversal buffers, which its main traversal overwrites afterwards),
    // stopped once it has reached the query's other sources
    std::vector<const int32_t *> tg;
    std::vector<int32_t> ntg;
    for (size_t k : need) {
        if (!npath[k]) continue;
        QueryWs &w = *items[k].w;
        const std::vector<int32_t> &src = *items[k].src;
        if ((s = dalloc(c, w.pc_src, sizeof(int32_t) * src.size())) != GH_OK) return s;
        GH_CUDA(cudaMemcpyAsync(w.pc_src.p, src.data(), sizeof(int32_t) * src.size(), cudaMemcpyHostToDevice, st));
        tg.push_back(ptr<int32_t>(w.pc_src) + 1);
        ntg.push_back((int32_t)src.size() - 1);
    }
    int cl = 8;   // the single-query cluster size of the meshes, when tuned and shared
    if (!mq.empty()) {
        std::lock_guard<std::mutex> lk(*mq[0]->rec_mu);
        if (mq[0]->bfs_cluster[0] != 0) cl = mq[0]->bfs_cluster[0];
    }
    for (DevMesh *x : mq)
        if (x != mq[0]) cl = 8;
    if (!mq.empty() && (s = run_bfs_fixed(c, mq, wq, sq, cl, &tg, &ntg)) != GH_OK) return s;
    std::vector<std::vector<int32_t>> lv(items.size());
    for (size_t k : need) {
        if (!npath[k]) continue;
        QueryWs &w = *items[k].w;
        const std::vector<int32_t> &src = *items[k].src;
        const int ns = (int)src.size();
        if ((s = dalloc(c, w.pc_lv, sizeof(int32_t) * ns)) != GH_OK) return s;
        k_pc_levels<<<1, 32, 0, st>>>(ptr<int32_t>(w.pc_src), ns, ptr<int32_t>(w.level), ptr<int32_t>(w.pc_lv));
        ++c->launches;
        lv[k].resize(ns);
        GH_CUDA(cudaMemcpyAsync(lv[k].data(), w.pc_lv.p, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost, st));
    }
    GH_CUDA(cudaStreamSynchronize(st));
    std::vector<std::vector<int32_t>> offs(items.size());
    for (size_t k : need) {
        QueryWs &w = *items[k].w;
        DevMesh &m = *items[k].m;
        const int form = items[k].p->form;
        const int fi = (form == GH_FORM_EDGE) ? 1 : 0;
        const int npc = npath[k] + ncyc[k];
        const int dim = (form == GH_FORM_EDGE) ? 1 : 3;
        // path constraints first (unreachable sources: empty), then the cycles
        std::vector<int32_t> &off = offs[k];
        off.assign(npc + 1, 0);
        for (int j = 0; j < npath[k]; ++j) off[j + 1] = off[j] + std::max(lv[k][j + 1], 0);
        const int nent_path = off[npath[k]];
        for (int j = 0; j < ncyc[k]; ++j) off[npath[k] + j + 1] = nent_path + m.cyc_off_h[fi][j + 1];
        const int nent = off[npc];
        const size_t ne1 = (size_t)std::max(nent, 1);
        const int64_t nvar = (form == GH_FORM_EDGE) ? m.ne : m.nf;
        const size_t es = w.fp64 ? sizeof(double) : sizeof(float);
        if ((s = dalloc(c, w.pc_off, sizeof(int32_t) * (npc + 1))) != GH_OK) return s;
        if ((s = dalloc(c, w.pc_var, sizeof(int32_t) * ne1)) != GH_OK) return s;
        if ((s = dalloc(c, w.pc_coef, sizeof(double) * ne1 * dim)) != GH_OK) return s;
        if ((s = dalloc(c, w.pc_entu, sizeof(int32_t) * ne1)) != GH_OK) return s;
        if ((s = dalloc(c, w.pc_uvar, sizeof(int32_t) * ne1)) != GH_OK) return s;
        if ((s = dalloc(c, w.pc_ucoef, sizeof(double) * ne1 * npc * dim)) != GH_OK) return s;
        if ((s = dalloc(c, w.pc_dinv, sizeof(double) * ne1)) != GH_OK) return s;
        if ((s = dalloc(c, w.pc_L, sizeof(double) * npc * npc)) != GH_OK) return s;
        if ((s = dalloc(c, w.pc_drop, sizeof(int32_t) * npc)) != GH_OK) return s;
        if ((s = dalloc(c, w.pc_meta, sizeof(int32_t) * 4)) != GH_OK) return s;
        if ((s = dalloc(c, w.pc_val, es * ne1 * dim)) != GH_OK) return s;
        if ((s = dalloc(c, w.pc_delta, es * ne1 * dim)) != GH_OK) return s;
        if ((s = dalloc(c, w.pc_map, sizeof(int32_t) * nvar)) != GH_OK) return s;
        GH_CUDA(cudaMemcpyAsync(w.pc_off.p, off.data(), sizeof(int32_t) * (npc + 1), cudaMemcpyHostToDevice, st));
        GH_CUDA(cudaMemsetAsync(w.pc_map.p, 0xff, sizeof(int32_t) * nvar, st));
        GH_CUDA(cudaMemsetAsync(w.pc_ucoef.p, 0, sizeof(double) * ne1 * npc * dim, st));
        if (npath[k]) {
            k_pc_paths<<<1, 32, 0, st>>>(ptr<int32_t>(w.pc_src), npath[k], ptr<int32_t>(w.pc_off),
                                         ptr<int32_t>(w.parent), ptr<int32_t>(w.pedge), ptr<int32_t>(m.edges),
                                         ptr<int32_t>(m.edge_face), ptr<double>(m.P), form, ptr<int32_t>(w.pc_var),
                                         ptr<double>(w.pc_coef));
            ++c->launches;
        }
        if (ncyc[k] && m.cyc_ent[fi] > 0) {
            GH_CUDA(cudaMemcpyAsync(ptr<int32_t>(w.pc_var) + nent_path, m.cyc_var[fi].p,
                                    sizeof(int32_t) * m.cyc_ent[fi], cudaMemcpyDeviceToDevice, st));
            GH_CUDA(cudaMemcpyAsync(ptr<double>(w.pc_coef) + (size_t)nent_path * dim, m.cyc_coef[fi].p,
                                    sizeof(double) * m.cyc_ent[fi] * dim, cudaMemcpyDeviceToDevice, st));
        }
        PcBuild b{npc, dim, nent, form, ptr<int32_t>(w.pc_off), ptr<int32_t>(w.pc_var), ptr<double>(w.pc_coef),
                  ptr<int32_t>(w.pc_entu), ptr<int32_t>(w.pc_uvar), ptr<int32_t>(w.pc_meta), ptr<int32_t>(w.pc_drop),
                  ptr<int32_t>(w.pc_map), ptr<double>(w.pc_ucoef), ptr<double>(w.pc_dinv), ptr<double>(w.pc_L)};
        k_pc_setup<<<1, PT, 0, st>>>(b, items[k].p->mu, ptr<int32_t>(m.edge_face), ptr<int32_t>(m.twin),
                                     ptr<double>(m.Af));
        ++c->launches;
        w.pc_n = npc;
        w.pc_ent = nent;
        w.pc_dim = dim;
    }
    GH_CUDA(cudaGetLastError());
    // the host copies of the offsets must outlive their transfers
    GH_CUDA(cudaStreamSynchronize(st));
    return GH_OK;
}

}  // namespace gh
