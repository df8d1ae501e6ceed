// The C-ABI of include/geoheat.h: contexts, resident meshes, solves (single
// and batched), intermediates for parity tests, error reporting.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cstddef>

#include "internal.cuh"

namespace gh {
struct Engine;
void engine_stop(Engine *e);
void engine_forget_mesh(Engine *e, DevMesh *m);
}

struct gh_ctx_s {
    gh::Ctx c;
    gh::Shared shared;
    std::mutex mu;
    std::vector<gh_mesh_s *> meshes;
    gh::Engine *engine = nullptr;   // serving workers, started by the first gh_submit
    std::mutex engine_mu;           // guards the start of the serving workers
    int serve_workers = 2, serve_max_batch = 32;
};

struct gh_mesh_s {
    gh_ctx_s *ctx = nullptr;
    gh::MeshH h;
};

namespace gh {

static thread_local std::string t_err;

void set_error(const std::string &msg) { t_err = msg; }

gh_status cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    if (e == cudaErrorMemoryAllocation) return GH_ENOMEM;
    return GH_EDEVICE;
}

gh_status dalloc(Ctx *c, DBuf &b, size_t bytes) {
    if (b.p && b.bytes >= bytes) return GH_OK;
    dfree(c, b);
    if (bytes == 0) bytes = 16;
    Shared *sh = c->shared;
    size_t cur = sh->in_use.load();
    do {
        if (sh->budget && cur + bytes > sh->budget) {
            set_error("device memory budget of the context exceeded (" + std::to_string(cur + bytes) + " > " +
                      std::to_string(sh->budget) + " bytes)");
            return GH_ENOMEM;
        }
    } while (!sh->in_use.compare_exchange_weak(cur, cur + bytes));
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        sh->in_use -= bytes;
        (void)cudaGetLastError();
        return cuda_fail(e, "cudaMalloc");
    }
    b.bytes = bytes;
    return GH_OK;
}

void dfree(Ctx *c, DBuf &b) {
    if (b.p) {
        cudaFree(b.p);
        c->shared->in_use -= b.bytes;
    }
    b.p = nullptr;
    b.bytes = 0;
}

int *dev_status(Ctx *c) { return c->status_dev; }

gh_status check_status(Ctx *c, const char *stage) {
    GH_CUDA(cudaStreamSynchronize(c->stream));
    GH_CUDA(cudaGetLastError());
    int s = 0;
    GH_CUDA(cudaMemcpy(&s, c->status_dev, sizeof(int), cudaMemcpyDeviceToHost));
    if (s == DEV_OK) return GH_OK;
    cudaMemset(c->status_dev, 0, sizeof(int));
    switch (s) {
    case DEV_EINVAL: set_error(std::string(stage) + ": invalid input (index out of range or repeated vertex in a face)"); return GH_EINVAL;
    case DEV_ENONMANIFOLD: set_error(std::string(stage) + ": mesh is not an oriented 2-manifold"); return GH_ENONMANIFOLD;
    case DEV_ETIMEOUT: set_error(std::string(stage) + ": a grid barrier wait ran out"); return GH_ETIMEOUT;
    case DEV_EINTERNAL: set_error(std::string(stage) + ": internal consistency check failed (breadth-first layout)"); return GH_EDEVICE;
    default: set_error(std::string(stage) + ": device error"); return GH_EDEVICE;
    }
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void free_ws(Ctx *c, QueryWs *w) {
    DBuf *all[] = {&w->level, &w->parent, &w->pedge, &w->order, &w->lorder, &w->pos, &w->key, &w->lvl_off, &w->meta, &w->twid, &w->gent,
                   &w->diag, &w->tiles, &w->ptile, &w->U0, &w->U1, &w->h, &w->g0, &w->g1, &w->l0, &w->l1, &w->z,
                   &w->w, &w->lam, &w->sz, &w->x, &w->inc, &w->d0, &w->d1, &w->n0, &w->n1, &w->resid, &w->e1, &w->actl,
                   &w->pc_src, &w->pc_lv, &w->pc_off, &w->pc_var, &w->pc_coef, &w->pc_entu, &w->pc_uvar,
                   &w->pc_ucoef, &w->pc_dinv, &w->pc_L, &w->pc_drop, &w->pc_meta, &w->pc_val, &w->pc_delta,
                   &w->pc_map};
    for (DBuf *b : all) dfree(c, *b);
}

// allocate (or keep) the workspace of one query for this mesh, precision and form
static gh_status ensure_ws(Ctx *c, const DevMesh &m, QueryWs &w, int fp64, int form, int iters) {
    const size_t es = fp64 ? sizeof(double) : sizeof(float);
    const size_t xs = fp64 ? sizeof(XVal<double>) : sizeof(XVal<float>);
    const int64_t nv = m.nv, nf = m.nf, ne = m.ne, nnz = 2 * m.ne;
    if (w.fp64 != fp64 || w.cap_nv != nv || w.cap_nf != nf || w.cap_ne != ne) {
        free_ws(c, &w);
        w.fp64 = fp64;
        w.cap_nv = nv;
        w.cap_nf = nf;
        w.cap_ne = ne;
        w.cap_nnz = nnz;
    }
    gh_status s;
#define A(buf, bytes) if ((s = dalloc(c, w.buf, (size_t)(bytes))) != GH_OK) return s
    A(level, 4 * nv); A(parent, 4 * nv); A(pedge, 4 * nv); A(order, 4 * nv); A(lorder, 4 * nv); A(pos, 4 * nv); A(key, 8 * nv);
    A(lvl_off, 4 * (nv + 2)); A(meta, 16);
    // padded so 16-byte aligned bulk copies of any row window stay inside the buffers
    A(gent, (nnz + 4) * (fp64 ? 16 : 8)); A(diag, es * (nv + 4));   // gent grows to the padded blocks
    A(ptile, 4 * (nv + 8));
    A(U0, xs * (nv + 1)); A(U1, xs * (nv + 1));   // + the zero slot
    A(h, es * 3 * nf);
    if (form == GH_FORM_FACE) {
        A(g0, es * 3 * nf); A(g1, es * 3 * nf); A(l0, es * 9 * nf); A(l1, es * 9 * nf);
    } else {
        A(z, es * 3 * nf); A(w, es * 3 * nf); A(lam, es * 3 * nf); A(sz, es * ne); A(x, es * ne);
    }
    A(inc, 8 * nv); A(d0, 8 * nv); A(d1, 8 * nv); A(n0, 4 * (nv + 1)); A(n1, 4 * (nv + 1));
    A(resid, 16 * std::max(iters, 1)); A(e1, 8); A(actl, sizeof(AdmmCtl));
#undef A
    return GH_OK;
}

gh_status validate_params(const gh_params *p) {
    if (!p) { set_error("params is NULL"); return GH_EINVAL; }
    if (p->gs_sweeps < 1) { set_error("gs_sweeps must be >= 1"); return GH_EINVAL; }
    if (p->admm_iters < 0) { set_error("admm_iters must be >= 0"); return GH_EINVAL; }
    if (!(p->mu > 0)) { set_error("mu must be > 0"); return GH_EINVAL; }
    if (p->form != GH_FORM_FACE && p->form != GH_FORM_EDGE) { set_error("form must be GH_FORM_FACE or GH_FORM_EDGE"); return GH_EINVAL; }
    if (!(p->t > 0) && !(p->m > 0)) { set_error("either t > 0 or m > 0 is required"); return GH_EINVAL; }
    if (p->early_stop != 0 && p->early_stop != 1) { set_error("early_stop must be 0 or 1"); return GH_EINVAL; }
    if (p->early_stop && !(p->eps1 >= 0 && p->eps2 >= 0 && p->eps1 < 1e300 && p->eps2 < 1e300)) {
        set_error("eps1 and eps2 must be finite and >= 0");
        return GH_EINVAL;
    }
    if (p->path_constraints != 0 && p->path_constraints != 1) {
        set_error("path_constraints must be 0 or 1");
        return GH_EINVAL;
    }
    if (p->cycle_constraints != 0 && p->cycle_constraints != 1) {
        set_error("cycle_constraints must be 0 or 1");
        return GH_EINVAL;
    }
    if (!(p->gs_tol >= 0 && p->gs_tol < 1e300)) { set_error("gs_tol must be finite and >= 0"); return GH_EINVAL; }
    if (p->gs_tol > 0 && p->gs_check < 1) { set_error("gs_check must be >= 1 when gs_tol > 0"); return GH_EINVAL; }
    if (p->gs_band < 0) { set_error("gs_band must be >= 0"); return GH_EINVAL; }
    return GH_OK;
}

// bytes one query's workspace needs
size_t ws_bytes(const DevMesh &m, int fp64, int form, int path_constraints) {
    const size_t es = fp64 ? 8 : 4, xs = fp64 ? 16 : 8;
    size_t nv = m.nv, nf = m.nf, ne = m.ne;
    // the level-ordered operator with a quarter more for the padding of its
    // tiles (a tile's rows are padded to its longest row)
    size_t b = nv * (6 * 4 + 8 + 4 + 4 + es + 8 + 4 + 2 * xs + 8 + 16 + 8) + 2 * ne * (fp64 ? 16 : 8) * 5 / 4 +
               es * 3 * nf;
    b += (form == GH_FORM_FACE) ? es * 24 * nf : es * (9 * nf + 2 * ne);
    // path constraints: the block's variable map and an allowance for the entries
    // (sources x sets; their allocations are checked against the budget anyway)
    if (path_constraints) b += 4 * ((form == GH_FORM_FACE) ? nf : ne) + (size_t)(kMaxPc + 1) * 64 * 1024;
    return b + (1 << 20);
}

// The diffusion of every query: gs_sweeps sweeps in one launch for all; the
// queries with gs_tol > 0 go in rounds of gs_check sweeps, each continuing
// the iteration of the last, until their heat residual E1 (eq.
// HeatSolutionError) is within gs_tol or gs_sweeps sweeps have run; every
// round is one launch for the queries still running.  ev0 / ev1 bracket all
// rounds.
static gh_status run_diffusion(Ctx *c, std::vector<Item> &items, std::vector<QueryWs *> &ws, cudaEvent_t ev0,
                               cudaEvent_t ev1) {
    const int K = (int)ws.size();
    std::vector<int> left(K);
    std::vector<QueryWs *> run;
    for (int q = 0; q < K; ++q) {
        ws[q]->gs_continue = 0;
        ws[q]->sweeps_run = 0;
        left[q] = items[q].p->gs_sweeps;
    }
    std::vector<int> active(K);
    for (int q = 0; q < K; ++q) active[q] = q;
    std::vector<double> e1(K, 0.0);
    bool first = true;
    while (!active.empty()) {
        run.clear();
        for (int q : active) {
            const gh_params *p = items[q].p;
            ws[q]->sweeps = (p->gs_tol > 0) ? std::min(p->gs_check, left[q]) : left[q];
            ws[q]->gs_band = p->gs_band;
            run.push_back(ws[q]);
        }
        gh_status s = run_gs(c, run, first ? ev0 : nullptr, nullptr);
        if (s != GH_OK) return s;
        first = false;
        std::vector<int> next;
        for (int q : active) {
            left[q] -= ws[q]->sweeps;
            ws[q]->sweeps_run += ws[q]->sweeps;
            ws[q]->gs_continue = 1;
            if (items[q].p->gs_tol > 0) {
                if ((s = run_heat_residual(c, *items[q].m, *ws[q])) != GH_OK) return s;
                GH_CUDA(cudaMemcpyAsync(&e1[q], ws[q]->e1.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
                next.push_back(q);
            }
        }
        if (next.empty()) break;
        GH_CUDA(cudaStreamSynchronize(c->stream));
        if ((s = check_status(c, "diffusion")) != GH_OK) return s;
        active.clear();
        for (int q : next)
            if (left[q] > 0 && !(e1[q] <= items[q].p->gs_tol)) active.push_back(q);
    }
    if (ev1) cudaEventRecord(ev1, c->stream);
    return GH_OK;
}

// The whole path for a list of queries, each with its own mesh, workspace,
// sources, parameters and (device) output; all of one precision.  One
// breadth-first launch and one diffusion launch (one per round with gs_tol)
// serve every query; the other stages run per query.  stage_ms6 (may be
// null) gets the stage times.
gh_status solve_items(Ctx *c, std::vector<Item> &items, double *stage_ms6) {
    const int K = (int)items.size();
    gh_status s = GH_OK;
    for (Item &it : items) {
        if (it.m->intrinsic && it.p->form == GH_FORM_FACE && (it.p->path_constraints || it.p->cycle_constraints)) {
            set_error("the constraints of Sec. 5 run on an intrinsic triangulation in the edge form only");
            return GH_EINVAL;
        }
        if ((s = ensure_ws(c, *it.m, *it.w, it.p->fp64, it.p->form, it.p->admm_iters)) != GH_OK) return s;
        it.w->diagnostics = it.p->diagnostics;
        it.w->sweeps = it.p->gs_sweeps;
    }
    std::vector<DevMesh *> meshes(K);
    std::vector<QueryWs *> ws(K);
    std::vector<std::vector<int32_t>> srcs(K);
    for (int q = 0; q < K; ++q) {
        meshes[q] = items[q].m;
        ws[q] = items[q].w;
        srcs[q] = *items[q].src;
    }
    cudaEvent_t ev[8];
    for (auto &e : ev) GH_CUDA(cudaEventCreate(&e));
    do {
        cudaEventRecord(ev[0], c->stream);
        if ((s = build_path_constraints(c, items)) != GH_OK) break;
        if ((s = run_bfs(c, meshes, ws, srcs)) != GH_OK) break;
        for (int q = 0; q < K && s == GH_OK; ++q) {
            const gh_params *p = items[q].p;
            const double t = (p->t > 0) ? p->t : p->m * items[q].m->hbar * items[q].m->hbar;
            s = build_layout(c, *items[q].m, *ws[q], t);
        }
        if (s != GH_OK) break;
        cudaEventRecord(ev[1], c->stream);
        if ((s = run_diffusion(c, items, ws, ev[6], ev[7])) != GH_OK) break;
        cudaEventRecord(ev[2], c->stream);
        // no host synchronisation here: a diffusion timeout leaves every index
        // in range, and the status word is read once the solve is done
        for (int q = 0; q < K && s == GH_OK; ++q) {
            if (items[q].p->diagnostics) s = run_heat_residual(c, *items[q].m, *ws[q]);
            if (s == GH_OK) s = run_normalize(c, *items[q].m, *ws[q]);
        }
        cudaEventRecord(ev[3], c->stream);
        for (int q = 0; q < K && s == GH_OK; ++q) {
            const gh_params *p = items[q].p;
            s = (p->form == GH_FORM_FACE) ? run_face_admm(c, *items[q].m, *ws[q], p)
                                          : run_edge_admm(c, *items[q].m, *ws[q], p);
        }
        cudaEventRecord(ev[4], c->stream);
        for (int q = 0; q < K && s == GH_OK; ++q) s = run_integrate(c, *items[q].m, *ws[q], items[q].d_out_dev);
        cudaEventRecord(ev[5], c->stream);
        if (s != GH_OK) break;
        if ((s = check_status(c, "solve")) != GH_OK) break;
        if (stage_ms6) {
            for (int i = 0; i < 5; ++i) {
                float x = 0;
                cudaEventElapsedTime(&x, ev[i], ev[i + 1]);
                stage_ms6[i] += x;
            }
            float xg = 0;
            cudaEventElapsedTime(&xg, ev[6], ev[7]);
            stage_ms6[5] += xg;
        }
    } while (false);
    for (auto &e : ev) cudaEventDestroy(e);
    return s;
}

// Run queries src[0..K) of one mesh through the whole path; d_out (device)
// gets K x nv.  Queries go in passes of as many as the budget (or 80% of
// free memory) allows, at most 64.
gh_status solve_core(Ctx *c, DevMesh &m, std::vector<QueryWs *> &pool, const std::vector<std::vector<int32_t>> &src,
                     const gh_params *p, double *d_out_dev, double *stage_ms6, int *last_k, double *d_out_host) {
    const int K = (int)src.size();
    size_t per = ws_bytes(m, p->fp64, p->form, p->path_constraints);
    size_t avail;
    if (c->shared->budget) {
        size_t used = c->shared->in_use.load();
        avail = c->shared->budget > used ? c->shared->budget - used : 0;
    } else {
        size_t fr = 0, tot = 0;
        GH_CUDA(cudaMemGetInfo(&fr, &tot));
        avail = (size_t)(0.8 * (double)fr);
    }
    for (QueryWs *w : pool) avail += w->level.p ? per : 0;  // workspaces already held are reusable
    int chunk = (int)std::min<size_t>(64, std::max<size_t>(1, avail / per));
    chunk = std::min(chunk, K);
    while ((int)pool.size() < chunk) pool.push_back(new QueryWs());
    double ms[6] = {0, 0, 0, 0, 0, 0};
    gh_status s = GH_OK;
    for (int q0 = 0; q0 < K && s == GH_OK; q0 += chunk) {
        int kq = std::min(chunk, K - q0);
        std::vector<Item> items(kq);
        for (int q = 0; q < kq; ++q)
            items[q] = Item{&m, pool[q], &src[q0 + q], p, d_out_dev ? d_out_dev + (size_t)(q0 + q) * m.nv : nullptr};
        s = solve_items(c, items, ms);
        // host output: straight from each workspace's distances (the next
        // chunk reuses the workspaces only after these copies, in stream order)
        for (int q = 0; q < kq && s == GH_OK && d_out_host; ++q) {
            cudaError_t e = cudaMemcpyAsync(d_out_host + (size_t)(q0 + q) * m.nv, pool[q]->d0.p,
                                            sizeof(double) * (size_t)m.nv, cudaMemcpyDeviceToHost, c->stream);
            if (e != cudaSuccess) s = cuda_fail(e, "copy of the distances to the host");
        }
    }
    if (s == GH_OK) {
        if (last_k) *last_k = std::min(K, chunk);
        if (stage_ms6) std::copy(ms, ms + 6, stage_ms6);
    }
    return s;
}

static gh_status solve_impl(gh_mesh_s *mh, const std::vector<std::vector<int32_t>> &src, const gh_params *p,
                            double *d_out_dev, double *d_out_host = nullptr) {
    double ms6[6];
    int lk = 0;
    gh_status s = solve_core(&mh->ctx->c, mh->h.m, mh->h.ws, src, p, d_out_dev, ms6, &lk, d_out_host);
    if (s == GH_OK) {
        mh->h.last_k = lk;
        std::copy(ms6, ms6 + 5, mh->h.stage_ms);
        mh->h.gs_kernel_ms = ms6[5];
    }
    return s;
}

gh_status check_pc_sources(const gh_params *p, const std::vector<int32_t> &set) {
    if (p->path_constraints && (int)set.size() > kMaxPc + 1) {
        set_error("path_constraints takes at most " + std::to_string(kMaxPc + 1) + " sources");
        return GH_EINVAL;
    }
    return GH_OK;
}

// sources of one set, validated, sorted and de-duplicated
gh_status prep_sources(const int32_t *src, int32_t nsrc, int64_t nv, std::vector<int32_t> &out) {
    if (!src || nsrc < 1) { set_error("a source set needs at least one vertex"); return GH_EINVAL; }
    out.resize(nsrc);
    if (is_device_ptr(src)) {
        GH_CUDA(cudaMemcpy(out.data(), src, sizeof(int32_t) * nsrc, cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(out.data(), src, sizeof(int32_t) * nsrc);
    }
    for (int32_t v : out)
        if (v < 0 || v >= nv) { set_error("source vertex " + std::to_string(v) + " outside [0, nv)"); return GH_EINVAL; }
    std::sort(out.begin(), out.end());
    out.erase(std::unique(out.begin(), out.end()), out.end());
    return GH_OK;
}

static gh_status solve_to(gh_mesh_s *mh, const std::vector<std::vector<int32_t>> &sets, const gh_params *p,
                          double *d_out) {
    Ctx *c = &mh->ctx->c;
    if (is_device_ptr(d_out)) return solve_impl(mh, sets, p, d_out);
    gh_status s = solve_impl(mh, sets, p, nullptr, d_out);
    const cudaError_t e = cudaStreamSynchronize(c->stream);
    if (s == GH_OK && e != cudaSuccess) s = cuda_fail(e, "copy of the distances to the host");
    return s;
}

}  // namespace gh

using namespace gh;

// accessors used by the serving engine (serve.cu)
gh::Ctx *gh_ctx_launcher(gh_ctx_s *ctx) { return &ctx->c; }
gh::Shared *gh_ctx_shared(gh_ctx_s *ctx) { return &ctx->shared; }
gh::Engine *&gh_ctx_engine(gh_ctx_s *ctx) { return ctx->engine; }
std::mutex &gh_ctx_engine_mutex(gh_ctx_s *ctx) { return ctx->engine_mu; }
int gh_ctx_serve_workers(gh_ctx_s *ctx) { return ctx->serve_workers; }
int gh_ctx_serve_max_batch(gh_ctx_s *ctx) { return ctx->serve_max_batch; }
gh::MeshH *gh_mesh_host(gh_mesh_s *m) { return &m->h; }
gh_ctx_s *gh_mesh_ctx(gh_mesh_s *m) { return m->ctx; }

extern "C" {

gh_status gh_serve_config(gh_ctx ctx, int32_t workers, int32_t max_batch) {
    if (!ctx) { set_error("ctx is NULL"); return GH_EINVAL; }
    if (workers < 1 || workers > 8 || max_batch < 1 || max_batch > 256) {
        set_error("workers must be 1..8 and max_batch 1..256");
        return GH_EINVAL;
    }
    std::lock_guard<std::mutex> lk(ctx->engine_mu);
    if (ctx->engine) { set_error("serving already started on this context"); return GH_EBUSY; }
    ctx->serve_workers = workers;
    ctx->serve_max_batch = max_batch;
    return GH_OK;
}

void gh_params_default(gh_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->m = 1.0;
    p->t = 0.0;
    p->gs_sweeps = 200;
    p->admm_iters = 10;
    p->mu = 100.0;
    p->form = GH_FORM_EDGE;
    p->fp64 = 0;
    p->diagnostics = 0;
    p->early_stop = 0;
    p->eps1 = 1e-5;
    p->eps2 = 1e-5;
    p->path_constraints = 0;
    p->cycle_constraints = 0;
    p->gs_tol = 0.0;
    p->gs_check = 100;
    p->gs_band = 0;
}

const char *gh_version(void) { return "geoheat 0.1 (sm_103a)"; }

const char *gh_last_error(void) { return t_err.c_str(); }

gh_status gh_ctx_create(int device, size_t hbm_budget_bytes, gh_ctx *out) {
    if (!out) { set_error("out is NULL"); return GH_EINVAL; }
    int n = 0;
    GH_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) { set_error("no such CUDA device"); return GH_EINVAL; }
    GH_CUDA(cudaSetDevice(device));
    auto *c = new gh_ctx_s();
    c->c.device = device;
    c->shared.budget = hbm_budget_bytes;
    c->c.shared = &c->shared;
    c->c.launches.p = &c->shared.launches;
    cudaError_t e = cudaDeviceGetAttribute(&c->c.num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->c.status_dev, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->c.status_dev, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->c.bar_dev, sizeof(GridBarrier));
    if (e == cudaSuccess) e = cudaMemset(c->c.bar_dev, 0, sizeof(GridBarrier));
    if (e != cudaSuccess) {
        if (c->c.status_dev) cudaFree(c->c.status_dev);
        if (c->c.bar_dev) cudaFree(c->c.bar_dev);
        delete c;
        return cuda_fail(e, "context setup");
    }
    *out = c;
    return GH_OK;
}

gh_status gh_mesh_free(gh_mesh mesh);

gh_status gh_ctx_destroy(gh_ctx ctx) {
    if (!ctx) return GH_EINVAL;
    if (ctx->engine) engine_stop(ctx->engine);
    ctx->engine = nullptr;
    std::vector<gh_mesh_s *> ms = ctx->meshes;
    for (gh_mesh_s *m : ms) gh_mesh_free(m);
    cudaFree(ctx->c.status_dev);
    cudaFree(ctx->c.bar_dev);
    delete ctx;
    return GH_OK;
}

gh_status gh_ctx_set_stream(gh_ctx ctx, void *stream) {
    if (!ctx) { set_error("ctx is NULL"); return GH_EINVAL; }
    ctx->c.stream = static_cast<cudaStream_t>(stream);
    return GH_OK;
}

gh_status gh_ctx_set_wait_limit(gh_ctx ctx, int64_t microseconds) {
    if (!ctx) { set_error("ctx is NULL"); return GH_EINVAL; }
    ctx->c.wait_limit_ns = microseconds > 0 ? (unsigned long long)microseconds * 1000ull : 2000000000ull;
    return GH_OK;
}

gh_status gh_ctx_memory(gh_ctx ctx, size_t *bytes) {
    if (!ctx || !bytes) { set_error("NULL argument"); return GH_EINVAL; }
    *bytes = ctx->shared.in_use.load();
    return GH_OK;
}

gh_status gh_ctx_stats(gh_ctx ctx, uint64_t *kernel_launches) {
    if (!ctx || !kernel_launches) { set_error("NULL argument"); return GH_EINVAL; }
    *kernel_launches = ctx->shared.launches.load();
    return GH_OK;
}

gh_status gh_mesh_load(gh_ctx ctx, const double *V, int64_t nv, const int32_t *F, int64_t nf, gh_mesh *out) {
    if (!ctx || !V || !F || !out) { set_error("NULL argument"); return GH_EINVAL; }
    if (nv < 3 || nf < 1) { set_error("a mesh needs nv >= 3 and nf >= 1"); return GH_EINVAL; }
    if (6 * nf >= (int64_t)INT32_MAX || nv >= (int64_t)INT32_MAX / 2) { set_error("mesh too large for 32-bit indices"); return GH_EINVAL; }
    std::lock_guard<std::mutex> lk(ctx->mu);
    GH_CUDA(cudaSetDevice(ctx->c.device));
    auto *mh = new gh_mesh_s();
    mh->ctx = ctx;
    mh->h.ctx = &ctx->c;
    mh->h.m.nv = nv;
    mh->h.m.nf = nf;
    gh_status s = build_mesh(&ctx->c, mh->h.m, V, F);
    if (s != GH_OK) {
        DevMesh &m = mh->h.m;
        DBuf *all[] = {&m.P, &m.F, &m.rowptr, &m.col, &m.col_edge, &m.edges, &m.face_edge, &m.face_sign, &m.edge_face,
                       &m.edge_slot, &m.twin, &m.Af, &m.Av, &m.theta, &m.ev, &m.gradop, &m.Aff, &m.face_rec32,
                   &m.face_rec64, &m.cyc_var[0], &m.cyc_var[1], &m.cyc_coef[0], &m.cyc_coef[1], &m.elen, &m.gradop64,
                   &m.evf64, &m.evf32};
        for (DBuf *b : all) dfree(&ctx->c, *b);
        delete mh;
        return s;
    }
    ctx->meshes.push_back(mh);
    *out = mh;
    return GH_OK;
}

gh_status gh_mesh_info(gh_mesh mesh, int64_t *nv, int64_t *ne, int64_t *nf, double *hbar) {
    if (!mesh) { set_error("mesh is NULL"); return GH_EINVAL; }
    if (nv) *nv = mesh->h.m.nv;
    if (ne) *ne = mesh->h.m.ne;
    if (nf) *nf = mesh->h.m.nf;
    if (hbar) *hbar = mesh->h.m.hbar;
    return GH_OK;
}

gh_status gh_mesh_tuning(gh_mesh mesh, int32_t *bfs_cluster) {
    if (!mesh || !bfs_cluster) { set_error("NULL argument"); return GH_EINVAL; }
    DevMesh &m = mesh->h.m;
    std::lock_guard<std::mutex> lk(*m.rec_mu);
    bfs_cluster[0] = m.bfs_cluster[0];
    bfs_cluster[1] = m.bfs_cluster[1];
    return GH_OK;
}

gh_status gh_mesh_intrinsic_delaunay(gh_mesh mesh, int64_t *flips) {
    if (!mesh) { set_error("mesh is NULL"); return GH_EINVAL; }
    std::lock_guard<std::mutex> lk(mesh->ctx->mu);
    if (mesh->h.inflight.load() > 0) { set_error("mesh has serving requests in flight"); return GH_EBUSY; }
    GH_CUDA(cudaSetDevice(mesh->ctx->c.device));
    return mesh_intrinsic_delaunay(&mesh->ctx->c, mesh->h.m, flips);
}

gh_status gh_mesh_set_tuning(gh_mesh mesh, int32_t kind, int32_t bfs_cluster) {
    if (!mesh) { set_error("mesh is NULL"); return GH_EINVAL; }
    if (kind != 0 && kind != 1) { set_error("kind must be 0 (single query) or 1 (batch)"); return GH_EINVAL; }
    if (bfs_cluster != 0 && bfs_cluster != 8 && bfs_cluster != 16) {
        set_error("bfs_cluster must be 0 (tune), 8 or 16");
        return GH_EINVAL;
    }
    GH_CUDA(cudaSetDevice(mesh->ctx->c.device));
    if (bfs_cluster != 0 && !bfs_cluster_supported(bfs_cluster)) {
        set_error("this device cannot place clusters of " + std::to_string(bfs_cluster) + " CTAs");
        return GH_EINVAL;
    }
    DevMesh &m = mesh->h.m;
    std::lock_guard<std::mutex> lk(*m.rec_mu);
    m.bfs_cluster[kind] = bfs_cluster;
    return GH_OK;
}

gh_status gh_mesh_free(gh_mesh mesh) {
    if (!mesh) return GH_EINVAL;
    if (mesh->h.inflight.load() > 0) { set_error("mesh has serving requests in flight"); return GH_EBUSY; }
    gh_ctx_s *ctx = mesh->ctx;
    Ctx *c = &ctx->c;
    {
        std::lock_guard<std::mutex> lk(ctx->engine_mu);
        if (ctx->engine) engine_forget_mesh(ctx->engine, &mesh->h.m);
    }
    cudaStreamSynchronize(c->stream);
    for (QueryWs *w : mesh->h.ws) {
        free_ws(c, w);
        delete w;
    }
    DevMesh &m = mesh->h.m;
    DBuf *all[] = {&m.P, &m.F, &m.rowptr, &m.col, &m.col_edge, &m.edges, &m.face_edge, &m.face_sign, &m.edge_face,
                   &m.edge_slot, &m.twin, &m.Af, &m.Av, &m.theta, &m.ev, &m.gradop, &m.Aff, &m.face_rec32,
                   &m.face_rec64, &m.cyc_var[0], &m.cyc_var[1], &m.cyc_coef[0], &m.cyc_coef[1], &m.elen, &m.gradop64,
                   &m.evf64, &m.evf32};
    for (DBuf *b : all) dfree(c, *b);
    auto it = std::find(ctx->meshes.begin(), ctx->meshes.end(), mesh);
    if (it != ctx->meshes.end()) ctx->meshes.erase(it);
    delete mesh;
    return GH_OK;
}

gh_status gh_solve(gh_mesh mesh, const int32_t *src, int32_t nsrc, const gh_params *params, double *d_out) {
    if (!mesh || !d_out) { set_error("NULL argument"); return GH_EINVAL; }
    gh_status s = validate_params(params);
    if (s != GH_OK) return s;
    std::lock_guard<std::mutex> lk(mesh->ctx->mu);
    GH_CUDA(cudaSetDevice(mesh->ctx->c.device));
    std::vector<std::vector<int32_t>> sets(1);
    if ((s = prep_sources(src, nsrc, mesh->h.m.nv, sets[0])) != GH_OK) return s;
    if ((s = check_pc_sources(params, sets[0])) != GH_OK) return s;
    return solve_to(mesh, sets, params, d_out);
}

gh_status gh_solve_batch(gh_mesh mesh, const int32_t *src_off, const int32_t *src, int32_t K, const gh_params *params,
                         double *d_out) {
    if (!mesh || !src_off || !src || !d_out || K < 1) { set_error("NULL argument or K < 1"); return GH_EINVAL; }
    gh_status s = validate_params(params);
    if (s != GH_OK) return s;
    std::lock_guard<std::mutex> lk(mesh->ctx->mu);
    GH_CUDA(cudaSetDevice(mesh->ctx->c.device));
    std::vector<std::vector<int32_t>> sets(K);
    for (int q = 0; q < K; ++q) {
        int32_t b = src_off[q], e = src_off[q + 1];
        if (b < 0 || e <= b) { set_error("src_off must be increasing and start at >= 0"); return GH_EINVAL; }
        if ((s = prep_sources(src + b, e - b, mesh->h.m.nv, sets[q])) != GH_OK) return s;
        if ((s = check_pc_sources(params, sets[q])) != GH_OK) return s;
    }
    return solve_to(mesh, sets, params, d_out);
}

gh_status gh_debug_size(gh_mesh mesh, int32_t query, int32_t what, int64_t *count, int32_t *elem_bytes) {
    if (!mesh || !count || !elem_bytes) { set_error("NULL argument"); return GH_EINVAL; }
    const DevMesh &m = mesh->h.m;
    QueryWs *w = (query >= 0 && query < (int)mesh->h.ws.size()) ? mesh->h.ws[query] : nullptr;
    bool need_q = !(what == GH_DUMP_EDGES || what == GH_DUMP_FACE_EDGE || what == GH_DUMP_FACE_SIGN ||
                    what == GH_DUMP_THETA || what == GH_DUMP_AV || what == GH_DUMP_AF || what == GH_DUMP_ROWPTR ||
                    what == GH_DUMP_COL || what == GH_DUMP_FACES || what == GH_DUMP_ELEN);
    if (need_q && (!w || !w->level.p)) { set_error("no such query in the last solve"); return GH_EINVAL; }
    int64_t n = 0;
    int32_t eb = 4;
    switch (what) {
    case GH_DUMP_LEVEL: case GH_DUMP_PARENT: n = m.nv; break;
    case GH_DUMP_ORDER: n = w->nreach; break;
    case GH_DUMP_LEVEL_OFF: n = w->nlev + 1; break;
    case GH_DUMP_U_MANT: n = m.nv; eb = 8; break;
    case GH_DUMP_U_EXP: n = m.nv; break;
    case GH_DUMP_H: n = 3 * m.nf; eb = 8; break;
    case GH_DUMP_G: if (w->form != GH_FORM_FACE) { set_error("last solve was not in the face form"); return GH_EINVAL; }
        n = 3 * m.nf; eb = 8; break;
    case GH_DUMP_X: if (w->form != GH_FORM_EDGE) { set_error("last solve was not in the edge form"); return GH_EINVAL; }
        n = m.ne; eb = 8; break;
    case GH_DUMP_D: n = m.nv; eb = 8; break;
    case GH_DUMP_EDGES: n = 2 * m.ne; break;
    case GH_DUMP_FACE_EDGE: case GH_DUMP_FACE_SIGN: n = 3 * m.nf; break;
    case GH_DUMP_THETA: n = m.ne; eb = 8; break;
    case GH_DUMP_AV: n = m.nv; eb = 8; break;
    case GH_DUMP_AF: n = m.nf; eb = 8; break;
    case GH_DUMP_ROWPTR: n = m.nv + 1; break;
    case GH_DUMP_COL: n = 2 * m.ne; break;
    case GH_DUMP_RESID: if (!w->diagnostics) { set_error("solve ran without diagnostics"); return GH_EINVAL; }
        n = 2 * w->admm_iters; eb = 8; break;
    case GH_DUMP_E1: if (!w->diagnostics) { set_error("solve ran without diagnostics"); return GH_EINVAL; }
        n = 1; eb = 8; break;
    case GH_DUMP_T: n = 1; eb = 8; break;
    case GH_DUMP_ITERS: n = 1; eb = 4; break;
    case GH_DUMP_GS_SWEEPS: n = 1; eb = 4; break;
    case GH_DUMP_PC_OFF: n = w->pc_n ? w->pc_n + 1 : 0; break;
    case GH_DUMP_PC_VAR: n = w->pc_ent; break;
    case GH_DUMP_PC_COEF: n = (int64_t)w->pc_ent * w->pc_dim; eb = 8; break;
    case GH_DUMP_FACES: n = 3 * m.nf; break;
    case GH_DUMP_ELEN: n = m.ne; eb = 8; break;
    default: set_error("unknown dump item"); return GH_EINVAL;
    }
    *count = n;
    *elem_bytes = eb;
    return GH_OK;
}

static gh_status copy_real(const void *dev, int fp64, int64_t n, double *out) {
    if (fp64) {
        GH_CUDA(cudaMemcpy(out, dev, sizeof(double) * n, cudaMemcpyDeviceToHost));
    } else {
        std::vector<float> tmp(n);
        GH_CUDA(cudaMemcpy(tmp.data(), dev, sizeof(float) * n, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < n; ++i) out[i] = tmp[i];
    }
    return GH_OK;
}

gh_status gh_debug_dump(gh_mesh mesh, int32_t query, int32_t what, void *out) {
    int64_t n = 0;
    int32_t eb = 0;
    gh_status s = gh_debug_size(mesh, query, what, &n, &eb);
    if (s != GH_OK) return s;
    if (!out) { set_error("out is NULL"); return GH_EINVAL; }
    std::lock_guard<std::mutex> lk(mesh->ctx->mu);
    Ctx *c = &mesh->ctx->c;
    GH_CUDA(cudaStreamSynchronize(c->stream));
    const DevMesh &m = mesh->h.m;
    QueryWs *w = (query >= 0 && query < (int)mesh->h.ws.size()) ? mesh->h.ws[query] : nullptr;
    auto cp = [&](const DBuf &b, size_t bytes) -> gh_status {
        GH_CUDA(cudaMemcpy(out, b.p, bytes, cudaMemcpyDeviceToHost));
        return GH_OK;
    };
    switch (what) {
    case GH_DUMP_LEVEL: return cp(w->level, 4 * n);
    case GH_DUMP_PARENT: return cp(w->parent, 4 * n);
    case GH_DUMP_ORDER: return cp(w->order, 4 * n);
    case GH_DUMP_LEVEL_OFF: return cp(w->lvl_off, 4 * n);
    case GH_DUMP_U_MANT:
    case GH_DUMP_U_EXP: {
        // state is in layout order; scatter back to vertex order
        std::vector<int32_t> pos(m.nv);
        GH_CUDA(cudaMemcpy(pos.data(), w->pos.p, 4 * m.nv, cudaMemcpyDeviceToHost));
        const DBuf &U = w->final_buf ? w->U1 : w->U0;
        std::vector<double> mant(m.nv, 0.0);
        std::vector<int32_t> ex(m.nv, kZeroExp);
        if (w->fp64) {
            std::vector<XVal<double>> u(w->nreach);
            GH_CUDA(cudaMemcpy(u.data(), U.p, sizeof(XVal<double>) * w->nreach, cudaMemcpyDeviceToHost));
            for (int64_t v = 0; v < m.nv; ++v) if (pos[v] >= 0) { mant[v] = u[pos[v]].m; ex[v] = u[pos[v]].e; }
        } else {
            std::vector<XVal<float>> u(w->nreach);
            GH_CUDA(cudaMemcpy(u.data(), U.p, sizeof(XVal<float>) * w->nreach, cudaMemcpyDeviceToHost));
            for (int64_t v = 0; v < m.nv; ++v) if (pos[v] >= 0) { mant[v] = u[pos[v]].m; ex[v] = u[pos[v]].e; }
        }
        if (what == GH_DUMP_U_MANT) std::memcpy(out, mant.data(), 8 * m.nv);
        else std::memcpy(out, ex.data(), 4 * m.nv);
        return GH_OK;
    }
    case GH_DUMP_H: return copy_real(w->h.p, w->fp64, n, (double *)out);
    case GH_DUMP_G: return copy_real(w->g0.p, w->fp64, n, (double *)out);
    case GH_DUMP_X: return copy_real(w->x.p, w->fp64, n, (double *)out);
    case GH_DUMP_D: return cp(w->d0, 8 * n);
    case GH_DUMP_EDGES: return cp(m.edges, 4 * n);
    case GH_DUMP_FACE_EDGE: return cp(m.face_edge, 4 * n);
    case GH_DUMP_FACE_SIGN: {
        std::vector<int8_t> sg(n);
        GH_CUDA(cudaMemcpy(sg.data(), m.face_sign.p, n, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < n; ++i) ((int32_t *)out)[i] = sg[i];
        return GH_OK;
    }
    case GH_DUMP_THETA: return cp(m.theta, 8 * n);
    case GH_DUMP_AV: return cp(m.Av, 8 * n);
    case GH_DUMP_AF: return cp(m.Af, 8 * n);
    case GH_DUMP_ROWPTR: return cp(m.rowptr, 4 * n);
    case GH_DUMP_COL: return cp(m.col, 4 * n);
    case GH_DUMP_RESID: return cp(w->resid, 8 * n);
    case GH_DUMP_E1: return cp(w->e1, 8);
    case GH_DUMP_T: std::memcpy(out, &w->t, 8); return GH_OK;
    case GH_DUMP_ITERS:
        GH_CUDA(cudaMemcpy(out, (const char *)w->actl.p + offsetof(AdmmCtl, iters_done), 4, cudaMemcpyDeviceToHost));
        return GH_OK;
    case GH_DUMP_GS_SWEEPS: std::memcpy(out, &w->sweeps_run, 4); return GH_OK;
    case GH_DUMP_PC_OFF: return n ? cp(w->pc_off, 4 * n) : GH_OK;
    case GH_DUMP_PC_VAR: return n ? cp(w->pc_var, 4 * n) : GH_OK;
    case GH_DUMP_PC_COEF: return n ? cp(w->pc_coef, 8 * n) : GH_OK;
    case GH_DUMP_FACES: return cp(m.F, 4 * n);
    case GH_DUMP_ELEN: return cp(m.elen, 8 * n);
    default: set_error("unknown dump item"); return GH_EINVAL;
    }
}

gh_status gh_stage_times(gh_mesh mesh, double *ms6) {
    if (!mesh || !ms6) { set_error("NULL argument"); return GH_EINVAL; }
    std::copy(mesh->h.stage_ms, mesh->h.stage_ms + 5, ms6);
    ms6[5] = mesh->h.gs_kernel_ms;
    return GH_OK;
}

}  // extern "C"
