// Serving: asynchronous requests with continuous batching.
//
// gh_submit queues a request and returns at once.  Worker threads (two by
// default), each with its own CUDA stream, status word and workspaces, take
// the pending requests as they arrive: a worker admits, in arrival order,
// the requests that share the mesh and parameters of the oldest pending one,
// as many as the memory budget (or the device's free memory) and the batch
// limit allow, and runs them as one batch: one breadth-first launch and one
// persistent diffusion launch for all of them, then the per-query stages.
// Requests that arrive while a batch is on the GPU join the next batch of
// whichever worker frees up first, so two batches' work overlaps on the
// device; each worker's diffusion launch takes a 1/workers share of the SMs
// so the two can be resident together.  Results are the same as a blocking
// gh_solve of the same request: the arithmetic of every vertex does not
// depend on the batch it ran in.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <stdexcept>
#include <thread>

#include "internal.cuh"

struct gh_mesh_s;
struct gh_ctx_s;

namespace gh {

struct Request {
    gh_req id = 0;
    gh_mesh_s *mesh = nullptr;
    std::vector<int32_t> src;
    gh_params p{};
    std::vector<double> d;
    int state = 0;          // 0 pending, 1 running, 2 done
    gh_status status = GH_OK;
    std::string err;
};

struct Worker {
    Ctx c;
    std::vector<QueryWs *> pool;
    DBuf dout;
    std::thread th;
};

struct Engine {
    gh_ctx_s *ctx = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::map<gh_req, Request *> all;
    gh_req next_id = 1;
    bool stop = false;
    int max_batch = 32;
    std::vector<Worker *> workers;
};

}  // namespace gh

// the parts of the context and mesh handles serving needs (defined in api.cu)
gh::Ctx *gh_ctx_launcher(gh_ctx_s *ctx);
gh::Shared *gh_ctx_shared(gh_ctx_s *ctx);
gh::Engine *&gh_ctx_engine(gh_ctx_s *ctx);
std::mutex &gh_ctx_engine_mutex(gh_ctx_s *ctx);
int gh_ctx_serve_workers(gh_ctx_s *ctx);
int gh_ctx_serve_max_batch(gh_ctx_s *ctx);
gh::MeshH *gh_mesh_host(gh_mesh_s *m);
gh_ctx_s *gh_mesh_ctx(gh_mesh_s *m);

namespace gh {

static bool same_batch(const Request *a, const Request *b) {
    return a->mesh == b->mesh && a->p.form == b->p.form && a->p.fp64 == b->p.fp64 &&
           a->p.gs_sweeps == b->p.gs_sweeps && a->p.admm_iters == b->p.admm_iters && a->p.mu == b->p.mu &&
           a->p.m == b->p.m && a->p.t == b->p.t && a->p.diagnostics == b->p.diagnostics;
}

static void worker_loop(Engine *E, Worker *W) {
    cudaSetDevice(W->c.device);
    while (true) {
        std::vector<Request *> batch;
        {
            std::unique_lock<std::mutex> lk(E->mu);
            E->cv_work.wait(lk, [&] { return E->stop || !E->pending.empty(); });
            if (E->stop && E->pending.empty()) return;
            Request *first = E->pending.front();
            DevMesh &m = gh_mesh_host(first->mesh)->m;
            // admission: requests whose workspaces fit next to what is held
            size_t per = ws_bytes(m, first->p.fp64, first->p.form);
            size_t avail;
            Shared *sh = W->c.shared;
            if (sh->budget) {
                size_t used = sh->in_use.load();
                avail = sh->budget > used ? sh->budget - used : 0;
            } else {
                size_t fr = 0, tot = 0;
                cudaMemGetInfo(&fr, &tot);
                avail = (size_t)(0.8 * (double)fr);
            }
            for (QueryWs *w : W->pool) avail += (w->level.p && w->cap_nv == m.nv) ? per : 0;
            size_t kmax = std::max<size_t>(1, std::min<size_t>((size_t)E->max_batch, avail / per));
            for (auto it = E->pending.begin(); it != E->pending.end() && batch.size() < kmax;) {
                if (same_batch(*it, first)) {
                    batch.push_back(*it);
                    (*it)->state = 1;
                    it = E->pending.erase(it);
                } else {
                    ++it;
                }
            }
        }
        Request *r0 = batch[0];
        DevMesh &m = gh_mesh_host(r0->mesh)->m;
        std::vector<std::vector<int32_t>> sets;
        for (Request *r : batch) sets.push_back(r->src);
        gh_status st = GH_OK;
        std::string err;
        try {
            st = dalloc(&W->c, W->dout, sizeof(double) * (size_t)m.nv * batch.size());
            if (st == GH_OK) st = solve_core(&W->c, m, W->pool, sets, &r0->p, ptr<double>(W->dout), nullptr, nullptr);
            if (st != GH_OK) err = gh_last_error();
        } catch (const std::exception &ex) {
            st = GH_EDEVICE;
            err = std::string("serving worker: ") + ex.what();
        }
        if (st == GH_OK) {
            for (size_t q = 0; q < batch.size() && st == GH_OK; ++q) {
                try {
                    batch[q]->d.resize(m.nv);
                } catch (const std::exception &ex) {
                    st = GH_ENOMEM;
                    err = "host memory for served distances";
                    break;
                }
                cudaError_t e = cudaMemcpyAsync(batch[q]->d.data(), ptr<double>(W->dout) + q * m.nv,
                                                sizeof(double) * m.nv, cudaMemcpyDeviceToHost, W->c.stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(W->c.stream);
                if (e != cudaSuccess) {
                    st = cuda_fail(e, "copy of served distances");
                    err = gh_last_error();
                }
            }
        }
        {
            std::lock_guard<std::mutex> lk(E->mu);
            for (Request *r : batch) {
                r->status = st;
                r->err = err;
                r->state = 2;
                gh_mesh_host(r->mesh)->inflight.fetch_sub(1);
            }
        }
        E->cv_done.notify_all();
    }
}

static gh_status engine_start(gh_ctx_s *ctx, Engine *&out) {
    Engine *E = new Engine();
    E->ctx = ctx;
    E->max_batch = gh_ctx_serve_max_batch(ctx);
    const int nw = gh_ctx_serve_workers(ctx);
    Ctx *base = gh_ctx_launcher(ctx);
    for (int i = 0; i < nw; ++i) {
        Worker *W = new Worker();
        W->c = *base;
        W->c.gs_share = nw;
        cudaError_t e = cudaStreamCreateWithFlags(&W->c.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMalloc((void **)&W->c.status_dev, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(W->c.status_dev, 0, sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc((void **)&W->c.bar_dev, sizeof(GridBarrier));
        if (e == cudaSuccess) e = cudaMemset(W->c.bar_dev, 0, sizeof(GridBarrier));
        if (e != cudaSuccess) {
            if (W->c.status_dev) cudaFree(W->c.status_dev);
            if (W->c.bar_dev) cudaFree(W->c.bar_dev);
            if (W->c.stream) cudaStreamDestroy(W->c.stream);
            delete W;
            out = E;   // the workers started so far keep serving
            return cuda_fail(e, "serving worker setup");
        }
        E->workers.push_back(W);
        W->th = std::thread(worker_loop, E, W);
    }
    out = E;
    return GH_OK;
}

void engine_stop(Engine *E) {
    {
        std::lock_guard<std::mutex> lk(E->mu);
        E->stop = true;
    }
    E->cv_work.notify_all();
    for (Worker *W : E->workers) {
        if (W->th.joinable()) W->th.join();
        for (QueryWs *w : W->pool) {
            free_ws(&W->c, w);
            delete w;
        }
        dfree(&W->c, W->dout);
        cudaStreamDestroy(W->c.stream);
        cudaFree(W->c.status_dev);
        cudaFree(W->c.bar_dev);
        delete W;
    }
    for (auto &kv : E->all) delete kv.second;
    delete E;
}

}  // namespace gh

using namespace gh;

extern "C" {

gh_status gh_submit(gh_ctx ctx, gh_mesh mesh, const int32_t *src, int32_t nsrc, const gh_params *params,
                    gh_req *out) {
    if (!ctx || !mesh || !out) { set_error("NULL argument"); return GH_EINVAL; }
    if (gh_mesh_ctx(mesh) != ctx) { set_error("mesh belongs to another context"); return GH_EINVAL; }
    gh_status s = validate_params(params);
    if (s != GH_OK) return s;
    auto *r = new Request();
    cudaSetDevice(gh_ctx_launcher(ctx)->device);
    if ((s = prep_sources(src, nsrc, gh_mesh_host(mesh)->m.nv, r->src)) != GH_OK) {
        delete r;
        return s;
    }
    r->mesh = mesh;
    r->p = *params;
    Engine *E = nullptr;
    {
        std::lock_guard<std::mutex> lk(gh_ctx_engine_mutex(ctx));
        Engine *&slot = gh_ctx_engine(ctx);
        if (!slot) {
            s = engine_start(ctx, slot);
            if (s != GH_OK && (!slot || slot->workers.empty())) {
                if (slot) { engine_stop(slot); slot = nullptr; }
                delete r;
                return s;
            }
        }
        E = slot;
    }
    {
        std::lock_guard<std::mutex> lk(E->mu);
        r->id = E->next_id++;
        E->all[r->id] = r;
        E->pending.push_back(r);
        gh_mesh_host(mesh)->inflight.fetch_add(1);
        *out = r->id;
    }
    E->cv_work.notify_one();
    return GH_OK;
}

static Engine *engine_of(gh_ctx ctx) {
    std::lock_guard<std::mutex> lk(gh_ctx_engine_mutex(ctx));
    return gh_ctx_engine(ctx);
}

gh_status gh_poll(gh_ctx ctx, gh_req req, int *done) {
    if (!ctx || !done) { set_error("NULL argument"); return GH_EINVAL; }
    Engine *E = engine_of(ctx);
    if (!E) { set_error("unknown request"); return GH_ENOTFOUND; }
    std::lock_guard<std::mutex> lk(E->mu);
    auto it = E->all.find(req);
    if (it == E->all.end()) { set_error("unknown request"); return GH_ENOTFOUND; }
    *done = it->second->state == 2;
    return GH_OK;
}

gh_status gh_wait(gh_ctx ctx, gh_req req, double *d_out, int64_t timeout_us) {
    if (!ctx || !d_out) { set_error("NULL argument"); return GH_EINVAL; }
    Engine *E = engine_of(ctx);
    if (!E) { set_error("unknown request"); return GH_ENOTFOUND; }
    Request *r = nullptr;
    {
        std::unique_lock<std::mutex> lk(E->mu);
        auto it = E->all.find(req);
        if (it == E->all.end()) { set_error("unknown request"); return GH_ENOTFOUND; }
        r = it->second;
        auto ready = [&] { return r->state == 2; };
        if (timeout_us < 0) {
            E->cv_done.wait(lk, ready);
        } else if (!E->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
            set_error("request not finished within the timeout");
            return GH_ETIMEOUT;
        }
        E->all.erase(it);
    }
    gh_status s = r->status;
    if (s != GH_OK) {
        set_error(r->err);
    } else if (is_device_ptr(d_out)) {
        cudaSetDevice(gh_ctx_launcher(ctx)->device);
        cudaError_t e = cudaMemcpy(d_out, r->d.data(), sizeof(double) * r->d.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) s = cuda_fail(e, "copy of served distances");
    } else {
        std::memcpy(d_out, r->d.data(), sizeof(double) * r->d.size());
    }
    delete r;
    return s;
}

}  // extern "C"
