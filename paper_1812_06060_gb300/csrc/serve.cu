// Serving: asynchronous requests with continuous batching.
//
// gh_submit queues a request and returns at once.  Worker threads (two by
// default), each with its own CUDA stream, status word and workspaces, take
// the pending requests as they arrive: a worker admits, in arrival order,
// the requests of the oldest pending one's precision and of a similar amount
// of work (vertices x sweeps within a factor of 4 of it) -- on any mesh, with
// any parameters -- as long as their workspaces fit the memory budget (or
// the device's free memory) and the batch limit, and runs them as one batch:
// one breadth-first launch and one persistent diffusion launch for all of
// them (every query with its own mesh and sweep count; with gs_tol, one
// launch per round for the queries still running), then the per-query
// stages.  Requests that arrive while a batch is on the GPU join the next
// batch of whichever worker frees up first: one worker's breadth-first,
// layout and ADMM work overlaps the other's diffusion, whose launch takes
// the whole GPU (a second diffusion launch waits until the first ends).  Results are the same as a
// blocking gh_solve of the same request: the arithmetic of every vertex does
// not depend on the batch it ran in.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <stdexcept>
#include <thread>
#include <tuple>

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
    int running = 0;                                      // workers with a batch on the GPU
    size_t reserved = 0;                                  // bytes admitted batches may still allocate
    // workspaces no batch is using, per (mesh, form, precision) of their last request
    std::map<std::tuple<DevMesh *, int, int>, std::vector<QueryWs *>> idle;
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

// device bytes a new batch may take (E->mu held): the budget less what the
// context holds, or 80% of the device's free memory without a budget, less
// what the batches admitted earlier may still allocate (a batch allocates
// after it leaves the lock, so its admitted bytes stay reserved until its
// solve has returned)
static size_t avail_bytes(Engine *E, Ctx *c) {
    Shared *sh = c->shared;
    size_t a;
    if (sh->budget) {
        size_t used = sh->in_use.load();
        a = sh->budget > used ? sh->budget - used : 0;
    } else {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            (void)cudaGetLastError();
            return 0;
        }
        a = (size_t)(0.8 * (double)fr);
    }
    return a > E->reserved ? a - E->reserved : 0;
}

// frees idle workspaces (E->mu held) until `need` bytes are available or
// none is left; returns the bytes available afterwards
static size_t release_idle(Engine *E, Worker *W, size_t need) {
    size_t avail = avail_bytes(E, &W->c);
    for (auto it = E->idle.begin(); it != E->idle.end() && avail < need;) {
        std::vector<QueryWs *> &v = it->second;
        while (!v.empty() && avail < need) {
            free_ws(&W->c, v.back());
            delete v.back();
            v.pop_back();
            avail = avail_bytes(E, &W->c);
        }
        it = v.empty() ? E->idle.erase(it) : std::next(it);
    }
    return avail;
}

static void worker_loop(Engine *E, Worker *W) {
    cudaSetDevice(W->c.device);
    while (true) {
        std::vector<Request *> batch;
        std::vector<QueryWs *> wsq;
        size_t batch_cost = 0;
        {
            std::unique_lock<std::mutex> lk(E->mu);
            while (true) {
                E->cv_work.wait(lk, [&] { return E->stop || !E->pending.empty(); });
                if (E->stop && E->pending.empty()) return;
                const int fp64 = E->pending.front()->p.fp64;
                auto work = [](const Request *r) {
                    return (double)gh_mesh_host(r->mesh)->m.nv * (double)std::max(1, r->p.gs_sweeps);
                };
                const double w0 = work(E->pending.front());
                // admission in arrival order: an idle workspace of the request's
                // mesh costs nothing, a new one its size (plus the growth of this
                // worker's output buffer); a request that does not fit waits
                size_t avail = avail_bytes(E, &W->c);
                size_t out_bytes = 0;
                batch_cost = 0;
                std::map<std::tuple<DevMesh *, int, int>, size_t> taken;
                for (auto it = E->pending.begin(); it != E->pending.end() && (int)batch.size() < E->max_batch;) {
                    Request *r = *it;
                    const double wr = work(r);
                    if (r->p.fp64 != fp64 || wr > 4.0 * w0 || 4.0 * wr < w0) {
                        ++it;
                        continue;
                    }
                    DevMesh *m = &gh_mesh_host(r->mesh)->m;
                    const auto key = std::make_tuple(m, r->p.form, fp64);
                    const size_t k = taken[key];
                    auto idl = E->idle.find(key);
                    const bool reuse = idl != E->idle.end() && k < idl->second.size();
                    const size_t ob = out_bytes + sizeof(double) * (size_t)m->nv;
                    const size_t grow = ob > W->dout.bytes ? ob - std::max(out_bytes, W->dout.bytes) : 0;
                    const size_t cost = (reuse ? 0 : ws_bytes(*m, fp64, r->p.form, r->p.path_constraints)) + grow;
                    if (cost > avail) {
                        if (!batch.empty()) break;   // the rest waits for the next batch
                        avail = release_idle(E, W, cost);
                        if (cost > avail) break;     // the oldest request waits for memory
                    }
                    avail -= cost;
                    batch_cost += cost;
                    out_bytes = ob;
                    taken[key] = k + 1;
                    batch.push_back(r);
                    r->state = 1;
                    it = E->pending.erase(it);
                }
                if (!batch.empty()) break;
                // nothing fits: wait for a running batch to give memory back; with
                // none running (and every idle workspace freed) the oldest
                // request can never fit and fails
                if (E->running == 0) {
                    Request *r = E->pending.front();
                    E->pending.pop_front();
                    r->status = GH_ENOMEM;
                    r->err = "the request's workspace does not fit the context's device memory budget";
                    r->state = 2;
                    gh_mesh_host(r->mesh)->inflight.fetch_sub(1);
                    E->cv_done.notify_all();
                    continue;
                }
                E->cv_work.wait(lk);
            }
            // the batch's workspaces: idle ones of its meshes first, then new ones
            for (Request *r : batch) {
                auto idl = E->idle.find(std::make_tuple(&gh_mesh_host(r->mesh)->m, r->p.form, r->p.fp64));
                if (idl != E->idle.end() && !idl->second.empty()) {
                    wsq.push_back(idl->second.back());
                    idl->second.pop_back();
                    if (idl->second.empty()) E->idle.erase(idl);
                } else {
                    wsq.push_back(new QueryWs());
                }
            }
            ++E->running;
            E->reserved += batch_cost;
        }
        gh_status st = GH_OK;
        std::string err;
        std::vector<size_t> off(batch.size() + 1, 0);
        for (size_t q = 0; q < batch.size(); ++q) off[q + 1] = off[q] + (size_t)gh_mesh_host(batch[q]->mesh)->m.nv;
        try {
            st = dalloc(&W->c, W->dout, sizeof(double) * off.back());
            if (st == GH_OK) {
                std::vector<Item> items(batch.size());
                for (size_t q = 0; q < batch.size(); ++q)
                    items[q] = Item{&gh_mesh_host(batch[q]->mesh)->m, wsq[q], &batch[q]->src, &batch[q]->p,
                                    ptr<double>(W->dout) + off[q]};
                st = solve_items(&W->c, items, nullptr);
            }
            if (st != GH_OK) err = gh_last_error();
        } catch (const std::exception &ex) {
            st = GH_EDEVICE;
            err = std::string("serving worker: ") + ex.what();
        }
        {
            // the batch's allocations are done (or failed): its reservation ends
            std::lock_guard<std::mutex> lk(E->mu);
            E->reserved -= std::min(E->reserved, batch_cost);
        }
        E->cv_work.notify_all();
        if (st == GH_OK) {
            try {
                for (size_t q = 0; q < batch.size(); ++q) batch[q]->d.resize(off[q + 1] - off[q]);
            } catch (const std::exception &ex) {
                st = GH_ENOMEM;
                err = "host memory for served distances";
            }
        }
        if (st == GH_OK) {
            cudaError_t e = cudaSuccess;
            for (size_t q = 0; q < batch.size() && e == cudaSuccess; ++q)
                e = cudaMemcpyAsync(batch[q]->d.data(), ptr<double>(W->dout) + off[q], sizeof(double) * (off[q + 1] - off[q]),
                                    cudaMemcpyDeviceToHost, W->c.stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(W->c.stream);
            if (e != cudaSuccess) {
                st = cuda_fail(e, "copy of served distances");
                err = gh_last_error();
            }
        }
        {
            std::lock_guard<std::mutex> lk(E->mu);
            for (size_t q = 0; q < batch.size(); ++q) {
                E->idle[std::make_tuple(&gh_mesh_host(batch[q]->mesh)->m, batch[q]->p.form, batch[q]->p.fp64)]
                    .push_back(wsq[q]);
                Request *r = batch[q];
                r->status = st;
                r->err = err;
                r->state = 2;
                gh_mesh_host(r->mesh)->inflight.fetch_sub(1);
            }
            --E->running;
        }
        E->cv_done.notify_all();
        E->cv_work.notify_all();   // memory came back: a waiting admission may fit now
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
        W->c.gs_share = 1;
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
    for (Worker *W : E->workers)
        if (W->th.joinable()) W->th.join();
    for (auto &kv : E->idle)
        for (QueryWs *w : kv.second) {
            free_ws(&E->workers[0]->c, w);
            delete w;
        }
    E->idle.clear();
    for (Worker *W : E->workers) {
        dfree(&W->c, W->dout);
        cudaStreamDestroy(W->c.stream);
        cudaFree(W->c.status_dev);
        cudaFree(W->c.bar_dev);
        delete W;
    }
    for (auto &kv : E->all) delete kv.second;
    delete E;
}

// A mesh is being freed (no request of it in flight): drop the workspaces
// the workers keep for it.
void engine_forget_mesh(Engine *E, DevMesh *m) {
    std::lock_guard<std::mutex> lk(E->mu);
    for (auto it = E->idle.begin(); it != E->idle.end();) {
        if (std::get<0>(it->first) != m || E->workers.empty()) {
            ++it;
            continue;
        }
        for (QueryWs *w : it->second) {
            free_ws(&E->workers[0]->c, w);
            delete w;
        }
        it = E->idle.erase(it);
    }
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
    if ((s = prep_sources(src, nsrc, gh_mesh_host(mesh)->m.nv, r->src)) != GH_OK ||
        (s = check_pc_sources(params, r->src)) != GH_OK) {
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
