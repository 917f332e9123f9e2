// Solve server (include/helm_server.h): request queue, batching, factor cache with HBM
// admission (server_cache.h), host worker threads.  Every solve is helm_solve /
// helm_adjoint_solve on a cached factor; each cache entry has its own CUDA stream, so the
// batches of different entries run concurrently.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>
#include <cuda_runtime.h>
#include "helm.h"
#include "helm_server.h"
#include "abi_internal.h"
#include "server_cache.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr size_t kMiB = (size_t)1 << 20;

struct Model {
    helm_grid grid{};
    double *m_dev = nullptr;
};

struct Slot {   // payload of a cache entry
    cudaStream_t st = nullptr;
    helm_op_t *op = nullptr;
    helm_factor_t *f = nullptr;
};

// right-hand sides the factor's refinement scratch is sized for
int scratch_cap(const Slot *sl) { return sl && sl->f ? sl->f->cap : 0; }

struct Pending {
    int64_t ticket;
    helm_request r;
    Clock::time_point arrival;
};

struct State {
    bool done = false;
    helm_request_info info{};
};

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

void destroy_slot(Slot *sl) {
    if (!sl) return;
    if (sl->st) cudaStreamSynchronize(sl->st);
    if (sl->f) helm_factor_destroy(sl->f);
    if (sl->op) helm_op_destroy(sl->op);
    if (sl->st) {
        cudaStreamSynchronize(sl->st);
        cudaStreamDestroy(sl->st);
    }
    delete sl;
}

}  // namespace

struct helm_server {
    helm_server_opts opts{};
    int device = 0;
    cudaStream_t st = nullptr;   // model uploads
    std::deque<Model> models;   // appended under the lock; workers copy an entry under it

    mutable std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_room;
    std::deque<Pending> queue;
    std::unordered_map<int64_t, State> states;
    std::unordered_map<helm_srv::Key, int, helm_srv::KeyHash> busy;   // entries a worker is using
    helm_srv::Cache cache{0};
    bool stop = false;
    int running = 0;   // batches between their reservation and their release
    int64_t next_ticket = 1;
    helm_server_counters stats{};
    std::vector<std::thread> workers;

    // device bytes as admission counts them (see helm_server.h)
    size_t factor_bytes(const helm_grid &g, int prec) const {
        const size_t N = (size_t)g.nx * g.nz, blk = (size_t)g.nz * g.nz * 8;
        const helm::GridGeom geom{g.nx, g.nz, g.lx / (g.nx - 1), g.lz / (g.nz - 1), g.lumping};
        if (helm::factor_picks_bcr(geom, (helm_prec)prec, HELM_FACTOR_AUTO)) {
            // block cyclic reduction: the inverses of every line and P, Q, W, V of the eliminated
            // ones, and as much again of working blocks while it factors (counted throughout)
            const size_t kept = ((size_t)g.nx + 4 * ((size_t)g.nx / 2 + 1)) * blk;
            return 2 * kept + 96 * N + 97 * kMiB;   // + the split-K tiles (32 MB kept, 64 MB while factoring)
        }
        return (size_t)g.nx * g.nz * g.nz * (prec == HELM_MIXED ? 8 : 16) + 96 * N + kMiB;
    }
    size_t scratch_bytes(const helm_grid &g, int prec, int nrhs) const {   // refinement scratch in the factor
        return prec == HELM_MIXED ? (size_t)g.nx * g.nz * nrhs * 64 + (size_t)nrhs * 16 : (size_t)nrhs * 16;
    }
    size_t staging_bytes(const helm_grid &g, int nrhs) const {   // device B and X of a batch
        return (size_t)g.nx * g.nz * nrhs * 32;
    }
    size_t footprint(const helm_grid &g, int prec, int nrhs) const {
        return factor_bytes(g, prec) + scratch_bytes(g, prec, nrhs) + staging_bytes(g, nrhs);
    }

    void worker_loop();
    void run_batch(const Model &md, std::vector<Pending> &batch, Slot *sl, bool hit,
                   std::vector<helm_request_info> &infos, helm_status &status);
};

namespace {
helm_srv::Key key_of(const helm_request &r) { return helm_srv::Key{r.model, r.omega, r.prec}; }
}

void helm_server::worker_loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        // the oldest request whose entry no other worker is using
        auto first = queue.end();
        for (auto it = queue.begin(); it != queue.end(); ++it)
            if (!busy.count(key_of(it->r))) { first = it; break; }
        if (first == queue.end()) {
            if (stop && queue.empty()) return;
            cv_work.wait(lk);
            continue;
        }
        const helm_srv::Key key = key_of(first->r);
        const int adjoint = first->r.adjoint != 0;
        const helm_grid g = models[key.model].grid;
        // the batch: later requests of the same key and direction, in arrival order, while the
        // batch stays within max_batch_rhs and its footprint within the budget
        std::vector<Pending> batch;
        int rhs = 0;
        for (auto it = first; it != queue.end();) {
            const bool same = key_of(it->r) == key && (it->r.adjoint != 0) == adjoint;
            if (same && (batch.empty() || (rhs + it->r.nrhs <= opts.max_batch_rhs &&
                                           footprint(g, key.prec, rhs + it->r.nrhs) <= cache.budget()))) {
                rhs += it->r.nrhs;
                batch.push_back(*it);
                it = queue.erase(it);
            } else {
                ++it;
            }
        }
        busy[key] = 1;
        const Model md = models[key.model];
        // room for the batch: its factor (on a miss), the growth of the factor's refinement
        // scratch and the device copies of B and X.  A worker that has to wait drops its pin,
        // so that two waiting workers never hold each other's room.
        helm_srv::Entry *entry = nullptr;
        size_t need = 0, grow = 0;
        std::vector<void *> victims;
        bool refuse = false;
        for (;;) {
            entry = cache.acquire(key);
            const int cap_old = entry ? scratch_cap(static_cast<Slot *>(entry->payload)) : 0;
            grow = rhs > cap_old ? scratch_bytes(g, key.prec, rhs) - scratch_bytes(g, key.prec, cap_old) : 0;
            need = (entry ? grow : factor_bytes(g, key.prec) + scratch_bytes(g, key.prec, rhs)) + staging_bytes(g, rhs);
            if (cache.reserve(need, &victims)) break;
            if (entry) cache.unpin(entry);
            if (running == 0) {
                // nothing else holds room: only this key's own entry (its scratch sized for an
                // earlier, larger batch) is in the way; drop it and rebuild (a batch's own
                // footprint is within the budget)
                if (void *p = cache.evict(key)) {
                    victims.push_back(p);
                    continue;
                }
                refuse = true;   // not reached: a batch's own footprint is within the budget
                break;
            }
            cv_room.wait(lk);
        }
        if (refuse) {
            stats.evictions += (int64_t)victims.size();
            busy.erase(key);
            for (const Pending &p : batch) {
                auto it = states.find(p.ticket);
                if (it != states.end()) {
                    it->second.info.status = HELM_ENOMEM;
                    it->second.done = true;
                }
                ++stats.completed;
            }
            lk.unlock();
            for (void *v : victims) destroy_slot(static_cast<Slot *>(v));
            lk.lock();
            cv_done.notify_all();
            cv_work.notify_all();
            continue;
        }
        ++running;
        const bool hit = entry != nullptr;
        cache.count(hit);
        stats.evictions += (int64_t)victims.size();
        Slot *sl = hit ? static_cast<Slot *>(entry->payload) : new Slot();
        const int cap_before = scratch_cap(sl);
        const auto t_start = Clock::now();
        lk.unlock();

        for (void *v : victims) destroy_slot(static_cast<Slot *>(v));
        std::vector<helm_request_info> infos(batch.size());
        helm_status status = HELM_OK;
        run_batch(md, batch, sl, hit, infos, status);
        const auto t_end = Clock::now();

        lk.lock();
        --running;
        cache.release(staging_bytes(g, rhs));
        // the scratch the factor actually holds now (it grows inside the solve)
        const int cap_after = scratch_cap(sl);
        const size_t grown = cap_after > cap_before ? scratch_bytes(g, key.prec, cap_after) -
                                                          scratch_bytes(g, key.prec, cap_before)
                                                    : 0;
        if (hit) {
            cache.grow(entry, grown);
            cache.release(grow - std::min(grow, grown));
            cache.unpin(entry);
        } else if (sl->f) {
            const size_t bytes = factor_bytes(g, key.prec) + scratch_bytes(g, key.prec, cap_after);
            const size_t reserved = factor_bytes(g, key.prec) + scratch_bytes(g, key.prec, rhs);
            cache.unpin(cache.insert(key, bytes, sl));
            cache.release(reserved - std::min(reserved, bytes));
            ++stats.factor_builds;
        } else {
            // the build failed: nothing stays resident
            cache.release(factor_bytes(g, key.prec) + scratch_bytes(g, key.prec, rhs));
            lk.unlock();
            destroy_slot(sl);
            lk.lock();
        }
        busy.erase(key);
        ++stats.batches;
        for (size_t b = 0; b < batch.size(); ++b) {
            helm_request_info &in = infos[b];
            in.cache_hit = hit ? 1 : 0;
            in.batch_rhs = rhs;
            in.queue_ms = ms_between(batch[b].arrival, t_start);
            in.total_ms = ms_between(batch[b].arrival, t_end);
            auto it = states.find(batch[b].ticket);
            if (it != states.end()) {
                it->second.info = in;
                it->second.done = true;
            }
            ++stats.completed;
            if (in.status == HELM_OK) stats.rhs_solved += batch[b].r.nrhs;
        }
        cv_done.notify_all();
        cv_room.notify_all();
        cv_work.notify_all();
    }
}

// One batch, outside the server lock: build the factor on a miss, copy the right-hand
// sides in, solve, copy the results out, all on the entry's stream.
void helm_server::run_batch(const Model &md, std::vector<Pending> &batch, Slot *sl, bool hit,
                            std::vector<helm_request_info> &infos, helm_status &status) {
    const helm_request &r0 = batch[0].r;
    const size_t N = (size_t)md.grid.nx * md.grid.nz;
    int rhs = 0;
    double rtol = r0.rtol;
    for (const Pending &p : batch) {
        rhs += p.r.nrhs;
        if (p.r.rtol < rtol) rtol = p.r.rtol;
    }
    cudaError_t e = cudaSuccess;
    helm_solve_info si{};
    helm_c128 *Bd = nullptr, *Xd = nullptr;
    if (!hit) {
        e = cudaStreamCreateWithFlags(&sl->st, cudaStreamNonBlocking);
        if (e != cudaSuccess) { helm_set_error("server: stream", e); status = HELM_ECUDA; goto out; }
        const double om = r0.omega;
        if ((status = helm_assemble(&md.grid, md.m_dev, &om, 1, sl->st, &sl->op)) != HELM_OK) goto out;
        if ((status = helm_factor(sl->op, (helm_prec)r0.prec, nullptr, &sl->f)) != HELM_OK) goto out;
    }
    if ((status = dev_alloc((void **)&Bd, rhs * N * sizeof(helm_c128), "server: allocate(B)", sl->st)) != HELM_OK ||
        (status = dev_alloc((void **)&Xd, rhs * N * sizeof(helm_c128), "server: allocate(X)", sl->st)) != HELM_OK)
        goto out;
    {
        size_t off = 0;
        for (const Pending &p : batch) {
            e = cudaMemcpyAsync(Bd + off, p.r.B, p.r.nrhs * N * sizeof(helm_c128), cudaMemcpyHostToDevice, sl->st);
            if (e != cudaSuccess) { helm_set_error("server: copy B", e); status = HELM_ECUDA; goto out; }
            off += (size_t)p.r.nrhs * N;
        }
    }
    status = r0.adjoint ? helm_adjoint_solve(sl->f, rhs, Bd, Xd, rtol, opts.max_iter, &si)
                        : helm_solve(sl->f, rhs, Bd, Xd, rtol, opts.max_iter, &si);
    if (status == HELM_OK || status == HELM_ENOCONV) {
        size_t off = 0;
        for (const Pending &p : batch) {
            e = cudaMemcpyAsync(p.r.X, Xd + off, p.r.nrhs * N * sizeof(helm_c128), cudaMemcpyDeviceToHost, sl->st);
            if (e != cudaSuccess) { helm_set_error("server: copy X", e); status = HELM_ECUDA; break; }
            off += (size_t)p.r.nrhs * N;
        }
    }
out:
    if (sl->st) {
        e = cudaStreamSynchronize(sl->st);
        if (e != cudaSuccess && status == HELM_OK) { helm_set_error("server: batch", e); status = HELM_ECUDA; }
    }
    if (Bd) dev_free(Bd, sl->st);
    if (Xd) dev_free(Xd, sl->st);
    for (helm_request_info &in : infos) {
        in.status = status;
        in.iters = si.iters;
        in.max_relres = si.max_relres;
    }
}

extern "C" helm_status helm_server_create(const helm_server_opts *opts, helm_server_t **out) {
    if (!out) { helm_set_msg("helm_server_create: NULL out"); return HELM_EINVAL; }
    *out = nullptr;
    helm_server_opts o{};
    if (opts) o = *opts;
    if (o.hbm_budget_bytes == 0) o.hbm_budget_bytes = (uint64_t)180 << 30;
    if (o.max_batch_rhs <= 0) o.max_batch_rhs = 128;
    if (o.workers <= 0) o.workers = 8;   // a factor build fills one cluster: several run at once
    if (o.max_iter <= 0) o.max_iter = 10;
    if (o.hbm_budget_bytes < kMiB) { helm_set_msg("helm_server_create: budget below 1 MiB"); return HELM_EINVAL; }
    keep_pool_memory();
    helm_server *s = new (std::nothrow) helm_server();
    if (!s) { helm_set_msg("helm_server_create: out of host memory"); return HELM_ENOMEM; }
    s->opts = o;
    s->cache = helm_srv::Cache((size_t)o.hbm_budget_bytes);
    s->stats.bytes_budget = o.hbm_budget_bytes;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        helm_set_error("helm_server_create", e);
        delete s;
        return HELM_ECUDA;
    }
    for (int w = 0; w < o.workers; ++w) s->workers.emplace_back([s]() { s->worker_loop(); });
    *out = s;
    return HELM_OK;
}

extern "C" helm_status helm_server_add_model(helm_server_t *s, const helm_grid *grid, const double *m_host,
                                             int32_t *model_id) {
    if (!s || !grid || !m_host || !model_id || grid->nx < 4 || grid->nz < 4 || !(grid->lx > 0) || !(grid->lz > 0)) {
        helm_set_msg("helm_server_add_model: bad arguments");
        return HELM_EINVAL;
    }
    const size_t N = (size_t)grid->nx * grid->nz;
    Model md;
    md.grid = *grid;
    helm_status st = dev_alloc((void **)&md.m_dev, N * sizeof(double), "helm_server_add_model: allocate(m)", s->st);
    if (st != HELM_OK) return st;
    cudaError_t e = cudaMemcpyAsync(md.m_dev, m_host, N * sizeof(double), cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) {
        helm_set_error("helm_server_add_model: copy m", e);
        dev_free(md.m_dev, s->st);
        return HELM_ECUDA;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->models.push_back(md);
    *model_id = (int32_t)s->models.size() - 1;
    return HELM_OK;
}

extern "C" uint64_t helm_server_footprint(const helm_server_t *s, int32_t model_id, int32_t prec, int32_t nrhs) {
    if (!s || nrhs < 1 || (prec != HELM_FP64 && prec != HELM_MIXED)) return 0;
    std::lock_guard<std::mutex> lk(s->mu);
    if (model_id < 0 || model_id >= (int32_t)s->models.size()) return 0;
    return s->footprint(s->models[model_id].grid, prec, nrhs);
}

extern "C" helm_status helm_server_submit(helm_server_t *s, const helm_request *req, int64_t *ticket) {
    if (!s || !req || !ticket || req->nrhs < 1 || !req->B || !req->X || !(req->omega > 0) ||
        (req->prec != HELM_FP64 && req->prec != HELM_MIXED) || !(req->rtol > 0)) {
        helm_set_msg("helm_server_submit: bad arguments");
        return HELM_EINVAL;
    }
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (req->model < 0 || req->model >= (int32_t)s->models.size()) {
        helm_set_msg("helm_server_submit: unknown model");
        return HELM_EINVAL;
    }
    if (s->footprint(s->models[req->model].grid, req->prec, req->nrhs) > s->cache.budget()) {
        ++s->stats.refused;
        helm_set_msg("helm_server_submit: request footprint above the HBM budget");
        return HELM_ENOMEM;
    }
    const int64_t t = s->next_ticket++;
    s->states.emplace(t, State{});
    s->queue.push_back(Pending{t, *req, now});
    ++s->stats.submitted;
    *ticket = t;
    s->cv_work.notify_one();
    return HELM_OK;
}

extern "C" helm_status helm_server_wait(helm_server_t *s, int64_t ticket, helm_request_info *info) {
    if (!s) { helm_set_msg("helm_server_wait: NULL server"); return HELM_EINVAL; }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->states.find(ticket);
    if (it == s->states.end()) {
        helm_set_msg("helm_server_wait: unknown ticket");
        return HELM_EINVAL;
    }
    s->cv_done.wait(lk, [&]() {
        auto jt = s->states.find(ticket);
        return jt == s->states.end() || jt->second.done;
    });
    it = s->states.find(ticket);
    if (it == s->states.end()) {   // waited for twice
        helm_set_msg("helm_server_wait: ticket already waited for");
        return HELM_EINVAL;
    }
    const helm_request_info in = it->second.info;
    s->states.erase(it);
    if (info) *info = in;
    return (helm_status)in.status;
}

extern "C" helm_status helm_server_stats(const helm_server_t *s, helm_server_counters *out) {
    if (!s || !out) { helm_set_msg("helm_server_stats: NULL argument"); return HELM_EINVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->cache_hits = (int64_t)s->cache.hits();
    out->entries = (int64_t)s->cache.entries();
    out->bytes_used = s->cache.used();
    out->bytes_peak = s->cache.peak();
    return HELM_OK;
}

extern "C" void helm_server_destroy(helm_server_t *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (std::thread &t : s->workers) t.join();
    std::vector<void *> slots;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        slots = s->cache.clear();
    }
    for (void *p : slots) destroy_slot(static_cast<Slot *>(p));
    for (Model &md : s->models) dev_free(md.m_dev, s->st);
    if (s->st) {
        cudaStreamSynchronize(s->st);
        cudaStreamDestroy(s->st);
    }
    delete s;
}
