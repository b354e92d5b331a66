// server.cu -- request loop for sweep points: admission by device-memory footprint,
// continuous batching (points that arrive while others run join at the next chunk
// boundary), per-point convergence test on the volume-averaged velocity, retirement,
// and submit-to-finish latency.
//
// Two threads, each with a private CUDA stream.  The admission thread takes queued points
// that fit the memory budget and builds them (geometry and memory, on its own stream) while
// the GPU steps the resident ones.  The worker owns one Batch per (storage, collision,
// layout) group.  Every chunk: take the points the admission thread has built, advance each
// group by check_interval steps (a captured graph ending in the FP64 reduction), read the
// per-point sums, retire.  check_interval is even, so that in-place (AA) groups are back in
// the arrangement of step 0 at every chunk boundary, where new points join them.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "batch.h"

using namespace lbm;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t id = 0;
    lbm_desc desc{};
    std::vector<lbm_sphere> spheres;
    std::vector<uint8_t> flags;
    std::vector<double> q, mrt;
    double tol = 1e-8;
    int64_t max_steps = 0;
    Clock::time_point t_submit, t_done;
    enum { QUEUED, RUNNING, DONE } state = QUEUED;
    bool cancel = false;      // retire at the next chunk boundary
    lbm_status result = LBM_OK;
    lbm_obs obs{};
    size_t bytes = 0;
    double U_old = 0.0;
    bool have_U = false;
};

}  // namespace

using GroupKey = std::tuple<int, int, int>;  // storage, collision, layout

struct lbm_server {
    lbm_server_opts opts{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_admit;
    std::deque<int64_t> queue;
    std::map<int64_t, Request> reqs;
    int64_t next_id = 1;
    bool stop = false;
    size_t used = 0;
    int device = 0;
    cudaStream_t stream = nullptr;   // stepping (worker)
    cudaStream_t astream = nullptr;  // instance builds (admission thread)
    int building = 0;                // points being built by the admission thread
    // points built and waiting to join their group at the next chunk boundary
    std::vector<std::pair<int64_t, std::unique_ptr<Instance>>> ready;
    std::map<GroupKey, std::unique_ptr<Batch>> groups;
    std::map<GroupKey, std::vector<int64_t>> members;  // request id per batch slot
    lbm_server_stats stats{};
    std::thread worker, admitter;

    void run();
    void admit_loop();
    void join_ready();
    int resident_count();
    void finish(Request &r, lbm_status st, const Instance *in);
};

void lbm_server::finish(Request &r, lbm_status st, const Instance *in)
{
    if (in) compute_obs(*in, 0.0, &r.obs);
    r.result = st;
    r.state = Request::DONE;
    r.t_done = Clock::now();
    used -= r.bytes;
    if (st == LBM_OK) ++stats.completed;
    else if (st == LBM_ERR_CANCELLED) ++stats.cancelled;
    else ++stats.failed;
}

int lbm_server::resident_count()
{
    int resident = (int)ready.size() + building;
    for (auto &g : groups) resident += g.second->size();
    return resident;
}

// Admission thread: builds the queued points that fit the memory budget and the resident
// cap, on its own stream, while the worker keeps the GPU stepping.
void lbm_server::admit_loop()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        cv_admit.wait(lk, [this] {
            if (stop) return true;
            if (queue.empty() || resident_count() >= opts.max_resident) return false;
            return used + reqs[queue.front()].bytes <= opts.hbm_budget_bytes;
        });
        if (stop) break;
        Request &r = reqs[queue.front()];
        queue.pop_front();
        used += r.bytes;
        r.state = Request::RUNNING;
        ++building;
        lbm_desc d = r.desc;
        d.spheres = r.spheres.empty() ? nullptr : r.spheres.data();
        d.flags = r.flags.empty() ? nullptr : r.flags.data();
        d.q = r.q.empty() ? nullptr : r.q.data();
        d.mrt_rates = r.mrt.empty() ? nullptr : r.mrt.data();
        const int64_t id = r.id;
        lk.unlock();
        std::unique_ptr<Instance> in;
        lbm_status st = Batch::make_instance(d, astream, &in);
        lk.lock();
        --building;
        Request &rr = reqs[id];
        if (st != LBM_OK) {
            finish(rr, st, nullptr);
            cv_done.notify_all();
            cv_admit.notify_all();
            continue;
        }
        ready.emplace_back(id, std::move(in));
        cv_work.notify_all();
    }
}

// Worker, at a chunk boundary (lock held): the built points join their groups.  Every
// group is in the arrangement of step 0 here (check_interval is even).
void lbm_server::join_ready()
{
    for (auto &p : ready) {
        Request &r = reqs[p.first];
        const lbm_desc &d = p.second->desc;
        const GroupKey key(d.storage, d.collision, d.layout);
        if (r.cancel) {  // cancelled while it was being built
            finish(r, LBM_ERR_CANCELLED, nullptr);
            continue;    // the instance frees its memory with ready below
        }
        auto &g = groups[key];
        if (!g) {
            g.reset(new Batch());
            g->init(stream, d.storage, d.collision, d.layout);
            if (d.block_cells > 0) g->set_block(d.block_cells);
        }
        lbm_status st = g->add(std::move(p.second));  // on failure the instance is freed
        if (st == LBM_OK) {
            st = g->init_equilibrium(g->size() - 1);
            if (st != LBM_OK) g->remove(g->size() - 1);
        }
        if (st != LBM_OK) {
            finish(r, st, nullptr);
            continue;
        }
        members[key].push_back(r.id);
    }
    ready.clear();
    cv_done.notify_all();
}

void lbm_server::run()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        join_ready();
        int resident = 0;
        for (auto &g : groups) resident += g.second->size();
        if (resident == 0) {
            if (stop && building == 0) break;
            cv_work.wait_for(lk, std::chrono::milliseconds(50));
            continue;
        }
        lk.unlock();
        TraceRange trace("lbm.server.chunk");
        const auto t0 = Clock::now();
        double updates = 0.0;
        for (auto &kv : groups) {
            Batch &b = *kv.second;
            if (b.size() == 0) continue;
            if (b.step(opts.check_interval) != LBM_OK) continue;
            updates += (double)b.fluid_cells() * opts.check_interval;
        }
        for (auto &kv : groups)
            if (kv.second->size()) kv.second->fetch_sums();
        const double dt = std::chrono::duration<double>(Clock::now() - t0).count();
        lk.lock();
        stats.fluid_updates += updates;
        stats.busy_seconds += dt;
        for (auto &kv : groups) {
            Batch &b = *kv.second;
            std::vector<int64_t> &ids = members[kv.first];
            for (int i = b.size() - 1; i >= 0; --i) {
                Request &r = reqs[ids[i]];
                Instance &in = b.at(i);
                const double U = in.sums[1] / (double)in.geo.ncells;
                lbm_status st = LBM_ERR_STATE;
                if (r.cancel) st = LBM_ERR_CANCELLED;
                else if (in.status & STATUS_DIVERGED) st = LBM_ERR_DIVERGED;
                else if (r.have_U && std::fabs(U - r.U_old) < r.tol * std::fabs(U)) st = LBM_OK;
                else if (in.steps >= r.max_steps) st = LBM_ERR_NOT_CONVERGED;
                r.U_old = U;
                r.have_U = true;
                if (st != LBM_ERR_STATE) {
                    finish(r, st, &in);
                    lk.unlock();
                    b.remove(i);
                    lk.lock();
                    ids.erase(ids.begin() + i);
                }
            }
        }
        stats.kernel_launches = 0;
        for (auto &kv : groups) stats.kernel_launches += kv.second->launches();
        cv_done.notify_all();
        cv_admit.notify_all();  // memory may have been freed
    }
}

extern "C" {

lbm_status lbm_server_create(const lbm_server_opts *opts, lbm_server **out)
{
    if (!out) return fail(LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!opts || opts->hbm_budget_bytes == 0) return fail(LBM_ERR_ARG, "hbm_budget_bytes must be > 0");
    lbm_server *s = new (std::nothrow) lbm_server();
    if (!s) return fail(LBM_ERR_NO_MEMORY, "host allocation failed");
    s->opts = *opts;
    if (s->opts.check_interval <= 0) s->opts.check_interval = 200;
    s->opts.check_interval += s->opts.check_interval & 1;  // even: AA groups back in step 0's arrangement
    if (s->opts.max_resident <= 0) s->opts.max_resident = 256;
    cudaGetDevice(&s->device);
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->astream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        if (s->stream) cudaStreamDestroy(s->stream);
        delete s;
        return cuda_fail(e, "cudaStreamCreate");
    }
    s->worker = std::thread([s] { s->run(); });
    s->admitter = std::thread([s] { s->admit_loop(); });
    *out = s;
    return LBM_OK;
}

lbm_status lbm_server_submit(lbm_server *s, const lbm_desc *desc, double tol, int64_t max_steps, int64_t *req_id)
{
    if (!s || !desc || !req_id) return fail(LBM_ERR_ARG, "NULL argument");
    if (!(tol > 0) || max_steps < 1) return fail(LBM_ERR_ARG, "tol must be > 0 and max_steps >= 1");
    lbm_status v = validate_desc(*desc);
    if (v != LBM_OK) return v;
    Request r;
    r.desc = *desc;
    const size_t n = (size_t)desc->nx * desc->ny * desc->nz;
    if (desc->spheres && desc->n_spheres > 0) r.spheres.assign(desc->spheres, desc->spheres + desc->n_spheres);
    if (desc->flags) r.flags.assign(desc->flags, desc->flags + n);
    if (desc->q) r.q.assign(desc->q, desc->q + (size_t)Q * n);
    if (desc->mrt_rates) r.mrt.assign(desc->mrt_rates, desc->mrt_rates + Q);
    r.desc.spheres = nullptr;
    r.desc.flags = nullptr;
    r.desc.q = nullptr;
    r.desc.mrt_rates = nullptr;
    r.tol = tol;
    r.max_steps = max_steps;
    r.bytes = Batch::footprint(r.desc);
    if (r.bytes > s->opts.hbm_budget_bytes) return fail(LBM_ERR_NO_MEMORY, "point alone exceeds the memory budget");
    std::lock_guard<std::mutex> lk(s->mu);
    r.id = s->next_id++;
    r.t_submit = Clock::now();
    *req_id = r.id;
    s->queue.push_back(r.id);
    s->reqs[r.id] = std::move(r);
    ++s->stats.submitted;
    s->cv_admit.notify_all();
    return LBM_OK;
}

lbm_status lbm_server_poll(lbm_server *s, int64_t req_id, lbm_obs *out, double *latency_s)
{
    if (!s) return fail(LBM_ERR_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return fail(LBM_ERR_ARG, "unknown request id");
    Request &r = it->second;
    if (r.state != Request::DONE) return fail(LBM_ERR_STATE, "request still queued or running");
    if (out) *out = r.obs;
    if (latency_s) *latency_s = std::chrono::duration<double>(r.t_done - r.t_submit).count();
    if (r.result == LBM_ERR_CANCELLED) set_error("request cancelled");
    else if (r.result != LBM_OK) set_error("request finished without converging");
    return r.result;
}

lbm_status lbm_server_drain(lbm_server *s, double timeout_s)
{
    if (!s) return fail(LBM_ERR_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto all_done = [s] {
        for (auto &kv : s->reqs)
            if (kv.second.state != Request::DONE) return false;
        return true;
    };
    if (timeout_s > 0) {
        if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), all_done))
            return fail(LBM_ERR_TIMEOUT, "drain timed out");
    } else {
        s->cv_done.wait(lk, all_done);
    }
    return LBM_OK;
}

lbm_status lbm_server_cancel(lbm_server *s, int64_t req_id)
{
    if (!s) return fail(LBM_ERR_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return fail(LBM_ERR_ARG, "unknown request id");
    Request &r = it->second;
    if (r.state == Request::DONE) return fail(LBM_ERR_STATE, "request already finished");
    if (r.state == Request::QUEUED) {  // never admitted: holds no memory
        for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
            if (*q == req_id) {
                s->queue.erase(q);
                break;
            }
        r.result = LBM_ERR_CANCELLED;
        r.state = Request::DONE;
        r.t_done = Clock::now();
        ++s->stats.cancelled;
        s->cv_done.notify_all();
        return LBM_OK;
    }
    r.cancel = true;  // being built or resident: retired at the next chunk boundary
    return LBM_OK;
}

lbm_status lbm_server_get_stats(lbm_server *s, lbm_server_stats *out)
{
    if (!s || !out) return fail(LBM_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->queued = (int64_t)s->queue.size();
    int64_t resident = 0;
    for (auto &kv : s->reqs)
        if (kv.second.state == Request::RUNNING) ++resident;
    out->resident = resident;
    out->mlups = s->stats.busy_seconds > 0 ? s->stats.fluid_updates / s->stats.busy_seconds / 1e6 : 0.0;
    return LBM_OK;
}

void lbm_server_destroy(lbm_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->queue.clear();
        for (auto &kv : s->reqs)
            if (kv.second.state == Request::QUEUED) kv.second.state = Request::DONE;
        // resident points are retired by the worker only on convergence: end them at the
        // next chunk boundary
        for (auto &kv : s->reqs) kv.second.max_steps = 0;
        s->cv_work.notify_all();
        s->cv_admit.notify_all();
    }
    if (s->admitter.joinable()) s->admitter.join();
    if (s->worker.joinable()) s->worker.join();
    s->ready.clear();
    s->groups.clear();
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->astream) cudaStreamDestroy(s->astream);
    delete s;
}

}  // extern "C"
