// mh_server: a request server over the whole path (Sec. 2: pack, count with
// the solid filter, mercy, SdBG) with continuous batching.
//
// Jobs (one read set, k, d) arrive at any time into one first-in first-out
// queue.  `slots` host threads, each driving a worker context of its own (its
// own stream and stream-ordered pool), take the queue's head when its
// mh_job_bytes estimate fits the HBM budget next to the jobs running and the
// results still held (or when nothing is held: a job larger than the budget
// runs alone).  Jobs that arrive while others run are admitted as slots and
// memory free up; their kernels overlap on the device, one stream per slot.
// A job's result stays resident, counted against the budget, until the
// client releases it (or at once with MH_SERVE_AUTO_RELEASE).  Every step of
// a job runs in the library's kernels; this file is host scheduling only.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "mh_internal.cuh"

using namespace mh;

namespace {

struct ServerJob {
    mh_read_set set{};
    int k = 0, d = 0;
    mh_job_info info{};
    mh_set_result result{nullptr, nullptr, nullptr, MH_OK};
    bool ended = false;
    bool held = false;  // its estimate counts against the budget
};

// Pools of worker contexts above this are trimmed after a job, so that one
// very large job does not keep its memory in a slot's pool.
constexpr uint64_t kTrimBytes = 8ull << 30;

}  // namespace

struct mh_server {
    int flags = 0;
    uint64_t budget = 0;
    std::vector<mh_ctx*> workers;
    std::vector<std::thread> threads;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> queue;
    std::map<uint64_t, ServerJob> jobs;  // node addresses stay valid until erased
    uint64_t next_id = 1;
    uint64_t held = 0, max_held = 0, running = 0;
    bool stop = false;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

    double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }

    // the queue's head may start (called with mu held)
    bool head_fits() {
        if (queue.empty()) return false;
        const uint64_t est = jobs[queue.front()].info.est_bytes;
        return held == 0 || held + est <= budget;
    }

    // frees an ended job's result and returns its bytes (mu held)
    void drop_result(ServerJob& j) {
        free_set_result(j.result);
        if (j.held) {
            held -= j.info.est_bytes;
            j.held = false;
        }
    }
};

namespace {

void serve_worker(mh_server* s, int slot) {
    mh_ctx* w = slot < (int)s->workers.size() ? s->workers[slot] : nullptr;
    for (;;) {
        ServerJob* j = nullptr;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            s->cv.wait(lock, [&] { return s->head_fits() || (s->stop && s->queue.empty()); });
            if (s->queue.empty()) return;  // stopping, nothing left
            const uint64_t id = s->queue.front();
            s->queue.pop_front();
            j = &s->jobs[id];
            j->held = true;
            s->held += j->info.est_bytes;
            s->max_held = std::max(s->max_held, s->held);
            s->running++;
            j->info.start_s = s->now();
            j->info.slot = slot;
        }
        s->cv.notify_all();  // the next job may fit beside this one
        mh_set_result r{nullptr, nullptr, nullptr, MH_OK};
        if (s->flags & MH_SERVE_DRY_RUN) {
            std::this_thread::sleep_for(std::chrono::microseconds(j->set.n_reads));
        } else {
            run_set_job(w, j->set, j->k, j->d, s->flags, r);
            if (j->info.est_bytes > kTrimBytes) mh_trim(w);
        }
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->running--;
            j->result = r;
            j->info.status = r.status;
            j->info.end_s = s->now();
            j->ended = true;
            // once the server is being destroyed no client reads results
            if ((s->flags & MH_SERVE_AUTO_RELEASE) || r.status != MH_OK || s->stop) s->drop_result(*j);
        }
        s->cv.notify_all();
    }
}

}  // namespace

extern "C" {

int mh_server_create(mh_ctx* ctx, int slots, uint64_t hbm_budget, int flags, mh_server** out) {
    if (!out || slots < 1 || slots > 64 || (!ctx && !(flags & MH_SERVE_DRY_RUN))) {
        if (ctx) ctx->last_error = "mh_server_create: need out, 1 <= slots <= 64, and a context unless dry run";
        return MH_EINVAL;
    }
    *out = nullptr;
    mh_server* s = new mh_server;
    s->flags = flags;
    if (flags & MH_SERVE_DRY_RUN) {
        s->budget = hbm_budget ? hbm_budget : ~0ull;
    } else {
        const uint64_t plan = ctx->budget ? ctx->budget : ctx->device_bytes / 20 * 17;
        s->budget = hbm_budget ? hbm_budget : plan;
        for (int i = 0; i < slots; i++) {
            mh_config cfg = {};
            cfg.device = ctx->device;
            cfg.with_mult = ctx->with_mult;
            mh_ctx* w = nullptr;
            const int rc = mh_create(&cfg, &w);
            if (rc != MH_OK) {
                for (mh_ctx* c : s->workers) mh_destroy(c);
                delete s;
                ctx->last_error = "mh_server_create: creating a worker context failed";
                return rc;
            }
            w->profile = ctx->profile;
            s->workers.push_back(w);
        }
    }
    try {
        for (int i = 0; i < slots; i++) s->threads.emplace_back(serve_worker, s, i);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->stop = true;
        }
        s->cv.notify_all();
        for (auto& t : s->threads) t.join();
        for (mh_ctx* c : s->workers) mh_destroy(c);
        delete s;
        return MH_EDEVICE;
    }
    *out = s;
    return MH_OK;
}

int mh_server_submit(mh_server* s, const mh_read_set* set, int k, int d, uint64_t* job) {
    if (!s || !set || !job || k < 2 || k > 127 || d < 1) return MH_EINVAL;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) return MH_EINVAL;
        const uint64_t id = s->next_id++;
        ServerJob& j = s->jobs[id];
        j.set = *set;
        j.k = k;
        j.d = d;
        j.info.submit_s = s->now();
        j.info.start_s = j.info.end_s = -1.0;
        j.info.slot = -1;
        j.info.status = MH_OK;
        j.info.est_bytes = mh_job_bytes(set, k);
        s->queue.push_back(id);
        *job = id;
    }
    s->cv.notify_all();
    return MH_OK;
}

int mh_server_wait(mh_server* s, uint64_t job, double timeout_s, mh_set_result* out, mh_job_info* info) {
    if (!s) return MH_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    // the record is looked up again after every wake-up: another thread may
    // have released it meanwhile
    auto ended = [&] {
        auto it = s->jobs.find(job);
        return it == s->jobs.end() || it->second.ended;
    };
    if (timeout_s < 0) {
        s->cv.wait(lock, ended);
    } else if (!s->cv.wait_for(lock, std::chrono::duration<double>(timeout_s), ended)) {
        return MH_ETIMEOUT;
    }
    auto it = s->jobs.find(job);
    if (it == s->jobs.end()) return MH_EINVAL;
    if (out) *out = it->second.result;
    if (info) *info = it->second.info;
    return MH_OK;
}

int mh_server_release(mh_server* s, uint64_t job) {
    if (!s) return MH_EINVAL;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        auto it = s->jobs.find(job);
        if (it == s->jobs.end() || !it->second.ended) return MH_EINVAL;
        s->drop_result(it->second);
        s->jobs.erase(it);
    }
    s->cv.notify_all();
    return MH_OK;
}

int mh_server_stats(mh_server* s, uint64_t* held_bytes, uint64_t* max_held_bytes, uint64_t* queued,
                    uint64_t* running) {
    if (!s) return MH_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    if (held_bytes) *held_bytes = s->held;
    if (max_held_bytes) *max_held_bytes = s->max_held;
    if (queued) *queued = s->queue.size();
    if (running) *running = s->running;
    return MH_OK;
}

int mh_server_reset_max(mh_server* s) {
    if (!s) return MH_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    s->max_held = s->held;
    return MH_OK;
}

mh_ctx* mh_server_context(mh_server* s, int slot) {
    if (!s || slot < 0 || slot >= (int)s->workers.size()) return nullptr;
    return s->workers[slot];
}

int mh_server_destroy(mh_server* s) {
    if (!s) return MH_EINVAL;
    {
        // no client can read the ended jobs' results any more: free them
        // now, so that the jobs still queued find room
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        for (auto& kv : s->jobs)
            if (kv.second.ended) s->drop_result(kv.second);
    }
    s->cv.notify_all();
    for (auto& t : s->threads) t.join();
    for (auto& kv : s->jobs) free_set_result(kv.second.result);
    for (mh_ctx* c : s->workers) mh_destroy(c);
    delete s;
    return MH_OK;
}

}  // extern "C"
