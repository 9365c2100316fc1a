// mh_run_batch: many independent read sets through the whole path at once.
//
// Every read set is an independent problem (the paper builds one graph per
// read set, Sec. 2).  A batch runs each set's pack, count, mercy and build
// as one job.  `workers` host threads each drive a worker context of the
// caller's context (its own blocking stream and stream-ordered pool), taking
// jobs largest first: the longest-processing-time order leaves the small
// jobs to fill the streams at the end.  A job starts when its estimated
// working set fits the memory plan next to the jobs in flight.  Jobs overlap
// on the device: while one job's thread waits on the device-to-host read
// that sizes an output, the other streams keep the SMs busy, and a small
// set's short kernels run beside a large set's.
//
// The autotuner times the scatter pass's tile shapes on the largest set of
// the first batch at a k with 1-word keys and keeps the fastest for the
// context.
#include <algorithm>
#include <condition_variable>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

#include "mh_internal.cuh"

namespace mh {
void profile_merge(mh_ctx* dst, mh_ctx* src);
}  // namespace mh

using namespace mh;

namespace {

constexpr int kSortShapes = 3;

// Peak device bytes of one job: counting dominates (keys, sort buffer, run
// slots and spectrum: about 48 bytes per window and key word), plus the
// packed reads, the host upload's staging pieces and a fixed margin.
uint64_t job_bytes(const mh_read_set& s, int k) {
    const uint64_t nw = (uint64_t)words_for(k);
    const uint64_t kk = (uint64_t)k * s.n_reads;
    const uint64_t win = s.n_bases > kk ? s.n_bases - kk : 0;
    return (64ull << 20) + 48 * nw * win + 2 * s.n_bases + (s.on_device ? 0 : (512ull << 20));
}

void free_result(mh_set_result& r) {
    mh_free_sdbg(r.sdbg);
    mh_free_kmers(r.mercy);
    mh_free_kmers(r.solid);
    r.sdbg = nullptr;
    r.mercy = r.solid = nullptr;
}

int run_job(mh_ctx* w, const mh_read_set& s, int k, int d, int flags, mh_set_result& r) {
    mh_reads* reads = nullptr;
    int rc = mh_pack_reads(w, s.ascii, s.n_bases, s.offs, s.n_reads, s.on_device, &reads);
    if (rc == MH_OK) rc = mh_count_kmers(w, reads, k, d, &r.solid);
    if (rc == MH_OK && (flags & MH_BATCH_MERCY)) rc = mh_mercy_kmers(w, reads, r.solid, &r.mercy);
    if (rc == MH_OK && (flags & MH_BATCH_BUILD)) rc = mh_build_sdbg(w, r.solid, r.mercy, &r.sdbg);
    mh_free_reads(reads);
    if (rc != MH_OK) free_result(r);
    r.status = rc;
    return rc;
}

// Count `s` once per tile shape on worker w (after one untimed count) and
// return the fastest shape.
int tune_shape(mh_ctx* w, const mh_read_set& s, int k, int d) {
    mh_reads* reads = nullptr;
    if (mh_pack_reads(w, s.ascii, s.n_bases, s.offs, s.n_reads, s.on_device, &reads) != MH_OK) return -1;
    cudaEvent_t a = nullptr, b = nullptr;
    int best = -1;
    float best_ms = 0.f;
    if (cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess) {
        for (int shape = -1; shape < kSortShapes; shape++) {
            w->sort_shape = shape < 0 ? 0 : shape;
            mh_kmers* solid = nullptr;
            cudaEventRecord(a, w->stream);
            const int rc = mh_count_kmers(w, reads, k, d, &solid);
            cudaEventRecord(b, w->stream);
            cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            mh_free_kmers(solid);
            if (rc != MH_OK) {
                best = -1;
                break;
            }
            if (shape >= 0 && (best < 0 || ms < best_ms)) {
                best = shape;
                best_ms = ms;
            }
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    mh_free_reads(reads);
    return best;
}

}  // namespace

extern "C" {

int mh_sort_shape(const mh_ctx* ctx) { return ctx ? ctx->sort_shape : -1; }

int mh_run_batch(mh_ctx* ctx, const mh_read_set* sets, int n_sets, int k, int d, int workers, int flags,
                 mh_set_result* out) {
    if (!ctx || n_sets < 0 || (n_sets && (!sets || !out)) || workers < 1 || workers > 64 || k < 2 || k > 127 ||
        d < 1) {
        if (ctx) ctx->last_error = "mh_run_batch: need ctx, sets, out, n_sets >= 0, 1 <= workers <= 64, "
                                   "2 <= k <= 127, d >= 1";
        return MH_EINVAL;
    }
    for (int i = 0; i < n_sets; i++) out[i] = mh_set_result{nullptr, nullptr, nullptr, MH_OK};
    if (n_sets == 0) return MH_OK;
    try {
        if (cudaSetDevice(ctx->device) != cudaSuccess) throw Error{MH_EDEVICE, "cudaSetDevice failed"};
        workers = std::min(workers, n_sets);
        while ((int)ctx->workers.size() < workers) {
            mh_config cfg = {};
            cfg.device = ctx->device;
            cfg.with_mult = ctx->with_mult;
            mh_ctx* w = nullptr;
            const int rc = mh_create(&cfg, &w);
            if (rc != MH_OK) throw Error{rc, "mh_run_batch: creating a worker context failed"};
            ctx->workers.push_back(w);
        }
        // the workers start after the work already queued on ctx's stream
        cudaEvent_t fence;
        MH_CUDA(cudaEventCreateWithFlags(&fence, cudaEventDisableTiming));
        MH_CUDA(cudaEventRecord(fence, ctx->stream));
        for (int i = 0; i < workers; i++) {
            mh_ctx* w = ctx->workers[i];
            w->profile = ctx->profile;
            cudaStreamWaitEvent(w->stream, fence, 0);
        }
        cudaEventDestroy(fence);

        std::vector<int> order(n_sets);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return sets[a].n_bases > sets[b].n_bases; });
        if ((flags & MH_BATCH_AUTOTUNE) && words_for(k) == 1 && ctx->tuned_k != k) {
            const int shape = tune_shape(ctx->workers[0], sets[order[0]], k, d);
            if (shape >= 0) {
                ctx->sort_shape = shape;
                ctx->tuned_k = k;
            }
        }
        for (int i = 0; i < workers; i++) ctx->workers[i]->sort_shape = ctx->sort_shape;

        const uint64_t plan = ctx->budget ? ctx->budget : ctx->device_bytes / 20 * 17;
        const uint64_t budget = plan > ctx->in_use ? plan - ctx->in_use : 0;
        std::mutex mu;
        std::condition_variable cv;
        int next = 0;
        uint64_t held = 0;
        auto body = [&](int wi) {
            mh_ctx* w = ctx->workers[wi];
            for (;;) {
                int j;
                uint64_t est;
                {
                    std::unique_lock<std::mutex> lock(mu);
                    cv.wait(lock, [&] {
                        return next >= n_sets || held == 0 || held + job_bytes(sets[order[next]], k) <= budget;
                    });
                    if (next >= n_sets) return;
                    j = order[next++];
                    est = job_bytes(sets[j], k);
                    held += est;
                }
                run_job(w, sets[j], k, d, flags, out[j]);
                {
                    std::lock_guard<std::mutex> lock(mu);
                    held -= est;
                }
                cv.notify_all();
            }
        };
        std::vector<std::thread> threads;
        threads.reserve(workers);
        try {
            for (int i = 0; i < workers; i++) threads.emplace_back(body, i);
        } catch (...) {
            // no more jobs start; the threads already running finish theirs
            {
                std::lock_guard<std::mutex> lock(mu);
                for (int i = next; i < n_sets; i++) out[order[i]].status = MH_EDEVICE;
                next = n_sets;
            }
            cv.notify_all();
            for (auto& t : threads) t.join();
            throw;
        }
        for (auto& t : threads) t.join();

        // ctx's stream waits for every worker's last kernel
        for (int i = 0; i < workers; i++) {
            mh_ctx* w = ctx->workers[i];
            cudaEvent_t done;
            MH_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
            MH_CUDA(cudaEventRecord(done, w->stream));
            MH_CUDA(cudaStreamWaitEvent(ctx->stream, done, 0));
            cudaEventDestroy(done);
            if (ctx->profile) profile_merge(ctx, w);
        }
    } catch (const Error& e) {
        ctx->last_error = e.msg;
        return e.code;
    } catch (const std::exception& e) {
        ctx->last_error = std::string("mh_run_batch: ") + e.what();
        return MH_EDEVICE;
    }
    for (int i = 0; i < n_sets; i++) {
        if (out[i].status != MH_OK) {
            ctx->last_error = "mh_run_batch: set " + std::to_string(i) + " failed";
            return out[i].status;
        }
    }
    ctx->last_error.clear();
    return MH_OK;
}

}  // extern "C"
