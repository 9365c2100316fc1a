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
// The autotuner counts the largest set of the first batch at a key width, k
// and size class once with each of a set of counting plans (route, scatter
// tile shape, unit or spread bits, out-of-core buckets when the set needs
// them) and keeps the fastest for the context.
#include <algorithm>
#include <condition_variable>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

#include "mh_internal.cuh"

namespace mh {
void profile_merge(mh_ctx* dst, mh_ctx* src);

void free_set_result(mh_set_result& r) {
    mh_free_sdbg(r.sdbg);
    mh_free_kmers(r.mercy);
    mh_free_kmers(r.solid);
    r.sdbg = nullptr;
    r.mercy = r.solid = nullptr;
}

int run_set_job(mh_ctx* w, const mh_read_set& s, int k, int d, int flags, mh_set_result& r) {
    NvtxRange nvtx("mh_set_job");
    mh_reads* reads = nullptr;
    int rc = mh_pack_reads(w, s.ascii, s.n_bases, s.offs, s.n_reads, s.on_device, &reads);
    if (rc == MH_OK) rc = mh_count_kmers(w, reads, k, d, &r.solid);
    if (rc == MH_OK && (flags & MH_BATCH_MERCY)) rc = mh_mercy_kmers(w, reads, r.solid, &r.mercy);
    if (rc == MH_OK && (flags & MH_BATCH_BUILD)) rc = mh_build_sdbg(w, r.solid, r.mercy, &r.sdbg);
    mh_free_reads(reads);
    if (rc != MH_OK) free_set_result(r);
    r.status = rc;
    return rc;
}
}  // namespace mh

// Peak device bytes of one job: counting dominates (keys, sort buffer, run
// slots and spectrum: about 48 bytes per window and key word), plus the
// packed reads, the host upload's staging pieces and a fixed margin.
extern "C" uint64_t mh_job_bytes(const mh_read_set* s, int k) {
    if (!s || k < 2 || k > 127) return 0;
    const uint64_t nw = (uint64_t)mh::words_for(k);
    const uint64_t kk = (uint64_t)k * s->n_reads;
    const uint64_t win = s->n_bases > kk ? s->n_bases - kk : 0;
    return (64ull << 20) + 48 * nw * win + 2 * s->n_bases + (s->on_device ? 0 : (512ull << 20));
}

using namespace mh;

namespace {

constexpr int kSortShapes = 3;

uint64_t job_bytes(const mh_read_set& s, int k) { return mh_job_bytes(&s, k); }


using Plan = std::vector<int>;  // path, sort_shape, unit_bits_delta, spread_bits_delta, bucket_bits

void apply_plan(mh_ctx* w, const Plan& p) {
    w->count_path = p[0];
    w->sort_shape = p[1];
    w->unit_bits_delta = p[2];
    w->spread_bits_delta = p[3];
    w->bucket_bits = p[4];
}

// The plans tried for a set: for 1-word keys the unit counting with each
// tile shape and unit bits one either side, and the spread route with its
// bits one digit either side; for wider keys the spread bits; and, when the
// memory plan splits the set into buckets, one bucket bit more.
std::vector<Plan> candidate_plans(int nw, int auto_buckets) {
    std::vector<Plan> c;
    if (nw == 1) {
        for (int shape = 0; shape < kSortShapes; shape++) c.push_back({0, shape, 0, 0, -1});
        c.push_back({0, 0, -1, 0, -1});
        c.push_back({0, 0, 1, 0, -1});
        for (int sb : {0, 8, -8}) c.push_back({1, 0, 0, sb, -1});
    } else {
        // wider keys: the unit route with its unit bits as planned and one
        // fewer or more, the spread route with its pass bits a digit apart
        for (int ubd : {0, -1, 1}) c.push_back({0, 0, ubd, 0, -1});
        for (int sb : {0, 8, -8}) c.push_back({1, 0, 0, sb, -1});
    }
    if (auto_buckets > 0 && auto_buckets < 6) {
        Plan p = c[0];
        p[4] = auto_buckets + 1;
        c.push_back(p);
    }
    return c;
}

// Count `s` on worker w once untimed, then once per candidate plan, and
// return the fastest plan (empty if a count failed).
Plan tune_plan(mh_ctx* w, const mh_read_set& s, int k, int d) {
    mh_reads* reads = nullptr;
    if (mh_pack_reads(w, s.ascii, s.n_bases, s.offs, s.n_reads, s.on_device, &reads) != MH_OK) return {};
    cudaEvent_t a = nullptr, b = nullptr;
    Plan best;
    float best_ms = 0.f;
    const Plan keep = {w->count_path, w->sort_shape, w->unit_bits_delta, w->spread_bits_delta, w->bucket_bits};
    if (cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess) {
        const int nw = words_for(k);
        const uint64_t kk = (uint64_t)k * s.n_reads;
        w->bucket_bits = -1;
        std::vector<Plan> cands = candidate_plans(nw, count_bucket_bits(w, s.n_bases > kk ? s.n_bases - kk : 0, nw));
        for (size_t i = 0; i <= cands.size(); i++) {
            apply_plan(w, i == 0 ? cands[0] : cands[i - 1]);  // the first count warms up
            mh_kmers* solid = nullptr;
            cudaEventRecord(a, w->stream);
            const int rc = mh_count_kmers(w, reads, k, d, &solid);
            cudaEventRecord(b, w->stream);
            cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            mh_free_kmers(solid);
            if (rc != MH_OK) {
                best.clear();
                break;
            }
            if (i > 0 && (best.empty() || ms < best_ms)) {
                best = cands[i - 1];
                best_ms = ms;
            }
        }
    }
    apply_plan(w, keep);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    mh_free_reads(reads);
    return best;
}

}  // namespace

extern "C" {

int mh_sort_shape(const mh_ctx* ctx) { return ctx ? ctx->sort_shape : -1; }

int mh_get_count_plan(const mh_ctx* ctx, mh_count_plan* out) {
    if (!ctx || !out) return MH_EINVAL;
    *out = mh_count_plan{ctx->count_path, ctx->sort_shape, ctx->unit_bits_delta, ctx->spread_bits_delta,
                         ctx->bucket_bits};
    return MH_OK;
}

int mh_set_count_plan(mh_ctx* ctx, const mh_count_plan* p) {
    if (!ctx || !p || p->path < -1 || p->path > 1 || p->sort_shape < -1 || p->sort_shape >= kSortShapes ||
        p->unit_bits_delta < -2 || p->unit_bits_delta > 2 ||
        (p->spread_bits_delta != 0 && p->spread_bits_delta != 8 && p->spread_bits_delta != -8) ||
        p->bucket_bits < -1 || p->bucket_bits > 6) {
        if (ctx) ctx->last_error = "mh_set_count_plan: a field out of range";
        return MH_EINVAL;
    }
    apply_plan(ctx, {p->path, p->sort_shape, p->unit_bits_delta, p->spread_bits_delta, p->bucket_bits});
    return MH_OK;
}

int mh_run_batch(mh_ctx* ctx, const mh_read_set* sets, int n_sets, int k, int d, int workers, int flags,
                 mh_set_result* out) {
    NvtxRange nvtx("mh_run_batch");
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
        if (flags & MH_BATCH_AUTOTUNE) {
            const mh_read_set& big = sets[order[0]];
            int cls = 0;
            while (cls < 63 && (2ull << cls) <= big.n_bases) cls++;
            const auto key = std::make_tuple(words_for(k), k, cls / 2);
            auto it = ctx->tuned.find(key);
            if (it == ctx->tuned.end()) {
                const Plan p = tune_plan(ctx->workers[0], big, k, d);
                if (!p.empty()) it = ctx->tuned.emplace(key, p).first;
            }
            if (it != ctx->tuned.end()) apply_plan(ctx, it->second);
        }
        for (int i = 0; i < workers; i++)
            apply_plan(ctx->workers[i], {ctx->count_path, ctx->sort_shape, ctx->unit_bits_delta,
                                         ctx->spread_bits_delta, ctx->bucket_bits});

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
                run_set_job(w, sets[j], k, d, flags, out[j]);
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
