// Job stream staged from pageable host memory through a ring of pooled jobs.
//
// Section 2.1 of the CrystalGPU paper: the GPU's DMA engines copy only from
// page-locked memory, so bytes an application holds in ordinary (pageable)
// memory are first copied into a pinned buffer -- by the driver, into its own
// staging buffer, unless the application stages them itself.  Section 3 keeps
// such pinned buffers in a pool allocated once, and Section 4.1 (Figure 4)
// overlaps the copies of some jobs with the kernels of others.
// crystal_stream_staged puts the three together for a stream of units in
// pageable memory: a fixed ring of jobs, each with its own pinned input and
// output, is created once; host copy threads take the units in order, copy
// each into the pinned input of a free job and submit it; a finished job goes
// back to the ring, and the copy thread that reuses it first moves the
// finished unit's result out to the caller's buffer.  The master thread only
// batches, launches and completes, as for any other job.
#include <stdint.h>
#include <string.h>
#include <time.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "crystal.h"
#include "crystal_internal.h"

using namespace crystal;

namespace {

uint64_t mono_ns() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (uint64_t)ts.tv_sec * 1000000000ull + (uint64_t)ts.tv_nsec;
}

struct Ring;

struct Ticket {
    Ring* ring;
    uint32_t job;
};

struct Ring {
    crystal_ctx* ctx = nullptr;
    const void* const* units = nullptr;
    const uint64_t* sizes = nullptr;
    uint32_t n = 0;
    int kind = 0;
    crystal_hash_params params{};
    uint64_t out_size = 0;
    uint8_t* outputs = nullptr;
    uint64_t out_stride = 0;
    crystal_request_result* res = nullptr;
    uint64_t t0 = 0;

    std::vector<crystal_task*> jobs;
    std::vector<int64_t> job_unit;  // unit whose result the job holds (-1: none)
    std::vector<Ticket> tickets;
    std::atomic<uint32_t> next{0};

    std::mutex mu;
    std::condition_variable cv_free, cv_done;
    std::deque<uint32_t> free_jobs;  // FIFO: jobs rotate in creation order, so
                                     // consecutive submits have adjacent buffers
    uint32_t finished = 0;
    uint32_t waiting = 0;  // copy threads waiting for a free job
};

// Used output bytes of a finished unit (never more than the job's buffer).
uint64_t used_bytes(int kind, uint64_t n, const uint8_t* out, uint64_t out_size) {
    if (kind_is_direct(kind)) return std::min<uint64_t>(digest_bytes_of(kind), out_size);
    if (!kind_is_sliding(kind)) return out_size;
    if (out_size < 8) return 0;
    uint32_t hdr[2];
    memcpy(hdr, out, 8);
    const uint64_t fixed = sliding_fixed_bytes(n);
    const uint64_t used = (hdr[1] & 1u) ? fixed : fixed + (4 + digest_bytes_of(kind)) * (uint64_t)hdr[0];
    return std::min(used, out_size);
}

// Copy the result a job holds to the caller's buffer (copy threads, or the
// caller's thread at the end; never while the job runs).
void retire(Ring* r, uint32_t j) {
    const int64_t u = r->job_unit[j];
    if (u < 0) return;
    r->job_unit[j] = -1;
    crystal_request_result& x = r->res[u];
    if (x.status != CRYSTAL_OK && x.status != CRYSTAL_EOVERFLOW) return;
    const uint8_t* out = static_cast<const uint8_t*>(crystal_task_host_out(r->jobs[j]));
    x.used_bytes = used_bytes(r->kind, r->sizes[u], out, r->out_size);
    if (r->outputs) memcpy(r->outputs + (uint64_t)u * r->out_stride, out, std::min(x.used_bytes, r->out_stride));
}

// A job back in the ring: wake a copy thread only if one waits, the caller
// only after the last unit (wake-ups cost system calls on the master thread).
void give_back(Ring* r, uint32_t j) {
    bool wake_copy, all_done;
    {
        std::lock_guard<std::mutex> lk(r->mu);
        r->free_jobs.push_back(j);
        ++r->finished;
        wake_copy = r->waiting > 0;
        all_done = r->finished == r->n;
    }
    if (wake_copy) r->cv_free.notify_one();
    if (all_done) r->cv_done.notify_all();
}

// Completion callback, on the master thread: record, hand the job back.  The
// job is still running until the callback returns; whoever takes it next
// waits for that (crystal_task_wait) before touching it.
void on_done(crystal_task*, int status, void* user) {
    Ticket* tk = static_cast<Ticket*>(user);
    Ring* r = tk->ring;
    const int64_t u = r->job_unit[tk->job];
    r->res[u].status = status;
    r->res[u].done_ns = mono_ns() - r->t0;
    give_back(r, tk->job);
}

void copy_thread(Ring* r) {
    for (;;) {
        const uint32_t u = r->next.fetch_add(1);
        if (u >= r->n) return;
        uint32_t j;
        {
            std::unique_lock<std::mutex> lk(r->mu);
            ++r->waiting;
            r->cv_free.wait(lk, [r] { return !r->free_jobs.empty(); });
            --r->waiting;
            j = r->free_jobs.front();
            r->free_jobs.pop_front();
        }
        crystal_task* t = r->jobs[j];
        if (r->job_unit[j] >= 0) crystal_task_wait(t, -1);  // its callback may still be returning
        retire(r, j);
        crystal_request_result& x = r->res[u];
        x.admit_ns = mono_ns() - r->t0;
        int st = crystal_task_resize(t, r->sizes[u], r->out_size);
        if (st == CRYSTAL_OK && r->sizes[u]) memcpy(crystal_task_host_in(t), r->units[u], r->sizes[u]);
        r->job_unit[j] = u;
        x.submit_ns = mono_ns() - r->t0;
        if (st == CRYSTAL_OK) st = crystal_task_submit(t, r->kind, &r->params, on_done, &r->tickets[j]);
        if (st != CRYSTAL_OK) {
            x.status = st;
            x.done_ns = mono_ns() - r->t0;
            r->job_unit[j] = -1;
            give_back(r, j);
        }
    }
}

}  // namespace

extern "C" {

int crystal_stream_staged(crystal_ctx* ctx, const void* const* units, const uint64_t* sizes, uint32_t n,
                          const crystal_stream_config* cfg, void* outputs, uint64_t out_stride,
                          crystal_request_result* results, uint64_t* wall_ns) {
    if (!ctx || !cfg || !results || (n && (!units || !sizes))) return CRYSTAL_EINVAL;
    if (cfg->reserved || (outputs && out_stride == 0)) return CRYSTAL_EINVAL;
    const int kind = cfg->kind;
    if (kind < CRYSTAL_KIND_NOP || kind > CRYSTAL_KIND_SHA1_SLIDING) return CRYSTAL_EINVAL;
    uint64_t max_in = 0;
    for (uint32_t i = 0; i < n; ++i) {
        if (sizes[i] && !units[i]) return CRYSTAL_EINVAL;
        max_in = std::max(max_in, sizes[i]);
    }
    crystal_config cc;
    if (crystal_get_config(ctx, &cc) != CRYSTAL_OK) return CRYSTAL_EINVAL;
    Ring r;
    r.ctx = ctx;
    r.units = units;
    r.sizes = sizes;
    r.n = n;
    r.kind = kind;
    crystal_params_default(&r.params);
    if (cfg->params) r.params = *cfg->params;
    r.out_size = cfg->out_size;
    r.outputs = static_cast<uint8_t*>(outputs);
    r.out_stride = out_stride;
    r.res = results;
    memset(results, 0, sizeof(crystal_request_result) * n);
    const uint32_t threads = std::min<uint32_t>(cfg->copy_threads ? cfg->copy_threads : 4, 64);
    uint32_t ring = cfg->ring_jobs ? cfg->ring_jobs
                                   : 3u * (uint32_t)cc.n_streams * std::min<uint32_t>(cc.max_batch_jobs, 4u);
    ring = std::max<uint32_t>(1, std::min<uint32_t>(ring, std::max<uint32_t>(n, 1)));
    // the ring: every job can take the largest unit, with its scratch reserved
    // so that a submit never waits for device memory
    const uint64_t scratch = crystal_scratch_bytes(kind, max_in, r.out_size, &r.params);
    int st = CRYSTAL_OK;
    for (uint32_t j = 0; j < ring && st == CRYSTAL_OK; ++j) {
        crystal_task* t = nullptr;
        st = crystal_task_create_ex(ctx, max_in, r.out_size, scratch, 0, &t);
        if (st == CRYSTAL_OK) r.jobs.push_back(t);
    }
    if (st != CRYSTAL_OK) {
        for (crystal_task* t : r.jobs) crystal_task_release(t);
        return st;
    }
    r.job_unit.assign(ring, -1);
    r.tickets.resize(ring);
    for (uint32_t j = 0; j < ring; ++j) {
        r.tickets[j] = Ticket{&r, j};
        r.free_jobs.push_back(j);
    }
    r.t0 = mono_ns();
    std::vector<std::thread> pool;
    try {
        for (uint32_t k = 0; k < threads; ++k) pool.emplace_back(copy_thread, &r);
    } catch (...) {
        r.next.store(n);  // threads already started stop at once
        for (auto& th : pool) th.join();
        for (crystal_task* t : r.jobs) crystal_task_release(t);
        return CRYSTAL_ENOMEM;
    }
    for (auto& th : pool) th.join();
    {
        std::unique_lock<std::mutex> lk(r.mu);
        r.cv_done.wait(lk, [&r] { return r.finished == r.n; });
    }
    for (uint32_t j = 0; j < ring; ++j) {
        if (r.job_unit[j] >= 0) crystal_task_wait(r.jobs[j], -1);
        retire(&r, j);
    }
    if (wall_ns) *wall_ns = mono_ns() - r.t0;
    for (crystal_task* t : r.jobs) crystal_task_release(t);
    int worst = CRYSTAL_OK;
    for (uint32_t i = 0; i < n; ++i)
        if (results[i].status < 0 && results[i].status != CRYSTAL_EOVERFLOW) worst = results[i].status;
    return worst;
}

}  // extern "C"
