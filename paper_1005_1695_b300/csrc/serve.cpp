// Serving loop: an open-loop stream of hashing requests over the job runtime.
//
// Section 2.2 of the CrystalGPU paper describes stream-processing
// applications: data units arrive continuously and each must be processed
// with low latency.  crystal_serve plays such a stream against a context:
// requests arrive at their given times, are admitted as soon as the
// context's pools can hold their buffers and scratch (admission by pool
// memory) -- in arrival order, except that while the oldest waiting request
// does not fit, later ones that do fit may pass it for a bounded time --
// have their bytes staged into the job's pinned buffer by copy threads, and
// are submitted; the master thread batches whatever is outstanding when a
// stream slot frees (continuous batching), so requests that arrive while
// others run join the next batch and overlap on the GPU.
// Completion callbacks record the times, optionally copy the result out,
// and release the job, which frees room for the next admission.
//
// Small requests can go through an input ring instead: one pinned block and
// one device block taken from the pools for the whole call, carved in
// admission order.  Their copy threads copy the bytes into the ring, so
// requests admitted one after another sit next to each other in host and in
// device memory, and the master merges their copies into one DMA transfer
// (each transfer costs a few microseconds beside its bytes, which for
// requests of a few hundred KiB is as much as the bytes themselves).
#include <stdint.h>
#include <string.h>
#include <time.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "crystal.h"
#include "crystal_internal.h"
#include "input_ring.h"

namespace {

// A blocked oldest request may be passed for this long by default
// (crystal_serve_config.bypass_ns), by up to this many candidates per pass.
constexpr uint64_t kDefaultBypassNs = 2000000;
constexpr uint32_t kBypassCandidates = 32;
// Requests up to this size go through the input ring when it is on
// (crystal_serve_config.ring_max_request = 0).
constexpr uint64_t kDefaultRingMaxRequest = 256 << 10;

uint64_t mono_ns() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (uint64_t)ts.tv_sec * 1000000000ull + (uint64_t)ts.tv_nsec;
}

struct Serve;

struct Ticket {
    Serve* s;
    uint32_t idx;
};

struct Serve {
    crystal_ctx* ctx = nullptr;
    const uint8_t* src = nullptr;
    const crystal_request* req = nullptr;
    crystal_request_result* res = nullptr;
    crystal_hash_params pd{}, ps{};
    uint8_t* capture = nullptr;
    uint64_t capture_bytes = 0;
    uint64_t t0 = 0;
    bool pinned_source = false;
    uint64_t bypass_ns = 0;  // how long the oldest waiting request may be passed
    std::vector<Ticket> tickets;
    // input ring (small requests): the pools' blocks, the size limit, and per
    // request its slot (offset, ticket) or crystal::InputRing::kNone
    crystal::InputRing ring;
    crystal::PoolPair ring_mem;
    uint64_t ring_max = 0;
    std::vector<uint64_t> ring_off, ring_seq;

    std::mutex mu;
    std::condition_variable cv_done, cv_work;
    std::deque<std::pair<uint32_t, crystal_task*>> work;
    uint32_t finished = 0;
    uint64_t last_done = 0;
    bool workers_stop = false;
    bool loop_waits = false;  // the admission loop is waiting on cv_done (under mu)

    const crystal_hash_params* params_for(int kind) const {
        return kind == CRYSTAL_KIND_MD5_SLIDING || kind == CRYSTAL_KIND_SHA1_SLIDING ? &ps : &pd;
    }

    // A request is done; wake the admission loop only if it waits for one
    // (a wake-up is a system call on the master thread's completion path).
    void finish(uint32_t i, int status) {
        const uint64_t t = mono_ns() - t0;
        bool wake;
        {
            std::lock_guard<std::mutex> lk(mu);
            res[i].status = status;
            res[i].done_ns = t;
            ++finished;
            if (t > last_done) last_done = t;
            wake = loop_waits;
        }
        if (wake) cv_done.notify_all();
    }
};

// Output bytes of a finished request that carry results.  Only called for a
// job that completed (OK or EOVERFLOW), whose header the kernels wrote; never
// more than the job's output buffer.
uint64_t used_bytes(int kind, uint64_t n, const uint8_t* out, uint64_t out_size) {
    const bool sha = kind == CRYSTAL_KIND_SHA1_DIRECT || kind == CRYSTAL_KIND_SHA1_SLIDING;
    const uint64_t D = sha ? 20 : 16;
    if (kind == CRYSTAL_KIND_MD5_DIRECT || kind == CRYSTAL_KIND_SHA1_DIRECT) return out_size < D ? 0 : D;
    if (kind != CRYSTAL_KIND_MD5_SLIDING && kind != CRYSTAL_KIND_SHA1_SLIDING) return out_size;
    if (out_size < 8) return 0;
    uint32_t hdr[2];
    memcpy(hdr, out, 8);
    const uint64_t fixed = 8 + 4 * ((n + 31) / 32);
    const uint64_t used = (hdr[1] & 1u) ? fixed : fixed + (4 + D) * (uint64_t)hdr[0];
    return used < out_size ? used : out_size;
}

// Completion callback, on the master thread.  A job that failed (a device
// or issue error, or cancellation) has no result: nothing is captured.
void on_done(crystal_task* t, int status, void* user) {
    Ticket* tk = static_cast<Ticket*>(user);
    Serve* s = tk->s;
    const uint32_t i = tk->idx;
    const crystal_request& r = s->req[i];
    const uint8_t* out = static_cast<const uint8_t*>(crystal_task_host_out(t));
    const bool has_result = status == CRYSTAL_OK || status == CRYSTAL_EOVERFLOW;
    const uint64_t used = has_result ? used_bytes(r.kind, r.size, out, r.out_size) : 0;
    s->res[i].used_bytes = used;
    if (used && r.capture_offset != UINT64_MAX && s->capture && r.capture_offset <= s->capture_bytes &&
        used <= s->capture_bytes - r.capture_offset)
        memcpy(s->capture + r.capture_offset, out, used);
    crystal_task_release(t);  // buffers back to the pools now (room for the next admission); handle later
    if (s->ring_off[i] != crystal::InputRing::kNone) s->ring.give_back(s->ring_seq[i]);
    s->finish(i, status);
}

void worker(Serve* s) {
    for (;;) {
        std::pair<uint32_t, crystal_task*> w;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [s] { return s->workers_stop || !s->work.empty(); });
            if (s->work.empty()) return;
            w = s->work.front();
            s->work.pop_front();
        }
        const crystal_request& r = s->req[w.first];
        if (s->ring_off[w.first] != crystal::InputRing::kNone) {
            if (r.size) memcpy(s->ring_mem.host + s->ring_off[w.first], s->src + r.src_offset, r.size);
        } else if (s->pinned_source) {
            crystal_task_bind_input(w.second, s->src + r.src_offset, r.size);
        } else if (r.size) {
            memcpy(crystal_task_host_in(w.second), s->src + r.src_offset, r.size);
        }
        s->res[w.first].submit_ns = mono_ns() - s->t0;
        const int st = crystal_task_submit(w.second, r.kind, s->params_for(r.kind), on_done, &s->tickets[w.first]);
        if (st != CRYSTAL_OK) {
            crystal_task_release(w.second);
            if (s->ring_off[w.first] != crystal::InputRing::kNone) s->ring.give_back(s->ring_seq[w.first]);
            s->finish(w.first, st);
        }
    }
}

}  // namespace

extern "C" {

int crystal_serve(crystal_ctx* ctx, const void* source, uint64_t source_bytes, const crystal_request* req,
                  uint32_t n, const crystal_serve_config* cfg, crystal_request_result* res, uint64_t* wall_ns) {
    if (!ctx || !req || !res || (!source && source_bytes)) return CRYSTAL_EINVAL;
    for (uint32_t i = 0; i < n; ++i) {
        const crystal_request& r = req[i];
        if (r.src_offset > source_bytes || r.size > source_bytes - r.src_offset) return CRYSTAL_EINVAL;
        if (r.kind < CRYSTAL_KIND_NOP || r.kind > CRYSTAL_KIND_SHA1_SLIDING) return CRYSTAL_EINVAL;
        if (i && r.arrival_ns < req[i - 1].arrival_ns) return CRYSTAL_EINVAL;
    }
    Serve s;
    s.ctx = ctx;
    s.src = static_cast<const uint8_t*>(source);
    s.req = req;
    s.res = res;
    crystal_params_default(&s.pd);
    crystal_params_default(&s.ps);
    uint32_t threads = 4;
    if (cfg) {
        if (cfg->direct_params) s.pd = *cfg->direct_params;
        if (cfg->sliding_params) s.ps = *cfg->sliding_params;
        s.capture = static_cast<uint8_t*>(cfg->capture);
        s.capture_bytes = cfg->capture_bytes;
        if (cfg->copy_threads) threads = cfg->copy_threads;
        s.pinned_source = cfg->flags & CRYSTAL_SERVE_SOURCE_PINNED;
    }
    s.bypass_ns = (cfg && (cfg->flags & CRYSTAL_SERVE_ARRIVAL_ORDER)) ? 0
                  : (cfg && cfg->bypass_ns) ? cfg->bypass_ns : kDefaultBypassNs;
    if (threads > 64) threads = 64;
    memset(res, 0, sizeof(crystal_request_result) * n);
    s.ring_off.assign(n, crystal::InputRing::kNone);
    s.ring_seq.assign(n, 0);
    if (cfg && cfg->ring_bytes) {
        const int rs = crystal::reserve_pool_pair(ctx, crystal::align_up(cfg->ring_bytes, 256), &s.ring_mem);
        if (rs != CRYSTAL_OK) return rs;
        s.ring.init(s.ring_mem.bytes);
        s.ring_max = cfg->ring_max_request ? cfg->ring_max_request : kDefaultRingMaxRequest;
    }
    s.tickets.resize(n);
    for (uint32_t i = 0; i < n; ++i) s.tickets[i] = Ticket{&s, i};
    std::vector<std::thread> pool;
    for (uint32_t k = 0; k < threads; ++k) pool.emplace_back(worker, &s);

    s.t0 = mono_ns();
    std::deque<uint32_t> fifo;  // arrived, not yet admitted (arrival order)
    uint32_t next = 0;
    uint32_t admitted = 0;      // admitted or refused at admission
    // Create request i's job; CRYSTAL_OK queues it for staging and submit.
    auto try_admit = [&](uint32_t i) {
        const crystal_request& r = req[i];
        const uint64_t scratch = crystal_scratch_bytes(r.kind, r.size, r.out_size, s.params_for(r.kind));
        crystal_task* t = nullptr;
        int st = CRYSTAL_EAGAIN;
        if (s.ring.enabled() && r.size <= s.ring_max) {
            uint64_t seq = 0;
            const uint64_t off = s.ring.take(r.size, &seq);
            if (off != crystal::InputRing::kNone) {
                st = crystal::task_create_borrowed(ctx, s.ring_mem.host + off, s.ring_mem.dev + off, r.size,
                                                   r.out_size, scratch, &t);
                if (st == CRYSTAL_OK) {
                    s.ring_off[i] = off;
                    s.ring_seq[i] = seq;
                } else {
                    s.ring.give_back(seq);
                }
            }
        }
        // not in the ring (too large, the ring full, or the pools): buffers of its own
        if (!t) st = crystal_task_create_ex(ctx, r.size, r.out_size, scratch,
                                            s.pinned_source ? CRYSTAL_TASK_EXTERNAL_INPUT : 0u, &t);
        if (st == CRYSTAL_OK) {
            ++admitted;
            res[i].admit_ns = mono_ns() - s.t0;
            {
                std::lock_guard<std::mutex> lk(s.mu);
                s.work.emplace_back(i, t);
            }
            s.cv_work.notify_one();
        }
        return st;
    };
    auto refuse = [&](uint32_t i, int st) {
        ++admitted;
        res[i].admit_ns = mono_ns() - s.t0;
        s.finish(i, st);
    };
    for (;;) {
        const uint64_t now = mono_ns() - s.t0;
        while (next < n && req[next].arrival_ns <= now) fifo.push_back(next++);
        // admission: the oldest waiting request first
        while (!fifo.empty()) {
            const uint32_t i = fifo.front();
            const int st = try_admit(i);
            if (st == CRYSTAL_OK) {
                fifo.pop_front();
                continue;
            }
            if (st != CRYSTAL_EAGAIN) {
                fifo.pop_front();
                refuse(i, st);
                continue;
            }
            uint32_t finished;
            {
                std::lock_guard<std::mutex> lk(s.mu);
                finished = s.finished;
            }
            if (finished == admitted) {  // nothing in flight: it can never fit
                fifo.pop_front();
                refuse(i, CRYSTAL_ENOMEM);
                continue;
            }
            // The oldest request waits for room.  While it is young, later
            // requests that fit now are admitted past it (a few candidates per
            // pass); once it has waited bypass_ns nothing passes it any more,
            // so completions free room for it and it cannot starve.
            if (now - std::min(now, req[i].arrival_ns) < s.bypass_ns) {
                size_t k = 1;
                for (uint32_t tried = 0; k < fifo.size() && tried < kBypassCandidates; ++tried) {
                    const uint32_t j = fifo[k];
                    const int sj = try_admit(j);
                    if (sj == CRYSTAL_EAGAIN) {
                        ++k;
                        continue;
                    }
                    fifo.erase(fifo.begin() + (std::ptrdiff_t)k);
                    if (sj != CRYSTAL_OK) refuse(j, sj);
                }
            }
            break;  // wait for a completion (or the next arrival)
        }
        std::unique_lock<std::mutex> lk(s.mu);
        if (s.finished == n) break;
        if (!fifo.empty()) {
            // blocked on pool room: wake on a completion or the next arrival
            const uint32_t before = s.finished;
            const uint64_t wait = next < n && req[next].arrival_ns > now ? req[next].arrival_ns - now : 200000;
            s.loop_waits = true;
            s.cv_done.wait_for(lk, std::chrono::nanoseconds(wait < 200000 ? wait : 200000),
                               [&] { return s.finished != before; });
            s.loop_waits = false;
        } else if (next < n) {
            const uint64_t due = req[next].arrival_ns;
            lk.unlock();
            const uint64_t t = mono_ns() - s.t0;
            if (due > t + 200000) {
                std::this_thread::sleep_for(std::chrono::nanoseconds(due - t - 100000));
            } else {
                while (mono_ns() - s.t0 < due) std::this_thread::yield();
            }
        } else {
            s.loop_waits = true;
            s.cv_done.wait(lk, [&] { return s.finished == n; });
            s.loop_waits = false;
            break;
        }
    }
    {
        std::lock_guard<std::mutex> lk(s.mu);
        s.workers_stop = true;
    }
    s.cv_work.notify_all();
    for (auto& th : pool) th.join();
    crystal::release_pool_pair(ctx, s.ring_mem);
    if (wall_ns) *wall_ns = s.last_done;
    int worst = CRYSTAL_OK;
    for (uint32_t i = 0; i < n; ++i)
        if (res[i].status < 0 && res[i].status != CRYSTAL_EOVERFLOW) worst = res[i].status;
    return worst;
}

}  // extern "C"
