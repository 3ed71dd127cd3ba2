// Job runtime: the CrystalGPU master module on one B300.
//
// Section 4.2 of the paper: a host master thread owns the GPU, jobs move
// through idle / outstanding / running states, the master takes outstanding
// jobs in FIFO order, runs each as copy-in / kernel / copy-out (Figure 4) on
// one of several streams so that the stages of different jobs overlap, finds
// completion by polling (Section 4.1: no completion interrupt) and runs the
// job's callback.  Section 3: job buffers come from a pool allocated once at
// init (one device arena, one pinned host arena) instead of per job.
//
// B300 specifics: the master groups the outstanding jobs it finds into one
// batch per stream slot, so a batch costs one descriptor upload and one
// persistent-kernel chain however many jobs it holds; with
// CRYSTAL_FLAG_GRAPHS that chain is a captured CUDA graph.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <string.h>
#include <time.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_set>
#include <vector>

#include "crystal.h"
#include "crystal_internal.h"

using namespace crystal;

namespace {

uint64_t now_ns() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (uint64_t)ts.tv_sec * 1000000000ull + (uint64_t)ts.tv_nsec;
}

enum TaskState : int { T_IDLE = 0, T_OUTSTANDING = 1, T_RUNNING = 2, T_DONE = 3 };

// Short polling windows before a thread blocks (the master when it runs out
// of work, a waiter before it sleeps): a thread wake-up costs tens of
// microseconds, comparable to a small job.
constexpr uint64_t kIdleSpinNs = 200000;
constexpr uint64_t kWaitSpinNs = 200000;

struct Slot {
    cudaStream_t stream = nullptr;
    uint32_t stream_index = 0;
    bool own_stream = false;  // slots beyond the first n_streams share a stream
    cudaEvent_t done = nullptr;
    crystal_batch* h_desc = nullptr;  // pinned
    uint8_t* h_desc_dev = nullptr;    // its device-visible address when mapped (descriptor fetched by the GPU)
    crystal_batch* d_desc = nullptr;  // device, inside the device arena
    uint64_t d_desc_off = 0;
    std::vector<crystal_task*> tasks;
    bool busy = false;
    uint64_t seq = 0;
    // [size class][has_direct | has_sliding << 1]
    cudaGraphExec_t graph[CRYSTAL_SIZE_CLASSES][4] = {};
};

thread_local const crystal_ctx* tl_callback_ctx = nullptr;

// NVTX ranges (header-only NVTX 3) around the master thread's work -- issuing
// a batch, completing one, capturing a graph -- so that a timeline tool
// (Nsight Systems, or ncu's NVTX filters) shows the runtime's stages beside
// the copies and kernels; without a tool attached each range costs a few
// nanoseconds.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace

struct crystal_task {
    crystal_ctx* ctx = nullptr;
    uint8_t* h_in = nullptr;
    uint8_t* h_out = nullptr;
    uint8_t* d_in = nullptr;
    uint8_t* d_out = nullptr;
    uint8_t* d_scratch = nullptr;
    uint8_t* d_reserved = nullptr;  // scratch reserved at create (crystal_task_create_ex)
    const uint8_t* h_in_ext = nullptr;  // caller memory bound as the input (crystal_task_bind_input)
    bool external_input = false;        // created without its own pinned input buffer
    bool borrowed_input = false;        // h_in / d_in lie in memory the job does not own (an input ring)
    bool one_block = false;             // d_in, d_out and d_reserved are one device allocation at d_in
    uint64_t h_in_off = 0, h_out_off = 0, d_in_off = 0, d_out_off = 0, d_scratch_off = 0, d_reserved_off = 0;
    uint64_t reserved_bytes = 0;
    uint64_t in_cap = 0, out_cap = 0, in_size = 0, out_size = 0, scratch_bytes = 0;
    int kind = 0;
    crystal_hash_params params{};
    crystal_callback cb = nullptr;
    void* user = nullptr;
    std::atomic<int> state{T_IDLE};  // written under the context lock; read lock-free by waiters
    int priority = 0;                 // higher is dispatched first (crystal_task_set_priority)
    int status = CRYSTAL_EINVAL;
    bool submitted_once = false;
    bool release_in_callback = false;
    uint64_t t_submit = 0, t_dispatch = 0, t_done = 0;
};

namespace {

// The outstanding queue (Section 4.2): FIFO within a priority, higher
// priorities first.  With every job at priority 0 it is the paper's FIFO.
class OutstandingQueue {
  public:
    bool empty() const { return n_ == 0; }
    size_t size() const { return n_; }
    crystal_task* front() const { return q_.begin()->second.front(); }
    void pop_front() {
        auto it = q_.begin();
        it->second.pop_front();
        if (it->second.empty()) q_.erase(it);
        --n_;
    }
    void push_back(crystal_task* t, int priority) {
        q_[priority].push_back(t);
        ++n_;
    }
    std::vector<crystal_task*> drain() {
        std::vector<crystal_task*> all;
        for (auto& kv : q_) all.insert(all.end(), kv.second.begin(), kv.second.end());
        q_.clear();
        n_ = 0;
        return all;
    }

  private:
    std::map<int, std::deque<crystal_task*>, std::greater<int>> q_;
    size_t n_ = 0;
};

}  // namespace

struct crystal_ctx {
    crystal_config cfg{};
    int device = 0;
    bool pooled = true;
    uint8_t* d_base = nullptr;
    bool own_d_base = false;
    crystal_arena* d_arena = nullptr;
    uint8_t* h_base = nullptr;
    crystal_arena* h_arena = nullptr;
    std::vector<Slot> slots;
    uint32_t next_slot = 0;
    uint32_t max_jobs = 64;
    uint64_t max_bytes = 32ull << 20;
    uint64_t region_bytes = 0;  // per slot: the batch descriptor (header + max_jobs units)
    bool h_mapped = false;      // the host pool is mapped into the device's address space
    LaunchGeom geom[CRYSTAL_SIZE_CLASSES];  // launch geometry per batch size class
    int64_t h_dev_delta = 0;    // device-visible address of a host-pool byte minus its address

    std::mutex mu;
    std::condition_variable cv_master;
    std::condition_variable cv_done;
    OutstandingQueue outstanding;
    std::deque<uint32_t> running;  // slot indices in dispatch order
    std::mutex tasks_mu;           // guards `tasks` only (not the queues), so that creating and
    std::unordered_set<crystal_task*> tasks;  // freeing jobs does not hold up submits and completion
    std::thread master;
    bool stop = false;
    bool accepting = true;                 // written under mu
    std::atomic<bool> accepting_fast{true};  // its copy for checks that need no lock
    uint64_t seq = 0;

    std::atomic<uint64_t> n_outstanding{0};  // mirrors outstanding.size() for the idle spin
    std::atomic<uint64_t> jobs_completed{0};
    std::atomic<uint64_t> batches{0};
    std::atomic<uint64_t> copies_dma{0};
    std::atomic<uint64_t> issue_ns{0}, complete_ns{0};  // master thread time issuing / completing batches
    std::atomic<uint64_t> create_ns{0}, create_calls{0}, create_eagain{0};  // crystal_task_create_ex
    std::atomic<uint64_t> graph_captures{0};
    uint64_t n_running_jobs = 0;
};

namespace {

// ---- buffers ------------------------------------------------------------------

int alloc_device(crystal_ctx* c, uint64_t bytes, uint8_t** p, uint64_t* off, int placement = CRYSTAL_ARENA_HIGHEST) {
    if (c->pooled) {
        int st = crystal_arena_alloc_at(c->d_arena, bytes, placement, off);
        if (st != CRYSTAL_OK) return st;
        *p = c->d_base + *off;
        return CRYSTAL_OK;
    }
    void* q = nullptr;
    if (cudaMalloc(&q, bytes ? bytes : 1) != cudaSuccess) {
        cudaGetLastError();
        return CRYSTAL_ENOMEM;
    }
    *p = (uint8_t*)q;
    return CRYSTAL_OK;
}

void free_device(crystal_ctx* c, uint8_t* p, uint64_t off) {
    if (!p) return;
    if (c->pooled) crystal_arena_free(c->d_arena, off);
    else cudaFree(p);
}

int alloc_host(crystal_ctx* c, uint64_t bytes, uint8_t** p, uint64_t* off, int placement = CRYSTAL_ARENA_HIGHEST) {
    if (c->pooled) {
        int st = crystal_arena_alloc_at(c->h_arena, bytes, placement, off);
        if (st != CRYSTAL_OK) return st;
        *p = c->h_base + *off;
        return CRYSTAL_OK;
    }
    void* q = nullptr;
    if (cudaHostAlloc(&q, bytes ? bytes : 1, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return CRYSTAL_ENOMEM;
    }
    *p = (uint8_t*)q;
    return CRYSTAL_OK;
}

void free_host(crystal_ctx* c, uint8_t* p, uint64_t off) {
    if (!p) return;
    if (c->pooled) crystal_arena_free(c->h_arena, off);
    else cudaFreeHost(p);
}

// Scratch a finished job gives back (none when it used its reserved scratch).
void free_job_scratch(crystal_ctx* c, crystal_task* t) {
    if (t->d_scratch && t->d_scratch != t->d_reserved) free_device(c, t->d_scratch, t->d_scratch_off);
    t->d_scratch = nullptr;
}

void free_task_buffers(crystal_task* t) {
    crystal_ctx* c = t->ctx;
    free_job_scratch(c, t);
    if (t->borrowed_input) t->h_in = t->d_in = nullptr;  // the ring's owner frees them
    if (t->one_block) {
        free_device(c, t->d_in, t->d_in_off);
        t->d_in = t->d_reserved = t->d_out = nullptr;
    }
    free_device(c, t->d_reserved, t->d_reserved_off);
    t->d_reserved = nullptr;
    free_device(c, t->d_in, t->d_in_off);
    free_device(c, t->d_out, t->d_out_off);
    free_host(c, t->h_in, t->h_in_off);
    free_host(c, t->h_out, t->h_out_off);
    t->d_in = t->d_out = t->h_in = t->h_out = nullptr;
}

// ---- parameters ---------------------------------------------------------------

int resolve_params(int kind, const crystal_hash_params* in, uint64_t n, uint64_t out_size,
                   crystal_hash_params* p) {
    crystal_params_default(p);
    if (in) {
        if (in->reserved != 0) return CRYSTAL_EINVAL;
        if (in->segment_bytes) p->segment_bytes = in->segment_bytes;
        if (in->window_bytes) p->window_bytes = in->window_bytes;
        if (in->chunk_segment_bytes) p->chunk_segment_bytes = in->chunk_segment_bytes;
        p->mask = in->mask;
        p->target = in->target;
    }
    if (kind == CRYSTAL_KIND_NOP) return CRYSTAL_OK;
    if (kind_is_direct(kind)) return out_size >= digest_bytes_of(kind) ? CRYSTAL_OK : CRYSTAL_EINVAL;
    if (kind_is_sliding(kind)) {
        if (p->window_bytes > kMaxWindow || n >= (1ull << 32)) return CRYSTAL_EINVAL;
        if (out_size < sliding_fixed_bytes(n) || out_size >= (1ull << 32)) return CRYSTAL_EINVAL;
        return CRYSTAL_OK;
    }
    return CRYSTAL_EINVAL;
}

// ---- issuing a batch --------------------------------------------------------------

// Fill the slot's pinned descriptor from its jobs: direct units first.  With
// the host pool mapped, a direct job's digest (its whole output) is written by
// the kernel straight into the job's pinned output buffer: no copy-out, which
// for a 16-byte result would cost a full DMA transfer.
bool digest_in_place(const crystal_ctx* c, const crystal_task* t) { return c->h_mapped && kind_is_direct(t->kind); }

void build_descriptor(const crystal_ctx* c, Slot& s, uint32_t* nd_out, uint32_t* ns_out) {
    crystal_unit* U = batch_units(s.h_desc);
    uint32_t k = 0;
    for (int pass = 0; pass < 2; ++pass) {
        for (crystal_task* t : s.tasks) {
            if (pass == 0 ? !kind_is_direct(t->kind) : !kind_is_sliding(t->kind)) continue;
            crystal_unit& x = U[k++];
            x.in = (uint64_t)t->d_in;
            x.n = t->in_size;
            x.out = digest_in_place(c, t) ? (uint64_t)t->h_out + (uint64_t)c->h_dev_delta : (uint64_t)t->d_out;
            x.scratch = (uint64_t)t->d_scratch;
            x.work_begin = 0;
            x.out_cap = (uint32_t)std::min<uint64_t>(t->out_size, 0xFFFFFFFFull);
            x.seg_bytes = pass == 0 ? t->params.segment_bytes : t->params.chunk_segment_bytes;
            x.window = (uint16_t)t->params.window_bytes;
            x.mask = t->params.mask;
            x.target = t->params.target;
            x.kind = (uint16_t)t->kind;
            x.seg_base = 0;
        }
        if (pass == 0) *nd_out = k;
    }
    *ns_out = k - *nd_out;
}

int launch_chain(crystal_batch* d, cudaStream_t st, bool direct, bool sliding, const LaunchGeom* g) {
    int r = CRYSTAL_OK;
    if (direct) {
        r = launch_direct_segments(d, st, g);
        if (r == CRYSTAL_OK) r = launch_direct_outer(d, st, g);
    }
    if (sliding && r == CRYSTAL_OK) {
        r = launch_sliding_windows(d, st, g);
        if (r == CRYSTAL_OK) r = launch_sliding_chunks(d, st, g);
        if (r == CRYSTAL_OK) r = launch_sliding_digests(d, st, g);
    }
    return r;
}

// Size class of a batch: the mean input bytes of its hashing jobs.
int size_class(const Slot& s) {
    uint64_t bytes = 0, n = 0;
    for (const crystal_task* t : s.tasks) {
        if (t->kind == CRYSTAL_KIND_NOP) continue;
        bytes += t->in_size;
        ++n;
    }
    const uint64_t mean = n ? bytes / n : 0;
    return mean < (64u << 10) ? 0 : mean < (1u << 20) ? 1 : 2;
}

int kernels_in_chain(bool direct, bool sliding) { return (direct ? 3 : 0) + (sliding ? 7 : 0); }

// Descriptor in, kernel chain, status back: the device side of one batch.
// With the slot's descriptor region mapped, the GPU fetches the descriptor
// and posts the status itself (two small kernels) instead of two DMA
// transfers of a few microseconds each.
int batch_sequence(crystal_ctx* c, Slot& s, bool direct, bool sliding, const LaunchGeom* g) {
    cudaStream_t st = s.stream;
    int r = CRYSTAL_OK;
    if (s.h_desc_dev) {
        r = launch_fetch_descriptor(s.h_desc_dev, s.d_desc, c->region_bytes, st);
    } else if (cudaMemcpyAsync(s.d_desc, s.h_desc, c->region_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        r = CRYSTAL_EDEVICE;
    }
    if (r == CRYSTAL_OK) r = launch_chain(s.d_desc, st, direct, sliding, g);
    if (r != CRYSTAL_OK) return r;
    if (s.h_desc_dev) {
        const uint64_t status_off = offsetof(crystal_batch, status);
        return launch_post_status(s.d_desc, reinterpret_cast<uint32_t*>(s.h_desc_dev + status_off), st);
    }
    return cudaMemcpyAsync(s.h_desc, s.d_desc, sizeof(crystal_batch), cudaMemcpyDeviceToHost, st) == cudaSuccess
               ? CRYSTAL_OK
               : CRYSTAL_EDEVICE;
}

// Capture batch_sequence of one slot as a graph.
int capture_graph(crystal_ctx* c, Slot& s, int cls, int variant) {
    NvtxRange range("crystal: capture batch graph");
    const bool direct = variant & 1, sliding = variant & 2;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return CRYSTAL_EDEVICE;
    tl_capturing = true;
    int r = batch_sequence(c, s, direct, sliding, &c->geom[cls]);
    tl_capturing = false;
    cudaError_t e = cudaStreamEndCapture(s.stream, &g);
    if (r != CRYSTAL_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return CRYSTAL_EDEVICE;
    }
    e = cudaGraphInstantiate(&s.graph[cls][variant], g, 0);
    cudaGraphDestroy(g);
    if (e == cudaSuccess) c->graph_captures.fetch_add(1, std::memory_order_relaxed);
    return e == cudaSuccess ? CRYSTAL_OK : CRYSTAL_EDEVICE;
}

// One copy of a batch: host range <-> device range, n bytes.
struct Run {
    const uint8_t* host;
    uint8_t* dev;
    uint64_t n;
};

// Copies of several jobs merged into one when their host ranges and their
// device ranges are both contiguous blocks at the same host-to-device offset
// (fewer, larger transfers: a DMA transfer costs a few microseconds whatever
// its size -- about 3.7 us on B300, so 256 KiB moves at 30 GB/s and 4 MiB at
// 53).  A job's block is its whole allocation, so a merged copy only ever
// covers memory of the merged jobs.
class RunBuilder {
  public:
    explicit RunBuilder(std::vector<Run>* out) : out_(out) {}
    // host/dev: the job's buffers; used: bytes that matter; block: allocated bytes
    void add(const uint8_t* host, uint8_t* dev, uint64_t used, uint64_t block, bool mergeable) {
        if (!used) return;
        const int64_t delta = (int64_t)((uint64_t)dev - (uint64_t)host);
        if (open_ && mergeable && delta == delta_) {
            if (host == hi_) {  // just above the run
                hi_ = host + block;
                end_ = host + used;
                return;
            }
            if (host + block == lo_) {  // just below the run
                lo_ = host;
                return;
            }
        }
        flush();
        if (!mergeable) {
            out_->push_back(Run{host, dev, used});
            return;
        }
        open_ = true;
        lo_ = host;
        hi_ = host + block;
        end_ = host + used;
        delta_ = delta;
    }
    void flush() {
        if (!open_) return;
        open_ = false;
        out_->push_back(Run{lo_, reinterpret_cast<uint8_t*>((uint64_t)lo_ + (uint64_t)delta_), (uint64_t)(end_ - lo_)});
    }

  private:
    std::vector<Run>* out_;
    bool open_ = false;
    const uint8_t* lo_ = nullptr;
    const uint8_t* hi_ = nullptr;   // end of the highest block in the run
    const uint8_t* end_ = nullptr;  // end of the bytes to copy (in the highest block)
    int64_t delta_ = 0;
};

bool dma(const Run& r, cudaMemcpyKind kind, cudaStream_t st) {
    if (kind == cudaMemcpyHostToDevice) return cudaMemcpyAsync(r.dev, r.host, r.n, kind, st) == cudaSuccess;
    return cudaMemcpyAsync(const_cast<uint8_t*>(r.host), r.dev, r.n, kind, st) == cudaSuccess;
}

// Issue copy-in, kernels and copy-out of the slot's jobs on its stream.
int issue(crystal_ctx* c, Slot& s) {
    NvtxRange range("crystal: issue batch");
    cudaStream_t st = s.stream;
    uint32_t nd = 0, ns = 0;
    build_descriptor(c, s, &nd, &ns);
    const bool hashing = nd + ns > 0;
    // The batch's copies in host-address order, so that the buffers of jobs
    // that sit next to each other in the pools merge into one transfer
    // whatever order the jobs were submitted in (the units' order in the
    // descriptor does not matter: every unit carries its own pointers).
    std::vector<Run> in_runs, out_runs;
    {
        struct Piece {
            const uint8_t* host;
            uint8_t* dev;
            uint64_t used, block;
            bool mergeable;
        };
        std::vector<Piece> pieces;
        pieces.reserve(s.tasks.size());
        auto build = [&](std::vector<Run>* runs) {
            std::sort(pieces.begin(), pieces.end(), [](const Piece& a, const Piece& b) { return a.host < b.host; });
            RunBuilder rb(runs);
            for (const Piece& q : pieces) rb.add(q.host, q.dev, q.used, q.block, q.mergeable);
            rb.flush();
            pieces.clear();
        };
        for (crystal_task* t : s.tasks) {
            const bool own = !t->h_in_ext;
            pieces.push_back(Piece{own ? t->h_in : t->h_in_ext, t->d_in, t->in_size,
                                   align_up(t->in_cap ? t->in_cap : 1, 256), own && c->pooled});
        }
        build(&in_runs);
        for (crystal_task* t : s.tasks) {
            if (digest_in_place(c, t)) continue;  // already in h_out when the batch completes
            pieces.push_back(Piece{t->h_out, t->d_out, t->out_size, align_up(t->out_cap ? t->out_cap : 1, 256),
                                   c->pooled});
        }
        build(&out_runs);
    }
    for (const Run& r : in_runs)
        if (!dma(r, cudaMemcpyHostToDevice, st)) return CRYSTAL_EDEVICE;
    if (hashing) {
        if (crystal_batch_plan(s.h_desc, nd, ns) != CRYSTAL_OK) return CRYSTAL_EINVAL;
        const int variant = (nd ? 1 : 0) | (ns ? 2 : 0);
        const int cls = size_class(s);
        if (c->cfg.flags & CRYSTAL_FLAG_GRAPHS) {
            cudaGraphExec_t& ge = s.graph[cls][variant];
            if (!ge && capture_graph(c, s, cls, variant) != CRYSTAL_OK) return CRYSTAL_EDEVICE;
            if (cudaGraphLaunch(ge, st) != cudaSuccess) return CRYSTAL_EDEVICE;
            g_kernel_launches.fetch_add((uint64_t)(kernels_in_chain(nd, ns) + (s.h_desc_dev ? 2 : 0)));
        } else {
            const int r = batch_sequence(c, s, nd > 0, ns > 0, &c->geom[cls]);
            if (r != CRYSTAL_OK) return r;
        }
    } else {
        // only dummy jobs: the "dummy kernel with insignificant execution
        // time" of the overhead experiment (Section 5.1)
        s.h_desc->status = 0;
        if (launch_nop(st) != CRYSTAL_OK) return CRYSTAL_EDEVICE;
    }
    for (const Run& r : out_runs)
        if (!dma(r, cudaMemcpyDeviceToHost, st)) return CRYSTAL_EDEVICE;
    c->copies_dma.fetch_add(in_runs.size() + out_runs.size());
    if (cudaEventRecord(s.done, st) != cudaSuccess) return CRYSTAL_EDEVICE;
    return CRYSTAL_OK;
}

int job_status(crystal_task* t, uint32_t dev_status) {
    if (dev_status) return CRYSTAL_EDEVICE;
    if (kind_is_sliding(t->kind)) {
        uint32_t flags;
        memcpy(&flags, t->h_out + 4, 4);
        if (flags & 1u) return CRYSTAL_EOVERFLOW;
    }
    return CRYSTAL_OK;
}

// Jobs released from their callbacks (their buffers are already back in the
// pools): out of the registry, handles freed.
void destroy_released(crystal_ctx* c, const std::vector<crystal_task*>& released) {
    if (released.empty()) return;
    {
        std::lock_guard<std::mutex> lk(c->tasks_mu);
        for (crystal_task* j : released) c->tasks.erase(j);
    }
    for (crystal_task* j : released) {
        free_task_buffers(j);
        delete j;
    }
}

// Finish the jobs of a slot: statuses, scratch back to the pool, callbacks,
// then the jobs' final states in one locked step, waiters, and the buffers
// of jobs released from their callbacks.  Called by the master thread
// without the lock held.
void finish_slot(crystal_ctx* c, Slot& s, int issue_status) {
    NvtxRange range("crystal: complete batch");
    const uint64_t t = now_ns();
    const uint32_t dev_status = s.h_desc ? s.h_desc->status : 0;
    std::vector<crystal_task*> jobs;
    jobs.swap(s.tasks);
    for (crystal_task* j : jobs) {
        j->status = issue_status != CRYSTAL_OK ? issue_status : job_status(j, dev_status);
        j->t_done = t;
        free_job_scratch(c, j);
    }
    for (crystal_task* j : jobs) {
        if (j->cb) {
            tl_callback_ctx = c;
            j->cb(j, j->status, j->user);
            tl_callback_ctx = nullptr;
        }
    }
    std::vector<crystal_task*> released;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        for (crystal_task* j : jobs) {
            c->n_running_jobs--;
            if (j->release_in_callback) released.push_back(j);
            else j->state = T_DONE;
        }
        s.busy = false;
    }
    c->jobs_completed.fetch_add(jobs.size());
    c->cv_done.notify_all();
    destroy_released(c, released);
}

bool take_batch(crystal_ctx* c, Slot& s) {
    // caller holds c->mu
    uint64_t bytes = 0;
    const uint32_t max_jobs = (c->cfg.flags & CRYSTAL_FLAG_NO_BATCH) ? 1 : c->max_jobs;
    while (!c->outstanding.empty() && s.tasks.size() < max_jobs) {
        crystal_task* t = c->outstanding.front();
        if (!s.tasks.empty() && bytes + t->in_size > c->max_bytes) break;
        c->outstanding.pop_front();
        c->n_outstanding.fetch_sub(1);
        bytes += t->in_size;
        t->state = T_RUNNING;
        s.tasks.push_back(t);
        c->n_running_jobs++;
    }
    return !s.tasks.empty();
}

// Cancel every outstanding job (shutdown): status ESHUTDOWN, callbacks run.
void cancel_outstanding(crystal_ctx* c) {
    std::vector<crystal_task*> cancel;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        cancel = c->outstanding.drain();
        c->n_outstanding.store(0);
        for (crystal_task* t : cancel) t->state = T_RUNNING;  // callbacks may release it
    }
    for (crystal_task* t : cancel) {
        free_job_scratch(c, t);
        t->status = CRYSTAL_ESHUTDOWN;
        t->t_done = now_ns();
        if (t->cb) {
            tl_callback_ctx = c;
            t->cb(t, t->status, t->user);
            tl_callback_ctx = nullptr;
        }
    }
    std::vector<crystal_task*> released;
    {
        std::lock_guard<std::mutex> g(c->mu);
        for (crystal_task* t : cancel) {
            if (t->release_in_callback) released.push_back(t);
            else t->state = T_DONE;
        }
    }
    c->cv_done.notify_all();
    destroy_released(c, released);
}

// The master thread (Section 4.2).  The running list and the slots' busy
// flags belong to this thread alone, so completion polling runs without the
// context lock; the lock is taken only to move jobs off the outstanding
// queue and to read the shutdown flag, so threads that create, submit and
// release jobs are not held up by the polling.
void master_loop(crystal_ctx* c) {
    cudaSetDevice(c->device);
    const bool sequential = c->cfg.flags & CRYSTAL_FLAG_NO_OVERLAP;
    for (;;) {
        bool progressed = false;
        // completion: every running slot whose event has fired.  A stream
        // completes its slots in dispatch order, so once a slot is not done
        // the later slots of its stream are not queried this pass (each query
        // takes the driver's context lock).
        uint64_t blocked = 0;  // streams with a slot still running, as bits (at most 64 streams)
        for (size_t i = 0; i < c->running.size();) {
            Slot& s = c->slots[c->running[i]];
            const uint64_t bit = 1ull << s.stream_index;
            if (blocked & bit) {
                ++i;
                continue;
            }
            const cudaError_t e = cudaEventQuery(s.done);
            if (e == cudaErrorNotReady) {
                blocked |= bit;
                ++i;
                continue;
            }
            c->running.erase(c->running.begin() + i);
            const uint64_t f0 = now_ns();
            if (e != cudaSuccess) cudaGetLastError();
            finish_slot(c, s, e == cudaSuccess ? CRYSTAL_OK : CRYSTAL_EDEVICE);
            c->complete_ns.fetch_add(now_ns() - f0, std::memory_order_relaxed);
            progressed = true;
        }
        bool stop;
        {
            std::lock_guard<std::mutex> lk(c->mu);
            stop = c->stop;
        }
        // cancellation on shutdown
        if (stop && c->n_outstanding.load() > 0) {
            cancel_outstanding(c);
            progressed = true;
        }
        // dispatch: from the outstanding queue (priority, then FIFO) into free slots
        while (c->n_outstanding.load() > 0) {
            const uint32_t ns = (uint32_t)c->slots.size();
            uint32_t pick = ns;
            for (uint32_t k = 0; k < ns; ++k) {
                const uint32_t cand = (c->next_slot + k) % ns;
                if (!c->slots[cand].busy) {
                    pick = cand;
                    break;
                }
            }
            if (pick == ns) break;
            Slot& s = c->slots[pick];
            {
                std::lock_guard<std::mutex> lk(c->mu);
                if (!take_batch(c, s)) break;
                s.busy = true;
                s.seq = ++c->seq;
            }
            c->next_slot = (pick + 1) % ns;
            const uint64_t t = now_ns();
            for (crystal_task* j : s.tasks) j->t_dispatch = t;
            int r = issue(c, s);
            c->issue_ns.fetch_add(now_ns() - t, std::memory_order_relaxed);
            c->batches.fetch_add(1);
            if (r != CRYSTAL_OK) {
                cudaGetLastError();
                cudaStreamSynchronize(s.stream);
                finish_slot(c, s, r);
            } else if (sequential) {
                cudaEventSynchronize(s.done);
                finish_slot(c, s, CRYSTAL_OK);
            } else {
                c->running.push_back(pick);
            }
            progressed = true;
        }
        if (progressed) continue;
        if (c->running.empty()) {
            if (stop && c->n_outstanding.load() == 0) break;
            // idle: poll for new jobs for a short while before sleeping, so a
            // job submitted soon after is dispatched without a thread wake-up
            const uint64_t t0 = now_ns();
            while (c->n_outstanding.load(std::memory_order_relaxed) == 0 && now_ns() - t0 < kIdleSpinNs)
                std::this_thread::yield();
            std::unique_lock<std::mutex> lk(c->mu);
            if (c->outstanding.empty() && !c->stop) c->cv_master.wait(lk);
        } else {
            // poll the running slots (Section 4.1: completion is found by polling)
            std::this_thread::yield();
        }
    }
}

void destroy_ctx(crystal_ctx* c) {
    for (Slot& s : c->slots) {
        for (auto& per_class : s.graph)
            for (auto& g : per_class)
                if (g) cudaGraphExecDestroy(g);
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream && s.own_stream) cudaStreamDestroy(s.stream);
        if (s.h_desc) cudaFreeHost(s.h_desc);
    }
    c->slots.clear();
    for (crystal_task* t : c->tasks) {
        if (!c->pooled) free_task_buffers(t);
        delete t;
    }
    c->tasks.clear();
    if (c->own_d_base && c->d_base) cudaFree(c->d_base);
    if (c->h_base) cudaFreeHost(c->h_base);
    crystal_arena_destroy(c->d_arena);
    crystal_arena_destroy(c->h_arena);
    delete c;
}

}  // namespace

extern "C" {

void crystal_config_default(crystal_config* cfg) {
    if (!cfg) return;
    memset(cfg, 0, sizeof *cfg);
    cfg->max_in_bytes = 64ull << 20;
    cfg->max_out_bytes = 16ull << 20;
    cfg->device_pool_bytes = 4ull << 30;
    cfg->host_pool_bytes = 1ull << 30;
    cfg->n_streams = 4;
    cfg->device = 0;
    cfg->flags = 0;
    cfg->max_batch_jobs = 64;
    cfg->max_batch_bytes = 32ull << 20;
}

int crystal_init(const crystal_config* user_cfg, crystal_ctx** out) {
    if (!user_cfg || !out) return CRYSTAL_EINVAL;
    *out = nullptr;
    crystal_config cfg;
    crystal_config_default(&cfg);
    const crystal_config& u = *user_cfg;
    if (u.max_in_bytes) cfg.max_in_bytes = u.max_in_bytes;
    if (u.max_out_bytes) cfg.max_out_bytes = u.max_out_bytes;
    if (u.device_pool_bytes) cfg.device_pool_bytes = u.device_pool_bytes;
    if (u.host_pool_bytes) cfg.host_pool_bytes = u.host_pool_bytes;
    cfg.device_arena = u.device_arena;
    if (u.n_streams) cfg.n_streams = u.n_streams;
    cfg.device = u.device;
    cfg.flags = u.flags;
    if (u.max_batch_jobs) cfg.max_batch_jobs = u.max_batch_jobs;
    if (u.max_batch_bytes) cfg.max_batch_bytes = u.max_batch_bytes;
    if (cfg.n_streams < 1 || cfg.n_streams > 64 || cfg.max_batch_jobs > 65536) return CRYSTAL_EINVAL;
    if (cfg.flags & ~(uint32_t)(CRYSTAL_FLAG_NO_POOL | CRYSTAL_FLAG_NO_OVERLAP | CRYSTAL_FLAG_NO_BATCH |
                                CRYSTAL_FLAG_GRAPHS))
        return CRYSTAL_EINVAL;
    if (cfg.device_arena && (reinterpret_cast<uint64_t>(cfg.device_arena) & 255)) return CRYSTAL_EINVAL;
    if (cudaSetDevice(cfg.device) != cudaSuccess) {
        cudaGetLastError();
        return CRYSTAL_EDEVICE;
    }
    crystal_ctx* c = new (std::nothrow) crystal_ctx;
    if (!c) return CRYSTAL_ENOMEM;
    c->cfg = cfg;
    c->device = cfg.device;
    c->pooled = !(cfg.flags & CRYSTAL_FLAG_NO_POOL);
    {
        const crystal_geometry defaults{};
        for (LaunchGeom& g : c->geom) {
            if (make_geometry(&defaults, &g) != CRYSTAL_OK) {
                delete c;
                return CRYSTAL_EDEVICE;
            }
        }
    }
    if (cfg.flags & CRYSTAL_FLAG_NO_OVERLAP) c->cfg.n_streams = 1;
    c->max_jobs = (cfg.flags & (CRYSTAL_FLAG_NO_BATCH | CRYSTAL_FLAG_NO_OVERLAP)) ? 1 : cfg.max_batch_jobs;
    c->max_bytes = cfg.max_batch_bytes;
    const uint32_t depth = (cfg.flags & CRYSTAL_FLAG_NO_OVERLAP) ? 1 : 2;  // slots per stream
    const uint32_t n_slots = (uint32_t)c->cfg.n_streams * depth;
    // per slot: the batch descriptor (header + max_jobs units)
    const uint64_t desc_bytes = align_up(crystal_batch_bytes(c->max_jobs), 256);
    c->region_bytes = desc_bytes;

    // device arena: job buffers (pooled mode), scratch and batch descriptors
    uint64_t d_bytes = cfg.device_pool_bytes;
    if (!c->pooled) d_bytes = desc_bytes * n_slots;  // descriptors only
    if (cfg.device_arena && c->pooled) {
        c->d_base = (uint8_t*)cfg.device_arena;
    } else {
        void* p = nullptr;
        if (cudaMalloc(&p, d_bytes) != cudaSuccess) {
            cudaGetLastError();
            destroy_ctx(c);
            return CRYSTAL_ENOMEM;
        }
        c->d_base = (uint8_t*)p;
        c->own_d_base = true;
    }
    if (crystal_arena_create(d_bytes, 256, &c->d_arena) != CRYSTAL_OK) {
        destroy_ctx(c);
        return CRYSTAL_ENOMEM;
    }
    if (c->pooled) {
        void* h = nullptr;
        if (cudaHostAlloc(&h, cfg.host_pool_bytes, cudaHostAllocMapped) != cudaSuccess) {
            cudaGetLastError();
            destroy_ctx(c);
            return CRYSTAL_ENOMEM;
        }
        c->h_base = (uint8_t*)h;
        if (crystal_arena_create(cfg.host_pool_bytes, 256, &c->h_arena) != CRYSTAL_OK) {
            destroy_ctx(c);
            return CRYSTAL_ENOMEM;
        }
        // the pool mapped into the device's address space: kernels write direct
        // digests into it
        int uva = 0;
        void* hd = nullptr;
        if (cudaDeviceGetAttribute(&uva, cudaDevAttrUnifiedAddressing, cfg.device) == cudaSuccess && uva &&
            cudaHostGetDevicePointer(&hd, h, 0) == cudaSuccess && hd) {
            c->h_mapped = true;
            c->h_dev_delta = (int64_t)((uint64_t)hd - (uint64_t)h);
        }
        cudaGetLastError();
    }
    c->slots.resize(n_slots);
    for (uint32_t i = 0; i < n_slots; ++i) {
        Slot& s = c->slots[i];
        if (i < (uint32_t)c->cfg.n_streams) {
            if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                destroy_ctx(c);
                return CRYSTAL_EDEVICE;
            }
            s.own_stream = true;
        } else {
            s.stream = c->slots[i % c->cfg.n_streams].stream;
        }
        s.stream_index = i % (uint32_t)c->cfg.n_streams;
        if (cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            destroy_ctx(c);
            return CRYSTAL_EDEVICE;
        }
        void* h = nullptr;
        if (cudaHostAlloc(&h, desc_bytes, cudaHostAllocMapped) != cudaSuccess) {
            cudaGetLastError();
            destroy_ctx(c);
            return CRYSTAL_ENOMEM;
        }
        memset(h, 0, desc_bytes);
        s.h_desc = (crystal_batch*)h;
        void* hd = nullptr;
        if (c->h_mapped && cudaHostGetDevicePointer(&hd, h, 0) == cudaSuccess && hd) s.h_desc_dev = (uint8_t*)hd;
        cudaGetLastError();
        if (crystal_arena_alloc(c->d_arena, desc_bytes, &s.d_desc_off) != CRYSTAL_OK) {
            destroy_ctx(c);
            return CRYSTAL_ENOMEM;
        }
        s.d_desc = (crystal_batch*)(c->d_base + s.d_desc_off);
    }
    try {
        c->master = std::thread(master_loop, c);
    } catch (...) {
        destroy_ctx(c);
        return CRYSTAL_ENOMEM;
    }
    *out = c;
    return CRYSTAL_OK;
}

int crystal_shutdown(crystal_ctx* c) {
    if (!c) return CRYSTAL_EINVAL;
    if (tl_callback_ctx == c) return CRYSTAL_EINVAL;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->accepting = false;
        c->accepting_fast.store(false);
        c->stop = true;
    }
    c->cv_master.notify_all();
    if (c->master.joinable()) c->master.join();
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    destroy_ctx(c);
    return CRYSTAL_OK;
}

int crystal_task_create(crystal_ctx* c, uint64_t in_size, uint64_t out_size, crystal_task** out) {
    return crystal_task_create_ex(c, in_size, out_size, 0, 0, out);
}

namespace {
int create_job(crystal_ctx* c, uint64_t in_size, uint64_t out_size, uint64_t scratch_bytes, uint32_t flags,
               crystal_task** out, uint8_t* borrowed_h_in = nullptr, uint8_t* borrowed_d_in = nullptr);

// create_job with the creation counters of crystal_stats
int counted_create(crystal_ctx* c, uint64_t in_size, uint64_t out_size, uint64_t scratch_bytes, uint32_t flags,
                   crystal_task** out, uint8_t* borrowed_h_in = nullptr, uint8_t* borrowed_d_in = nullptr) {
    const uint64_t t0 = now_ns();
    const int st = create_job(c, in_size, out_size, scratch_bytes, flags, out, borrowed_h_in, borrowed_d_in);
    c->create_ns.fetch_add(now_ns() - t0, std::memory_order_relaxed);
    c->create_calls.fetch_add(1, std::memory_order_relaxed);
    if (st == CRYSTAL_EAGAIN) c->create_eagain.fetch_add(1, std::memory_order_relaxed);
    return st;
}
}  // namespace

int crystal_task_create_ex(crystal_ctx* c, uint64_t in_size, uint64_t out_size, uint64_t scratch_bytes,
                           uint32_t flags, crystal_task** out) {
    if (!c) return CRYSTAL_EINVAL;
    return counted_create(c, in_size, out_size, scratch_bytes, flags, out);
}

}  // extern "C"

namespace {

int create_job(crystal_ctx* c, uint64_t in_size, uint64_t out_size, uint64_t scratch_bytes, uint32_t flags,
               crystal_task** out, uint8_t* borrowed_h_in, uint8_t* borrowed_d_in) {
    if (!out) return CRYSTAL_EINVAL;
    if ((borrowed_d_in != nullptr) != (borrowed_h_in != nullptr) || (borrowed_d_in && flags)) return CRYSTAL_EINVAL;
    if (flags & ~(uint32_t)CRYSTAL_TASK_EXTERNAL_INPUT) return CRYSTAL_EINVAL;
    *out = nullptr;
    if (in_size > c->cfg.max_in_bytes || out_size > c->cfg.max_out_bytes) return CRYSTAL_EINVAL;
    if (!c->accepting_fast.load()) return CRYSTAL_ESHUTDOWN;
    if (!c->pooled) cudaSetDevice(c->device);
    crystal_task* t = new (std::nothrow) crystal_task;
    if (!t) return CRYSTAL_ENOMEM;
    t->ctx = c;
    t->in_cap = t->in_size = in_size;
    t->out_cap = t->out_size = out_size;
    t->external_input = flags & CRYSTAL_TASK_EXTERNAL_INPUT;
    if (borrowed_d_in) {
        t->borrowed_input = true;
        t->h_in = borrowed_h_in;
        t->d_in = borrowed_d_in;
    }
    // inputs from the bottom of the arenas, outputs and scratch from the top
    int st = CRYSTAL_OK;
    if (t->borrowed_input) {
        // input buffers given; output and scratch below
    } else if (!t->external_input && c->pooled) {
        // the pinned input at the same arena offset as the device input when
        // that range is free: jobs with adjacent device inputs then have
        // adjacent pinned inputs too, at one host-to-device distance, and a
        // batch copies them in one transfer whatever order they were made in
        st = alloc_device(c, in_size, &t->d_in, &t->d_in_off, CRYSTAL_ARENA_LOWEST);
        if (st == CRYSTAL_OK) {
            if (crystal_arena_alloc_exact(c->h_arena, t->d_in_off, in_size) == CRYSTAL_OK) {
                t->h_in_off = t->d_in_off;
                t->h_in = c->h_base + t->h_in_off;
            } else {
                st = alloc_host(c, in_size, &t->h_in, &t->h_in_off, CRYSTAL_ARENA_LOWEST);
            }
        }
    } else if (!t->external_input) {
        st = alloc_host(c, in_size, &t->h_in, &t->h_in_off, CRYSTAL_ARENA_LOWEST);
    }
    if (st == CRYSTAL_OK) st = alloc_host(c, out_size, &t->h_out, &t->h_out_off, CRYSTAL_ARENA_HIGHEST);
    if (st == CRYSTAL_OK && t->external_input && c->pooled) {
        // an external input is copied on its own (never merged with its
        // neighbours), so the job's device input, output and scratch are one
        // block: one allocation and one free instead of three
        const uint64_t in_b = align_up(in_size ? in_size : 1, 256), out_b = align_up(out_size ? out_size : 1, 256);
        st = alloc_device(c, in_b + out_b + scratch_bytes, &t->d_in, &t->d_in_off, CRYSTAL_ARENA_HIGHEST);
        if (st == CRYSTAL_OK) {
            t->one_block = true;
            t->d_out = t->d_in + in_b;
            if (scratch_bytes) {
                t->d_reserved = t->d_out + out_b;
                t->reserved_bytes = scratch_bytes;
            }
        }
    } else {
        if (st == CRYSTAL_OK && !t->d_in) st = alloc_device(c, in_size, &t->d_in, &t->d_in_off, CRYSTAL_ARENA_LOWEST);
        if (st == CRYSTAL_OK) st = alloc_device(c, out_size, &t->d_out, &t->d_out_off, CRYSTAL_ARENA_HIGHEST);
        if (st == CRYSTAL_OK && scratch_bytes) {
            st = alloc_device(c, scratch_bytes, &t->d_reserved, &t->d_reserved_off);
            if (st == CRYSTAL_OK) t->reserved_bytes = scratch_bytes;
        }
    }
    if (st != CRYSTAL_OK) {
        free_task_buffers(t);
        delete t;
        return st;
    }
    std::lock_guard<std::mutex> lk(c->tasks_mu);
    c->tasks.insert(t);
    *out = t;
    return CRYSTAL_OK;
}

}  // namespace

extern "C" {

void* crystal_task_host_in(crystal_task* t) { return t ? t->h_in : nullptr; }
void* crystal_task_host_out(crystal_task* t) { return t ? t->h_out : nullptr; }
uint64_t crystal_task_device_in(crystal_task* t) { return t ? (uint64_t)t->d_in : 0; }
uint64_t crystal_task_device_out(crystal_task* t) { return t ? (uint64_t)t->d_out : 0; }

int crystal_task_resize(crystal_task* t, uint64_t in_size, uint64_t out_size) {
    if (!t) return CRYSTAL_EINVAL;
    std::lock_guard<std::mutex> lk(t->ctx->mu);
    if (t->state == T_OUTSTANDING || t->state == T_RUNNING) return CRYSTAL_EINVAL;
    if (in_size > t->in_cap || out_size > t->out_cap) return CRYSTAL_EINVAL;
    t->in_size = in_size;
    t->out_size = out_size;
    return CRYSTAL_OK;
}

int crystal_task_submit(crystal_task* t, int kind, const crystal_hash_params* params, crystal_callback cb,
                        void* user) {
    if (!t) return CRYSTAL_EINVAL;
    if (t->external_input && !t->h_in_ext && t->in_size) return CRYSTAL_EINVAL;
    crystal_ctx* c = t->ctx;
    crystal_hash_params p;
    int st = resolve_params(kind, params, t->in_size, t->out_size, &p);
    if (st != CRYSTAL_OK) return st;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        if (!c->accepting) return CRYSTAL_ESHUTDOWN;
        if (t->state == T_OUTSTANDING || t->state == T_RUNNING) return CRYSTAL_EINVAL;
    }
    const uint64_t scratch = crystal_scratch_bytes(kind, t->in_size, t->out_size, &p);
    uint8_t* d_scratch = nullptr;
    uint64_t d_scratch_off = 0;
    if (scratch && scratch <= t->reserved_bytes) {
        d_scratch = t->d_reserved;
        d_scratch_off = t->d_reserved_off;
    } else if (scratch) {
        if (!c->pooled) cudaSetDevice(c->device);
        st = alloc_device(c, scratch, &d_scratch, &d_scratch_off);
        if (st != CRYSTAL_OK) return st == CRYSTAL_ENOMEM ? CRYSTAL_ENOMEM : CRYSTAL_EAGAIN;
    }
    {
        std::lock_guard<std::mutex> lk(c->mu);
        if (!c->accepting) {
            if (d_scratch != t->d_reserved) free_device(c, d_scratch, d_scratch_off);
            return CRYSTAL_ESHUTDOWN;
        }
        t->kind = kind;
        t->params = p;
        t->cb = cb;
        t->user = user;
        t->d_scratch = d_scratch;
        t->d_scratch_off = d_scratch_off;
        t->scratch_bytes = scratch;
        t->status = CRYSTAL_PENDING;
        t->state = T_OUTSTANDING;
        t->submitted_once = true;
        t->release_in_callback = false;
        t->t_submit = now_ns();
        t->t_dispatch = t->t_done = 0;
        c->outstanding.push_back(t, t->priority);
        c->n_outstanding.fetch_add(1);
    }
    c->cv_master.notify_one();
    return CRYSTAL_OK;
}

int crystal_task_submit_many(crystal_task* const* tasks, uint32_t n, int kind, const crystal_hash_params* params,
                             crystal_callback cb, void* user) {
    if (!tasks && n) return CRYSTAL_EINVAL;
    if (n == 0) return CRYSTAL_OK;
    crystal_ctx* c = tasks[0] ? tasks[0]->ctx : nullptr;
    if (!c) return CRYSTAL_EINVAL;
    std::vector<crystal_hash_params> ps(n);
    std::vector<uint64_t> scratch(n, 0);
    for (uint32_t i = 0; i < n; ++i) {
        crystal_task* t = tasks[i];
        if (!t || t->ctx != c) return CRYSTAL_EINVAL;
        if (t->external_input && !t->h_in_ext && t->in_size) return CRYSTAL_EINVAL;
        int st = resolve_params(kind, params, t->in_size, t->out_size, &ps[i]);
        if (st != CRYSTAL_OK) return st;
        scratch[i] = crystal_scratch_bytes(kind, t->in_size, t->out_size, &ps[i]);
    }
    {
        std::lock_guard<std::mutex> lk(c->mu);
        if (!c->accepting) return CRYSTAL_ESHUTDOWN;
        for (uint32_t i = 0; i < n; ++i) {
            if (tasks[i]->state == T_OUTSTANDING || tasks[i]->state == T_RUNNING) return CRYSTAL_EINVAL;
            for (uint32_t j = 0; j < i; ++j)
                if (tasks[j] == tasks[i]) return CRYSTAL_EINVAL;
        }
    }
    if (!c->pooled) cudaSetDevice(c->device);
    std::vector<uint8_t*> dp(n, nullptr);
    std::vector<uint64_t> doff(n, 0);
    auto undo = [&](uint32_t upto) {
        for (uint32_t j = 0; j < upto; ++j)
            if (dp[j] && dp[j] != tasks[j]->d_reserved) free_device(c, dp[j], doff[j]);
    };
    for (uint32_t i = 0; i < n; ++i) {
        if (!scratch[i]) continue;
        if (scratch[i] <= tasks[i]->reserved_bytes) {
            dp[i] = tasks[i]->d_reserved;
            doff[i] = tasks[i]->d_reserved_off;
            continue;
        }
        int st = alloc_device(c, scratch[i], &dp[i], &doff[i]);
        if (st != CRYSTAL_OK) {
            undo(i);
            return st == CRYSTAL_ENOMEM ? CRYSTAL_ENOMEM : CRYSTAL_EAGAIN;
        }
    }
    {
        std::lock_guard<std::mutex> lk(c->mu);
        if (!c->accepting) {
            undo(n);
            return CRYSTAL_ESHUTDOWN;
        }
        const uint64_t now = now_ns();
        for (uint32_t i = 0; i < n; ++i) {
            crystal_task* t = tasks[i];
            t->kind = kind;
            t->params = ps[i];
            t->cb = cb;
            t->user = user;
            t->d_scratch = dp[i];
            t->d_scratch_off = doff[i];
            t->scratch_bytes = scratch[i];
            t->status = CRYSTAL_PENDING;
            t->state = T_OUTSTANDING;
            t->submitted_once = true;
            t->release_in_callback = false;
            t->t_submit = now;
            t->t_dispatch = t->t_done = 0;
            c->outstanding.push_back(t, t->priority);
        }
        c->n_outstanding.fetch_add(n);
    }
    c->cv_master.notify_one();
    return CRYSTAL_OK;
}

int crystal_task_bind_input(crystal_task* t, const void* host, uint64_t size) {
    if (!t) return CRYSTAL_EINVAL;
    std::lock_guard<std::mutex> lk(t->ctx->mu);
    if (t->state == T_OUTSTANDING || t->state == T_RUNNING) return CRYSTAL_EINVAL;
    if (!host) {
        if (t->external_input) return CRYSTAL_EINVAL;  // it has no buffer of its own to go back to
        t->h_in_ext = nullptr;
        return CRYSTAL_OK;
    }
    if (size > t->in_cap) return CRYSTAL_EINVAL;
    t->h_in_ext = static_cast<const uint8_t*>(host);
    t->in_size = size;
    return CRYSTAL_OK;
}

int crystal_host_register(void* host, uint64_t bytes) {
    if (!host || !bytes) return CRYSTAL_EINVAL;
    if (cudaHostRegister(host, bytes, cudaHostRegisterMapped | cudaHostRegisterPortable) != cudaSuccess) {
        cudaGetLastError();
        return CRYSTAL_EDEVICE;
    }
    return CRYSTAL_OK;
}

int crystal_host_unregister(void* host) {
    if (!host) return CRYSTAL_EINVAL;
    if (cudaHostUnregister(host) != cudaSuccess) {
        cudaGetLastError();
        return CRYSTAL_EDEVICE;
    }
    return CRYSTAL_OK;
}

int crystal_task_set_priority(crystal_task* t, int priority) {
    if (!t) return CRYSTAL_EINVAL;
    std::lock_guard<std::mutex> lk(t->ctx->mu);
    if (t->state == T_OUTSTANDING || t->state == T_RUNNING) return CRYSTAL_EINVAL;
    t->priority = priority;
    return CRYSTAL_OK;
}

int crystal_task_poll(crystal_task* t) {
    if (!t) return CRYSTAL_EINVAL;
    std::lock_guard<std::mutex> lk(t->ctx->mu);
    if (!t->submitted_once) return CRYSTAL_EINVAL;
    if (t->state != T_DONE) return CRYSTAL_PENDING;
    return t->status;
}

int crystal_task_wait(crystal_task* t, int64_t timeout_ns) {
    if (!t) return CRYSTAL_EINVAL;
    crystal_ctx* c = t->ctx;
    if (tl_callback_ctx == c) return CRYSTAL_EINVAL;
    {
        const uint64_t spin = timeout_ns >= 0 && (uint64_t)timeout_ns < kWaitSpinNs ? (uint64_t)timeout_ns : kWaitSpinNs;
        const uint64_t t0 = now_ns();
        while (t->state.load() != T_DONE && now_ns() - t0 < spin) std::this_thread::yield();
    }
    std::unique_lock<std::mutex> lk(c->mu);
    if (!t->submitted_once) return CRYSTAL_EINVAL;
    auto done = [t] { return t->state == T_DONE; };
    if (timeout_ns < 0) {
        c->cv_done.wait(lk, done);
    } else if (!c->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), done)) {
        return CRYSTAL_ETIMEDOUT;
    }
    return t->status;
}

int crystal_task_wait_many(crystal_task* const* tasks, uint32_t n, int64_t timeout_ns) {
    if (n == 0) return CRYSTAL_OK;
    if (!tasks || !tasks[0]) return CRYSTAL_EINVAL;
    crystal_ctx* c = tasks[0]->ctx;
    if (tl_callback_ctx == c) return CRYSTAL_EINVAL;
    for (uint32_t i = 0; i < n; ++i) {
        if (!tasks[i] || tasks[i]->ctx != c) return CRYSTAL_EINVAL;
    }
    // jobs finish roughly in array order: advance past the finished prefix
    uint32_t first = 0;
    auto all_done = [&] {
        while (first < n && tasks[first]->state.load() == T_DONE) ++first;
        return first == n;
    };
    {
        const uint64_t spin = timeout_ns >= 0 && (uint64_t)timeout_ns < kWaitSpinNs ? (uint64_t)timeout_ns : kWaitSpinNs;
        const uint64_t t0 = now_ns();
        while (!all_done() && now_ns() - t0 < spin) std::this_thread::yield();
    }
    std::unique_lock<std::mutex> lk(c->mu);
    for (uint32_t i = 0; i < n; ++i) {
        if (!tasks[i]->submitted_once) return CRYSTAL_EINVAL;
    }
    if (timeout_ns < 0) {
        c->cv_done.wait(lk, all_done);
    } else if (!c->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), all_done)) {
        return CRYSTAL_ETIMEDOUT;
    }
    for (uint32_t i = 0; i < n; ++i) {
        if (tasks[i]->status != CRYSTAL_OK) return tasks[i]->status;
    }
    return CRYSTAL_OK;
}

int crystal_task_release(crystal_task* t) {
    if (!t) return CRYSTAL_EINVAL;
    crystal_ctx* c = t->ctx;
    std::unique_lock<std::mutex> lk(c->mu);
    if (t->state == T_RUNNING && tl_callback_ctx == c) {
        // from the job's own callback: its buffers go back to the pools now
        // (the caller may count on the room, e.g. to admit the next job); the
        // handle itself is freed by the master after the callback returns
        t->release_in_callback = true;
        lk.unlock();
        free_task_buffers(t);
        return CRYSTAL_OK;
    }
    if (t->state == T_OUTSTANDING || t->state == T_RUNNING) return CRYSTAL_EINVAL;
    lk.unlock();
    {
        std::lock_guard<std::mutex> g(c->tasks_mu);
        c->tasks.erase(t);
    }
    if (!c->pooled) cudaSetDevice(c->device);
    free_task_buffers(t);
    delete t;
    return CRYSTAL_OK;
}

int crystal_task_timing(crystal_task* t, uint64_t* submit_ns, uint64_t* dispatch_ns, uint64_t* done_ns) {
    if (!t) return CRYSTAL_EINVAL;
    std::lock_guard<std::mutex> lk(t->ctx->mu);
    if (submit_ns) *submit_ns = t->t_submit;
    if (dispatch_ns) *dispatch_ns = t->t_dispatch;
    if (done_ns) *done_ns = t->t_done;
    return CRYSTAL_OK;
}

int crystal_task_timing_many(crystal_task* const* tasks, uint32_t n, uint64_t* out) {
    if (n == 0) return CRYSTAL_OK;
    if (!tasks || !out) return CRYSTAL_EINVAL;
    for (uint32_t i = 0; i < n; ++i) {
        crystal_task* t = tasks[i];
        if (!t) return CRYSTAL_EINVAL;
        std::lock_guard<std::mutex> lk(t->ctx->mu);
        out[3 * (uint64_t)i + 0] = t->t_submit;
        out[3 * (uint64_t)i + 1] = t->t_dispatch;
        out[3 * (uint64_t)i + 2] = t->t_done;
    }
    return CRYSTAL_OK;
}

int crystal_set_geometry(crystal_ctx* c, int size_class, const crystal_geometry* g) {
    if (!c || size_class < -1 || size_class >= CRYSTAL_SIZE_CLASSES) return CRYSTAL_EINVAL;
    const crystal_geometry defaults{};
    // resolved against the context's device; the caller's current device is kept
    int prev = 0;
    const bool restore = cudaGetDevice(&prev) == cudaSuccess && prev != c->device;
    if (restore) cudaSetDevice(c->device);
    LaunchGeom lg;
    const int st = make_geometry(g ? g : &defaults, &lg);
    if (restore) cudaSetDevice(prev);
    if (st != CRYSTAL_OK) return st;
    // idle: the master issues nothing (issuing needs an outstanding job), so
    // no graph is in use or being captured while they are dropped here
    std::lock_guard<std::mutex> lk(c->mu);
    if (!c->outstanding.empty() || c->n_running_jobs) return CRYSTAL_EINVAL;
    for (int k = 0; k < CRYSTAL_SIZE_CLASSES; ++k) {
        if (size_class != -1 && k != size_class) continue;
        c->geom[k] = lg;
        for (Slot& s : c->slots)
            for (auto& ge : s.graph[k])
                if (ge) {
                    cudaGraphExecDestroy(ge);
                    ge = nullptr;
                }
    }
    return CRYSTAL_OK;
}

int crystal_get_geometry(crystal_ctx* c, int size_class, crystal_geometry* out) {
    if (!c || !out || size_class < 0 || size_class >= CRYSTAL_SIZE_CLASSES) return CRYSTAL_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    describe_geometry(c->geom[size_class], out);
    return CRYSTAL_OK;
}

int crystal_get_config(crystal_ctx* c, crystal_config* out) {
    if (!c || !out) return CRYSTAL_EINVAL;
    *out = c->cfg;
    out->max_batch_jobs = c->max_jobs;
    return CRYSTAL_OK;
}

int crystal_get_stats(crystal_ctx* c, crystal_stats* out) {
    if (!c || !out) return CRYSTAL_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    out->jobs_completed = c->jobs_completed.load();
    out->batches_launched = c->batches.load();
    out->device_pool_bytes = c->pooled ? c->cfg.device_pool_bytes : 0;
    out->device_pool_used = c->pooled ? crystal_arena_used(c->d_arena) : 0;
    out->host_pool_bytes = c->pooled ? c->cfg.host_pool_bytes : 0;
    out->host_pool_used = c->pooled ? crystal_arena_used(c->h_arena) : 0;
    out->jobs_outstanding = c->outstanding.size();
    out->jobs_running = c->n_running_jobs;
    out->copies_dma = c->copies_dma.load();
    out->master_issue_ns = c->issue_ns.load();
    out->master_complete_ns = c->complete_ns.load();
    out->create_ns = c->create_ns.load();
    out->create_calls = c->create_calls.load();
    out->create_eagain = c->create_eagain.load();
    out->graph_captures = c->graph_captures.load();
    return CRYSTAL_OK;
}

int crystal_prepare_graphs(crystal_ctx* c) {
    if (!c) return CRYSTAL_EINVAL;
    if (!(c->cfg.flags & CRYSTAL_FLAG_GRAPHS)) return CRYSTAL_OK;
    int prev = 0;
    const bool restore = cudaGetDevice(&prev) == cudaSuccess && prev != c->device;
    if (restore) cudaSetDevice(c->device);
    int r = CRYSTAL_OK;
    {
        // idle: the master issues nothing while no job is outstanding, so the
        // slots' streams and graphs are this thread's for the duration
        std::lock_guard<std::mutex> lk(c->mu);
        if (!c->outstanding.empty() || c->n_running_jobs || c->stop) {
            r = CRYSTAL_EINVAL;
        } else {
            for (Slot& s : c->slots)
                for (int cls = 0; cls < CRYSTAL_SIZE_CLASSES && r == CRYSTAL_OK; ++cls)
                    for (int variant = 1; variant < 4 && r == CRYSTAL_OK; ++variant)
                        if (!s.graph[cls][variant]) r = capture_graph(c, s, cls, variant);
        }
    }
    if (restore) cudaSetDevice(prev);
    return r;
}

}  // extern "C"

namespace crystal {

int reserve_pool_pair(crystal_ctx* c, uint64_t bytes, PoolPair* out) {
    if (!c || !out || !bytes || !c->pooled) return CRYSTAL_EINVAL;
    PoolPair p{};
    p.bytes = bytes;
    int st = alloc_host(c, bytes, &p.host, &p.host_off, CRYSTAL_ARENA_LOWEST);
    if (st != CRYSTAL_OK) return st;
    st = alloc_device(c, bytes, &p.dev, &p.dev_off, CRYSTAL_ARENA_LOWEST);
    if (st != CRYSTAL_OK) {
        free_host(c, p.host, p.host_off);
        return st;
    }
    *out = p;
    return CRYSTAL_OK;
}

void release_pool_pair(crystal_ctx* c, const PoolPair& p) {
    if (!c || !p.host) return;
    free_device(c, p.dev, p.dev_off);
    free_host(c, p.host, p.host_off);
}

int task_create_borrowed(crystal_ctx* c, uint8_t* h_in, uint8_t* d_in, uint64_t in_size, uint64_t out_size,
                         uint64_t scratch_bytes, crystal_task** out) {
    if (!c || !h_in || !d_in) return CRYSTAL_EINVAL;
    return counted_create(c, in_size, out_size, scratch_bytes, 0, out, h_in, d_in);
}

}  // namespace crystal
