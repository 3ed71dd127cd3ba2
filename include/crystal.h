/*
 * crystal.h -- C ABI of the B300 CrystalGPU hashing library (libcrystal.so).
 *
 * The library runs a stream of host data units through MD5 direct hashing
 * and MD5 sliding-window hashing on one GPU, behind the job abstraction of
 * the CrystalGPU paper (Gharaibeh, Al-Kiswany, Ripeanu):
 *   - Section 3, Figure 2: a job carries host and device input/output
 *     buffers, their sizes, the kernel to run and a completion callback;
 *   - Section 3, Figure 3: init / finalize / job_get / job_put / job_submit /
 *     job_synch / job_query;
 *   - Section 4.2: one host master thread per GPU, idle / outstanding /
 *     running job queues, jobs interleaved over a copy-in / kernel /
 *     copy-out pipeline (Figure 4), completion found by polling because the
 *     GPU runtime has no completion interrupt (Section 4.1).
 * Every call below names the paper passage it follows.  All sizes are bytes.
 * Every function returns a status (CRYSTAL_OK or a negative error) unless it
 * says otherwise; no function throws, aborts or prints.
 *
 * Two layers:
 *   1. the job runtime (crystal_init ... crystal_shutdown), which owns a
 *      device pool, a pinned host pool, the streams and the master thread;
 *   2. the stateless batch launchers (crystal_launch_*), which run the
 *      kernels of one batch on caller-owned device memory and a caller
 *      stream.  The runtime is built on them.
 */
#ifndef CRYSTAL_H
#define CRYSTAL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
enum {
    CRYSTAL_OK = 0,
    CRYSTAL_PENDING = 1,      /* job submitted and not finished (job_query false) */
    CRYSTAL_EINVAL = -1,      /* bad argument, or a call not allowed in this state */
    CRYSTAL_EAGAIN = -2,      /* pool has no room now; retry after a release */
    CRYSTAL_ENOMEM = -3,      /* allocation failed at init / unpooled create */
    CRYSTAL_ETIMEDOUT = -4,   /* bounded wait ran out */
    CRYSTAL_EOVERFLOW = -5,   /* sliding output buffer too small for the chunk records */
    CRYSTAL_ESHUTDOWN = -6,   /* context is shutting down */
    CRYSTAL_EDEVICE = -7      /* CUDA error, or a device-side status word was set */
};

/* ---- job kinds (the kernel_func of Figure 2, chosen by id) -------------- */
enum {
    CRYSTAL_KIND_NOP = 0,          /* dummy kernel of Section 5.1: copy in, empty kernel, copy out */
    CRYSTAL_KIND_MD5_DIRECT = 1,   /* direct hashing (Section 5.2, Figure 6) */
    CRYSTAL_KIND_MD5_SLIDING = 2,  /* sliding-window hashing (Section 2.2, content-addressable storage) */
    CRYSTAL_KIND_SHA1_DIRECT = 3,  /* the same with SHA-1 (FIPS 180-4), the hash of Section 5.2's runs */
    CRYSTAL_KIND_SHA1_SLIDING = 4
};

/* ---- context flags ------------------------------------------------------ */
enum {
    /* Allocate each job's device and pinned host buffers at crystal_task_create
     * (cudaMalloc / cudaHostAlloc) and free them at release: the per-job
     * allocation the paper's buffer pool removes (Section 3, Section 5.2). */
    CRYSTAL_FLAG_NO_POOL = 1u,
    /* One stream, one job at a time, the master waits for each job to finish
     * before issuing the next: no copy/compute overlap (Section 4.1). */
    CRYSTAL_FLAG_NO_OVERLAP = 2u,
    /* One job per kernel launch (no grouping of outstanding jobs). */
    CRYSTAL_FLAG_NO_BATCH = 4u,
    /* Replay each batch's descriptor upload and kernel chain as a captured
     * CUDA graph instead of individual launches. */
    CRYSTAL_FLAG_GRAPHS = 8u
};

/* crystal_init's argument.  Zero fields take the defaults listed. */
typedef struct crystal_config {
    uint64_t max_in_bytes;      /* largest job input (init's max_input_size, Figure 3); default 64 MiB */
    uint64_t max_out_bytes;     /* largest job output (init's max_output_size); default 16 MiB */
    uint64_t device_pool_bytes; /* device arena for job buffers and scratch; default 4 GiB */
    uint64_t host_pool_bytes;   /* pinned host arena for job buffers; default 1 GiB */
    void* device_arena;         /* optional caller-owned device memory of device_pool_bytes
                                   (must stay valid until shutdown); NULL: the library
                                   allocates it with one cudaMalloc */
    int32_t n_streams;          /* streams the master interleaves jobs over; default 4 */
    int32_t device;             /* CUDA device ordinal; default 0 */
    uint32_t flags;             /* CRYSTAL_FLAG_* */
    uint32_t max_batch_jobs;    /* outstanding jobs grouped into one launch; default 64 */
    uint64_t max_batch_bytes;   /* input bytes grouped into one launch; default 32 MiB */
} crystal_config;

/* Hash parameters of one job.  A NULL params pointer means all defaults
 * (crystal_params_default).  A zero size field takes its default; mask and
 * target are always taken as given (mask = 0, target = 0 marks every window). */
typedef struct crystal_hash_params {
    uint32_t segment_bytes;       /* direct: segment size S; default 4096; >= 1 */
    uint32_t window_bytes;        /* sliding: window w; default 20; 1..55 (one MD5 block) */
    uint32_t mask;                /* sliding: boundary mask; default 0x1FFF */
    uint32_t target;              /* sliding: boundary target; default 0x1FFF */
    uint32_t chunk_segment_bytes; /* sliding: S of each chunk's direct hash; default 4096 */
    uint32_t reserved;            /* must be 0 */
} crystal_hash_params;

typedef struct crystal_ctx crystal_ctx;   /* opaque: pools, streams, master thread */
typedef struct crystal_task crystal_task; /* opaque: one job (Figure 2's job_t) */

/* Completion callback (Figure 2's callback_func).  Runs on the master thread
 * (Section 4.2) once the job's output is in host memory.  It may read the
 * output and call crystal_task_release on this job; it must not block, and
 * crystal_task_wait called from it returns CRYSTAL_EINVAL. */
typedef void (*crystal_callback)(crystal_task* task, int status, void* user);

/* Fill *cfg / *p with the defaults above. */
void crystal_config_default(crystal_config* cfg);
void crystal_params_default(crystal_hash_params* p);

/* init(max_input_size, max_output_size), Figure 3 / Section 3: creates the
 * buffer pool (one device arena, one pinned host arena), the streams and the
 * master thread.  *out receives the context.  Errors: EINVAL (bad field),
 * ENOMEM (an allocation failed; nothing is left allocated), EDEVICE. */
int crystal_init(const crystal_config* cfg, crystal_ctx** out);

/* finalize(), Figure 3: stops accepting jobs, lets in-flight jobs finish,
 * cancels outstanding ones (their status becomes ESHUTDOWN and their
 * callbacks run), frees every pool and stream.  Jobs not yet released are
 * freed too; their handles become invalid. */
int crystal_shutdown(crystal_ctx* ctx);

/* job_get(), Figure 3: takes a job from the pool with a pinned host input of
 * in_size bytes, a pinned host output of out_size bytes and device buffers of
 * the same sizes.  in_size <= max_in_bytes, out_size <= max_out_bytes.
 * Errors: EINVAL, EAGAIN (pool full now), ENOMEM (unpooled mode), ESHUTDOWN. */
int crystal_task_create(crystal_ctx* ctx, uint64_t in_size, uint64_t out_size, crystal_task** out);

/* crystal_task_create with two extensions.
 *  - scratch_bytes of device scratch are reserved for the job (see
 *    crystal_scratch_bytes): a later submit whose kind needs no more than that
 *    takes no device memory, so a job that was created can always be
 *    submitted.  This is how a serving loop admits a request against the
 *    device pool (admission by pool memory).  Returned at release.
 *  - flags CRYSTAL_TASK_EXTERNAL_INPUT: the job gets no pinned input buffer of
 *    its own (crystal_task_host_in returns NULL); its input must be bound
 *    with crystal_task_bind_input before each submit. */
#define CRYSTAL_TASK_EXTERNAL_INPUT 1u
int crystal_task_create_ex(crystal_ctx* ctx, uint64_t in_size, uint64_t out_size, uint64_t scratch_bytes,
                           uint32_t flags, crystal_task** out);

/* Bind caller memory as the job's input for the next submits (Figure 2's
 * h_input pointed at application memory): the copy-in reads size bytes from
 * host (size <= the job's input capacity), which must stay valid and
 * unchanged until the job completes.  For the copy to run asynchronously
 * the memory must be page-locked (crystal_host_register, or cudaHostAlloc);
 * Section 2.1: data in pinned memory from the beginning saves the driver's
 * extra copy.  host = NULL returns to the job's own input buffer (EINVAL for a
 * job created with CRYSTAL_TASK_EXTERNAL_INPUT).  Not while the job runs. */
int crystal_task_bind_input(crystal_task* task, const void* host, uint64_t size);

/* Page-lock (and unlock) caller host memory for the GPU's DMA engines
 * (cudaHostRegister / cudaHostUnregister).  EDEVICE on failure. */
int crystal_host_register(void* host, uint64_t bytes);
int crystal_host_unregister(void* host);

/* h_input / h_output of Figure 2.  The application writes the input before
 * submit and reads the output after completion until release; it must not
 * touch either while the job runs.  NULL for a NULL task. */
void* crystal_task_host_in(crystal_task* task);
void* crystal_task_host_out(crystal_task* task);

/* Device addresses of d_input / d_output (Figure 2), for inspection. */
uint64_t crystal_task_device_in(crystal_task* task);
uint64_t crystal_task_device_out(crystal_task* task);

/* Shrink the sizes the next submit uses (input_size / output_size of
 * Figure 2) without giving the buffers back: in_size and out_size must not
 * exceed the sizes the job was created with.  Not while the job runs. */
int crystal_task_resize(crystal_task* task, uint64_t in_size, uint64_t out_size);

/* job_submit(), Figure 3: queues the job on the shared outstanding queue
 * (Section 4.2).  kind is a CRYSTAL_KIND_*, params may be NULL (defaults).
 * cb (may be NULL) runs on completion with user.  Errors: EINVAL (bad kind,
 * params or out_size below what the kind needs: 16 for direct, the fixed
 * sliding header + bitmap for sliding), EAGAIN (no device room for the job's
 * scratch now), ESHUTDOWN.  A job may be submitted again after it finished. */
int crystal_task_submit(crystal_task* task, int kind, const crystal_hash_params* params,
                        crystal_callback cb, void* user);

/* Submit n jobs at once, in array order, with one kind, params, callback
 * and user pointer: the batch-processing case of Section 2.2 (many
 * independent jobs available at once).  Either every job is queued
 * (CRYSTAL_OK) or none is (the first error is returned and no job changes
 * state). */
int crystal_task_submit_many(crystal_task* const* tasks, uint32_t n, int kind,
                             const crystal_hash_params* params, crystal_callback cb, void* user);

/* Priority of the job's next submits (default 0).  The master thread takes
 * outstanding jobs highest priority first and in submission order within a
 * priority (all jobs at 0: the paper's FIFO, Section 4.2; priority-based
 * scheduling is the extension its Section 7 names).  A deadline scheduler
 * maps earlier deadlines to higher priorities.  Not while the job is queued
 * or running. */
int crystal_task_set_priority(crystal_task* task, int priority);

/* job_query(), Figure 3: CRYSTAL_PENDING while queued or running, otherwise
 * the job's final status (CRYSTAL_OK, CRYSTAL_EOVERFLOW, CRYSTAL_EDEVICE,
 * CRYSTAL_ESHUTDOWN).  EINVAL for a job never submitted. */
int crystal_task_poll(crystal_task* task);

/* job_synch(), Figure 3, bounded: blocks until the job finished or
 * timeout_ns elapsed (timeout_ns < 0: no bound).  Returns the job's final
 * status, CRYSTAL_ETIMEDOUT, or CRYSTAL_EINVAL (never submitted, or called
 * from a completion callback). */
int crystal_task_wait(crystal_task* task, int64_t timeout_ns);

/* job_synch() over a set of jobs (no counterpart in the paper, which waits
 * job by job): blocks until every job of tasks[0..n) finished or timeout_ns
 * elapsed (one bound for the whole call; < 0: no bound).  All jobs must
 * belong to one context and have been submitted.  Returns CRYSTAL_OK when all
 * finished with CRYSTAL_OK, else the first non-OK final status in array
 * order; CRYSTAL_ETIMEDOUT if some job had not finished in time;
 * CRYSTAL_EINVAL for tasks == NULL with n > 0, a NULL or never-submitted job,
 * jobs of two contexts, or a call from a completion callback.  One call
 * replaces n calls of crystal_task_wait when a caller needs all of them. */
int crystal_task_wait_many(crystal_task* const* tasks, uint32_t n, int64_t timeout_ns);

/* job_put(), Figure 3: returns the job's buffers to the pool.  EINVAL while
 * the job is queued or running, except from the job's own completion
 * callback: there the buffers return to the pools at once (the output must
 * not be touched after the call) and the handle is freed when the callback
 * returns. */
int crystal_task_release(crystal_task* task);

/* Host clock stamps (nanoseconds, CLOCK_MONOTONIC) of the job's last run:
 * submit, dispatch by the master thread, completion seen by the master.
 * Any pointer may be NULL. */
int crystal_task_timing(crystal_task* task, uint64_t* submit_ns, uint64_t* dispatch_ns,
                        uint64_t* done_ns);

/* crystal_task_timing of n jobs at once: out[3 i], out[3 i + 1], out[3 i + 2]
 * = submit, dispatch, done stamps of tasks[i] (out holds 3 n values, caller
 * owned).  CRYSTAL_EINVAL for NULL arrays with n > 0 or a NULL job (out is
 * then partly written). */
int crystal_task_timing_many(crystal_task* const* tasks, uint32_t n, uint64_t* out);

/* The configuration a context runs with, written to *out (defaults filled
 * in; n_streams is 1 under CRYSTAL_FLAG_NO_OVERLAP, max_batch_jobs 1 under
 * CRYSTAL_FLAG_NO_BATCH or CRYSTAL_FLAG_NO_OVERLAP).  EINVAL for NULL. */
int crystal_get_config(crystal_ctx* ctx, crystal_config* out);

/* Launch geometry of the hashing kernels (the paper has no counterpart: it
 * leaves the kernel to the application).  The runtime sorts each batch into
 * one of CRYSTAL_SIZE_CLASSES classes by the mean input size of its hashing
 * jobs (< 64 KiB, < 1 MiB, >= 1 MiB) and launches the batch with that class's
 * geometry, which an autotuner may set from measurements.  Zero fields take
 * the defaults; CTAs per SM are capped at what fits.  Results never depend on
 * the geometry (every kernel walks its work in a grid-stride loop). */
typedef struct crystal_geometry {
    uint32_t seg_threads;        /* segment digests: threads per CTA, 64, 128 or 256 (0: 128) */
    uint32_t seg_ctas_per_sm;    /* segment digests: CTAs per SM (0: as many as fit) */
    uint32_t win_ctas_per_sm;    /* window kernel: CTAs per SM (0: as many as fit) */
    uint32_t win_registers;      /* w = 20 MD5 window kernel: 32 or 64 registers per thread (0: 32) */
    uint32_t digest_ctas_per_sm; /* chunk segment digests: CTAs per SM (0: as many as fit) */
    uint32_t reserved;           /* must be 0 */
} crystal_geometry;
#define CRYSTAL_SIZE_CLASSES 3

/* Set the geometry of size class size_class (0..2; -1: every class) of a
 * context; g NULL restores the defaults.  Only while the context is idle (no
 * job outstanding or running): EINVAL otherwise, or for a bad class or field;
 * the class's captured graphs are dropped and re-captured on next use. */
int crystal_set_geometry(crystal_ctx* ctx, int size_class, const crystal_geometry* g);

/* With CRYSTAL_FLAG_GRAPHS each stream slot replays one captured graph per
 * batch size class and kind mix, captured the first time a batch of that
 * shape lands on that slot -- a few hundred microseconds of master-thread time
 * inside whatever stream meets it first.  crystal_prepare_graphs captures
 * every graph not captured yet now, on the calling thread, so that a stream
 * that follows pays none of it (a set-up step like the pools of crystal_init;
 * crystal_set_geometry drops the graphs of the classes it changes, so call it
 * again after that).  The context must be idle (no outstanding or running
 * job): EINVAL otherwise; CRYSTAL_OK with nothing done without
 * CRYSTAL_FLAG_GRAPHS; EDEVICE if a capture fails. */
int crystal_prepare_graphs(crystal_ctx* ctx);

/* The geometry class size_class (0..2) runs with, resolved (threads per CTA
 * and CTAs per SM as launched, register budget 32 or 64), written to *out.
 * EINVAL for NULL or a bad class. */
int crystal_get_geometry(crystal_ctx* ctx, int size_class, crystal_geometry* out);

/* Counters of a context. */
typedef struct crystal_stats {
    uint64_t jobs_completed;
    uint64_t batches_launched;
    uint64_t device_pool_bytes, device_pool_used;
    uint64_t host_pool_bytes, host_pool_used;
    uint64_t jobs_outstanding, jobs_running;
    uint64_t copies_dma;  /* job-buffer copies issued to the DMA engines (merged runs count once) */
    uint64_t master_issue_ns;    /* master-thread time spent issuing batches (copies, launches) */
    uint64_t master_complete_ns; /* master-thread time spent completing batches (statuses, callbacks) */
    uint64_t create_ns;          /* time spent inside crystal_task_create[_ex] (all threads) */
    uint64_t create_calls;       /* calls of crystal_task_create[_ex] */
    uint64_t create_eagain;      /* of which returned CRYSTAL_EAGAIN (pool full) */
    uint64_t graph_captures;     /* batch graphs captured and instantiated (CRYSTAL_FLAG_GRAPHS) */
} crystal_stats;
int crystal_get_stats(crystal_ctx* ctx, crystal_stats* out);

/* Worst-case output size of a job: the digest size (16 MD5, 20 SHA-1) for
 * direct; for sliding the header, the bitmap and one record per possible
 * chunk (n - w + 2 of them, the case mask = 0).  in_size for NOP.  0 on a
 * bad kind. */
uint64_t crystal_out_bytes(int kind, uint64_t in_size, const crystal_hash_params* params);

/* Output size of an MD5 sliding job with room for max_chunks chunk records
 * (20 bytes each), and of a sliding job of any kind (4 + digest bytes each;
 * 0 for a kind that is not sliding). */
uint64_t crystal_sliding_out_bytes(uint64_t in_size, uint64_t max_chunks);
uint64_t crystal_out_bytes_for_chunks(int kind, uint64_t in_size, uint64_t max_chunks);

/* Static text for a status code. */
const char* crystal_strerror(int status);

/* Kernel launches this process made through the library (all contexts and
 * launchers; a graph replay counts each kernel node). */
uint64_t crystal_kernel_launches(void);

/* Microbenchmark of the integer pipes the hashing kernels are bound by (the
 * paper has no counterpart; it gives the integer roofline its measured
 * denominator).  Launches one kernel of ctas_per_sm x SMs CTAs of 256 threads
 * on `stream` that runs `iters` iterations on register data only -- no memory
 * is read, and d_sink (4 bytes of device memory) is written only if the
 * result equals `magic`, so no work can be optimised away.  Time it with
 * events on `stream`.  *work (may be NULL) receives the work the launch
 * performs: windows for the two window kinds (each a 20-byte window's hash up
 * to its first digest word, eight per thread per iteration, message words
 * shared from a ring of registers as the window kernel shares them), single
 * instructions for the others (eight independent chains per thread).
 * EINVAL for a bad kind, iters = 0, ctas_per_sm outside 1..64 or a NULL
 * d_sink; EDEVICE on a launch error. */
enum {
    CRYSTAL_PROBE_MD5_WINDOWS = 0,  /* MD5 window hash, w = 20, as k_sliding_windows<20> computes it */
    CRYSTAL_PROBE_SHA1_WINDOWS = 1, /* SHA-1 window hash, w = 20 */
    CRYSTAL_PROBE_LOP3 = 2,         /* three-input logic op (integer ALU pipe) */
    CRYSTAL_PROBE_SHF = 3,          /* funnel shift / rotate (integer ALU pipe) */
    CRYSTAL_PROBE_IADD3 = 4,        /* three-input add */
    CRYSTAL_PROBE_IMAD = 5,         /* integer multiply-add (FMA pipe) */
    CRYSTAL_PROBE_LOP3_IMAD = 6     /* LOP3 and IMAD alternately: two pipes at once */
};
int crystal_alu_probe(int kind, uint32_t ctas_per_sm, uint32_t iters, uint32_t magic, uint32_t* d_sink,
                      void* stream, uint64_t* work);

/* The baseline of the overhead experiment (Section 5.1, Figure 5): one job
 * issued without the framework -- copy in_size bytes h_in -> d_in, launch a
 * kernel that does nothing, copy out_size bytes d_out -> h_out, all on
 * `stream`, then wait for the stream.  Host buffers should be page-locked.
 * CRYSTAL_KIND_NOP jobs through the runtime do the same three stages, so the
 * difference of the two times is the framework's own cost. */
int crystal_direct_job(const void* h_in, void* d_in, uint64_t in_size, void* h_out, const void* d_out,
                       uint64_t out_size, void* stream);

/* ---- output layouts (what the kernels write) ----------------------------
 * direct  : digest Direct(u, S) = H(H(seg_0) || ... || H(seg_{m-1})) of D bytes,
 *           m = max(1, ceil(n / S)); the last segment may be short.  H is
 *           MD5 (D = 16) or SHA-1 (D = 20) by kind.
 * sliding : u32 n_chunks | u32 flags | u32 bitmap[ceil(n/32)] |
 *           u32 chunk_end[n_chunks] | u8 digest[n_chunks][D]
 *           bit i of the bitmap (word i/32, bit i%32) is set iff
 *           i <= n - w and (LE32(H(u[i, i+w))[0..3]) & mask) == target;
 *           chunk ends are the sorted set {i + w : bit i} U {n};
 *           digest[k] = Direct(u[end_{k-1}, end_k), chunk_segment_bytes),
 *           end_{-1} = 0.  If the records do not fit in out_size, flags bit 0
 *           is set, n_chunks holds the count needed and no record is written.
 * nop     : a kernel that does nothing runs; out_size bytes are copied back.
 */

/* ---- stateless batch launchers ------------------------------------------
 * One batch = a device-resident crystal_batch header followed by n_units
 * crystal_unit records (direct units first, then sliding units).  Build it on
 * the host with crystal_batch_plan, copy it to the device, then launch.
 * Every pointer inside is a device address.  Kernels read the header from
 * device memory, so one launch sequence (or one captured graph) serves any
 * batch that fits the launch's grid-independent limits.
 */
typedef struct crystal_unit {
    uint64_t in;         /* device address of the unit's bytes (any alignment) */
    uint64_t n;          /* unit length */
    uint64_t out;        /* device address of the unit's output (4-byte aligned) */
    uint64_t scratch;    /* device address of the unit's scratch (16-byte aligned) */
    uint64_t work_begin; /* filled by crystal_batch_plan: first global work item */
    uint32_t out_cap;    /* output bytes available */
    uint32_t seg_bytes;  /* direct: S; sliding: chunk S */
    uint16_t window;     /* sliding: w */
    uint16_t kind;       /* a direct or a sliding CRYSTAL_KIND_* (MD5 or SHA-1) */
    uint32_t mask, target;
    uint32_t seg_base;   /* sliding: written by the kernels (first chunk segment of
                            this unit among the batch's chunk segments) */
} crystal_unit;

typedef struct crystal_batch {
    uint32_t n_direct;          /* units [0, n_direct) are direct */
    uint32_t n_sliding;         /* units [n_direct, n_direct + n_sliding) are sliding */
    uint64_t direct_segments;   /* total segments over the direct units */
    uint64_t sliding_tiles;     /* total window tiles over the sliding units */
    uint32_t window_max;        /* largest window among the sliding units */
    uint32_t status;            /* device status word: 0, or a bit set by a kernel that met
                                   an inconsistent record (the record is skipped) */
    uint64_t sliding_tiles_w20; /* tiles of the sliding units with w = 20, which the
                                   planner places first */
    uint64_t chunk_segments;    /* written by the kernels: chunk segments of the batch */
    uint64_t sliding_tiles_md5; /* tiles of the MD5 sliding units (w = 20 first, then other
                                   windows); the SHA-1 sliding units follow */
    uint64_t direct_segments_md5; /* segments of the MD5 direct units, which come before the
                                     SHA-1 direct units (header is 64 bytes) */
    /* crystal_unit units[n_direct + n_sliding] follow */
} crystal_batch;

/* Offsets processed by one window tile of the sliding kernel (256 threads x
 * 8 windows).  The planner counts a sliding unit's work in these tiles. */
#ifndef CRYSTAL_SLIDING_TILE
#define CRYSTAL_SLIDING_TILE 2048u
#endif

/* Scratch bytes one unit needs: 16 * ceil(n/S) for direct; for sliding the
 * per-chunk segment table and digests for as many chunks as out_size holds.
 * 0 for NOP or on a bad argument. */
uint64_t crystal_scratch_bytes(int kind, uint64_t n, uint64_t out_size, const crystal_hash_params* params);

/* Host-side planning of a batch in host memory (the header followed by the
 * unit records, units filled by the caller except work_begin and seg_base):
 * checks every unit (kinds in order, sizes, windows 1..55, out_cap large
 * enough, 16-byte aligned scratch), orders the units (stable; each record
 * keeps its own pointers, so results do not depend on the order): MD5 direct
 * before SHA-1 direct; MD5 sliding with w = 20, other MD5 sliding, SHA-1
 * sliding; fills work_begin and the header's totals.  The buffer is then copied to the device as is.  Returns
 * CRYSTAL_OK or CRYSTAL_EINVAL. */
int crystal_batch_plan(crystal_batch* batch_host, uint32_t n_direct, uint32_t n_sliding);

/* Bytes of a batch buffer holding n_units records. */
uint64_t crystal_batch_bytes(uint32_t n_units);

/* Launch the kernels of a device-resident batch on a CUDA stream
 * (cudaStream_t passed as void*; NULL = legacy default stream).  Asynchronous;
 * errors are launch errors only (CRYSTAL_EDEVICE).  The kernels may read up
 * to 15 bytes before a unit's first byte and after its last byte inside the
 * same 16-byte-aligned block; those bytes never affect a result.
 *   crystal_launch_direct          segment MD5s then the digest of digests
 *   crystal_launch_direct_segments segment MD5s into scratch only
 *   crystal_launch_direct_outer    digest of digests from scratch only
 *   crystal_launch_sliding         window bitmap, chunk ends, chunk digests
 *   crystal_launch_sliding_windows window MD5s and the boundary bitmap only
 *   crystal_launch_sliding_chunks  chunk ends and chunk segment tables only
 *   crystal_launch_sliding_digests chunk segment MD5s and chunk digests only
 *   crystal_launch_batch           everything the batch holds */
int crystal_launch_direct(const crystal_batch* batch_dev, void* stream);
int crystal_launch_direct_segments(const crystal_batch* batch_dev, void* stream);
int crystal_launch_direct_outer(const crystal_batch* batch_dev, void* stream);
int crystal_launch_sliding(const crystal_batch* batch_dev, void* stream);
int crystal_launch_sliding_windows(const crystal_batch* batch_dev, void* stream);
int crystal_launch_sliding_chunks(const crystal_batch* batch_dev, void* stream);
int crystal_launch_sliding_digests(const crystal_batch* batch_dev, void* stream);
int crystal_launch_batch(const crystal_batch* batch_dev, void* stream);

/* ---- serving loop --------------------------------------------------------
 * crystal_serve plays an open-loop stream of requests against a context
 * (stream-processing applications, Section 2.2: data units arrive
 * continuously and each needs low latency).  Request i arrives arrival_ns
 * after the call starts; requests are admitted as soon as the context's pools
 * can hold the job's buffers and scratch (crystal_task_create_ex), oldest
 * first: while the oldest waiting request does not fit, later requests that
 * fit may be admitted past it until it has waited bypass_ns (then nothing
 * passes it, so room frees up for it and it cannot starve);
 * CRYSTAL_SERVE_ARRIVAL_ORDER admits strictly in arrival order instead.
 * Copy threads stage the request's bytes from
 * `source` into the job's pinned input (or, with CRYSTAL_SERVE_SOURCE_PINNED,
 * bind the job's input to them) and submit it; with ring_bytes > 0, requests
 * of at most ring_max_request bytes are instead copied into an input ring
 * (ring_bytes of pinned host pool and ring_bytes of device pool, reserved for
 * the call; EAGAIN / ENOMEM if the pools cannot hold it, EINVAL for a context
 * without pools, CRYSTAL_FLAG_NO_POOL) in admission order,
 * so neighbouring requests' copies merge into one DMA transfer -- a request
 * that finds the ring full gets buffers of its own as before; the master thread
 * batches whatever is outstanding (continuous batching).  On completion the
 * used output bytes of a request with capture_offset != UINT64_MAX are copied
 * to capture + capture_offset (if they fit), and the job is released.  A
 * request that can never fit the pools fails with CRYSTAL_ENOMEM.
 * Returns CRYSTAL_OK when every request finished with OK or EOVERFLOW,
 * otherwise the last other error; per-request results are in `res`;
 * *wall_ns receives the time of the last completion. */
typedef struct crystal_request {
    uint64_t arrival_ns;     /* arrival time after the start of the call (non-decreasing) */
    uint64_t src_offset;     /* the request's bytes are source[src_offset, src_offset + size) */
    uint64_t size;
    uint64_t out_size;       /* output bytes reserved for the job */
    uint64_t capture_offset; /* UINT64_MAX: output not copied out */
    int32_t kind;            /* CRYSTAL_KIND_* */
    uint32_t reserved;
} crystal_request;

typedef struct crystal_request_result {
    int32_t status;
    uint32_t reserved;
    uint64_t admit_ns;   /* buffers obtained (after any wait for pool room) */
    uint64_t submit_ns;  /* bytes staged, job submitted */
    uint64_t done_ns;    /* completion seen by the master thread */
    uint64_t used_bytes; /* output bytes that carry results */
} crystal_request_result;

#define CRYSTAL_SERVE_SOURCE_PINNED 1u
#define CRYSTAL_SERVE_ARRIVAL_ORDER 2u
typedef struct crystal_serve_config {
    uint32_t copy_threads;                      /* staging threads; default 4 */
    uint32_t flags;                             /* CRYSTAL_SERVE_SOURCE_PINNED: `source` is page-locked;
                                                   jobs read their input from it directly
                                                   (crystal_task_bind_input) and nothing is staged */
    const crystal_hash_params* direct_params;   /* NULL: defaults */
    const crystal_hash_params* sliding_params;  /* NULL: defaults */
    void* capture;                              /* host buffer for captured outputs, or NULL */
    uint64_t capture_bytes;
    uint64_t bypass_ns;                         /* how long later requests may pass a blocked oldest
                                                   request; default (0) 2 ms */
    uint64_t ring_bytes;                        /* input ring for small requests; 0 = none */
    uint64_t ring_max_request;                  /* largest request staged in the ring; default (0)
                                                   256 KiB */
} crystal_serve_config;

int crystal_serve(crystal_ctx* ctx, const void* source, uint64_t source_bytes, const crystal_request* requests,
                  uint32_t n, const crystal_serve_config* cfg, crystal_request_result* results, uint64_t* wall_ns);

/* ---- a job stream staged from pageable memory -----------------------------
 * Section 2.1: the DMA engines copy only from page-locked memory, so bytes an
 * application holds in ordinary (pageable) memory must first be copied into a
 * pinned buffer; Section 3 keeps pinned job buffers in a pool allocated once,
 * and Section 4.1 / Figure 4 overlaps the copies of some jobs with the kernels
 * of others.  crystal_stream_staged hashes units[0..n) (pageable or pinned
 * host memory, sizes[i] bytes each, read-only during the call) through a ring
 * of ring_jobs jobs created at the start of the call (each with a pinned
 * input of the largest unit's size, a pinned output of out_size bytes and its
 * device scratch reserved) and released at its end:
 *   - copy_threads host threads take the units in index order, copy each into
 *     the pinned input of a free job (FIFO over the ring) and submit it;
 *   - the master thread batches the submitted jobs as for any other job;
 *   - a finished job returns to the ring; the thread that takes it next first
 *     copies the finished unit's used output bytes (at most out_stride) to
 *     outputs + i * out_stride (outputs may be NULL: results not kept).
 * results[i] receives the unit's status, admit_ns (a ring job taken),
 * submit_ns (bytes staged, job submitted), done_ns (completion seen by the
 * master) relative to the call's start, and used_bytes.  *wall_ns (may be
 * NULL) receives the time from the start to the last result copied out.
 * ring_jobs 0 = 3 x n_streams x min(max_batch_jobs, 4) (at most n); the
 * context's pools must hold the ring (host: ring x (largest unit + out_size);
 * device: the same plus each job's scratch, crystal_scratch_bytes).
 * Returns CRYSTAL_OK when every unit finished with OK or EOVERFLOW, else the
 * last other per-unit error; EINVAL for bad arguments (NULL arrays, a unit
 * larger than the context's max_in_bytes, out_size above max_out_bytes, a
 * bad kind or params); EAGAIN / ENOMEM if the pools cannot hold the ring (no
 * unit is then processed). */
typedef struct crystal_stream_config {
    int32_t kind;                       /* CRYSTAL_KIND_* of every unit */
    uint32_t copy_threads;              /* staging threads; default 4, at most 64 */
    uint32_t ring_jobs;                 /* jobs in the ring; 0 = the default above */
    uint32_t reserved;                  /* must be 0 */
    uint64_t out_size;                  /* output bytes of each job */
    const crystal_hash_params* params;  /* NULL: defaults */
} crystal_stream_config;

int crystal_stream_staged(crystal_ctx* ctx, const void* const* units, const uint64_t* sizes, uint32_t n,
                          const crystal_stream_config* cfg, void* outputs, uint64_t out_stride,
                          crystal_request_result* results, uint64_t* wall_ns);

/* ---- direct hashing that allocates nothing --------------------------------
 * The paper has no counterpart to this call; it serves callers that cannot
 * allocate device memory where they hash: a thread on a storage or network
 * data path with a fixed latency budget (cudaMalloc and cudaFree can
 * synchronise the whole device and take milliseconds), or a process whose
 * free device memory already belongs to another allocator, so that a new
 * cudaMalloc would fail.
 *
 * crystal_md5_direct_noalloc hashes n_units units of unit_bytes each, lying
 * back to back from d_in (device memory), with direct hashing at segment size
 * segment_bytes, and writes unit u's 16-byte digest at d_digests + 16 u
 * (device memory, 4-byte aligned).  It is asynchronous on `stream`
 * (cudaStream_t as void*).  Its batch descriptor and segment digests live in
 * a fixed device array of CRYSTAL_NOALLOC_SCRATCH_BYTES inside the library,
 * which every GPU that loads the library holds until the process exits; the
 * call itself allocates nothing.
 *   - Limit: align_up(64 + 64 n_units, 256) + 16 n_units ceil(unit_bytes /
 *     segment_bytes) (a unit of 0 bytes counts one segment) must not exceed
 *     CRYSTAL_NOALLOC_SCRATCH_BYTES; a larger request returns CRYSTAL_EINVAL
 *     and launches nothing.
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current); make that first call before
 *     any stream capture.  A failed lookup returns CRYSTAL_EDEVICE.
 *   - Every call on a device shares the one array and leaves its contents
 *     behind; each call rewrites everything it reads before reading it.
 *     Calls whose work overlaps on the GPU (different streams, or different
 *     host threads without ordering between them) race on the array and give
 *     wrong digests: order them, e.g. issue them on one stream.
 * Returns CRYSTAL_OK (also for n_units = 0), CRYSTAL_EINVAL (NULL pointers,
 * segment_bytes = 0, misaligned d_digests, or the size limit) or
 * CRYSTAL_EDEVICE (launch failure; a launch error already pending on the
 * calling thread from earlier work is reported this way too, and cleared,
 * before anything is queued; if the descriptor kernel fails to launch, the
 * hashing kernels are not queued). */
#define CRYSTAL_NOALLOC_SCRATCH_BYTES (8u << 20)
int crystal_md5_direct_noalloc(const void* d_in, uint64_t unit_bytes, uint32_t n_units, uint32_t segment_bytes,
                               void* d_digests, void* stream);

/* Host-side arena allocator the pools use (exposed for tests; no GPU
 * needed).  Offsets are relative to 0; alignment is a power of two; the
 * arena's size is rounded down to a multiple of it. */
typedef struct crystal_arena crystal_arena;
int crystal_arena_create(uint64_t bytes, uint64_t alignment, crystal_arena** out);
int crystal_arena_alloc(crystal_arena* a, uint64_t bytes, uint64_t* offset);  /* best fit */
/* Placement-controlled allocation: best fit, the lowest-addressed free block
 * that fits (from its bottom), or the highest-addressed one (from its top).
 * The job runtime takes inputs from the bottom and outputs and scratch from
 * the top, so jobs created one after another get adjacent inputs and adjacent
 * outputs and a batch's copies can be merged. */
enum { CRYSTAL_ARENA_BEST_FIT = 0, CRYSTAL_ARENA_LOWEST = 1, CRYSTAL_ARENA_HIGHEST = 2 };
int crystal_arena_alloc_at(crystal_arena* a, uint64_t bytes, int placement, uint64_t* offset);
/* Allocate exactly [offset, offset + bytes rounded up): CRYSTAL_OK if that
 * range is free, else EAGAIN (EINVAL for an offset off the alignment).  The
 * runtime places a job's pinned input at the offset of its device input, so
 * that jobs with adjacent inputs can be copied by one transfer. */
int crystal_arena_alloc_exact(crystal_arena* a, uint64_t offset, uint64_t bytes);
int crystal_arena_free(crystal_arena* a, uint64_t offset);
uint64_t crystal_arena_used(crystal_arena* a);
uint64_t crystal_arena_largest_free(crystal_arena* a);
void crystal_arena_destroy(crystal_arena* a);

#ifdef __cplusplus
}
#endif
#endif /* CRYSTAL_H */
