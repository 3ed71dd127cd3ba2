// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstddef>

#include "crystal.h"

namespace crystal {

extern std::atomic<uint64_t> g_kernel_launches;
// Set while this thread captures a graph: captured launches are counted when
// the graph is replayed, not when it is captured.
extern thread_local bool tl_capturing;

// Grid and CTA shape of each kernel of a batch (kernels.cu): resolved from a
// crystal_geometry against the kernels' occupancy on the current device.
struct LaunchGeom {
    int sms = 0;
    int seg_threads = 128;  // K1 threads per CTA: 64, 128 or 256
    int seg_per_sm = 0, seg_blocks = 0, seg_sha1_blocks = 0;
    int win20_wide = 0;  // 1: the 64-register instance of the w = 20 MD5 window kernel
    int win_per_sm = 0, win20_blocks = 0, win_blocks = 0, win_sha1_blocks = 0;
    int digest_per_sm = 0, digest_blocks = 0;
    int outer_blocks = 0, unit_blocks = 0;
};
int make_geometry(const crystal_geometry* in, LaunchGeom* out);  // EINVAL / EDEVICE
void describe_geometry(const LaunchGeom& g, crystal_geometry* out);

// Kernel launchers on a device-resident batch (kernels.cu); geom NULL: the
// device's default geometry.
int launch_direct_segments(crystal_batch* b, cudaStream_t s, const LaunchGeom* geom = nullptr);
int launch_direct_outer(crystal_batch* b, cudaStream_t s, const LaunchGeom* geom = nullptr);
int launch_sliding_windows(crystal_batch* b, cudaStream_t s, const LaunchGeom* geom = nullptr);
int launch_sliding_chunks(crystal_batch* b, cudaStream_t s, const LaunchGeom* geom = nullptr);
int launch_sliding_digests(crystal_batch* b, cudaStream_t s, const LaunchGeom* geom = nullptr);  // two kernels
int launch_nop(cudaStream_t s);                                 // the dummy kernel

// The batch descriptor fetched by the GPU from mapped pinned memory (bytes a
// multiple of 16), and its status word posted back to mapped pinned memory:
// no DMA transfer for either.
int launch_fetch_descriptor(const void* host_dev, crystal_batch* dst, uint64_t bytes, cudaStream_t s);
int launch_post_status(const crystal_batch* d, uint32_t* host_status_dev, cudaStream_t s);

inline crystal_unit* batch_units(crystal_batch* b) {
    return reinterpret_cast<crystal_unit*>(reinterpret_cast<uint8_t*>(b) + sizeof(crystal_batch));
}

// A pinned-host block and a device block of the same size, both taken from
// the context's pools (host from the pinned arena, device from the device
// arena); given back with release_pool_pair.  EINVAL for a context without
// pools.
struct PoolPair {
    uint8_t* host = nullptr;
    uint8_t* dev = nullptr;
    uint64_t host_off = 0, dev_off = 0, bytes = 0;
};
int reserve_pool_pair(crystal_ctx* c, uint64_t bytes, PoolPair* out);
void release_pool_pair(crystal_ctx* c, const PoolPair& p);

// A job whose input lies in memory the caller keeps (h_in page-locked, d_in
// device memory, in_size bytes each; e.g. slots of an input ring made from a
// PoolPair): only its output and scratch come from the pools, and releasing
// it leaves the input memory alone.  Jobs whose inputs sit next to each other
// at one host-to-device distance have their copies merged like pooled jobs
// (a job's block is in_size rounded up to 256 bytes, so the caller keeps the
// inputs 256-byte aligned and the padding its own).
int task_create_borrowed(crystal_ctx* c, uint8_t* h_in, uint8_t* d_in, uint64_t in_size, uint64_t out_size,
                         uint64_t scratch_bytes, crystal_task** out);

constexpr uint32_t kMaxWindow = 55;  // a window message fits one MD5 block

inline bool kind_is_direct(int k) { return k == CRYSTAL_KIND_MD5_DIRECT || k == CRYSTAL_KIND_SHA1_DIRECT; }
inline bool kind_is_sliding(int k) { return k == CRYSTAL_KIND_MD5_SLIDING || k == CRYSTAL_KIND_SHA1_SLIDING; }
inline bool kind_is_sha1(int k) { return k == CRYSTAL_KIND_SHA1_DIRECT || k == CRYSTAL_KIND_SHA1_SLIDING; }
inline uint64_t digest_bytes_of(int k) { return kind_is_sha1(k) ? 20 : 16; }

inline uint64_t segments_of(uint64_t n, uint64_t S) { return n == 0 ? 1 : (n + S - 1) / S; }
inline uint64_t bitmap_words(uint64_t n) { return (n + 31) / 32; }
inline uint64_t sliding_fixed_bytes(uint64_t n) { return 8 + 4 * bitmap_words(n); }
inline uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) & ~(a - 1); }

}  // namespace crystal

static_assert(sizeof(crystal_unit) == 64, "unit record is 64 bytes");
static_assert(sizeof(crystal_batch) == 64, "batch header is 64 bytes");

