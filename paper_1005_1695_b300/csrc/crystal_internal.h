// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstddef>

#include "crystal.h"

namespace crystal {

extern std::atomic<uint64_t> g_kernel_launches;

// Kernel launchers on a device-resident batch (kernels.cu).
int launch_direct_segments(crystal_batch* b, cudaStream_t s);
int launch_direct_outer(crystal_batch* b, cudaStream_t s);
int launch_sliding_windows(crystal_batch* b, cudaStream_t s);
int launch_sliding_chunks(crystal_batch* b, cudaStream_t s);
int launch_sliding_digests(crystal_batch* b, cudaStream_t s);  // two kernels
int launch_nop(cudaStream_t s);                                 // the dummy kernel

// Copies made by the SMs instead of the DMA engines (runtime.cu decides which):
// piece i moves n bytes from src to dst, either address may be mapped pinned
// host memory.  The table lives in device memory; chunks of kCopyChunk bytes
// of every piece are spread over the CTAs of one launch.
constexpr uint64_t kCopyChunk = 16384;
struct CopyPiece {
    uint64_t src, dst, n;
    uint64_t first_chunk;  // chunks of the pieces before this one
};
struct CopyTable {
    uint32_t n_pieces;
    uint32_t reserved;
    uint64_t n_chunks;  // chunks of all pieces
    CopyPiece piece[1];  // n_pieces used (the table is allocated for the slot's maximum)
};
inline uint64_t copy_table_bytes(uint32_t max_pieces) {
    return 16 + 32ull * (max_pieces ? max_pieces : 1);
}
int launch_copy_pieces(const CopyTable* table, cudaStream_t s);
// The batch descriptor fetched by the GPU from mapped pinned memory (bytes a
// multiple of 16), and its status word posted back to mapped pinned memory:
// no DMA transfer for either.
int launch_fetch_descriptor(const void* host_dev, crystal_batch* dst, uint64_t bytes, cudaStream_t s);
int launch_post_status(const crystal_batch* d, uint32_t* host_status_dev, cudaStream_t s);

inline crystal_unit* batch_units(crystal_batch* b) {
    return reinterpret_cast<crystal_unit*>(reinterpret_cast<uint8_t*>(b) + sizeof(crystal_batch));
}

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
static_assert(sizeof(crystal::CopyPiece) == 32 && offsetof(crystal::CopyTable, piece) == 16, "copy table layout");
