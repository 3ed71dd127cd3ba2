// Hashing kernels of one batch (sm_103a) and their stateless launchers.
//
//   k_direct_segments  K1  one MD5 per segment of every direct unit
//   k_direct_outer     K2  MD5 over each unit's concatenated segment digests
//   k_sliding_windows  K3  digest of every w-byte window, boundary bitmap
//                          (MD5 with w = 20, MD5 with any w in 1..55, SHA-1)
//   k_sliding_chunks   K4  chunk ends from the bitmap, per-chunk segment table
//   k_chunk_seg_scan   K4b where each unit's chunk segments start in the batch
//   k_chunk_segments   K5a one MD5 per segment of every chunk
//   k_chunk_outer      K5b MD5 over each chunk's segment digests
//
// Direct hashing is StoreGPU's direct hashing (Section 5.2, Figure 6 of the
// CrystalGPU paper; the paper's CPU post-processing step, the hash of the
// digests, runs on the GPU here as K2).  Sliding-window hashing is the
// content-defined chunking of content-addressable storage (Section 2.2).
//
// Every kernel is persistent: a fixed grid sized to the device walks the work
// of whatever batch the device-resident header describes, so one launch
// sequence (or one captured graph) serves every batch.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <thread>

#include "crystal.h"
#include "crystal_internal.h"
#include "digest_device.cuh"
#include "md5_device.cuh"
#include "sha1_device.cuh"

namespace crystal {

std::atomic<uint64_t> g_kernel_launches{0};
thread_local bool tl_capturing = false;

namespace {

constexpr int kTile = CRYSTAL_SLIDING_TILE;  // window offsets per tile
constexpr int kWinThreads = 256;             // 8 warps x kWinPerThread windows x 32 lanes
constexpr int kWinPerThread = kTile / kWinThreads;
static_assert(kWinPerThread * kWinThreads == kTile && kWinPerThread <= 32, "tile layout");
// Staged words per tile: the tile's offsets + up to 54 halo bytes + 15 alignment
// bytes, rounded up to whole 16-byte vectors, plus room for the last window's
// word reads.
constexpr int kStageWords = 4 * ((kTile + 69 + 15) / 16) + 4;

constexpr int kChunkThreads = 512;
constexpr int kDigestThreads = 256;
constexpr int kChunkSegThreads = 128;  // K5a: 5 CTAs per SM at <= 102 registers
constexpr int kScanThreads = 1024;

constexpr uint32_t kDevBadRecord = 1u;

// Whether each kernel puts the round-function add on the FMA pipe (see
// md5::add_on_fma): throughput-bound kernels do; the serial digest-of-digests
// chains may prefer the lower-latency ALU add.
#ifndef CRYSTAL_FMA_SEGMENTS
#define CRYSTAL_FMA_SEGMENTS 1
#endif
#ifndef CRYSTAL_FMA_OUTER
#define CRYSTAL_FMA_OUTER 1
#endif

__device__ __forceinline__ crystal_unit* units_of(crystal_batch* b) {
    return reinterpret_cast<crystal_unit*>(reinterpret_cast<uint8_t*>(b) + sizeof(crystal_batch));
}

// Last unit in [lo, lo + cnt) whose work_begin <= g (units with no work share
// their successor's begin, so the last one is the owner).
__device__ __forceinline__ uint32_t owner_of(const crystal_unit* U, uint32_t cnt, uint64_t g) {
    uint32_t lo = 0, hi = cnt;  // answer in [lo, hi)
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (U[mid].work_begin <= g) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool is_sha1(const crystal_unit& X) {
    return X.kind == CRYSTAL_KIND_SHA1_DIRECT || X.kind == CRYSTAL_KIND_SHA1_SLIDING;
}

// Digest bytes of a unit's hash, and bytes per chunk record (u32 end + digest).
__device__ __forceinline__ uint32_t digest_bytes(const crystal_unit& X) { return is_sha1(X) ? 20u : 16u; }
__device__ __forceinline__ uint32_t record_bytes(const crystal_unit& X) { return 4u + digest_bytes(X); }

// Digest of [p, p + len) with the unit's hash, stored at dst (4-byte aligned).
// ANY: the single-path loader for messages that rarely start 16-byte aligned.
template <bool FMA, bool ANY = false>
__device__ __forceinline__ void digest_to(const crystal_unit& X, const uint8_t* p, uint64_t len, uint8_t* dst,
                                          uint32_t one) {
    uint32_t st[5];
    if (is_sha1(X)) {
        if constexpr (ANY) digest_global_any<SHA1Hash, FMA>(p, len, st, one);
        else digest_global<SHA1Hash, FMA>(p, len, st, one);
        store_digest<SHA1Hash>(dst, st);
    } else {
        if constexpr (ANY) digest_global_any<MD5Hash, FMA>(p, len, st, one);
        else digest_global<MD5Hash, FMA>(p, len, st, one);
        store_digest<MD5Hash>(dst, st);
    }
}

__device__ __forceinline__ uint64_t num_segments(uint64_t n, uint32_t S) {
    return n == 0 ? 1 : (n + S - 1) / S;
}

// ---- K1: segment digests of direct units ------------------------------------

// One instance per hash: MD5 units are [0, direct_segments_md5) of the
// segment space (the planner puts them first), SHA-1 units the rest.  NT
// threads per CTA (64, 128 or 256: a launch-geometry choice), compiled for
// 640 resident threads per SM at least.
template <class H, int NT>
__global__ void __launch_bounds__(NT, 640 / NT) k_direct_segments(crystal_batch* B, uint32_t one) {
    const uint32_t nd = B->n_direct;
    const bool sha = H::kWords == 5;
    const uint64_t lo = sha ? B->direct_segments_md5 : 0;
    const uint64_t hi = sha ? B->direct_segments : B->direct_segments_md5;
    const crystal_unit* U = units_of(B);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t g = lo + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < hi; g += stride) {
        const uint32_t u = owner_of(U, nd, g);
        const crystal_unit X = U[u];
        const uint64_t j = g - X.work_begin;
        const uint64_t off = j * X.seg_bytes;
        const uint64_t len = X.n > off ? (X.n - off < X.seg_bytes ? X.n - off : X.seg_bytes) : 0;
        uint32_t st[5];
        digest_global<H, CRYSTAL_FMA_SEGMENTS>(reinterpret_cast<const uint8_t*>(X.in) + off, len, st, one);
        store_digest<H>(reinterpret_cast<uint8_t*>(X.scratch) + (uint64_t)H::kBytes * j, st);
    }
}

// ---- K2: digest of digests -------------------------------------------------

__global__ void __launch_bounds__(kDigestThreads) k_direct_outer(crystal_batch* B, uint32_t one) {
    const uint32_t nd = B->n_direct;
    const crystal_unit* U = units_of(B);
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < nd; u += gridDim.x * blockDim.x) {
        const crystal_unit X = U[u];
        const uint64_t m = num_segments(X.n, X.seg_bytes);
        digest_to<CRYSTAL_FMA_OUTER>(X, reinterpret_cast<const uint8_t*>(X.scratch), digest_bytes(X) * m,
                                     reinterpret_cast<uint8_t*>(X.out), one);
    }
    __threadfence_system();  // out may be mapped host memory (the runtime writes digests in place)
}

// ---- K3: window digests and boundary bitmap ---------------------------------

// Message block of the window starting at staged byte p.  W > 0: the window
// length is the compile-time constant W (constant padding words fold away);
// W == 0: the length w is taken at run time.
template <int W>
__device__ __forceinline__ void window_block(const uint32_t* sw, uint32_t p, uint32_t w,
                                             uint32_t (&X)[16]) {
    const uint32_t q = p >> 2;
    const uint32_t sh = (p & 3) * 8;
    if constexpr (W > 0) {
        constexpr int full = W / 4;
        constexpr int part = W % 4;
#pragma unroll
        for (int k = 0; k < 16; ++k) X[k] = 0;
#pragma unroll
        for (int k = 0; k < full; ++k) X[k] = __funnelshift_r(sw[q + k], sw[q + k + 1], sh);
        if constexpr (part > 0) {
            const uint32_t v = __funnelshift_r(sw[q + full], sw[q + full + 1], sh);
            X[full] = (v & ((1u << (8 * part)) - 1u)) | (0x80u << (8 * part));
        } else {
            X[full] = 0x80u;
        }
        X[14] = 8u * W;
        X[15] = 0;
    } else {
#pragma unroll
        for (int k = 0; k < 14; ++k) {
            const int have = (int)w - 4 * k;
            uint32_t v = 0;
            if (have > 0) {
                v = __funnelshift_r(sw[q + k], sw[q + k + 1], sh);
                if (have < 4) v &= (1u << (8 * have)) - 1u;
            }
            if (have >= 0 && have < 4) v |= 0x80u << (8 * have);
            X[k] = v;
        }
        X[14] = 8u * w;
        X[15] = 0;
    }
}

// LE32 of digest bytes 0..3 of the one-block message X (MD5 layout: little-
// endian words, bit length in word 14).  For SHA-1 the words are turned
// big-endian and the length moved to word 15 first.
template <class H>
__device__ __forceinline__ uint32_t window_first_word(uint32_t (&X)[16], uint32_t w, uint32_t one) {
    if constexpr (H::kWords == 5) {
#pragma unroll
        for (int k = 0; k < 14; ++k) X[k] = sha1::bswap(X[k]);
        X[14] = 0;
        X[15] = 8u * w;
        return sha1::bswap(sha1::first_word_one_block(X, one));
    } else {
        return md5::first_word_one_block(X, one);
    }
}

template <int W, class H>
__device__ __forceinline__ uint32_t tile_windows(const uint32_t* sw, uint32_t delta, uint32_t lim, uint32_t w,
                                                 uint32_t mask, uint32_t target, uint32_t one) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warp = threadIdx.x >> 5;
    uint32_t A[kWinPerThread];
#pragma unroll
    for (int r = 0; r < kWinPerThread; ++r) {
        const uint32_t rel = warp * (32 * kWinPerThread) + r * 32 + lane;
        uint32_t X[16];
        window_block<W>(sw, rel + delta, w, X);
        A[r] = window_first_word<H>(X, w, one);
    }
    // ballots only after every window of the thread is hashed: a ballot per
    // window was measured 9% slower (each one is a warp-wide sync point)
    uint32_t mine = 0;  // lane r ends up holding bitmap word r of this warp
#pragma unroll
    for (int r = 0; r < kWinPerThread; ++r) {
        const uint32_t rel = warp * (32 * kWinPerThread) + r * 32 + lane;
        const bool hit = (rel + w <= lim) && ((A[r] & mask) == target);
        const uint32_t word = __ballot_sync(0xffffffffu, hit);
        if (lane == (uint32_t)r) mine = word;
    }
    return mine;
}

// Hit mask of a lane's eight windows past the unit's last full window
// (rel0 + 4 j + 20 > lim) cleared, ORed over the four lanes of its group and
// moved to lane g (the layout of tile_windows).
__device__ __forceinline__ uint32_t gather_group_mask(uint32_t m, uint32_t rel0, uint32_t lim) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t sub = lane & 3;
    const int32_t room = (int32_t)lim - (int32_t)(rel0 + 20);
    const uint32_t valid = room < 0 ? 0u : min(8u, (uint32_t)room / 4 + 1);
    m &= valid ? (0x11111111u >> (4 * (8 - valid))) << sub : 0u;
    m |= __shfl_xor_sync(0xffffffffu, m, 1);
    m |= __shfl_xor_sync(0xffffffffu, m, 2);
    return __shfl_sync(0xffffffffu, m, (lane & 7) * 4);
}

// SHA-1 form of tile_windows20 (same lanes and windows).  SHA-1 reads its
// message words big-endian, so the staged words are byte-swapped once each
// and shifted into place from the high end (one swap per window instead of
// five), and the boundary test compares the big-endian first digest word
// against the byte-swapped mask and target: (bswap(x) & m) == t exactly when
// (x & bswap(m)) == bswap(t).
__device__ __forceinline__ uint32_t tile_windows20_sha1(const uint32_t* s, uint32_t sh, uint32_t rel0, uint32_t lim,
                                                        uint32_t mask, uint32_t target, uint32_t one) {
    const uint32_t sub = threadIdx.x & 3;
    const uint32_t bmask = sha1::bswap(mask), btarget = sha1::bswap(target);
    uint32_t M[5];  // big-endian message words 0..4 of the current window
    uint32_t raw = sha1::bswap(s[0]);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const uint32_t nxt = sha1::bswap(s[k + 1]);
        M[k] = __funnelshift_l(nxt, raw, sh);
        raw = nxt;
    }
    uint32_t m = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        uint32_t W[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) W[k] = 0;
#pragma unroll
        for (int k = 0; k < 5; ++k) W[k] = M[k];
        W[5] = 0x80000000u;
        W[15] = 8u * 20;
        const uint32_t A = sha1::first_word_one_block(W, one);
        m |= (uint32_t)((A & bmask) == btarget) << (sub + 4 * j);
        if (j < 7) {
#pragma unroll
            for (int k = 0; k < 4; ++k) M[k] = M[k + 1];
            const uint32_t nxt = sha1::bswap(s[j + 6]);
            M[4] = __funnelshift_l(nxt, raw, sh);
            raw = nxt;
        }
    }
    return gather_group_mask(m, rel0, lim);
}

// The tile with the common 20-byte window.  Lane (g, s) = (lane / 4, lane % 4)
// of a warp hashes the windows at offsets 32 g + s + 4 j, j = 0..7, of the
// warp's 256: consecutive windows of a thread are one word apart, so they
// share the byte phase and all but one message word, and the thread shifts
// 12 words into place for its 8 windows instead of 40.  Each hit becomes bit
// s + 4 j of the thread's mask; the four lanes of a group then OR their masks
// into bitmap word g, which is moved to lane g (the layout of tile_windows).
template <class H>
__device__ __forceinline__ uint32_t tile_windows20(const uint32_t* sw, uint32_t delta, uint32_t lim, uint32_t mask,
                                                   uint32_t target, uint32_t one) {
    static_assert(kWinPerThread == 8 && kWinThreads == 256, "lane layout assumes 8 warps x 8 windows");
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t sub = lane & 3;
    const uint32_t rel0 = warp * 256 + (lane >> 2) * 32 + sub;
    const uint32_t p = rel0 + delta;
    const uint32_t* s = sw + (p >> 2);
    const uint32_t sh = (p & 3) * 8;
    if constexpr (H::kWords == 5) return tile_windows20_sha1(s, sh, rel0, lim, mask, target, one);
    uint32_t M[5];  // message words 0..4 of the current window
    uint32_t raw = s[0];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const uint32_t nxt = s[k + 1];
        M[k] = __funnelshift_r(raw, nxt, sh);
        raw = nxt;
    }
    uint32_t m = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        uint32_t X[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) X[k] = 0;
#pragma unroll
        for (int k = 0; k < 5; ++k) X[k] = M[k];
        X[5] = 0x80u;
        X[14] = 8u * 20;
        const uint32_t A = window_first_word<H>(X, 20u, one);
        m |= (uint32_t)((A & mask) == target) << (sub + 4 * j);
        if (j < 7) {
#pragma unroll
            for (int k = 0; k < 4; ++k) M[k] = M[k + 1];
            const uint32_t nxt = s[j + 6];
            M[4] = __funnelshift_r(raw, nxt, sh);
            raw = nxt;
        }
    }
    // windows past the unit's last full window do not count
    return gather_group_mask(m, rel0, lim);
}

// What every thread of a CTA needs to know about one tile, worked out once by
// thread 0 (the unit that owns it, the staging source, the output words).
struct TileInfo {
    uint64_t src;     // 16-byte aligned address of the first vector to stage
    uint64_t out;     // address of the tile's first bitmap word
    uint32_t nvec;    // 16-byte vectors to stage
    uint32_t delta;   // byte offset of the tile's first window in the staged data
    uint32_t lim;     // bytes of the unit from the tile's first window on (at most 2 tiles)
    uint32_t words;   // bitmap words of the tile that lie inside the unit
    uint32_t mask, target, w, pad;
};

__device__ __forceinline__ void describe_tile(TileInfo& I, const crystal_unit* U, uint32_t ns, uint64_t g) {
    const crystal_unit X = U[owner_of(U, ns, g)];
    const uint64_t base = (g - X.work_begin) * (uint64_t)kTile;
    const uint64_t a = X.in + base;
    const uint32_t delta = (uint32_t)(a & 15);
    const uint64_t left = X.n - base;
    const uint64_t span = (uint64_t)(kTile + X.window - 1);
    const uint64_t want = left < span ? left : span;
    const uint64_t words_left = ((X.n + 31) >> 5) - (base >> 5);
    I.src = a - delta;
    I.out = X.out + 8 + 4 * (base >> 5);
    I.nvec = (uint32_t)((delta + want + 15) >> 4);
    I.delta = delta;
    I.lim = left < (uint64_t)(2 * kTile) ? (uint32_t)left : (uint32_t)(2 * kTile);
    I.words = words_left < (uint64_t)(kTile / 32) ? (uint32_t)words_left : (uint32_t)(kTile / 32);
    I.mask = X.mask;
    I.target = X.target;
    I.w = X.window;
}

// Copy one described tile's bytes into smem (vectors past the unit's end are
// not loaded).
__device__ __forceinline__ void stage_described(uint32_t* sw, const TileInfo& I) {
    const uint32_t nvec = I.nvec;
    const uint64_t src = I.src;
    for (uint32_t v = threadIdx.x; v < nvec; v += blockDim.x) cp_async16(sw + 4 * v, src + 16ull * v);
}

// Instances (the planner orders the sliding units this way):
//   <20, MD5>: tiles [0, sliding_tiles_w20), MD5 units with w = 20;
//   <0, MD5>:  tiles [sliding_tiles_w20, sliding_tiles_md5), other MD5 units;
//   <0, SHA1>: tiles [sliding_tiles_md5, sliding_tiles), SHA-1 units, any w.
// The next tile's bytes are copied into the other half of a double buffer
// while the current tile is hashed.  A CTA's tiles are described in chunks of
// kDescChunk, one tile per thread of the first two warps (each finds its
// tile's unit by binary search), into a double-buffered table: chunk c + 1 is
// written at the first tile of chunk c, into the half that chunk c - 1 used
// and the previous iteration's closing barrier retired; it is first read a
// chunk later.  No thread does per-tile bookkeeping for the others.
// Resident CTAs per SM the window kernel is compiled for (sets its register
// budget: 65536 / (256 * blocks)).  Eight (32 registers) was measured fastest
// on B300 with 2048-offset tiles (8 windows per thread).
#ifndef CRYSTAL_WIN_MIN_BLOCKS
#define CRYSTAL_WIN_MIN_BLOCKS 8
#endif
constexpr uint32_t kDescChunk = 64;
static_assert(kDescChunk <= kWinThreads, "one describing thread per tile of a chunk");

template <int W, class H, int MINB>
__global__ void __launch_bounds__(kWinThreads, MINB) k_sliding_windows(crystal_batch* B, uint32_t one) {
    __shared__ __align__(16) uint32_t sw[2][kStageWords];
    __shared__ TileInfo desc[2][kDescChunk];
    const uint32_t ns = B->n_sliding;
    const crystal_unit* U = units_of(B) + B->n_direct;
    const bool sha = H::kWords == 5;
    const uint64_t lo = sha ? B->sliding_tiles_md5 : (W == 20 ? 0 : B->sliding_tiles_w20);
    const uint64_t hi = sha ? B->sliding_tiles : (W == 20 ? B->sliding_tiles_w20 : B->sliding_tiles_md5);
    const uint64_t G = gridDim.x;
    const uint64_t t0 = lo + blockIdx.x;  // the CTA's tile k is t0 + k G
    if (t0 >= hi) return;
    // describe the CTA's tiles [c kDescChunk, (c + 1) kDescChunk) into desc[c & 1]
    auto describe_chunk = [&](uint32_t c) {
        if (threadIdx.x < kDescChunk) {
            const uint64_t g = t0 + ((uint64_t)c * kDescChunk + threadIdx.x) * G;
            if (g < hi) describe_tile(desc[c & 1][threadIdx.x], U, ns, g);
        }
    };
    describe_chunk(0);
    __syncthreads();
    stage_described(sw[0], desc[0][0]);
    cp_async_commit();
    int buf = 0;
    uint32_t k = 0;
    for (uint64_t t = t0; t < hi; t += G, ++k) {
        if (k % kDescChunk == 0) describe_chunk(k / kDescChunk + 1);
        const uint32_t k1 = k + 1;
        if (t + G < hi) stage_described(sw[buf ^ 1], desc[(k1 / kDescChunk) & 1][k1 % kDescChunk]);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const TileInfo& I = desc[(k / kDescChunk) & 1][k % kDescChunk];
        const uint32_t delta = I.delta, lim = I.lim;
        const uint32_t w = W > 0 ? (uint32_t)W : I.w;
        uint32_t mine;
        if constexpr (W == 20) {
            mine = tile_windows20<H>(sw[buf], delta, lim, I.mask, I.target, one);
        } else if (H::kWords == 5 && w == 20) {
            // SHA-1 units with the common window: padding words fold at compile time
            mine = tile_windows20<H>(sw[buf], delta, lim, I.mask, I.target, one);
        } else {
            mine = tile_windows<W, H>(sw[buf], delta, lim, w, I.mask, I.target, one);
        }
        const uint32_t lane = threadIdx.x & 31;
        if (lane < (uint32_t)kWinPerThread) {
            const uint32_t word = (threadIdx.x >> 5) * kWinPerThread + lane;
            if (word < I.words) reinterpret_cast<uint32_t*>(I.out)[word] = mine;
        }
        __syncthreads();
        buf ^= 1;
    }
    cp_async_wait<0>();
}

// ---- K4: chunk ends and per-chunk segment table ------------------------------

template <int NT>
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t* sh, uint64_t& total) {
    // sh holds NT/32 + 1 entries
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint64_t s = lane < NT / 32 ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < NT / 32) sh[lane] = s;  // inclusive warp totals
    }
    __syncthreads();
    const uint64_t before = (warp > 0 ? sh[warp - 1] : 0) + x - v;
    total = sh[NT / 32 - 1];
    __syncthreads();
    return before;
}

__device__ __forceinline__ uint64_t warp_sum(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ uint64_t warp_inclusive_scan(uint64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Exclusive scan of one value per warp over the block's warps: returns this
// warp's start; total receives the block's sum.  sh holds NT/32 + 1 entries.
template <int NT>
__device__ __forceinline__ uint64_t warp_starts(uint64_t warp_total, uint64_t* sh, uint64_t& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = NT / 32;
    if (lane == 0) sh[warp] = warp_total;
    __syncthreads();
    if (warp == 0) {
        const uint64_t v = lane < NW ? sh[lane] : 0;
        const uint64_t x = warp_inclusive_scan(v);
        if (lane < NW) sh[lane] = x - v;
        if (lane == NW - 1) sh[NW] = x;
    }
    __syncthreads();
    const uint64_t start = sh[warp];
    total = sh[NW];
    __syncthreads();
    return start;
}

// Bitmap words a warp reads per pass iteration: each lane loads four 16-byte
// vectors, vector r of the warp covering words [128 r, 128 r + 128).
constexpr uint32_t kChunkWarpWords = 512;

// Words [j, j + 4) of the bitmap, zero past `words`; j is a multiple of 4, so
// every such group has the alignment `al` (address mod 16) of the bitmap,
// which picks the widest load allowed (the output buffer is only 4-byte
// aligned in general).
__device__ __forceinline__ uint4 bitmap_vec(const uint32_t* bm, uint64_t j, uint64_t words, uint32_t al) {
    if (j + 4 <= words) {
        if (al == 0) return *reinterpret_cast<const uint4*>(bm + j);
        if ((al & 7) == 0) {
            const uint2 a = *reinterpret_cast<const uint2*>(bm + j);
            const uint2 b = *reinterpret_cast<const uint2*>(bm + j + 2);
            return make_uint4(a.x, a.y, b.x, b.y);
        }
        return make_uint4(bm[j], bm[j + 1], bm[j + 2], bm[j + 3]);
    }
    uint4 v = make_uint4(0, 0, 0, 0);
    if (j < words) v.x = bm[j];
    if (j + 1 < words) v.y = bm[j + 1];
    if (j + 2 < words) v.z = bm[j + 2];
    return v;
}

__device__ __forceinline__ uint32_t popc4(uint4 v) {
    return __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
}

// One CTA per sliding unit.  Each warp owns a contiguous range of bitmap words
// (then of chunks) and reads it kChunkWarpWords words per iteration with
// vector loads (coalesced, four in flight per lane); prefix counts inside a
// warp come from shuffles, across warps from one scan of the warp totals.
__global__ void __launch_bounds__(kChunkThreads) k_sliding_chunks(crystal_batch* B) {
    __shared__ uint64_t sh[kChunkThreads / 32 + 1];
    constexpr uint32_t NW = kChunkThreads / 32;
    const uint32_t ns = B->n_sliding;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    crystal_unit* U = units_of(B) + B->n_direct;
    for (uint32_t u = blockIdx.x; u < ns; u += gridDim.x) {
        const crystal_unit X = U[u];
        const uint64_t n = X.n;
        const uint64_t words = (n + 31) >> 5;
        const uint64_t fixed = 8 + 4 * words;
        uint32_t* hdr = reinterpret_cast<uint32_t*>(X.out);
        const uint32_t* bm = hdr + 2;
        const uint32_t al = (uint32_t)(reinterpret_cast<uint64_t>(bm) & 15);
        uint32_t* seg_prefix = reinterpret_cast<uint32_t*>(X.scratch);
        if (X.out_cap < fixed) {
            if (threadIdx.x == 0) {
                atomicOr(&B->status, kDevBadRecord);
                U[u].seg_base = 0;
            }
            continue;
        }
        const uint64_t cap = (X.out_cap - fixed) / record_bytes(X);
        // pass 1: boundaries per warp range (ranges are whole iterations)
        const uint64_t iters = (words + NW * kChunkWarpWords - 1) / (NW * kChunkWarpWords);
        const uint64_t w0 = (uint64_t)warp * iters * kChunkWarpWords;
        const uint64_t w1 = min(words, w0 + iters * kChunkWarpWords);
        uint32_t cnt = 0;
        for (uint64_t j0 = w0; j0 < w1; j0 += kChunkWarpWords) {
            uint4 v[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) v[r] = bitmap_vec(bm, j0 + 128 * r + 4 * lane, w1, al);
#pragma unroll
            for (int r = 0; r < 4; ++r) cnt += popc4(v[r]);
        }
        uint64_t pop;
        uint64_t k = warp_starts<kChunkThreads>(warp_sum(cnt), sh, pop);
        bool last_set = false;
        if (n >= X.window) {
            const uint64_t i = n - X.window;
            last_set = (bm[i >> 5] >> (i & 31)) & 1u;
        }
        const uint64_t n_chunks = pop + (last_set ? 0 : 1);
        const bool fits = n_chunks <= cap;
        if (threadIdx.x == 0) {
            hdr[0] = (uint32_t)n_chunks;
            hdr[1] = fits ? 0u : 1u;
        }
        if (!fits) {
            if (threadIdx.x == 0) {
                seg_prefix[0] = 0;  // no chunk segments to hash
                U[u].seg_base = 0;
            }
            __syncthreads();
            continue;
        }
        // pass 2: chunk ends, in bit order
        uint32_t* ends = hdr + 2 + words;
        for (uint64_t j0 = w0; j0 < w1; j0 += kChunkWarpWords) {
            uint4 v[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) v[r] = bitmap_vec(bm, j0 + 128 * r + 4 * lane, w1, al);
            // per-vector counts fit 16 bits even summed over the warp (<= 4096)
            const uint32_t c01 = popc4(v[0]) | (popc4(v[1]) << 16);
            const uint32_t c23 = popc4(v[2]) | (popc4(v[3]) << 16);
            const uint32_t i01 = (uint32_t)warp_inclusive_scan(c01);
            const uint32_t i23 = (uint32_t)warp_inclusive_scan(c23);
            const uint32_t t01 = __shfl_sync(0xffffffffu, i01, 31), t23 = __shfl_sync(0xffffffffu, i23, 31);
            const uint32_t tot[4] = {t01 & 0xffffu, t01 >> 16, t23 & 0xffffu, t23 >> 16};
            const uint32_t exc[4] = {(i01 - c01) & 0xffffu, (i01 - c01) >> 16, (i23 - c23) & 0xffffu,
                                     (i23 - c23) >> 16};
            uint64_t before = k;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                uint64_t pos = before + exc[r];
                const uint32_t x4[4] = {v[r].x, v[r].y, v[r].z, v[r].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    uint32_t x = x4[e];
                    const uint64_t j = j0 + 128 * r + 4 * lane + e;
                    while (x) {
                        const int b = __ffs(x) - 1;
                        x &= x - 1;
                        ends[pos++] = (uint32_t)(32 * j + b + X.window);
                    }
                }
                before += tot[r];
            }
            k = before;
        }
        if (threadIdx.x == 0 && !last_set) ends[n_chunks - 1] = (uint32_t)n;
        __syncthreads();
        // pass 3: segments per chunk, exclusive prefix into the scratch table
        const uint32_t S = X.seg_bytes;
        const uint64_t cper = (((n_chunks + NW - 1) / NW) + 31) & ~uint64_t(31);
        const uint64_t c0 = min(n_chunks, (uint64_t)warp * cper), c1 = min(n_chunks, c0 + cper);
        uint64_t segs = 0;
        for (uint64_t c = c0 + lane; c < c1; c += 32) segs += num_segments(ends[c] - (c ? ends[c - 1] : 0u), S);
        uint64_t total_segs;
        uint64_t run = warp_starts<kChunkThreads>(warp_sum(segs), sh, total_segs);
        for (uint64_t b0 = c0; b0 < c1; b0 += 32) {
            const uint64_t c = b0 + lane;
            const uint64_t m = c < c1 ? num_segments(ends[c] - (c ? ends[c - 1] : 0u), S) : 0;
            const uint64_t incl = warp_inclusive_scan(m);
            if (c < c1) seg_prefix[c] = (uint32_t)(run + incl - m);
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (threadIdx.x == 0) {
            seg_prefix[n_chunks] = (uint32_t)total_segs;
            U[u].seg_base = (uint32_t)total_segs;  // a count here; k_chunk_seg_scan makes it a start
        }
        __syncthreads();
    }
}

// ---- K4b: where each unit's chunk segments start ---------------------------

// One block: turns the per-unit chunk-segment counts K4 left in seg_base into
// exclusive starts and stores the batch total.
__global__ void __launch_bounds__(kScanThreads) k_chunk_seg_scan(crystal_batch* B) {
    __shared__ uint64_t scan_sh[kScanThreads / 32 + 1];
    const uint32_t ns = B->n_sliding;
    crystal_unit* U = units_of(B) + B->n_direct;
    uint64_t carry = 0;
    for (uint32_t lo = 0; lo < ns; lo += kScanThreads) {
        const uint32_t i = lo + threadIdx.x;
        const uint64_t v = i < ns ? U[i].seg_base : 0;
        uint64_t total;
        const uint64_t before = block_exclusive_scan<kScanThreads>(v, scan_sh, total);
        if (i < ns) U[i].seg_base = (uint32_t)(carry + before);
        carry += total;
    }
    if (threadIdx.x == 0) {
        if (carry >> 32) {  // starts no longer fit 32 bits: hash no chunk segment, flag the batch
            atomicOr(&B->status, kDevBadRecord);
            carry = 0;
        }
        B->chunk_segments = carry;
    }
}

// Scratch of a sliding unit: u32 seg_prefix[cap + 1], then 16-byte aligned
// segment digests.
__device__ __forceinline__ uint8_t* chunk_digest_area(const crystal_unit& X, uint64_t cap) {
    return reinterpret_cast<uint8_t*>(X.scratch) + ((4 * (cap + 1) + 15) & ~uint64_t(15));
}

// ---- K5a: chunk segment digests ---------------------------------------------

// One thread per chunk segment of the whole batch: the unit comes from the
// starts K4b wrote, the chunk from the unit's segment table.  Neighbouring
// lanes hash neighbouring segments, which keeps the DRAM streams of a warp
// close together (dealing segments round-robin over CTAs was measured twice as
// slow).  Chunks start at arbitrary byte offsets, hence the single-path
// loader; the kernel is bound by the integer ALU pipe (staging its blocks
// through shared memory to have more in flight was measured slower).
#ifndef CRYSTAL_DIGEST_MIN_BLOCKS
#define CRYSTAL_DIGEST_MIN_BLOCKS 5
#endif
__global__ void __launch_bounds__(kChunkSegThreads, CRYSTAL_DIGEST_MIN_BLOCKS) k_chunk_segments(crystal_batch* B,
                                                                                          uint32_t one) {
    const uint32_t ns = B->n_sliding;
    const crystal_unit* U = units_of(B) + B->n_direct;
    const uint64_t total = B->chunk_segments;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
        uint32_t lo = 0, hi = ns;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (U[mid].seg_base <= g) lo = mid; else hi = mid;
        }
        const crystal_unit X = U[lo];
        const uint32_t t = (uint32_t)(g - X.seg_base);
        const uint64_t words = (X.n + 31) >> 5;
        const uint64_t fixed = 8 + 4 * words;
        const uint32_t* hdr = reinterpret_cast<const uint32_t*>(X.out);
        const uint32_t n_chunks = hdr[0];
        const uint64_t cap = (X.out_cap - fixed) / record_bytes(X);
        const uint32_t* ends = hdr + 2 + words;
        const uint32_t* seg_prefix = reinterpret_cast<const uint32_t*>(X.scratch);
        uint32_t clo = 0, chi = n_chunks;  // chunk: last with seg_prefix[c] <= t
        while (chi - clo > 1) {
            const uint32_t mid = (clo + chi) >> 1;
            if (seg_prefix[mid] <= t) clo = mid; else chi = mid;
        }
        const uint32_t S = X.seg_bytes;
        const uint64_t start = clo == 0 ? 0 : ends[clo - 1];
        const uint64_t end = ends[clo];
        const uint64_t off = start + (uint64_t)(t - seg_prefix[clo]) * S;
        const uint64_t len = end > off ? (end - off < S ? end - off : S) : 0;
        digest_to<CRYSTAL_FMA_SEGMENTS, true>(X, reinterpret_cast<const uint8_t*>(X.in) + off, len,
                                              chunk_digest_area(X, cap) + (uint64_t)digest_bytes(X) * t, one);
    }
}

// ---- K5b: chunk digests ------------------------------------------------------

__global__ void __launch_bounds__(kDigestThreads) k_chunk_outer(crystal_batch* B, uint32_t one) {
    const uint32_t ns = B->n_sliding;
    const crystal_unit* U = units_of(B) + B->n_direct;
    for (uint32_t u = blockIdx.x; u < ns; u += gridDim.x) {
        const crystal_unit X = U[u];
        const uint64_t words = (X.n + 31) >> 5;
        const uint64_t fixed = 8 + 4 * words;
        if (X.out_cap < fixed) continue;
        uint32_t* hdr = reinterpret_cast<uint32_t*>(X.out);
        if (hdr[1] & 1u) continue;
        const uint32_t n_chunks = hdr[0];
        const uint64_t cap = (X.out_cap - fixed) / record_bytes(X);
        const uint32_t* seg_prefix = reinterpret_cast<const uint32_t*>(X.scratch);
        const uint8_t* dig = chunk_digest_area(X, cap);
        uint8_t* out_dig = reinterpret_cast<uint8_t*>(hdr + 2 + words + n_chunks);
        const uint64_t D = digest_bytes(X);
        for (uint32_t c = threadIdx.x; c < n_chunks; c += blockDim.x) {
            const uint32_t s0 = seg_prefix[c], s1 = seg_prefix[c + 1];
            digest_to<CRYSTAL_FMA_OUTER>(X, dig + D * s0, D * (s1 - s0), out_dig + D * c, one);
        }
    }
}

// ---- batch descriptor in, status out, without DMA ------------------------------

__global__ void __launch_bounds__(256) k_fetch_descriptor(const uint4* __restrict__ src, uint4* __restrict__ dst,
                                                          uint32_t n16) {
    constexpr int kIn = 4;  // loads in flight per thread
    for (uint32_t b = 0; b < n16; b += kIn * blockDim.x) {
        uint4 v[kIn];
#pragma unroll
        for (int k = 0; k < kIn; ++k) {
            const uint32_t i = b + k * blockDim.x + threadIdx.x;
            if (i < n16) v[k] = src[i];
        }
#pragma unroll
        for (int k = 0; k < kIn; ++k) {
            const uint32_t i = b + k * blockDim.x + threadIdx.x;
            if (i < n16) dst[i] = v[k];
        }
    }
}

__global__ void k_post_status(const crystal_batch* d, uint32_t* host_status) {
    *host_status = d->status;
    __threadfence_system();
}

// ---- the dummy kernel of the overhead experiment ----------------------------

__global__ void k_nop() {}

// ---- integer-pipe microbenchmarks (crystal_alu_probe) --------------------------
//
// Register-resident loops that measure what the hashing kernels are bound by:
// the window hash itself with no memory traffic or bookkeeping (kinds MD5 and
// SHA-1: eight 20-byte windows per thread per iteration, their message words
// taken from a 12-word ring of registers the way the window kernel shares
// them), and single-instruction chains that load one pipe (LOP3, funnel shift,
// three-input add, integer multiply-add), or two alternately.  Eight
// independent chains per thread keep every scheduler supplied.  The result is
// written only if it equals `magic`, so no work can be dropped.

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

template <class H>
__device__ __forceinline__ uint32_t probe_windows(uint32_t (&M)[12], uint32_t one) {
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        uint32_t X[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) X[k] = 0;
#pragma unroll
        for (int k = 0; k < 5; ++k) X[k] = M[j + k];
        X[5] = 0x80u;
        X[14] = 8u * 20;
        acc ^= window_first_word<H>(X, 20u, one);
    }
    return acc;
}

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) k_alu_probe(uint32_t iters, uint32_t one, uint32_t magic,
                                                             uint32_t* sink) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    if constexpr (KIND == CRYSTAL_PROBE_MD5_WINDOWS || KIND == CRYSTAL_PROBE_SHA1_WINDOWS) {
        uint32_t M[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) M[k] = tid * 0x9E3779B9u + (uint32_t)k * 0x85EBCA6Bu;
        for (uint32_t it = 0; it < iters; ++it) {
            const uint32_t a = KIND == CRYSTAL_PROBE_MD5_WINDOWS ? probe_windows<MD5Hash>(M, one)
                                                                : probe_windows<SHA1Hash>(M, one);
#pragma unroll
            for (int k = 0; k < 12; ++k) M[k] += a;
            acc ^= a;
        }
    } else {
        uint32_t x[kProbeChains];
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) x[c] = tid + (uint32_t)c * 0x01000193u;
        const uint32_t y = tid ^ 0x5bd1e995u, z = tid * 3u + 1u;
        for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
            for (int r = 0; r < 8; ++r) {
#pragma unroll
                for (int c = 0; c < kProbeChains; ++c) {
                    uint32_t v = x[c];
                    if constexpr (KIND == CRYSTAL_PROBE_LOP3) {
                        asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(v) : "r"(y), "r"(z));
                    } else if constexpr (KIND == CRYSTAL_PROBE_SHF) {
                        asm volatile("shf.l.wrap.b32 %0, %0, %0, 7;" : "+r"(v));
                    } else if constexpr (KIND == CRYSTAL_PROBE_IADD3) {
                        asm volatile("{\n\t.reg .u32 t;\n\tadd.u32 t, %0, %1;\n\tadd.u32 %0, t, %2;\n\t}"
                                     : "+r"(v) : "r"(y), "r"(z));
                    } else if constexpr (KIND == CRYSTAL_PROBE_IMAD) {
                        asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(v) : "r"(one), "r"(z));
                    } else {  // CRYSTAL_PROBE_LOP3_IMAD: one of each, alternately
                        if (r & 1) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(v) : "r"(one), "r"(z));
                        else asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(v) : "r"(y), "r"(z));
                    }
                    x[c] = v;
                }
            }
        }
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) acc ^= x[c];
    }
    if (acc == magic) sink[0] = acc;
}

// ---- launch geometry -----------------------------------------------------------

// The window-kernel instances (SHA-1 needs more registers for its 16-word
// schedule: four CTAs per SM).  The w = 20 MD5 instance also exists at a
// 64-register budget (four CTAs per SM), a launch-geometry choice.
constexpr auto kWin20 = k_sliding_windows<20, MD5Hash, CRYSTAL_WIN_MIN_BLOCKS>;
constexpr auto kWin20Wide = k_sliding_windows<20, MD5Hash, 4>;
constexpr auto kWinAny = k_sliding_windows<0, MD5Hash, CRYSTAL_WIN_MIN_BLOCKS>;
#ifndef CRYSTAL_SHA1_WIN_MIN_BLOCKS
#define CRYSTAL_SHA1_WIN_MIN_BLOCKS 4
#endif
constexpr auto kWinSha1 = k_sliding_windows<0, SHA1Hash, CRYSTAL_SHA1_WIN_MIN_BLOCKS>;

template <class H>
const void* seg_kernel(int threads) {
    return threads == 64 ? (const void*)k_direct_segments<H, 64>
                         : threads == 256 ? (const void*)k_direct_segments<H, 256> : (const void*)k_direct_segments<H, 128>;
}

// Resident CTAs per SM of each kernel at each choice, per device.
struct Occupancy {
    int sms = 0;
    int seg[3] = {}, seg_sha1[3] = {};  // 64, 128, 256 threads
    int win20 = 0, win20_wide = 0, win = 0, win_sha1 = 0, digest = 0;
};

constexpr int kMaxDevices = 64;
Occupancy g_occ[kMaxDevices];
std::once_flag g_occ_once[kMaxDevices];

int resident(const void* fn, int threads) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, 0);
    return occ > 0 ? occ : 1;
}

int seg_index(int threads) { return threads == 64 ? 0 : threads == 256 ? 2 : 1; }

const Occupancy* occupancy() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::call_once(g_occ_once[dev], [dev] {
        Occupancy o;
        cudaDeviceGetAttribute(&o.sms, cudaDevAttrMultiProcessorCount, dev);
        for (int t : {64, 128, 256}) {
            o.seg[seg_index(t)] = resident(seg_kernel<MD5Hash>(t), t);
            o.seg_sha1[seg_index(t)] = resident(seg_kernel<SHA1Hash>(t), t);
        }
        o.win20 = resident((const void*)kWin20, kWinThreads);
        o.win20_wide = resident((const void*)kWin20Wide, kWinThreads);
        o.win = resident((const void*)kWinAny, kWinThreads);
        o.win_sha1 = resident((const void*)kWinSha1, kWinThreads);
        o.digest = resident((const void*)k_chunk_segments, kChunkSegThreads);
        g_occ[dev] = o;
    });
    return g_occ[dev].sms > 0 ? &g_occ[dev] : nullptr;
}

// CTAs per SM: the request (0 = as many as fit), never more than fit.
int per_sm(uint32_t want, int fit) { return want == 0 || (int)want > fit ? fit : (int)want; }

LaunchGeom g_default[kMaxDevices];
std::once_flag g_default_once[kMaxDevices];

const LaunchGeom* default_geometry() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::call_once(g_default_once[dev], [] {
        int d = 0;
        cudaGetDevice(&d);
        crystal_geometry zero{};
        make_geometry(&zero, &g_default[d]);
    });
    return g_default[dev].sms > 0 ? &g_default[dev] : nullptr;
}

// Passed to every hashing kernel as its `one` argument (see md5::add_on_fma).
uint32_t g_one = 1;

// After each launch: a launch error stops the sequence, so a kernel that
// depends on a failed one is never queued behind it.
int launched(int kernels) {
    if (cudaGetLastError() != cudaSuccess) return CRYSTAL_EDEVICE;
    if (!tl_capturing) g_kernel_launches.fetch_add((uint64_t)kernels, std::memory_order_relaxed);
    return CRYSTAL_OK;
}

const LaunchGeom* resolve(const LaunchGeom* g) { return g ? g : default_geometry(); }

template <class H>
void launch_seg(const LaunchGeom* g, int blocks, crystal_batch* b, cudaStream_t s) {
    switch (g->seg_threads) {
        case 64: k_direct_segments<H, 64><<<blocks, 64, 0, s>>>(b, g_one); break;
        case 256: k_direct_segments<H, 256><<<blocks, 256, 0, s>>>(b, g_one); break;
        default: k_direct_segments<H, 128><<<blocks, 128, 0, s>>>(b, g_one); break;
    }
}

}  // namespace

int make_geometry(const crystal_geometry* in, LaunchGeom* out) {
    if (!in || !out) return CRYSTAL_EINVAL;
    if (in->reserved) return CRYSTAL_EINVAL;
    const int threads = in->seg_threads ? (int)in->seg_threads : 128;
    if (threads != 64 && threads != 128 && threads != 256) return CRYSTAL_EINVAL;
    if (in->win_registers && in->win_registers != 32 && in->win_registers != 64) return CRYSTAL_EINVAL;
    if (in->seg_ctas_per_sm > 64 || in->win_ctas_per_sm > 64 || in->digest_ctas_per_sm > 64) return CRYSTAL_EINVAL;
    const Occupancy* o = occupancy();
    if (!o) return CRYSTAL_EDEVICE;
    LaunchGeom g;
    g.sms = o->sms;
    g.seg_threads = threads;
    g.seg_per_sm = per_sm(in->seg_ctas_per_sm, o->seg[seg_index(threads)]);
    g.seg_blocks = o->sms * g.seg_per_sm;
    g.seg_sha1_blocks = o->sms * per_sm(in->seg_ctas_per_sm, o->seg_sha1[seg_index(threads)]);
    g.win20_wide = in->win_registers == 64;
    g.win_per_sm = per_sm(in->win_ctas_per_sm, g.win20_wide ? o->win20_wide : o->win20);
    g.win20_blocks = o->sms * g.win_per_sm;
    g.win_blocks = o->sms * per_sm(in->win_ctas_per_sm, o->win);
    g.win_sha1_blocks = o->sms * per_sm(in->win_ctas_per_sm, o->win_sha1);
    g.digest_per_sm = per_sm(in->digest_ctas_per_sm, o->digest);
    g.digest_blocks = o->sms * g.digest_per_sm;
    g.outer_blocks = o->sms * 2;
    g.unit_blocks = o->sms * 2;
    *out = g;
    return CRYSTAL_OK;
}

void describe_geometry(const LaunchGeom& g, crystal_geometry* out) {
    out->seg_threads = (uint32_t)g.seg_threads;
    out->seg_ctas_per_sm = (uint32_t)g.seg_per_sm;
    out->win_ctas_per_sm = (uint32_t)g.win_per_sm;
    out->win_registers = g.win20_wide ? 64u : 32u;
    out->digest_ctas_per_sm = (uint32_t)g.digest_per_sm;
    out->reserved = 0;
}

int launch_nop(cudaStream_t s) {
    k_nop<<<1, 32, 0, s>>>();
    return launched(1);
}

int launch_fetch_descriptor(const void* host_dev, crystal_batch* dst, uint64_t bytes, cudaStream_t s) {
    if ((bytes & 15) || ((uint64_t)host_dev & 15) || ((uint64_t)dst & 15)) return CRYSTAL_EINVAL;
    k_fetch_descriptor<<<1, 256, 0, s>>>(static_cast<const uint4*>(host_dev), reinterpret_cast<uint4*>(dst),
                                         (uint32_t)(bytes / 16));
    return launched(1);
}

int launch_post_status(const crystal_batch* d, uint32_t* host_status_dev, cudaStream_t s) {
    k_post_status<<<1, 1, 0, s>>>(d, host_status_dev);
    return launched(1);
}

int launch_direct_segments(crystal_batch* b, cudaStream_t s, const LaunchGeom* geom) {
    const LaunchGeom* g = resolve(geom);
    if (!g) return CRYSTAL_EDEVICE;
    launch_seg<MD5Hash>(g, g->seg_blocks, b, s);
    if (launched(1) != CRYSTAL_OK) return CRYSTAL_EDEVICE;
    launch_seg<SHA1Hash>(g, g->seg_sha1_blocks, b, s);
    return launched(1);
}

int launch_direct_outer(crystal_batch* b, cudaStream_t s, const LaunchGeom* geom) {
    const LaunchGeom* g = resolve(geom);
    if (!g) return CRYSTAL_EDEVICE;
    k_direct_outer<<<g->outer_blocks, kDigestThreads, 0, s>>>(b, g_one);
    return launched(1);
}

int launch_sliding_windows(crystal_batch* b, cudaStream_t s, const LaunchGeom* geom) {
    const LaunchGeom* g = resolve(geom);
    if (!g) return CRYSTAL_EDEVICE;
    if (g->win20_wide) kWin20Wide<<<g->win20_blocks, kWinThreads, 0, s>>>(b, g_one);
    else kWin20<<<g->win20_blocks, kWinThreads, 0, s>>>(b, g_one);
    if (launched(1) != CRYSTAL_OK) return CRYSTAL_EDEVICE;
    kWinAny<<<g->win_blocks, kWinThreads, 0, s>>>(b, g_one);
    if (launched(1) != CRYSTAL_OK) return CRYSTAL_EDEVICE;
    kWinSha1<<<g->win_sha1_blocks, kWinThreads, 0, s>>>(b, g_one);
    return launched(1);
}

int launch_sliding_chunks(crystal_batch* b, cudaStream_t s, const LaunchGeom* geom) {
    const LaunchGeom* g = resolve(geom);
    if (!g) return CRYSTAL_EDEVICE;
    k_sliding_chunks<<<g->unit_blocks, kChunkThreads, 0, s>>>(b);
    if (launched(1) != CRYSTAL_OK) return CRYSTAL_EDEVICE;
    k_chunk_seg_scan<<<1, kScanThreads, 0, s>>>(b);
    return launched(1);
}

int launch_sliding_digests(crystal_batch* b, cudaStream_t s, const LaunchGeom* geom) {
    const LaunchGeom* g = resolve(geom);
    if (!g) return CRYSTAL_EDEVICE;
    k_chunk_segments<<<g->digest_blocks, kChunkSegThreads, 0, s>>>(b, g_one);
    if (launched(1) != CRYSTAL_OK) return CRYSTAL_EDEVICE;
    k_chunk_outer<<<g->unit_blocks, kDigestThreads, 0, s>>>(b, g_one);
    return launched(1);
}

// ---- direct hashing that allocates nothing ------------------------------------
//
// Some callers cannot allocate device memory on their data path: a host
// thread in a storage or network data path with a fixed latency budget
// (cudaMalloc and cudaFree may synchronise the whole device and take
// milliseconds), or a process whose free device memory has all been handed
// to another allocator, so a new cudaMalloc would fail.  For them the batch
// descriptor and the segment digests of crystal_md5_direct_noalloc live in
// this fixed array instead of caller-allocated scratch.  Every GPU that loads
// the library holds it until the process exits.

static __device__ __align__(256) uint8_t g_noalloc_scratch[CRYSTAL_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of g_noalloc_scratch per device, looked up once per device.
uint8_t* g_noalloc_addr[kMaxDevices];
std::once_flag g_noalloc_once[kMaxDevices];
cudaError_t g_noalloc_err[kMaxDevices];

// Writes the batch header and one record per unit (units back to back in
// d_in, digests of unit u at d_out + 16u) into the fixed array.
__global__ void k_noalloc_describe(crystal_batch* B, uint64_t in, uint64_t unit_bytes, uint32_t n_units,
                                   uint32_t seg_bytes, uint64_t out, uint64_t digests) {
    const uint64_t m = num_segments(unit_bytes, seg_bytes);
    crystal_unit* U = units_of(B);
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n_units; u += gridDim.x * blockDim.x) {
        crystal_unit x;
        x.in = in + (uint64_t)u * unit_bytes;
        x.n = unit_bytes;
        x.out = out + 16ull * u;
        x.scratch = digests + 16ull * m * u;
        x.work_begin = m * u;
        x.out_cap = 16;
        x.seg_bytes = seg_bytes;
        x.window = 0;
        x.kind = CRYSTAL_KIND_MD5_DIRECT;
        x.mask = 0;
        x.target = 0;
        x.seg_base = 0;
        U[u] = x;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        B->n_direct = n_units;
        B->n_sliding = 0;
        B->direct_segments = m * n_units;
        B->direct_segments_md5 = m * n_units;
        B->sliding_tiles = 0;
        B->window_max = 0;
        B->status = 0;
        B->sliding_tiles_w20 = 0;
        B->chunk_segments = 0;
        B->sliding_tiles_md5 = 0;
    }
}

}  // namespace

}  // namespace crystal

using namespace crystal;

extern "C" {

int crystal_md5_direct_noalloc(const void* d_in, uint64_t unit_bytes, uint32_t n_units, uint32_t segment_bytes,
                               void* d_digests, void* stream) {
    if (n_units == 0) return CRYSTAL_OK;
    if (!d_in || !d_digests || segment_bytes == 0 || (reinterpret_cast<uint64_t>(d_digests) & 3))
        return CRYSTAL_EINVAL;
    const uint64_t m = segments_of(unit_bytes, segment_bytes);
    const uint64_t desc = align_up(crystal_batch_bytes(n_units), 256);
    // bound every term before multiplying so the size test cannot wrap
    if (m > CRYSTAL_NOALLOC_SCRATCH_BYTES || n_units > CRYSTAL_NOALLOC_SCRATCH_BYTES) return CRYSTAL_EINVAL;
    if (desc + 16 * m * (uint64_t)n_units > CRYSTAL_NOALLOC_SCRATCH_BYTES) return CRYSTAL_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CRYSTAL_EDEVICE;
    std::call_once(g_noalloc_once[dev], [dev] {
        void* p = nullptr;
        g_noalloc_err[dev] = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        g_noalloc_addr[dev] = g_noalloc_err[dev] == cudaSuccess ? static_cast<uint8_t*>(p) : nullptr;
    });
    if (g_noalloc_err[dev] != cudaSuccess || !g_noalloc_addr[dev]) return CRYSTAL_EDEVICE;
    const LaunchGeom* g = default_geometry();
    if (!g) return CRYSTAL_EDEVICE;
    crystal_batch* B = reinterpret_cast<crystal_batch*>(g_noalloc_addr[dev]);
    const uint64_t digests = reinterpret_cast<uint64_t>(g_noalloc_addr[dev]) + desc;
    cudaStream_t s = (cudaStream_t)stream;
    const int threads = 256;
    const int blocks = (int)((n_units + threads - 1) / threads < 1024 ? (n_units + threads - 1) / threads : 1024);
    // a launch error left pending by earlier work on this thread is reported
    // (and cleared) here, before anything is queued
    if (cudaGetLastError() != cudaSuccess) return CRYSTAL_EDEVICE;
    k_noalloc_describe<<<blocks, threads, 0, s>>>(B, reinterpret_cast<uint64_t>(d_in), unit_bytes, n_units,
                                                   segment_bytes, reinterpret_cast<uint64_t>(d_digests), digests);
    // the hashing kernels read the descriptor this launch writes: queue them
    // only if it was queued
    if (launched(1) != CRYSTAL_OK) return CRYSTAL_EDEVICE;
    launch_seg<MD5Hash>(g, g->seg_blocks, B, s);
    if (launched(1) != CRYSTAL_OK) return CRYSTAL_EDEVICE;
    k_direct_outer<<<g->outer_blocks, kDigestThreads, 0, s>>>(B, g_one);
    return launched(1);
}

int crystal_launch_direct_segments(const crystal_batch* b, void* stream) {
    if (!b) return CRYSTAL_EINVAL;
    return launch_direct_segments(const_cast<crystal_batch*>(b), (cudaStream_t)stream);
}

int crystal_launch_direct_outer(const crystal_batch* b, void* stream) {
    if (!b) return CRYSTAL_EINVAL;
    return launch_direct_outer(const_cast<crystal_batch*>(b), (cudaStream_t)stream);
}

int crystal_launch_direct(const crystal_batch* b, void* stream) {
    int st = crystal_launch_direct_segments(b, stream);
    if (st != CRYSTAL_OK) return st;
    return crystal_launch_direct_outer(b, stream);
}

int crystal_launch_sliding_windows(const crystal_batch* b, void* stream) {
    if (!b) return CRYSTAL_EINVAL;
    return launch_sliding_windows(const_cast<crystal_batch*>(b), (cudaStream_t)stream);
}

int crystal_launch_sliding_chunks(const crystal_batch* b, void* stream) {
    if (!b) return CRYSTAL_EINVAL;
    return launch_sliding_chunks(const_cast<crystal_batch*>(b), (cudaStream_t)stream);
}

int crystal_launch_sliding_digests(const crystal_batch* b, void* stream) {
    if (!b) return CRYSTAL_EINVAL;
    return launch_sliding_digests(const_cast<crystal_batch*>(b), (cudaStream_t)stream);
}

int crystal_launch_sliding(const crystal_batch* b, void* stream) {
    int st = crystal_launch_sliding_windows(b, stream);
    if (st == CRYSTAL_OK) st = crystal_launch_sliding_chunks(b, stream);
    if (st == CRYSTAL_OK) st = crystal_launch_sliding_digests(b, stream);
    return st;
}

int crystal_launch_batch(const crystal_batch* b, void* stream) {
    int st = crystal_launch_direct(b, stream);
    if (st == CRYSTAL_OK) st = crystal_launch_sliding(b, stream);
    return st;
}

uint64_t crystal_kernel_launches(void) { return g_kernel_launches.load(std::memory_order_relaxed); }

int crystal_alu_probe(int kind, uint32_t ctas_per_sm, uint32_t iters, uint32_t magic, uint32_t* d_sink,
                      void* stream, uint64_t* work) {
    if (!d_sink || ctas_per_sm == 0 || ctas_per_sm > 64 || iters == 0) return CRYSTAL_EINVAL;
    const LaunchGeom* g = default_geometry();
    if (!g) return CRYSTAL_EDEVICE;
    const uint32_t blocks = (uint32_t)g->sms * ctas_per_sm;
    const uint64_t threads = (uint64_t)blocks * kProbeThreads;
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t units;
    switch (kind) {
        case CRYSTAL_PROBE_MD5_WINDOWS:
            k_alu_probe<CRYSTAL_PROBE_MD5_WINDOWS><<<blocks, kProbeThreads, 0, s>>>(iters, g_one, magic, d_sink);
            units = threads * iters * 8;  // windows
            break;
        case CRYSTAL_PROBE_SHA1_WINDOWS:
            k_alu_probe<CRYSTAL_PROBE_SHA1_WINDOWS><<<blocks, kProbeThreads, 0, s>>>(iters, g_one, magic, d_sink);
            units = threads * iters * 8;
            break;
        case CRYSTAL_PROBE_LOP3:
            k_alu_probe<CRYSTAL_PROBE_LOP3><<<blocks, kProbeThreads, 0, s>>>(iters, g_one, magic, d_sink);
            units = threads * iters * 8 * kProbeChains;  // instructions (per thread)
            break;
        case CRYSTAL_PROBE_SHF:
            k_alu_probe<CRYSTAL_PROBE_SHF><<<blocks, kProbeThreads, 0, s>>>(iters, g_one, magic, d_sink);
            units = threads * iters * 8 * kProbeChains;
            break;
        case CRYSTAL_PROBE_IADD3:
            k_alu_probe<CRYSTAL_PROBE_IADD3><<<blocks, kProbeThreads, 0, s>>>(iters, g_one, magic, d_sink);
            units = threads * iters * 8 * kProbeChains;
            break;
        case CRYSTAL_PROBE_IMAD:
            k_alu_probe<CRYSTAL_PROBE_IMAD><<<blocks, kProbeThreads, 0, s>>>(iters, g_one, magic, d_sink);
            units = threads * iters * 8 * kProbeChains;
            break;
        case CRYSTAL_PROBE_LOP3_IMAD:
            k_alu_probe<CRYSTAL_PROBE_LOP3_IMAD><<<blocks, kProbeThreads, 0, s>>>(iters, g_one, magic, d_sink);
            units = threads * iters * 8 * kProbeChains;
            break;
        default:
            return CRYSTAL_EINVAL;
    }
    if (work) *work = units;
    return launched(1);
}

int crystal_direct_job(const void* h_in, void* d_in, uint64_t in_size, void* h_out, const void* d_out,
                       uint64_t out_size, void* stream) {
    if ((in_size && (!h_in || !d_in)) || (out_size && (!h_out || !d_out))) return CRYSTAL_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (in_size && cudaMemcpyAsync(d_in, h_in, in_size, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return CRYSTAL_EDEVICE;
    if (launch_nop(s) != CRYSTAL_OK) return CRYSTAL_EDEVICE;
    if (out_size && cudaMemcpyAsync(h_out, d_out, out_size, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return CRYSTAL_EDEVICE;
    // poll for completion, as the runtime's master thread does
    cudaError_t e;
    while ((e = cudaStreamQuery(s)) == cudaErrorNotReady) std::this_thread::yield();
    return e == cudaSuccess ? CRYSTAL_OK : CRYSTAL_EDEVICE;
}

}  // extern "C"
