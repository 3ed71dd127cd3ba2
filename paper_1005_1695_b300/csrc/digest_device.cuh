// Hash-generic message digests over global memory, for MD5 and SHA-1.
//
// One thread hashes one message (a segment, a chunk segment or a list of
// digests): whole 64-byte blocks are loaded with 16-byte vector loads (the
// next block's loads in flight while the current one compresses), words are
// shifted into place when the message does not start on a 16-byte boundary,
// and the tail block gets the padding and the 64-bit bit length.  The hash
// type supplies the state, the compression, the word byte order (MD5 reads
// little-endian words, SHA-1 big-endian) and where the length goes.
#pragma once

#include <stdint.h>

#include "md5_device.cuh"
#include "sha1_device.cuh"

namespace crystal {

// 16-byte asynchronous global -> shared copy (L2 only), its commit and wait.
__device__ __forceinline__ void cp_async16(void* smem_dst, uint64_t gmem_src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

struct MD5Hash {
    static constexpr int kWords = 4;
    static constexpr int kBytes = 16;
    __device__ static void init(uint32_t (&st)[5]) {
        st[0] = md5::kIV0;
        st[1] = md5::kIV1;
        st[2] = md5::kIV2;
        st[3] = md5::kIV3;
        st[4] = 0;
    }
    template <bool FMA>
    __device__ static void compress(uint32_t (&st)[5], uint32_t (&X)[16], uint32_t one) {
        uint32_t s4[4] = {st[0], st[1], st[2], st[3]};
        md5::compress<FMA>(s4, X, one);
        st[0] = s4[0];
        st[1] = s4[1];
        st[2] = s4[2];
        st[3] = s4[3];
    }
    __device__ static uint32_t word(uint32_t memory_order) { return memory_order; }
    __device__ static void length(uint32_t (&X)[16], uint64_t bits) {
        X[14] = (uint32_t)bits;
        X[15] = (uint32_t)(bits >> 32);
    }
    // digest word i in memory byte order
    __device__ static uint32_t out_word(uint32_t s) { return s; }
};

struct SHA1Hash {
    static constexpr int kWords = 5;
    static constexpr int kBytes = 20;
    __device__ static void init(uint32_t (&st)[5]) {
        st[0] = sha1::kH0;
        st[1] = sha1::kH1;
        st[2] = sha1::kH2;
        st[3] = sha1::kH3;
        st[4] = sha1::kH4;
    }
    template <bool FMA>
    __device__ static void compress(uint32_t (&st)[5], uint32_t (&X)[16], uint32_t one) {
        sha1::compress(st, X, one);
    }
    __device__ static uint32_t word(uint32_t memory_order) { return sha1::bswap(memory_order); }
    __device__ static void length(uint32_t (&X)[16], uint64_t bits) {
        X[14] = (uint32_t)(bits >> 32);
        X[15] = (uint32_t)bits;
    }
    __device__ static uint32_t out_word(uint32_t s) { return sha1::bswap(s); }
};

// Tail of a message of len bytes whose last len mod 64 bytes start at ta:
// those bytes, then 0x80, zeros and the 64-bit bit length.
template <class H, bool FMA>
__device__ __forceinline__ void digest_tail(uint64_t ta, uint64_t len, uint32_t (&st)[5], uint32_t (&X)[16],
                                            uint32_t one) {
    const uint32_t rem = (uint32_t)(len & 63);
    const uint32_t sh = (uint32_t)(ta & 3) * 8;
    const uint32_t* q = reinterpret_cast<const uint32_t*>(ta & ~uint64_t(3));
    const uint32_t nwords = ((uint32_t)(ta & 3) + rem + 3) >> 2;  // aligned words holding tail bytes
    uint32_t x[17];
#pragma unroll
    for (int k = 0; k < 17; ++k) x[k] = (uint32_t)k < nwords ? md5::ldg32(q + k) : 0u;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        uint32_t w = __funnelshift_r(x[k], x[k + 1], sh);
        const int have = (int)rem - 4 * k;  // message bytes in this word
        if (have <= 0) {
            w = 0;
        } else if (have < 4) {
            w &= (1u << (8 * have)) - 1u;
        }
        if (have >= 0 && have < 4) w |= 0x80u << (8 * have);
        X[k] = H::word(w);
    }
    const uint64_t bits = len << 3;
    if (rem < 56) {
        H::length(X, bits);
        H::template compress<FMA>(st, X, one);
    } else {
        H::template compress<FMA>(st, X, one);
#pragma unroll
        for (int k = 0; k < 16; ++k) X[k] = 0;
        H::length(X, bits);
        H::template compress<FMA>(st, X, one);
    }
}

// Digest of len bytes at p (any alignment) in global memory into st[0..kWords).
// Bytes outside [p, p + len) are read only inside aligned 16-byte blocks that
// also hold a byte of the message, and never used.
template <class H, bool FMA = true>
__device__ __forceinline__ void digest_global(const uint8_t* p, uint64_t len, uint32_t (&st)[5], uint32_t one) {
    H::init(st);
    const uint64_t addr = reinterpret_cast<uint64_t>(p);
    const uint64_t full = len >> 6;
    uint32_t X[16];
    if ((addr & 15) == 0) {
        const uint8_t* q = p;
        uint4 nx[4];
        if (full) {
#pragma unroll
            for (int v = 0; v < 4; ++v) nx[v] = md5::ldg_stream16(q + 16 * v);
        }
        for (uint64_t blk = 0; blk < full; ++blk) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                X[4 * v + 0] = H::word(nx[v].x);
                X[4 * v + 1] = H::word(nx[v].y);
                X[4 * v + 2] = H::word(nx[v].z);
                X[4 * v + 3] = H::word(nx[v].w);
            }
            q += 64;
            if (blk + 1 < full) {
#pragma unroll
                for (int v = 0; v < 4; ++v) nx[v] = md5::ldg_stream16(q + 16 * v);
            }
            H::template compress<FMA>(st, X, one);
        }
    } else {
        // Five aligned 16-byte loads cover the block (each holds at least one
        // byte of it); whole words are shifted into place by a two-level select
        // on (addr mod 16) / 4, the rest by a funnel shift.
        const uint32_t o = (uint32_t)(addr & 15);
        const uint32_t wq = o >> 2;
        const uint32_t sh = (o & 3) * 8;
        const uint8_t* q = reinterpret_cast<const uint8_t*>(addr - o);
        uint4 nx[5];
        if (full) {
#pragma unroll
            for (int v = 0; v < 5; ++v) nx[v] = md5::ldg_stream16(q + 16 * v);
        }
        for (uint64_t blk = 0; blk < full; ++blk) {
            uint32_t w[20];
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                w[4 * v + 0] = nx[v].x;
                w[4 * v + 1] = nx[v].y;
                w[4 * v + 2] = nx[v].z;
                w[4 * v + 3] = nx[v].w;
            }
            q += 64;
            if (blk + 1 < full) {
#pragma unroll
                for (int v = 0; v < 5; ++v) nx[v] = md5::ldg_stream16(q + 16 * v);
            }
            uint32_t y1[19];
#pragma unroll
            for (int k = 0; k < 19; ++k) y1[k] = (wq & 1) ? w[k + 1] : w[k];
            uint32_t y[17];
#pragma unroll
            for (int k = 0; k < 17; ++k) y[k] = (wq & 2) ? y1[k + 2] : y1[k];
#pragma unroll
            for (int k = 0; k < 16; ++k) X[k] = H::word(__funnelshift_r(y[k], y[k + 1], sh));
            H::template compress<FMA>(st, X, one);
        }
    }
    digest_tail<H, FMA>(addr + (full << 6), len, st, X, one);
}

// digest_global for messages that mostly start off a 16-byte boundary (chunk
// segments start wherever a content-defined cut fell): one code path for
// every alignment, so the lanes of a warp never split between an aligned and
// an unaligned loop.  Each block is assembled from five aligned 16-byte
// vectors (the fifth is loaded only when the start is unaligned, so no vector
// without a message byte is read).
template <class H, bool FMA = true>
__device__ __forceinline__ void digest_global_any(const uint8_t* p, uint64_t len, uint32_t (&st)[5], uint32_t one) {
    H::init(st);
    const uint64_t addr = reinterpret_cast<uint64_t>(p);
    const uint64_t full = len >> 6;
    const uint32_t o = (uint32_t)(addr & 15);
    const uint32_t wq = o >> 2;
    const uint32_t sh = (o & 3) * 8;
    const uint8_t* q = reinterpret_cast<const uint8_t*>(addr - o);
    uint32_t X[16];
    uint4 nx[5];
    if (full) {
#pragma unroll
        for (int v = 0; v < 4; ++v) nx[v] = md5::ldg_stream16(q + 16 * v);
        nx[4] = o ? md5::ldg_stream16(q + 64) : make_uint4(0, 0, 0, 0);
    }
    for (uint64_t blk = 0; blk < full; ++blk) {
        uint32_t w[20];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            w[4 * v + 0] = nx[v].x;
            w[4 * v + 1] = nx[v].y;
            w[4 * v + 2] = nx[v].z;
            w[4 * v + 3] = nx[v].w;
        }
        q += 64;
        if (blk + 1 < full) {
#pragma unroll
            for (int v = 0; v < 4; ++v) nx[v] = md5::ldg_stream16(q + 16 * v);
            nx[4] = o ? md5::ldg_stream16(q + 64) : make_uint4(0, 0, 0, 0);
        }
        uint32_t y1[19];
#pragma unroll
        for (int k = 0; k < 19; ++k) y1[k] = (wq & 1) ? w[k + 1] : w[k];
        uint32_t y[17];
#pragma unroll
        for (int k = 0; k < 17; ++k) y[k] = (wq & 2) ? y1[k + 2] : y1[k];
#pragma unroll
        for (int k = 0; k < 16; ++k) X[k] = H::word(__funnelshift_r(y[k], y[k + 1], sh));
        H::template compress<FMA>(st, X, one);
    }
    digest_tail<H, FMA>(addr + (full << 6), len, st, X, one);
}

// Store a digest (memory byte order) at a 4-byte aligned address.
template <class H>
__device__ __forceinline__ void store_digest(uint8_t* dst, const uint32_t (&st)[5]) {
    uint32_t* d = reinterpret_cast<uint32_t*>(dst);
#pragma unroll
    for (int i = 0; i < H::kWords; ++i) d[i] = H::out_word(st[i]);
}

}  // namespace crystal
