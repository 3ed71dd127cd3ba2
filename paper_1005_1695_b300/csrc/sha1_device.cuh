// SHA-1 device core for sm_103a (FIPS 180-4, sections 5.1.1 and 6.1.2).
//
// Message words are big-endian; the 16-word schedule is kept in a circular
// window in registers (W[t mod 16]), extended in place from step 16 on.  All
// 80 steps are unrolled at compile time so the round function and constant
// of each step are fixed and padding words known at compile time fold away.
#pragma once

#include <stdint.h>

#include <utility>

// Which adds of a step issue on the FMA pipe: 0 none (the compiler's choice),
// 1 the add of the round function f, 2 that and the add of a <<< 5.  SHA-1's
// two rotates and its logic op only run on the integer ALU pipe; on B300, 1
// was measured 1.2% faster than 0 in the window kernel and 4.6% in the chunk
// digests, and 2 slower than both.
#ifndef CRYSTAL_SHA1_FMA
#define CRYSTAL_SHA1_FMA 1
#endif

namespace crystal {
namespace sha1 {

// x * one + y issued on the FMA pipe (`one` is a run-time 1 the compiler
// cannot fold), leaving the integer ALU pipe to the rotates and logic ops.
__device__ __forceinline__ uint32_t add_fma(uint32_t x, uint32_t one, uint32_t y) {
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(x), "r"(one), "r"(y));
    return d;
}

constexpr uint32_t kH0 = 0x67452301u;
constexpr uint32_t kH1 = 0xefcdab89u;
constexpr uint32_t kH2 = 0x98badcfeu;
constexpr uint32_t kH3 = 0x10325476u;
constexpr uint32_t kH4 = 0xc3d2e1f0u;

// FIPS 180-4 4.2.1: one constant per 20 steps.
__host__ __device__ constexpr uint32_t kK(int t) {
    return t < 20 ? 0x5a827999u : t < 40 ? 0x6ed9eba1u : t < 60 ? 0x8f1bbcdcu : 0xca62c1d6u;
}

__device__ __forceinline__ uint32_t rotl(uint32_t x, int s) { return __funnelshift_l(x, x, s); }

__device__ __forceinline__ uint32_t bswap(uint32_t x) { return __byte_perm(x, 0, 0x0123); }

// Step t: schedule word (extended from step 16 on), round function
// Ch / Parity / Maj / Parity, then (a, b, c, d, e) <- (T, a, b<<<30, c, d).
template <int T>
__device__ __forceinline__ void step(uint32_t& a, uint32_t& b, uint32_t& c, uint32_t& d, uint32_t& e,
                                     uint32_t (&W)[16], uint32_t one) {
    if constexpr (T >= 16) {
        W[T & 15] = rotl(W[(T - 3) & 15] ^ W[(T - 8) & 15] ^ W[(T - 14) & 15] ^ W[T & 15], 1);
    }
    uint32_t f;
    if constexpr (T < 20) {
        f = d ^ (b & (c ^ d));            // Ch
    } else if constexpr (T < 40 || T >= 60) {
        f = b ^ c ^ d;                    // Parity
    } else {
        f = (b & c) | (d & (b | c));      // Maj
    }
    uint32_t t;
    if constexpr (CRYSTAL_SHA1_FMA == 2) {
        t = add_fma(rotl(a, 5), one, add_fma(f, one, e + (kK(T) + W[T & 15])));
    } else if constexpr (CRYSTAL_SHA1_FMA == 1) {
        t = add_fma(f, one, rotl(a, 5) + (e + (kK(T) + W[T & 15])));
    } else {
        t = rotl(a, 5) + f + (e + (kK(T) + W[T & 15]));
    }
    e = d;
    d = c;
    c = rotl(b, 30);
    b = a;
    a = t;
}

template <int... T>
__device__ __forceinline__ void steps_seq(std::integer_sequence<int, T...>, uint32_t& a, uint32_t& b, uint32_t& c,
                                          uint32_t& d, uint32_t& e, uint32_t (&W)[16], uint32_t one) {
    (step<T>(a, b, c, d, e, W, one), ...);
}

// One block: W holds the 16 big-endian message words and is consumed.
__device__ __forceinline__ void compress(uint32_t (&st)[5], uint32_t (&W)[16], uint32_t one) {
    uint32_t a = st[0], b = st[1], c = st[2], d = st[3], e = st[4];
    steps_seq(std::make_integer_sequence<int, 80>{}, a, b, c, d, e, W, one);
    st[0] += a;
    st[1] += b;
    st[2] += c;
    st[3] += d;
    st[4] += e;
}

// H0 of a one-block message (W consumed), i.e. big-endian digest bytes 0..3.
__device__ __forceinline__ uint32_t first_word_one_block(uint32_t (&W)[16], uint32_t one) {
    uint32_t a = kH0, b = kH1, c = kH2, d = kH3, e = kH4;
    steps_seq(std::make_integer_sequence<int, 80>{}, a, b, c, d, e, W, one);
    return kH0 + a;
}

}  // namespace sha1
}  // namespace crystal
