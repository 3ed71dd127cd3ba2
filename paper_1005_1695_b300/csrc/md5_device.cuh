// MD5 device core for sm_103a (RFC 1321, section 3).
//
// Every step is unrolled at compile time: the additive constant, the
// rotation and the message-word index of step I are template constants, so
// message words that are known at compile time (the padding words of a
// short fixed-length message) fold into immediates and their adds vanish.
// Rotations are single funnel shifts; the round functions are single
// three-input logic ops.
#pragma once

#include <stdint.h>

#include <utility>

namespace crystal {
namespace md5 {

// RFC 1321 3.4: T[1..64], written out as the RFC tabulates them.
__host__ __device__ constexpr uint32_t kT(int i) {
    constexpr uint32_t t[64] = {
        0xd76aa478u, 0xe8c7b756u, 0x242070dbu, 0xc1bdceeeu, 0xf57c0fafu, 0x4787c62au, 0xa8304613u,
        0xfd469501u, 0x698098d8u, 0x8b44f7afu, 0xffff5bb1u, 0x895cd7beu, 0x6b901122u, 0xfd987193u,
        0xa679438eu, 0x49b40821u, 0xf61e2562u, 0xc040b340u, 0x265e5a51u, 0xe9b6c7aau, 0xd62f105du,
        0x02441453u, 0xd8a1e681u, 0xe7d3fbc8u, 0x21e1cde6u, 0xc33707d6u, 0xf4d50d87u, 0x455a14edu,
        0xa9e3e905u, 0xfcefa3f8u, 0x676f02d9u, 0x8d2a4c8au, 0xfffa3942u, 0x8771f681u, 0x6d9d6122u,
        0xfde5380cu, 0xa4beea44u, 0x4bdecfa9u, 0xf6bb4b60u, 0xbebfbc70u, 0x289b7ec6u, 0xeaa127fau,
        0xd4ef3085u, 0x04881d05u, 0xd9d4d039u, 0xe6db99e5u, 0x1fa27cf8u, 0xc4ac5665u, 0xf4292244u,
        0x432aff97u, 0xab9423a7u, 0xfc93a039u, 0x655b59c3u, 0x8f0ccc92u, 0xffeff47du, 0x85845dd1u,
        0x6fa87e4fu, 0xfe2ce6e0u, 0xa3014314u, 0x4e0811a1u, 0xf7537e82u, 0xbd3af235u, 0x2ad7d2bbu,
        0xeb86d391u};
    return t[i];
}

// Left-rotation of step i: four amounts per round, cycled.
__host__ __device__ constexpr int kRot(int i) {
    constexpr int r[16] = {7, 12, 17, 22, 5, 9, 14, 20, 4, 11, 16, 23, 6, 10, 15, 21};
    return r[(i >> 4) * 4 + (i & 3)];
}

// Message word of step i: X[i], X[5i+1], X[3i+5], X[7i] (mod 16) by round.
__host__ __device__ constexpr int kWord(int i) {
    return i < 16 ? i : i < 32 ? (5 * i + 1) & 15 : i < 48 ? (3 * i + 5) & 15 : (7 * i) & 15;
}

constexpr uint32_t kIV0 = 0x67452301u;
constexpr uint32_t kIV1 = 0xefcdab89u;
constexpr uint32_t kIV2 = 0x98badcfeu;
constexpr uint32_t kIV3 = 0x10325476u;

__device__ __forceinline__ uint32_t rotl(uint32_t x, int s) { return __funnelshift_l(x, x, s); }

// x * one + y with `one` a run-time 1 the compiler cannot see through: the
// add then issues as an integer multiply-add on the FMA pipe instead of the
// integer ALU pipe.  On sm_103a the ALU pipe takes one warp instruction every
// two cycles per scheduler and bounds this hash; moving the add that joins
// the round function into the running sum to the FMA pipe was measured
// faster (moving the other adds, or the rotate, was measured slower in the
// window kernel).
__device__ __forceinline__ uint32_t add_on_fma(uint32_t x, uint32_t one, uint32_t y) {
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(x), "r"(one), "r"(y));
    return d;
}

// One step: b' = b + ((a + f(b,c,d) + X[k] + T[i]) <<< s), then the register
// names rotate (a, b, c, d) <- (d, b', b, c).  The sum not involving b is
// formed first so the dependent chain through b is f -> add -> rotate -> add.
template <int I, bool FMA = true>
__device__ __forceinline__ void step(uint32_t& a, uint32_t& b, uint32_t& c, uint32_t& d,
                                     const uint32_t (&X)[16], uint32_t one) {
    uint32_t f;
    if constexpr (I < 16) {
        f = d ^ (b & (c ^ d));          // F = (b & c) | (~b & d)
    } else if constexpr (I < 32) {
        f = c ^ (d & (b ^ c));          // G = (b & d) | (c & ~d)
    } else if constexpr (I < 48) {
        f = b ^ c ^ d;                  // H
    } else {
        f = c ^ (b | ~d);               // I
    }
    uint32_t t;
    if constexpr (FMA) {
        const uint32_t pre = a + (kT(I) + X[kWord(I)]);
        t = add_on_fma(f, one, pre);
    } else {
        const uint32_t pre = a + (kT(I) + X[kWord(I)]);
        t = pre + f;
    }
    const uint32_t nb = b + rotl(t, kRot(I));
    a = d;
    d = c;
    c = b;
    b = nb;
}

template <bool FMA, int... I>
__device__ __forceinline__ void steps_seq(std::integer_sequence<int, I...>, uint32_t& a, uint32_t& b,
                                          uint32_t& c, uint32_t& d, const uint32_t (&X)[16], uint32_t one) {
    (step<I, FMA>(a, b, c, d, X, one), ...);
}

// The first N steps of the compression function.  FMA: the round-function
// add goes to the FMA pipe (more throughput when many chains share the ALU
// pipe); without it every add stays on the ALU pipe (lower latency for a
// single chain).
template <int N, bool FMA = true>
__device__ __forceinline__ void steps(uint32_t& a, uint32_t& b, uint32_t& c, uint32_t& d,
                                      const uint32_t (&X)[16], uint32_t one) {
    steps_seq<FMA>(std::make_integer_sequence<int, N>{}, a, b, c, d, X, one);
}

// Full compression of one 16-word block into the chaining state.
template <bool FMA = true>
__device__ __forceinline__ void compress(uint32_t (&st)[4], const uint32_t (&X)[16], uint32_t one) {
    uint32_t a = st[0], b = st[1], c = st[2], d = st[3];
    steps<64, FMA>(a, b, c, d, X, one);
    st[0] += a;
    st[1] += b;
    st[2] += c;
    st[3] += d;
}

// First digest word of a one-block message: after step 61 the register A
// holds its final value (steps 62..64 only update D, C, B), so three steps
// are skipped.  Returns A + IV_A, i.e. LE32 of digest bytes 0..3.
__device__ __forceinline__ uint32_t first_word_one_block(const uint32_t (&X)[16], uint32_t one) {
    uint32_t a = kIV0, b = kIV1, c = kIV2, d = kIV3;
    steps<61>(a, b, c, d, X, one);
    return kIV0 + b;
}

__device__ __forceinline__ void init(uint32_t (&st)[4]) {
    st[0] = kIV0;
    st[1] = kIV1;
    st[2] = kIV2;
    st[3] = kIV3;
}

// ---- loads ----------------------------------------------------------------

__device__ __forceinline__ uint4 ldg_stream16(const void* p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ uint32_t ldg32(const uint32_t* p) { return __ldg(p); }

}  // namespace md5
}  // namespace crystal
