/*
 * CPU oracle for the CrystalGPU hashing hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * restatement of what the GPU path computes.  It is linked only by the test
 * suite, by the package's smoke check and by the benchmark's CPU-baseline
 * leg.  It shares no code, header, table or constant generator with the CUDA
 * path, and it never reads anything the CUDA path produced.
 *
 * What it computes (all arithmetic is unsigned 32-bit, no floating point on
 * the data path):
 *
 *   oracle_md5        MD5 as defined by RFC 1321 (section 3: padding, length,
 *                     4 rounds x 16 steps with F, G, H, I).  The sine-derived
 *                     constant table T[i] = floor(2^32 * |sin(i+1)|) is
 *                     computed at load time from that closed form, not typed.
 *   oracle_direct     StoreGPU-style "direct hashing" (named in Section 5.2 of
 *                     the CrystalGPU paper, defined here by its usual reading):
 *                     MD5 of each fixed-size segment, then one MD5 over the
 *                     concatenation of the segment digests.
 *   oracle_sliding    "sliding-window hashing" (the hashing-based primitives of
 *                     Section 2.2, content-addressable storage): MD5 of every
 *                     w-byte window, a boundary bit where the first digest
 *                     word matches a mask/target, cut positions at the end of
 *                     each marked window, and a direct hash per chunk.
 *   oracle_sha1       SHA-1 as defined by FIPS 180-4 (section 5.1.1 padding,
 *                     section 6.1.2: 80 steps over a 16-word message schedule
 *                     extended by the one-bit left rotation of the XOR of
 *                     four earlier words; big-endian words and length).  The
 *                     paper's own measurements use SHA-1 (Section 5.2).
 *   oracle_task       one job of the paper's job abstraction (Section 3,
 *                     Figures 2 and 3) executed synchronously: input bytes in,
 *                     output buffer in the library's documented layout out.
 *
 * Readings taken where the paper is silent (the paper gives no hash
 * definitions at all; it measures SHA1, the target here is MD5):
 *   - a segment shorter than S at the end of a unit is hashed as it is;
 *   - a unit with n <= S (including n = 0) has exactly one segment and still
 *     gets the outer MD5 over that single 16-byte digest;
 *   - the "first digest word" is the little-endian 32-bit word of digest
 *     bytes 0..3 (MD5's register A after the feed-forward);
 *   - the cut for a marked window at offset i is placed at i + w; the cut set
 *     is {i + w : bit i set} united with {n}, duplicates removed;
 *   - windows never cross unit edges; a unit with n < w has no windows and a
 *     single chunk [0, n);
 *   - the chunk digest is the segmented direct hash with S_chunk.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- MD5, RFC 1321 ------------------------------------------------------ */

/* T[i] = floor(4294967296 * |sin(i + 1)|), i = 0..63, radians (RFC 1321 3.4). */
static uint32_t T[64];

/* Per-round left-rotation amounts (RFC 1321 3.4, rounds 1..4). */
static const int ROT[4][4] = {
    {7, 12, 17, 22},
    {5, 9, 14, 20},
    {4, 11, 16, 23},
    {6, 10, 15, 21},
};

__attribute__((constructor)) static void oracle_init_table(void) {
    for (int i = 0; i < 64; i++) {
        double v = fabs(sin((double)(i + 1))) * 4294967296.0;
        T[i] = (uint32_t)floor(v);
    }
}

static uint32_t rotl32(uint32_t x, int s) { return (x << s) | (x >> (32 - s)); }

/* The four auxiliary functions of RFC 1321 3.4. */
static uint32_t fF(uint32_t x, uint32_t y, uint32_t z) { return (x & y) | (~x & z); }
static uint32_t fG(uint32_t x, uint32_t y, uint32_t z) { return (x & z) | (y & ~z); }
static uint32_t fH(uint32_t x, uint32_t y, uint32_t z) { return x ^ y ^ z; }
static uint32_t fI(uint32_t x, uint32_t y, uint32_t z) { return y ^ (x | ~z); }

/* One 64-byte block through the four rounds (RFC 1321 3.4).  Step i of round
 * r uses message word X[k] with k = i (r=0), 5i+1 (r=1), 3i+5 (r=2), 7i (r=3)
 * modulo 16, constant T[16r + i] and rotation ROT[r][i mod 4]; the registers
 * rotate (a, b, c, d) <- (d, a', b, c) after every step. */
static void md5_block(uint32_t st[4], const uint8_t blk[64]) {
    uint32_t X[16];
    for (int j = 0; j < 16; j++) {
        X[j] = (uint32_t)blk[4 * j] | ((uint32_t)blk[4 * j + 1] << 8) |
               ((uint32_t)blk[4 * j + 2] << 16) | ((uint32_t)blk[4 * j + 3] << 24);
    }
    uint32_t a = st[0], b = st[1], c = st[2], d = st[3];
    for (int r = 0; r < 4; r++) {
        for (int i = 0; i < 16; i++) {
            uint32_t f;
            int k;
            switch (r) {
            case 0: f = fF(b, c, d); k = i; break;
            case 1: f = fG(b, c, d); k = (5 * i + 1) % 16; break;
            case 2: f = fH(b, c, d); k = (3 * i + 5) % 16; break;
            default: f = fI(b, c, d); k = (7 * i) % 16; break;
            }
            uint32_t na = b + rotl32(a + f + X[k] + T[16 * r + i], ROT[r][i % 4]);
            a = d;
            d = c;
            c = b;
            b = na;
        }
    }
    st[0] += a;
    st[1] += b;
    st[2] += c;
    st[3] += d;
}

/* MD5 of len bytes (RFC 1321 3.1-3.5): append 0x80, zero-fill to 56 mod 64,
 * append the bit length as 64-bit little-endian, run every block from the
 * initial registers A=67452301 B=efcdab89 C=98badcfe D=10325476 (as the RFC
 * writes them, low byte first: 01 23 45 67 / 89 ab cd ef / fe dc ba 98 /
 * 76 54 32 10), output A, B, C, D low byte first. */
void oracle_md5(const uint8_t* msg, uint64_t len, uint8_t out[16]) {
    uint32_t st[4] = {0x67452301u, 0xefcdab89u, 0x98badcfeu, 0x10325476u};
    uint64_t full = len / 64;
    for (uint64_t b = 0; b < full; b++) md5_block(st, msg + 64 * b);
    uint8_t tail[128];
    uint64_t rem = len - 64 * full;
    memset(tail, 0, sizeof tail);
    if (rem) memcpy(tail, msg + 64 * full, (size_t)rem);
    tail[rem] = 0x80;
    uint64_t tail_len = (rem < 56) ? 64 : 128;
    uint64_t bits = len * 8;
    for (int j = 0; j < 8; j++) tail[tail_len - 8 + j] = (uint8_t)(bits >> (8 * j));
    md5_block(st, tail);
    if (tail_len == 128) md5_block(st, tail + 64);
    for (int j = 0; j < 4; j++) {
        out[4 * j + 0] = (uint8_t)(st[j]);
        out[4 * j + 1] = (uint8_t)(st[j] >> 8);
        out[4 * j + 2] = (uint8_t)(st[j] >> 16);
        out[4 * j + 3] = (uint8_t)(st[j] >> 24);
    }
}

/* Copy of the constant table, for the pin against the closed form. */
void oracle_md5_table(uint32_t out[64]) { memcpy(out, T, sizeof T); }

/* ---- SHA-1, FIPS 180-4 --------------------------------------------------- */

static uint32_t rotl32s(uint32_t x, int s) { return (x << s) | (x >> (32 - s)); }

/* One 512-bit block (FIPS 180-4 6.1.2): schedule W[0..79], then 80 steps
 * with Ch (0..19), Parity (20..39), Maj (40..59), Parity (60..79) and the
 * four constants of section 4.2.1. */
static void sha1_block(uint32_t H[5], const uint8_t blk[64]) {
    static const uint32_t K4[4] = {0x5a827999u, 0x6ed9eba1u, 0x8f1bbcdcu, 0xca62c1d6u};
    uint32_t W[80];
    for (int t = 0; t < 16; t++) {
        W[t] = ((uint32_t)blk[4 * t] << 24) | ((uint32_t)blk[4 * t + 1] << 16) |
               ((uint32_t)blk[4 * t + 2] << 8) | (uint32_t)blk[4 * t + 3];
    }
    for (int t = 16; t < 80; t++) W[t] = rotl32s(W[t - 3] ^ W[t - 8] ^ W[t - 14] ^ W[t - 16], 1);
    uint32_t a = H[0], b = H[1], c = H[2], d = H[3], e = H[4];
    for (int t = 0; t < 80; t++) {
        uint32_t f;
        if (t < 20) f = (b & c) ^ (~b & d);
        else if (t < 40) f = b ^ c ^ d;
        else if (t < 60) f = (b & c) ^ (b & d) ^ (c & d);
        else f = b ^ c ^ d;
        uint32_t T = rotl32s(a, 5) + f + e + K4[t / 20] + W[t];
        e = d;
        d = c;
        c = rotl32s(b, 30);
        b = a;
        a = T;
    }
    H[0] += a;
    H[1] += b;
    H[2] += c;
    H[3] += d;
    H[4] += e;
}

/* SHA-1 of len bytes (FIPS 180-4 5.1.1, 5.3.1, 6.1): append 0x80, zeros to
 * 56 mod 64, the 64-bit big-endian bit length; initial H of section 5.3.1;
 * digest = H0..H4, each big-endian. */
void oracle_sha1(const uint8_t* msg, uint64_t len, uint8_t out[20]) {
    uint32_t H[5] = {0x67452301u, 0xefcdab89u, 0x98badcfeu, 0x10325476u, 0xc3d2e1f0u};
    uint64_t full = len / 64;
    for (uint64_t b = 0; b < full; b++) sha1_block(H, msg + 64 * b);
    uint8_t tail[128];
    uint64_t rem = len - 64 * full;
    memset(tail, 0, sizeof tail);
    if (rem) memcpy(tail, msg + 64 * full, (size_t)rem);
    tail[rem] = 0x80;
    uint64_t tail_len = (rem < 56) ? 64 : 128;
    uint64_t bits = len * 8;
    for (int j = 0; j < 8; j++) tail[tail_len - 1 - j] = (uint8_t)(bits >> (8 * j));
    sha1_block(H, tail);
    if (tail_len == 128) sha1_block(H, tail + 64);
    for (int j = 0; j < 5; j++) {
        out[4 * j + 0] = (uint8_t)(H[j] >> 24);
        out[4 * j + 1] = (uint8_t)(H[j] >> 16);
        out[4 * j + 2] = (uint8_t)(H[j] >> 8);
        out[4 * j + 3] = (uint8_t)(H[j]);
    }
}

/* ---- hash selection ------------------------------------------------------ */

enum { HASH_MD5 = 0, HASH_SHA1 = 1 };

uint32_t oracle_digest_bytes(int hash) { return hash == HASH_SHA1 ? 20 : 16; }

static void digest(int hash, const uint8_t* msg, uint64_t len, uint8_t* out) {
    if (hash == HASH_SHA1) oracle_sha1(msg, len, out);
    else oracle_md5(msg, len, out);
}

/* ---- direct hashing ----------------------------------------------------- */

/* Number of segments of a unit of n bytes at segment size S (n = 0 counts as
 * one empty segment). */
uint64_t oracle_num_segments(uint64_t n, uint64_t S) {
    if (n == 0) return 1;
    return (n + S - 1) / S;
}

/* Direct(u, S) = H(H(seg_0) || H(seg_1) || ... || H(seg_{m-1})) for the hash
 * H (MD5 or SHA-1).  Returns 0, or -1 on a bad argument / allocation failure. */
int oracle_direct_hash(int hash, const uint8_t* u, uint64_t n, uint64_t S, uint8_t* out) {
    if (S == 0) return -1;
    const uint64_t D = oracle_digest_bytes(hash);
    uint64_t m = oracle_num_segments(n, S);
    uint8_t* cat = (uint8_t*)malloc((size_t)(D * m));
    if (!cat) return -1;
    for (uint64_t i = 0; i < m; i++) {
        uint64_t off = i * S;
        uint64_t len = (n - off < S) ? (n - off) : S;
        digest(hash, u + off, len, cat + D * i);
    }
    digest(hash, cat, D * m, out);
    free(cat);
    return 0;
}

int oracle_direct(const uint8_t* u, uint64_t n, uint64_t S, uint8_t out[16]) {
    return oracle_direct_hash(HASH_MD5, u, n, S, out);
}

/* ---- sliding-window hashing --------------------------------------------- */

/* Boundary bitmap: bit i (word i/32, bit i%32) is set iff window u[i, i+w)
 * exists (i <= n - w) and (LE32(MD5(window)[0..3]) & mask) == target.
 * The bitmap has ceil(n/32) words; all other bits are zero. */
void oracle_sliding_bitmap_hash(int hash, const uint8_t* u, uint64_t n, uint32_t w, uint32_t mask,
                                uint32_t target, uint32_t* bitmap) {
    uint64_t words = (n + 31) / 32;
    memset(bitmap, 0, (size_t)(4 * words));
    if (w == 0 || n < w) return;
    uint8_t h[20];
    for (uint64_t i = 0; i + w <= n; i++) {
        digest(hash, u + i, w, h);
        uint32_t word0 = (uint32_t)h[0] | ((uint32_t)h[1] << 8) | ((uint32_t)h[2] << 16) |
                         ((uint32_t)h[3] << 24);
        if ((word0 & mask) == target) bitmap[i / 32] |= 1u << (i % 32);
    }
}

void oracle_sliding_bitmap(const uint8_t* u, uint64_t n, uint32_t w, uint32_t mask, uint32_t target,
                           uint32_t* bitmap) {
    oracle_sliding_bitmap_hash(HASH_MD5, u, n, w, mask, target, bitmap);
}

/* Chunk ends from a bitmap: the sorted cut set {i + w : bit i} U {n} with
 * duplicates removed.  Writes up to cap ends; returns the number of chunks. */
uint64_t oracle_chunk_ends(const uint32_t* bitmap, uint64_t n, uint32_t w, uint32_t* ends,
                           uint64_t cap) {
    uint64_t k = 0;
    uint64_t last = 0;
    int have_last = 0;
    for (uint64_t i = 0; i < n; i++) {
        if (bitmap[i / 32] & (1u << (i % 32))) {
            uint64_t c = i + w;
            if (have_last && c == last) continue;
            if (k < cap) ends[k] = (uint32_t)c;
            k++;
            last = c;
            have_last = 1;
        }
    }
    if (!(have_last && last == n)) {
        if (k < cap) ends[k] = (uint32_t)n;
        k++;
    }
    return k;
}

/* ---- one job, output in the library's layout ----------------------------- */

enum { KIND_NOP = 0, KIND_MD5_DIRECT = 1, KIND_MD5_SLIDING = 2, KIND_SHA1_DIRECT = 3, KIND_SHA1_SLIDING = 4 };

/*
 * Runs one job synchronously and fills out[0 .. out_size).
 *   direct : out = Direct(u, seg_bytes) (16 bytes).
 *   sliding: out = u32 n_chunks | u32 flags | u32 bitmap[ceil(n/32)] |
 *            u32 chunk_end[n_chunks] | u8 digest[n_chunks][D]
 *            where digest[k] = Direct(u[c_{k-1}, c_k), chunk_seg_bytes) and D
 *            is the digest size (16 for MD5, 20 for SHA-1; kinds 3 and 4 are
 *            the SHA-1 counterparts of kinds 1 and 2).
 *            If the records do not fit, flags bit 0 is set, n_chunks still
 *            holds the needed count and no records are written.
 * Returns 0 on success, 1 on overflow, -1 on a bad argument.
 */
int oracle_task(int kind, const uint8_t* u, uint64_t n, uint32_t seg_bytes, uint32_t window,
                uint32_t mask, uint32_t target, uint32_t chunk_seg_bytes, uint8_t* out,
                uint64_t out_size) {
    const int hash = (kind == KIND_SHA1_DIRECT || kind == KIND_SHA1_SLIDING) ? HASH_SHA1 : HASH_MD5;
    const uint64_t D = oracle_digest_bytes(hash);
    if (kind == KIND_MD5_DIRECT || kind == KIND_SHA1_DIRECT) {
        if (out_size < D) return -1;
        return oracle_direct_hash(hash, u, n, seg_bytes, out);
    }
    if (kind != KIND_MD5_SLIDING && kind != KIND_SHA1_SLIDING) return -1;
    if (window == 0 || chunk_seg_bytes == 0) return -1;
    uint64_t words = (n + 31) / 32;
    uint64_t fixed = 8 + 4 * words;
    if (out_size < fixed) return -1;
    uint32_t* bitmap = (uint32_t*)malloc((size_t)(4 * words + 4));
    if (!bitmap) return -1;
    oracle_sliding_bitmap_hash(hash, u, n, window, mask, target, bitmap);
    uint64_t count = oracle_chunk_ends(bitmap, n, window, NULL, 0);
    uint64_t cap = (out_size - fixed) / (4 + D);
    uint32_t flags = 0;
    uint32_t hdr[2];
    hdr[0] = (uint32_t)count;
    memcpy(out + 8, bitmap, (size_t)(4 * words));
    free(bitmap);
    int status = 0;
    if (count > cap) {
        flags = 1;
        status = 1;
    } else {
        uint32_t* ends = (uint32_t*)malloc((size_t)(4 * count));
        if (!ends) return -1;
        /* recompute from the copied bitmap so the ends follow the stored bits */
        uint32_t* bm = (uint32_t*)malloc((size_t)(4 * words + 4));
        if (!bm) { free(ends); return -1; }
        memcpy(bm, out + 8, (size_t)(4 * words));
        oracle_chunk_ends(bm, n, window, ends, count);
        free(bm);
        uint8_t* rec = out + fixed;
        memcpy(rec, ends, (size_t)(4 * count));
        uint8_t* dig = rec + 4 * count;
        uint64_t start = 0;
        for (uint64_t k = 0; k < count; k++) {
            if (oracle_direct_hash(hash, u + start, ends[k] - start, chunk_seg_bytes, dig + D * k) != 0) {
                free(ends);
                return -1;
            }
            start = ends[k];
        }
        free(ends);
    }
    hdr[1] = flags;
    memcpy(out, hdr, 8);
    return status;
}
