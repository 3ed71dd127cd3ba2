// Host-side planning of a batch and the arena allocator behind the pools.
//
// The arena is the bookkeeping of the paper's buffer pool (Section 3: buffers
// pre-allocated once at init and handed out by job_get / job_put): one large
// region, carved into 256-byte-aligned blocks, best fit, freed blocks merged
// with their free neighbours.  It holds offsets only, so the same code serves
// the device arena and the pinned host arena, and runs without a GPU.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <unordered_map>

#include "crystal.h"
#include "crystal_internal.h"

using namespace crystal;

// Free blocks are indexed three ways: by offset (to merge neighbours), by
// (length, offset) (best fit), and in 64 buckets of lengths [2^k, 2^(k+1)),
// each ordered by offset, so that the lowest or highest block that fits is
// found from the first or last entry of the buckets that surely fit plus a
// short walk of the one bucket that may not -- not by walking every free
// block in address order.
struct crystal_arena {
    uint64_t size = 0;
    uint64_t align = 256;
    uint64_t used = 0;
    std::map<uint64_t, uint64_t> free_by_off;             // offset -> length
    std::set<std::pair<uint64_t, uint64_t>> free_by_len;  // (length, offset)
    std::set<uint64_t> bucket[64];                        // offsets of free blocks, by floor(log2 length)
    std::unordered_map<uint64_t, uint64_t> live;          // offset -> length
    std::mutex mu;

    static int bucket_of(uint64_t len) { return 63 - __builtin_clzll(len); }
    void insert_free(uint64_t off, uint64_t len) {
        free_by_off.emplace(off, len);
        free_by_len.emplace(len, off);
        bucket[bucket_of(len)].insert(off);
    }
    void erase_free(std::map<uint64_t, uint64_t>::iterator it) {
        free_by_len.erase({it->second, it->first});
        bucket[bucket_of(it->second)].erase(it->first);
        free_by_off.erase(it);
    }
    // Lowest (highest) free block of at least `want` bytes: buckets above
    // want's own hold only blocks that fit, so their first (last) offset is a
    // candidate; in want's own bucket, walk in offset order to the first block
    // that fits, stopping once past the best candidate.  false: none fits.
    bool extreme_fit(uint64_t want, bool lowest, uint64_t* off) const {
        const int kw = bucket_of(want);
        bool found = false;
        uint64_t best = 0;
        auto better = [&](uint64_t o) { return !found || (lowest ? o < best : o > best); };
        for (int k = kw + 1; k < 64; ++k) {
            if (bucket[k].empty()) continue;
            const uint64_t o = lowest ? *bucket[k].begin() : *bucket[k].rbegin();
            if (better(o)) {
                best = o;
                found = true;
            }
        }
        auto fits = [&](uint64_t o) { return free_by_off.find(o)->second >= want; };
        if (lowest) {
            for (auto it = bucket[kw].begin(); it != bucket[kw].end() && better(*it); ++it)
                if (fits(*it)) {
                    best = *it;
                    found = true;
                    break;
                }
        } else {
            for (auto it = bucket[kw].rbegin(); it != bucket[kw].rend() && better(*it); ++it)
                if (fits(*it)) {
                    best = *it;
                    found = true;
                    break;
                }
        }
        if (found) *off = best;
        return found;
    }
};

extern "C" {

int crystal_arena_create(uint64_t bytes, uint64_t alignment, crystal_arena** out) {
    if (!out || bytes == 0 || alignment == 0 || (alignment & (alignment - 1))) return CRYSTAL_EINVAL;
    bytes &= ~(alignment - 1);  // whole aligned blocks only, so blocks taken from the top stay aligned
    if (bytes == 0) return CRYSTAL_EINVAL;
    crystal_arena* a = new (std::nothrow) crystal_arena;
    if (!a) return CRYSTAL_ENOMEM;
    a->size = bytes;
    a->align = alignment;
    a->insert_free(0, bytes);
    *out = a;
    return CRYSTAL_OK;
}

int crystal_arena_alloc_at(crystal_arena* a, uint64_t bytes, int placement, uint64_t* offset) {
    if (!a || !offset || placement < CRYSTAL_ARENA_BEST_FIT || placement > CRYSTAL_ARENA_HIGHEST)
        return CRYSTAL_EINVAL;
    const uint64_t want = align_up(bytes ? bytes : 1, a->align);
    if (want < bytes) return CRYSTAL_EAGAIN;  // overflow
    std::lock_guard<std::mutex> lk(a->mu);
    uint64_t off = 0, len = 0;
    if (placement == CRYSTAL_ARENA_BEST_FIT) {
        auto it = a->free_by_len.lower_bound({want, 0});
        if (it == a->free_by_len.end()) return CRYSTAL_EAGAIN;
        len = it->first;
        off = it->second;
    } else {
        if (!a->extreme_fit(want, placement == CRYSTAL_ARENA_LOWEST, &off)) return CRYSTAL_EAGAIN;
        len = a->free_by_off.find(off)->second;
    }
    a->erase_free(a->free_by_off.find(off));
    uint64_t at = off;
    if (placement == CRYSTAL_ARENA_HIGHEST) {
        at = off + len - want;  // top of the block; the rest stays free below it
        if (len > want) a->insert_free(off, len - want);
    } else if (len > want) {
        a->insert_free(off + want, len - want);
    }
    a->live.emplace(at, want);
    a->used += want;
    *offset = at;
    return CRYSTAL_OK;
}

int crystal_arena_alloc_exact(crystal_arena* a, uint64_t offset, uint64_t bytes) {
    if (!a || (offset & (a->align - 1))) return CRYSTAL_EINVAL;
    const uint64_t want = align_up(bytes ? bytes : 1, a->align);
    if (want < bytes || offset > a->size || want > a->size - offset) return CRYSTAL_EAGAIN;
    std::lock_guard<std::mutex> lk(a->mu);
    auto it = a->free_by_off.upper_bound(offset);  // the free block starting at or below offset
    if (it == a->free_by_off.begin()) return CRYSTAL_EAGAIN;
    --it;
    const uint64_t off = it->first, len = it->second;
    if (off + len < offset + want) return CRYSTAL_EAGAIN;
    a->erase_free(it);
    if (offset > off) a->insert_free(off, offset - off);
    if (off + len > offset + want) a->insert_free(offset + want, off + len - offset - want);
    a->live.emplace(offset, want);
    a->used += want;
    return CRYSTAL_OK;
}

int crystal_arena_alloc(crystal_arena* a, uint64_t bytes, uint64_t* offset) {
    return crystal_arena_alloc_at(a, bytes, CRYSTAL_ARENA_BEST_FIT, offset);
}

int crystal_arena_free(crystal_arena* a, uint64_t offset) {
    if (!a) return CRYSTAL_EINVAL;
    std::lock_guard<std::mutex> lk(a->mu);
    auto lv = a->live.find(offset);
    if (lv == a->live.end()) return CRYSTAL_EINVAL;
    uint64_t off = lv->first, len = lv->second;
    a->live.erase(lv);
    a->used -= len;
    auto next = a->free_by_off.lower_bound(off);
    if (next != a->free_by_off.end() && next->first == off + len) {
        len += next->second;
        a->erase_free(next);
    }
    auto prev = a->free_by_off.lower_bound(off);
    if (prev != a->free_by_off.begin()) {
        --prev;
        if (prev->first + prev->second == off) {
            off = prev->first;
            len += prev->second;
            a->erase_free(prev);
        }
    }
    a->insert_free(off, len);
    return CRYSTAL_OK;
}

uint64_t crystal_arena_used(crystal_arena* a) {
    if (!a) return 0;
    std::lock_guard<std::mutex> lk(a->mu);
    return a->used;
}

uint64_t crystal_arena_largest_free(crystal_arena* a) {
    if (!a) return 0;
    std::lock_guard<std::mutex> lk(a->mu);
    return a->free_by_len.empty() ? 0 : a->free_by_len.rbegin()->first;
}

void crystal_arena_destroy(crystal_arena* a) { delete a; }

// ---- parameters and sizes -----------------------------------------------------

void crystal_params_default(crystal_hash_params* p) {
    if (!p) return;
    p->segment_bytes = 4096;
    p->window_bytes = 20;
    p->mask = 0x1FFF;
    p->target = 0x1FFF;
    p->chunk_segment_bytes = 4096;
    p->reserved = 0;
}

uint64_t crystal_sliding_out_bytes(uint64_t in_size, uint64_t max_chunks) {
    return sliding_fixed_bytes(in_size) + 20 * max_chunks;
}

uint64_t crystal_out_bytes_for_chunks(int kind, uint64_t in_size, uint64_t max_chunks) {
    if (!kind_is_sliding(kind)) return 0;
    return sliding_fixed_bytes(in_size) + (4 + digest_bytes_of(kind)) * max_chunks;
}

uint64_t crystal_out_bytes(int kind, uint64_t in_size, const crystal_hash_params* params) {
    crystal_hash_params p;
    crystal_params_default(&p);
    if (params) {
        if (params->window_bytes) p.window_bytes = params->window_bytes;
    }
    if (kind == CRYSTAL_KIND_NOP) return in_size;
    if (kind_is_direct(kind)) return digest_bytes_of(kind);
    if (kind_is_sliding(kind)) {
        const uint64_t windows = in_size >= p.window_bytes ? in_size - p.window_bytes + 1 : 0;
        return crystal_out_bytes_for_chunks(kind, in_size, windows + 1);
    }
    return 0;
}

uint64_t crystal_scratch_bytes(int kind, uint64_t n, uint64_t out_size, const crystal_hash_params* params) {
    crystal_hash_params p;
    crystal_params_default(&p);
    if (params) {
        if (params->segment_bytes) p.segment_bytes = params->segment_bytes;
        if (params->chunk_segment_bytes) p.chunk_segment_bytes = params->chunk_segment_bytes;
    }
    const uint64_t D = digest_bytes_of(kind);
    if (kind_is_direct(kind)) return D * segments_of(n, p.segment_bytes);
    if (kind_is_sliding(kind)) {
        const uint64_t fixed = sliding_fixed_bytes(n);
        if (out_size < fixed) return 0;
        const uint64_t cap = (out_size - fixed) / (4 + D);
        const uint64_t table = align_up(4 * (cap + 1), 16);
        const uint64_t chunk_segments = cap + (n + p.chunk_segment_bytes - 1) / p.chunk_segment_bytes + 1;
        return table + D * chunk_segments;
    }
    return 0;
}

uint64_t crystal_batch_bytes(uint32_t n_units) {
    return sizeof(crystal_batch) + (uint64_t)n_units * sizeof(crystal_unit);
}

int crystal_batch_plan(crystal_batch* b, uint32_t n_direct, uint32_t n_sliding) {
    if (!b) return CRYSTAL_EINVAL;
    crystal_unit* U = batch_units(b);
    uint64_t segs = 0, tiles = 0;
    uint32_t wmax = 0;
    for (uint32_t i = 0; i < n_direct; ++i) {
        const crystal_unit& x = U[i];
        if (!kind_is_direct(x.kind) || x.seg_bytes == 0 || x.out_cap < digest_bytes_of(x.kind)) return CRYSTAL_EINVAL;
        if ((x.scratch & 15) || (x.out & 3) || !x.scratch || !x.out || (!x.in && x.n)) return CRYSTAL_EINVAL;
    }
    // MD5 direct units first (stable): one segment kernel instance per hash
    std::stable_partition(U, U + n_direct, [](const crystal_unit& x) { return !kind_is_sha1(x.kind); });
    uint64_t segs_md5 = 0;
    for (uint32_t i = 0; i < n_direct; ++i) {
        crystal_unit& x = U[i];
        x.work_begin = segs;
        segs += segments_of(x.n, x.seg_bytes);
        if (!kind_is_sha1(x.kind)) segs_md5 = segs;
    }
    crystal_unit* S = U + n_direct;
    for (uint32_t i = 0; i < n_sliding; ++i) {
        const crystal_unit& x = S[i];
        if (!kind_is_sliding(x.kind) || x.seg_bytes == 0) return CRYSTAL_EINVAL;
        if (x.window == 0 || x.window > kMaxWindow || x.n >= (1ull << 32)) return CRYSTAL_EINVAL;
        if (x.out_cap < sliding_fixed_bytes(x.n)) return CRYSTAL_EINVAL;
        if ((x.scratch & 15) || (x.out & 3) || !x.scratch || !x.out || (!x.in && x.n)) return CRYSTAL_EINVAL;
    }
    // order (stable): MD5 with w = 20, other MD5, SHA-1 -- the window kernel
    // has one instance for each group
    auto group = [](const crystal_unit& x) {
        return kind_is_sha1(x.kind) ? 2 : (x.window == 20 ? 0 : 1);
    };
    std::stable_sort(S, S + n_sliding,
                     [&](const crystal_unit& a, const crystal_unit& b) { return group(a) < group(b); });
    uint64_t tiles_w20 = 0, tiles_md5 = 0;
    for (uint32_t i = 0; i < n_sliding; ++i) {
        crystal_unit& x = S[i];
        x.work_begin = tiles;
        x.seg_base = 0;
        tiles += (x.n + CRYSTAL_SLIDING_TILE - 1) / CRYSTAL_SLIDING_TILE;
        if (group(x) == 0) tiles_w20 = tiles;
        if (group(x) <= 1) tiles_md5 = tiles;
        if (x.window > wmax) wmax = x.window;
    }
    if (tiles_md5 < tiles_w20) tiles_md5 = tiles_w20;
    b->n_direct = n_direct;
    b->n_sliding = n_sliding;
    b->direct_segments = segs;
    b->sliding_tiles = tiles;
    b->window_max = wmax;
    b->status = 0;
    b->sliding_tiles_w20 = tiles_w20;
    b->sliding_tiles_md5 = tiles_md5;
    b->direct_segments_md5 = segs_md5;
    b->chunk_segments = 0;
    return CRYSTAL_OK;
}

const char* crystal_strerror(int status) {
    switch (status) {
    case CRYSTAL_OK: return "ok";
    case CRYSTAL_PENDING: return "pending";
    case CRYSTAL_EINVAL: return "invalid argument or state";
    case CRYSTAL_EAGAIN: return "pool has no room now";
    case CRYSTAL_ENOMEM: return "allocation failed";
    case CRYSTAL_ETIMEDOUT: return "timed out";
    case CRYSTAL_EOVERFLOW: return "output buffer too small for the chunk records";
    case CRYSTAL_ESHUTDOWN: return "context is shutting down";
    case CRYSTAL_EDEVICE: return "CUDA or device-side error";
    default: return "unknown status";
    }
}

}  // extern "C"
