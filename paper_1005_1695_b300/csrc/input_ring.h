// Input ring of the serving loop (host-only; no CUDA).
//
// Slots of 256-byte-aligned sizes are handed out in admission order, each
// directly after the newest live slot, wrapping to the start when the end is
// reached, and are reclaimed in the same order: a finished slot is reused
// once every older slot has finished too (the newest slot, given back, is
// free at once).  Offsets are relative to the ring's memory; the caller maps
// them onto a pinned block and a device block of the same size.
// Thread-safe: admission takes slots while completion callbacks give them
// back.
#pragma once

#include <stdint.h>

#include <deque>
#include <mutex>

namespace crystal {

class InputRing {
  public:
    static constexpr uint64_t kNone = UINT64_MAX;
    void init(uint64_t bytes) { bytes_ = bytes; }
    bool enabled() const { return bytes_ != 0; }
    // A slot for `size` bytes: its offset, and its ticket in *seq; kNone when
    // the ring has no room.
    uint64_t take(uint64_t size, uint64_t* seq) {
        if (size > bytes_) return kNone;  // also keeps the rounding below from wrapping
        const uint64_t b = ((size ? size : 1) + 255) & ~(uint64_t)255;
        std::lock_guard<std::mutex> lk(mu_);
        uint64_t off = kNone;
        if (live_.empty()) {
            if (b <= bytes_) off = 0;
        } else {
            const uint64_t first = live_.front().off;
            const uint64_t end = live_.back().off + live_.back().len;
            if (live_.back().off >= first) {  // live slots run from first up to end
                if (end + b <= bytes_) off = end;
                else if (b <= first) off = 0;
            } else if (end + b <= first) {    // wrapped: the gap is [end, first)
                off = end;
            }
        }
        if (off == kNone) return kNone;
        live_.push_back(Slot{off, b, false});
        *seq = front_seq_ + live_.size() - 1;
        return off;
    }
    // The slot's job finished (or was never submitted): reclaim it and every
    // finished slot behind it.
    void give_back(uint64_t seq) {
        std::lock_guard<std::mutex> lk(mu_);
        if (seq < front_seq_ || seq - front_seq_ >= live_.size()) return;
        if (seq - front_seq_ == live_.size() - 1 && live_.size() > 1) {
            live_.pop_back();  // the newest slot: its room is free at once
            return;
        }
        live_[seq - front_seq_].done = true;
        while (!live_.empty() && live_.front().done) {
            live_.pop_front();
            ++front_seq_;
        }
    }
    uint64_t live_slots() {
        std::lock_guard<std::mutex> lk(mu_);
        return live_.size();
    }

  private:
    struct Slot {
        uint64_t off, len;
        bool done;
    };
    std::mutex mu_;
    std::deque<Slot> live_;   // slots in use, oldest first
    uint64_t front_seq_ = 0;  // ticket of live_.front()
    uint64_t bytes_ = 0;
};

}  // namespace crystal
