// sx_sched.h -- the host-side scheduling of the serving loop (sx_server.cpp), free of CUDA so
// that it is tested on the host: the arena allocator of the server's device memory, admission of
// waiting requests, and the sharing of one step's byte budget between the active requests.
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <deque>
#include <map>
#include <vector>

#include "sx.h"

namespace sx {
namespace sched {

constexpr size_t kAlign = 256;

// Bytes an allocation of `bytes` takes: a multiple of kAlign, at least kAlign.
inline size_t arena_bytes(size_t bytes) {
    bytes = (bytes + kAlign - 1) / kAlign * kAlign;
    return bytes ? bytes : kAlign;
}

// First-fit allocator over [0, size) with an address-ordered, coalescing free list.  Offsets are
// multiples of kAlign.
class Arena {
  public:
    explicit Arena(size_t size) : size_(size) {
        if (size) free_[0] = size;
    }
    bool alloc(size_t bytes, size_t *off) {
        bytes = arena_bytes(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = arena_bytes(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }
    size_t size() const { return size_; }
    size_t free_blocks() const { return free_.size(); }

  private:
    size_t size_;
    size_t used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

// The work a request still has, as the step planner sees it.
struct Want {
    uint64_t key;        // the caller's handle for the request
    uint64_t admit_seq;  // order of admission (ties)
    uint64_t per;        // bytes per element of the current phase (> 0)
    uint64_t remaining;  // elements of the current phase not yet launched (> 0)
    uint64_t later;      // bytes of the phases after the current one
    uint64_t phase_bytes() const { return remaining * per; }
    uint64_t total_bytes() const { return remaining * per + later; }
};

// Grants are whole multiples of 64 elements (tiles keep their vector alignment), at least 64.
inline uint64_t whole_units(uint64_t elems) { return std::max<uint64_t>(elems / 64 * 64, 64); }

// Orders `w` by `policy` (SX_SERVE_POLICY_*) and returns, in that order, the elements of its
// current phase each request gets in a step of `budget` bytes, never more than it has left:
//   SRPT         shortest remaining work (all phases) first; each request in that order gets all
//                of its current phase's remaining work until the budget is spent.
//   FAIR         water-filling: requests with less remaining work in their phase than an equal
//                share get all of it; the others split the rest equally.
//   SHORT_FIRST  requests whose whole remaining work is at most a quarter of the budget go
//                first, shortest first, and get all of it; the rest of the budget goes to the
//                others in admission order.
// The first request in the order always gets at least 64 elements (or all it has), so a step
// is never empty; the bytes granted exceed the budget by less than 64 elements' worth per
// request served.
inline std::vector<uint64_t> plan_step(int policy, uint64_t budget, std::vector<Want> &w) {
    std::vector<uint64_t> grant(w.size(), 0);
    if (policy == SX_SERVE_POLICY_FAIR) {
        std::sort(w.begin(), w.end(), [](const Want &a, const Want &b) { return a.phase_bytes() < b.phase_bytes(); });
        for (size_t i = 0; i < w.size(); ++i) {
            grant[i] = std::min(w[i].remaining, whole_units(budget / (w.size() - i) / w[i].per));
            budget -= std::min(budget, grant[i] * w[i].per);
        }
        return grant;
    }
    if (policy == SX_SERVE_POLICY_SRPT) {
        std::sort(w.begin(), w.end(), [](const Want &a, const Want &b) {
            if (a.total_bytes() != b.total_bytes()) return a.total_bytes() < b.total_bytes();
            return a.admit_seq < b.admit_seq;
        });
    } else {
        const uint64_t short_bytes = budget / 4;
        std::sort(w.begin(), w.end(), [short_bytes](const Want &a, const Want &b) {
            const bool sa = a.total_bytes() <= short_bytes, sb = b.total_bytes() <= short_bytes;
            if (sa != sb) return sa;
            if (sa) return a.total_bytes() < b.total_bytes();
            return a.admit_seq < b.admit_seq;
        });
    }
    for (size_t i = 0; i < w.size() && budget > 0; ++i) {
        grant[i] = std::min(w[i].remaining, whole_units(budget / w[i].per));
        budget -= std::min(budget, grant[i] * w[i].per);
    }
    return grant;
}

// One admission pass over `waiting` (arrival order) into `active`, at most `slots` active and at
// most kAdmitTries requests looked at: `fits(q)` admits q if its arrays fit (taking the memory).
// A later request may pass one that does not fit, but a request passed kMaxBypass times blocks
// the queue until it fits (no starvation).  Returns true if another pass should follow at once
// (the look-ahead ran out with room left).  Q has an int `bypassed`.
constexpr size_t kAdmitTries = 64;
constexpr int kMaxBypass = 64;

template <class Q, class Fits>
bool admission_pass(std::deque<Q *> &waiting, std::vector<Q *> &active, size_t slots, Fits fits) {
    std::vector<Q *> passed;  // waiting requests a later one may overtake in this pass
    size_t tried = 0;
    for (auto it = waiting.begin(); it != waiting.end() && tried < kAdmitTries; ++tried) {
        if (active.size() >= slots) break;
        Q *q = *it;
        if (fits(q)) {
            for (Q *p : passed) p->bypassed++;
            active.push_back(q);
            it = waiting.erase(it);
            continue;
        }
        if (q->bypassed >= kMaxBypass) break;  // it has waited long enough: nobody passes it any more
        passed.push_back(q);
        ++it;
    }
    return !waiting.empty() && active.size() < slots && tried >= kAdmitTries;
}

}  // namespace sched
}  // namespace sx
