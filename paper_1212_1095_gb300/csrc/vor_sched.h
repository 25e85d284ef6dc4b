// vor_sched.h -- host-side core of the request server: memory arenas and
// the wave planner.  No CUDA here, so the scheduling rules can be exercised
// on a machine without a GPU.
//
// Arena: first-fit allocator over a fixed range [0, size) (a device or a
// pinned host block allocated once), with coalescing of free neighbours.
//
// plan_wave: continuous batching.  Given the pending requests in arrival
// order, it takes the longest prefix that fits the limits of one wave (a
// request count, a site count) and whose memory, as computed by the caller,
// fits the largest free block of the arena.  Taking a prefix keeps the
// arrival order (no request is overtaken, so none starves); a request that
// alone exceeds the arena is refused at submission, never planned.
#pragma once

#include <cstdint>
#include <functional>
#include <map>
#include <vector>

namespace vor {

class Arena {
public:
    explicit Arena(uint64_t size = 0, uint64_t align = 256) { reset(size, align); }

    void reset(uint64_t size, uint64_t align = 256) {
        size_ = size;
        align_ = align ? align : 1;
        free_.clear();
        used_.clear();
        if (size_ > 0) free_[0] = size_;
    }

    uint64_t round(uint64_t bytes) const { return (bytes + align_ - 1) / align_ * align_; }

    // first fit; returns false when no free block holds the request
    bool alloc(uint64_t bytes, uint64_t *off) {
        const uint64_t need = round(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < need) continue;
            const uint64_t at = it->first, left = it->second - need;
            free_.erase(it);
            if (left) free_[at + need] = left;
            used_[at] = need;
            *off = at;
            return true;
        }
        return false;
    }

    // returns false for an offset that is not allocated
    bool release(uint64_t off) {
        auto u = used_.find(off);
        if (u == used_.end()) return false;
        uint64_t at = off, len = u->second;
        used_.erase(u);
        auto next = free_.lower_bound(at);
        if (next != free_.end() && next->first == at + len) {
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == at) {
                at = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        free_[at] = len;
        return true;
    }

    uint64_t size() const { return size_; }
    uint64_t free_bytes() const {
        uint64_t t = 0;
        for (const auto &f : free_) t += f.second;
        return t;
    }
    uint64_t largest_free() const {
        uint64_t m = 0;
        for (const auto &f : free_) m = f.second > m ? f.second : m;
        return m;
    }
    size_t blocks_used() const { return used_.size(); }
    size_t blocks_free() const { return free_.size(); }

private:
    uint64_t size_ = 0, align_ = 256;
    std::map<uint64_t, uint64_t> free_;   // offset -> length
    std::map<uint64_t, uint64_t> used_;   // offset -> length
};

struct WaveLimits {
    int max_requests;
    int64_t max_sites;
};

// Number of pending requests (a prefix of sizes[], in arrival order) that
// form the next wave: the longest prefix with at most lim.max_requests
// requests and lim.max_sites sites (a single request may exceed max_sites)
// whose bytes(k) fits in `room` bytes.  0 when even the first does not fit.
inline int plan_wave(const std::vector<int64_t> &sizes, const WaveLimits &lim, uint64_t room,
                     const std::function<uint64_t(int)> &bytes) {
    int take = 0;
    int64_t sites = 0;
    const int n = (int)sizes.size();
    for (int k = 1; k <= n && k <= lim.max_requests; k++) {
        sites += sizes[k - 1];
        if (k > 1 && sites > lim.max_sites) break;
        if (bytes(k) > room) break;
        take = k;
    }
    return take;
}

}  // namespace vor
