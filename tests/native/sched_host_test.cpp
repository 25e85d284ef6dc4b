// Host-only checks of the request server's arena and wave planner
// (paper_1212_1095_gb300/csrc/vor_sched.h).  Prints "ok" and exits 0 when
// every check holds; prints the failing check and exits 1 otherwise.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "vor_sched.h"

#define CHECK(c)                                                        \
    do {                                                                \
        if (!(c)) {                                                     \
            std::printf("check failed at line %d: %s\n", __LINE__, #c); \
            std::exit(1);                                               \
        }                                                               \
    } while (0)

using vor::Arena;
using vor::plan_wave;
using vor::WaveLimits;

static void arena_basics() {
    Arena a(4096, 256);
    uint64_t x, y, z, w;
    CHECK(a.alloc(1, &x) && x == 0);               // rounded up to 256
    CHECK(a.alloc(300, &y) && y == 256);           // 512 bytes
    CHECK(a.alloc(1024, &z) && z == 768);
    CHECK(a.free_bytes() == 4096 - 256 - 512 - 1024);
    CHECK(!a.alloc(4096, &w));                     // does not fit
    CHECK(a.release(y));
    CHECK(!a.release(y));                          // double free is refused
    CHECK(!a.release(12345));                      // unknown offset
    CHECK(a.alloc(512, &w) && w == 256);           // first fit reuses the hole
    CHECK(a.release(x) && a.release(w) && a.release(z));
    CHECK(a.free_bytes() == 4096 && a.blocks_free() == 1 && a.largest_free() == 4096);
}

static void arena_random_no_leak() {
    std::mt19937_64 g(1212);
    Arena a(1 << 20, 256);
    std::vector<std::pair<uint64_t, uint64_t>> live;   // offset, rounded length
    for (int it = 0; it < 20000; it++) {
        if (live.empty() || g() % 3 != 0) {
            const uint64_t len = 1 + g() % 20000;
            uint64_t off;
            if (a.alloc(len, &off)) {
                const uint64_t r = a.round(len);
                CHECK(off % 256 == 0 && off + r <= a.size());
                for (auto &l : live) CHECK(off + r <= l.first || l.first + l.second <= off);
                live.push_back({off, r});
            } else {
                CHECK(a.largest_free() < a.round(len));
            }
        } else {
            const size_t k = g() % live.size();
            CHECK(a.release(live[k].first));
            live[k] = live.back();
            live.pop_back();
        }
        uint64_t used = 0;
        for (auto &l : live) used += l.second;
        CHECK(used + a.free_bytes() == a.size());
    }
    for (auto &l : live) CHECK(a.release(l.first));
    CHECK(a.free_bytes() == a.size() && a.blocks_free() == 1 && a.blocks_used() == 0);
}

static void planner() {
    // 100 bytes per site: the prefix stops where memory, count or sites run out
    auto bytes_of = [](const std::vector<int64_t> &s) {
        return [&s](int k) -> uint64_t {
            uint64_t t = 0;
            for (int j = 0; j < k; j++) t += 100 * (uint64_t)s[j];
            return t;
        };
    };
    std::vector<int64_t> s = {10, 20, 30, 40};
    CHECK(plan_wave(s, WaveLimits{8, 1000}, 1e9, bytes_of(s)) == 4);
    CHECK(plan_wave(s, WaveLimits{2, 1000}, 1e9, bytes_of(s)) == 2);      // request limit
    CHECK(plan_wave(s, WaveLimits{8, 60}, 1e9, bytes_of(s)) == 3);        // site limit
    CHECK(plan_wave(s, WaveLimits{8, 1000}, 3000, bytes_of(s)) == 2);     // memory
    CHECK(plan_wave(s, WaveLimits{8, 1000}, 999, bytes_of(s)) == 0);      // first does not fit
    std::vector<int64_t> big = {5000, 1};
    CHECK(plan_wave(big, WaveLimits{8, 100}, 1e9, bytes_of(big)) == 1);   // alone above the site limit
    std::vector<int64_t> none;
    CHECK(plan_wave(none, WaveLimits{8, 100}, 1e9, bytes_of(none)) == 0);
    // arrival order is kept: a small request behind a big one waits for it
    std::vector<int64_t> order = {50, 1, 1};
    CHECK(plan_wave(order, WaveLimits{8, 1000}, 4000, bytes_of(order)) == 0);
}

int main() {
    arena_basics();
    arena_random_no_leak();
    planner();
    std::printf("ok\n");
    return 0;
}
