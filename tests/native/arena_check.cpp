// Host-only check of the serving arena (csrc/arena.h) against a unit-occupancy
// model: a seeded random sequence of allocations and releases, after each step
// the allocator's offset, usage, high-water mark, free-range count and largest
// free range must equal the model's (first fit = lowest run of enough free
// units, which holds only if released ranges are fully coalesced).
#include <stdint.h>
#include <stdio.h>

#include <vector>

#include "arena.h"

static uint64_t rng_state = 0x9E3779B97F4A7C15ull;
static uint64_t next_u64()
{
    // splitmix64
    uint64_t z = (rng_state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

#define CHECK(c)                                                  \
    do {                                                          \
        if (!(c)) {                                               \
            fprintf(stderr, "FAIL line %d: %s\n", __LINE__, #c); \
            return 1;                                             \
        }                                                         \
    } while (0)

int main()
{
    const int64_t align = 256, units = 512;
    ctm::Arena a(units * align + 100, align);  // the ragged tail is cut off
    CHECK(a.size() == units * align);
    std::vector<int> occ(units, 0);
    std::vector<std::pair<int64_t, int64_t>> live;  // offset, units
    int64_t used = 0, peak = 0;
    for (int step = 0; step < 20000; ++step) {
        const bool do_alloc = live.empty() || (next_u64() % 100) < 55;
        if (do_alloc) {
            const int64_t bytes = 1 + (int64_t)(next_u64() % (40 * align));
            const int64_t need = (bytes + align - 1) / align;
            int64_t expect = -1;
            for (int64_t i = 0, run = 0; i < units; ++i) {
                run = occ[i] ? 0 : run + 1;
                if (run == need) { expect = i - need + 1; break; }
            }
            const int64_t off = a.alloc(bytes);
            CHECK((expect < 0 && off < 0) || off == expect * align);
            if (off >= 0) {
                for (int64_t i = 0; i < need; ++i) occ[expect + i] = 1;
                live.push_back({off, need});
                used += need;
                if (used > peak) peak = used;
            }
        } else {
            const size_t k = (size_t)(next_u64() % live.size());
            CHECK(a.release(live[k].first));
            CHECK(!a.release(live[k].first));  // a second release is refused
            for (int64_t i = 0; i < live[k].second; ++i) occ[live[k].first / align + i] = 0;
            used -= live[k].second;
            live[k] = live.back();
            live.pop_back();
        }
        int64_t runs = 0, longest = 0;
        for (int64_t i = 0, run = 0; i < units; ++i) {
            if (!occ[i]) {
                if (run == 0) ++runs;
                ++run;
                if (run > longest) longest = run;
            } else {
                run = 0;
            }
        }
        CHECK(a.used() == used * align);
        CHECK(a.peak() == peak * align);
        CHECK(a.free_ranges() == runs);
        CHECK(a.largest_free() == longest * align);
        CHECK(a.live_blocks() == (int64_t)live.size());
    }
    for (auto &b : live) CHECK(a.release(b.first));
    CHECK(a.used() == 0 && a.free_ranges() == 1 && a.largest_free() == a.size());
    CHECK(a.release(12345) == false);
    CHECK(a.alloc(a.size() + 1) == -1);
    CHECK(a.alloc(a.size()) == 0);
    printf("OK\n");
    return 0;
}
