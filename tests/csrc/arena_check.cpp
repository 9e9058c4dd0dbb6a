// Test-only driver: random allocate/release sequences on fhp::Arena, checking
// that live blocks never overlap, stay aligned and inside the arena, and that
// the free space is whole again once everything is released.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "../../paper_1208_2428_gb300/csrc/fhp_arena.h"

int main() {
    std::mt19937_64 rng(12345);
    const size_t cap = 64u << 20;
    fhp::Arena a(cap);
    struct Blk { size_t off, bytes; };
    std::vector<Blk> live;
    for (int it = 0; it < 200000; ++it) {
        if (live.empty() || rng() % 3) {
            size_t bytes = 1 + rng() % (1u << (rng() % 20));
            size_t off = a.allocate(bytes);
            if (off == SIZE_MAX) {
                if (a.largest_free() >= fhp::Arena::round(bytes)) { std::printf("FAIL: refused with room\n"); return 1; }
                continue;
            }
            if (off % fhp::Arena::kAlign || off + fhp::Arena::round(bytes) > a.capacity()) { std::printf("FAIL: bounds\n"); return 1; }
            for (const Blk& b : live) {
                size_t e1 = off + fhp::Arena::round(bytes), e2 = b.off + fhp::Arena::round(b.bytes);
                if (off < e2 && b.off < e1) { std::printf("FAIL: overlap\n"); return 1; }
            }
            live.push_back({off, bytes});
        } else {
            size_t i = rng() % live.size();
            if (!a.release(live[i].off, live[i].bytes)) { std::printf("FAIL: release\n"); return 1; }
            live[i] = live.back();
            live.pop_back();
        }
        size_t used = 0;
        for (const Blk& b : live) used += fhp::Arena::round(b.bytes);
        if (used != a.used()) { std::printf("FAIL: accounting\n"); return 1; }
    }
    for (const Blk& b : live) a.release(b.off, b.bytes);
    if (a.used() != 0 || a.free_ranges() != 1 || a.largest_free() != a.capacity()) { std::printf("FAIL: not coalesced\n"); return 1; }
    if (a.release(0, 256)) { std::printf("FAIL: double release accepted\n"); return 1; }
    std::printf("ok\n");
    return 0;
}
