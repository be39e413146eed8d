// Randomised check of the serving form's host-side allocator (arena.h):
// blocks are 256-byte aligned, inside the reservation and disjoint; the byte
// count in use is exact; frees coalesce (after freeing everything one block
// spans the whole reservation); high allocations come from the top.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "../paper_2112_00821_b300/csrc/arena.h"

int main()
{
    using fmh::Arena;
    std::mt19937_64 rng(12345);
    for (int round = 0; round < 50; ++round) {
        const size_t cap = (size_t)(1 + rng() % 64) << 20 | (rng() % 4096);   // unaligned on purpose
        Arena a;
        a.init(cap, nullptr);
        const size_t usable = cap & ~(size_t)255;
        if (a.capacity() != usable) { std::printf("capacity %zu != %zu\n", a.capacity(), usable); return 1; }
        struct B { size_t off, size; };
        std::vector<B> live;
        size_t used = 0;
        for (int step = 0; step < 4000; ++step) {
            if (!live.empty() && (rng() % 3 == 0)) {
                const size_t i = rng() % live.size();
                a.release(live[i].off);
                used -= live[i].size;
                live.erase(live.begin() + i);
            } else {
                const bool high = rng() % 2;
                const size_t want = 1 + rng() % (usable / 8 + 1);
                const size_t off = a.alloc(want, high);
                if (off == SIZE_MAX) continue;
                const size_t size = fmh::align_up(want);
                if (off % 256 || off + size > usable) { std::printf("bad block %zu+%zu\n", off, size); return 1; }
                for (const B& b : live)
                    if (off < b.off + b.size && b.off < off + size) {
                        std::printf("overlap %zu+%zu with %zu+%zu\n", off, size, b.off, b.size);
                        return 1;
                    }
                if (high) {
                    // nothing free above a high block's end within the same free run
                    bool above = false;
                    for (const B& b : live) above = above || b.off >= off + size;
                    if (!above && off + size != usable) {
                        std::printf("high block %zu+%zu not at the top of %zu\n", off, size, usable);
                        return 1;
                    }
                }
                live.push_back({off, size});
                used += size;
            }
            if (a.used() != used) { std::printf("used %zu != %zu\n", a.used(), used); return 1; }
        }
        for (const B& b : live) a.release(b.off);
        if (a.used() != 0) { std::printf("used %zu after freeing all\n", a.used()); return 1; }
        if (a.alloc(usable) != 0) { std::printf("free runs did not coalesce\n"); return 1; }
    }
    std::printf("ok\n");
    return 0;
}
