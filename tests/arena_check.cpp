// Host harness for the serving arena (paper_1205_1098_gb300/csrc/arena.h):
// a seeded random sequence of allocations and releases checked against a
// model that marks every 256-byte granule.  Prints "ok" and exits 0, or
// prints the first violation and exits 1.
#include <cstdio>
#include <cstdint>
#include <vector>
#include "arena.h"

namespace {

uint64_t state = 0x9E3779B97F4A7C15ull;
uint64_t next_u64() {                       // SplitMix64
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int fail(const char* what, long a, long b) {
    std::printf("violation: %s (%ld, %ld)\n", what, a, b);
    return 1;
}

}  // namespace

int main() {
    const size_t G = bto::kArenaGranule, cap = 4096 * G + 100;   // capacity rounds down to 4096 granules
    bto::Arena A(cap);
    if (A.capacity() != 4096 * G) return fail("capacity not rounded down", (long)A.capacity(), 0);
    std::vector<int> owner(4096, -1);        // model: which live block holds each granule
    struct Live { size_t off, bytes; };
    std::vector<Live> live;
    size_t used = 0, peak = 0;
    for (int step = 0; step < 200000; step++) {
        const bool do_alloc = live.empty() || (next_u64() % 100) < 55;
        if (do_alloc) {
            const size_t bytes = 1 + next_u64() % (64 * G);
            const size_t need = (bytes + G - 1) / G;
            // First fit in the model: the lowest run of `need` free granules.
            long first = -1;
            for (size_t g = 0, run = 0; g < owner.size(); g++) {
                run = owner[g] < 0 ? run + 1 : 0;
                if (run == need) { first = (long)(g + 1 - need); break; }
            }
            size_t off = 0;
            const bool ok = A.alloc(bytes, &off);
            if (ok != (first >= 0)) return fail("fit disagrees with the model", ok, first);
            if (!ok) continue;
            if ((long)(off / G) != first || off % G) return fail("not the first fit", (long)off, first);
            for (size_t g = off / G; g < off / G + need; g++) owner[g] = (int)live.size();
            live.push_back({off, bytes});
            used += need * G;
            peak = used > peak ? used : peak;
        } else {
            const size_t k = next_u64() % live.size();
            const Live b = live[k];
            A.release(b.off, b.bytes);
            const size_t need = (b.bytes + G - 1) / G;
            for (size_t g = b.off / G; g < b.off / G + need; g++) owner[g] = -1;
            live[k] = live.back();
            live.pop_back();
            for (size_t g = 0; g < owner.size(); g++)        // reindex the moved block
                if (owner[g] == (int)live.size()) owner[g] = (int)k;
            used -= need * G;
        }
        if (A.used() != used) return fail("used bytes", (long)A.used(), (long)used);
        if (A.peak() != peak) return fail("peak bytes", (long)A.peak(), (long)peak);
        // Free blocks are maximal: as many as the model's free runs.
        size_t runs = 0;
        for (size_t g = 0; g < owner.size(); g++)
            if (owner[g] < 0 && (g == 0 || owner[g - 1] >= 0)) runs++;
        if (A.free_blocks() != runs) return fail("free blocks not coalesced", (long)A.free_blocks(), (long)runs);
    }
    for (const Live& b : live) A.release(b.off, b.bytes);
    size_t off = 1;
    if (A.used() != 0 || A.free_blocks() != 1 || !A.alloc(4096 * G, &off) || off != 0)
        return fail("arena not whole after releasing everything", (long)A.free_blocks(), (long)off);
    std::printf("ok\n");
    return 0;
}
