// Argument validation shared by the entry points.
#pragma once
#include "internal.cuh"
#include <algorithm>

namespace bto {

// Collects the first failing argument (1-based position) of a call.
struct Check {
    int pos = 0;
    bto_status st = BTO_OK;
    bool ok() const { return st == BTO_OK; }
    void fail(int p, bto_status s = BTO_ERR_INVALID_VALUE) {
        if (st == BTO_OK) { st = s; pos = p; }
    }
    void size(int p, int64_t v) { if (v < 0) fail(p); }
    void ld(int p, int64_t ld, int64_t m) { if (ld < std::max<int64_t>(1, m)) fail(p); }
    // Pointer must be non-NULL when `needed`, and aligned to its element size.
    void ptr(int p, const void* x, bool needed, size_t align = 8) {
        if (needed && !x) fail(p);
        else if (x && (reinterpret_cast<uintptr_t>(x) % align)) fail(p);
    }
    void finite_scalar(int, double) {}
    // Output [o, o+no) must not overlap input [i, i+ni).
    void disjoint(int p, const void* o, size_t no, const void* i, size_t ni) {
        if (overlap(o, no, i, ni)) fail(p);
    }
    void ws(int p, const void* w, size_t bytes, const WsLayout& L) {
        if (L.total == 0) return;
        if (!w || (reinterpret_cast<uintptr_t>(w) & 255u) || bytes < L.total)
            fail(p, BTO_ERR_WORKSPACE);
    }
    bto_status finish() {
        if (st != BTO_OK) set_invalid_arg(pos);
        return st;
    }
};

inline size_t vbytes(int64_t len) { return len > 0 ? (size_t)len * sizeof(double) : 0; }

}  // namespace bto
