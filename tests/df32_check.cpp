// Host checks of the double-float building blocks (csrc/df32.cuh) against
// exact arithmetic: the FP64 split, TwoSum, TwoProduct and a dot product
// accumulated with df_mac, measured against a sum in a type of at least 113 significand bits.
// Prints "ok" and exits 0, or the first violation and exits 1.
#include <cstdio>
#include <cstdint>
#include <cmath>
#include <cstring>
#include "df32.cuh"

using namespace bto::df;

// A type with at least 113 significand bits for the exact reference sums.
#if defined(__x86_64__)
typedef __float128 quad;
#else
typedef long double quad;        // IEEE binary128 on AArch64 Linux
#endif

namespace {

uint64_t state = 0x243F6A8885A308D3ull;
uint64_t next_u64() {                       // SplitMix64
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double unit() { return (double)(next_u64() >> 11) * 0x1.0p-53; }      // [0, 1)

int fail(const char* what, double a, double b) {
    std::printf("violation: %s (%.17g, %.17g)\n", what, a, b);
    return 1;
}

}  // namespace

int main() {
    // Split: random significands over the whole supported exponent range.
    for (int i = 0; i < 2000000; i++) {
        const int ex = -74 + (int)(next_u64() % 202);                  // -74 .. 127
        double x = std::ldexp(1.0 + unit(), ex);
        if (next_u64() & 1) x = -x;
        if (!split_ok(x)) return fail("split_ok rejects a supported value", x, ex);
        const f2 v = split_f64(x);
        if (!std::isfinite(v.hi) || !std::isfinite(v.lo)) return fail("non-finite part", x, v.hi);
        const double err = x - ((double)v.hi + (double)v.lo);          // exact: the parts are bit subsets of x
        if (std::fabs(err) > std::ldexp(std::fabs(x), -47)) return fail("split error above 2^-47", x, err);
        if (v.lo != 0.0f && std::fabs((double)v.lo) > std::ldexp(std::fabs((double)v.hi), -23))
            return fail("lo not below hi's last bit", v.hi, v.lo);
    }
    // Exact cases: FP32 values and integers below 2^48; zero; out-of-range values refused.
    for (int i = 0; i < 200000; i++) {
        const float f = (float)((unit() - 0.5) * std::ldexp(1.0, (int)(next_u64() % 60) - 30));
        const f2 v = split_f64((double)f);
        if (v.hi != f || v.lo != 0.0f) return fail("FP32 value not exact", f, v.lo);
        const double k = (double)(next_u64() >> 16);
        const f2 w = split_f64(k);
        if ((double)w.hi + (double)w.lo != k) return fail("integer below 2^48 not exact", k, w.lo);
    }
    if (split_f64(0.0).hi != 0.0f || split_f64(-0.0).lo != 0.0f || !split_ok(0.0)) return fail("zero", 0, 0);
    if (split_ok(1e39) || split_ok(1e-23) || split_ok(INFINITY)) return fail("range check", 1e39, 1e-23);
    // TwoSum and TwoProduct: exact in double for operands within 2^±10.
    for (int i = 0; i < 2000000; i++) {
        const float a = (float)std::ldexp(unit() - 0.5, (int)(next_u64() % 20) - 10);
        const float b = (float)std::ldexp(unit() - 0.5, (int)(next_u64() % 20) - 10);
        const f2 s = two_sum(a, b);
        if ((double)s.hi + (double)s.lo != (double)a + (double)b) return fail("two_sum not exact", a, b);
        if (s.hi != a + b) return fail("two_sum high part is not the rounded sum", a, b);
        const f2 p = two_prod(a, b);
        if ((double)p.hi + (double)p.lo != (double)a * (double)b) return fail("two_prod not exact", a, b);
    }
    // Dot products of U[-1, 1) vectors: double-float against a 113-bit sum.
    for (int trial = 0; trial < 20; trial++) {
        const int n = 16384;
        f2 acc = {0.0f, 0.0f};
        quad exact = 0, mag = 0;
        for (int i = 0; i < n; i++) {
            const double a = 2 * unit() - 1, p = 2 * unit() - 1;
            acc = df_mac(acc, split_f64(a), split_f64(p));
            exact += (quad)a * (quad)p;
            mag += (quad)std::fabs(a * p);
        }
        const double err = std::fabs((double)((quad)to_f64(acc) - exact));
        // Relative to the sum of magnitudes (the condition-free bound): within 1e-13.
        if (err > 1e-13 * (double)mag) return fail("dot product error", err, (double)mag);
    }
    // The sweep split: hi + lo is x with its 6 lowest fraction bits cleared
    // (47 significant bits), exactly, over 2^-100 <= |x| < 2^128 and for zero.
    for (int i = 0; i < 2000000; i++) {
        const int ex = -100 + (int)(next_u64() % 228);                 // -100 .. 127
        double x = std::ldexp(1.0 + unit(), ex);
        if (next_u64() & 1) x = -x;
        float hi, lo;
        split_double(x, hi, lo);
        const uint64_t kept = bits_of(x) & ~0x3full;
        double want;
        std::memcpy(&want, &kept, sizeof want);
        if ((double)hi + (double)lo != want) return fail("sweep split is not x truncated to 47 bits", x, lo);
        if (std::fabs(x - want) >= std::ldexp(std::fabs(x), -46)) return fail("sweep split error", x, want);
        if (lo != 0.0f && std::fabs((double)lo) >= std::ldexp(std::fabs((double)hi), -23))
            return fail("sweep split lo not below hi's last bit", hi, lo);
        if ((std::signbit(hi) != std::signbit(x)) || (lo != 0.0f && std::signbit(lo) != std::signbit(x)))
            return fail("sweep split sign", x, lo);
    }
    for (int i = 0; i < 200000; i++) {
        const float f = (float)((unit() - 0.5) * std::ldexp(1.0, (int)(next_u64() % 60) - 30));
        float hi, lo;
        split_double((double)f, hi, lo);
        if (hi != f || lo != 0.0f) return fail("sweep split: FP32 value not exact", f, lo);
        const double k = (double)(next_u64() >> 17);                   // below 2^47
        split_double(next_u64() & 1 ? -k : k, hi, lo);
        if (std::fabs((double)hi + (double)lo) != k) return fail("sweep split: integer below 2^47 not exact", k, lo);
    }
    {
        float hi, lo;
        split_double(0.0, hi, lo);
        if (hi != 0.0f || lo != 0.0f || std::signbit(hi)) return fail("sweep split of +0", hi, lo);
        split_double(-0.0, hi, lo);
        if (hi != 0.0f || lo != 0.0f || !std::signbit(hi)) return fail("sweep split of -0", hi, lo);
    }
    // FP64 subnormals whose high word is zero apart from the sign: near zero.
    for (int i = 0; i < 200000; i++) {
        const uint64_t u = (next_u64() & 0xffffffffull) | ((next_u64() & 1) << 63);
        double x;
        std::memcpy(&x, &u, sizeof x);
        float hi, lo;
        split_double(x, hi, lo);
        if (!(std::fabs((double)hi) + std::fabs((double)lo) < std::ldexp(1.0, -145)))
            return fail("sweep split of a small subnormal is not near zero", x, hi);
    }
    // Flushed below 2^-127; not finite from 2^128 up and for Inf and NaN.
    for (int i = 0; i < 200000; i++) {
        const int ex = -1022 + (int)(next_u64() % (1022 - 128));        // -1022 .. -129
        double x = std::ldexp(1.0 + unit(), ex);
        if (next_u64() & 1) x = -x;
        float hi, lo;
        split_double(x, hi, lo);
        if (!(std::fabs((double)hi) + std::fabs((double)lo) < std::ldexp(1.0, -145)))
            return fail("sweep split does not flush below 2^-127", x, hi);
        const double big = std::ldexp(1.0 + unit(), 128 + (int)(next_u64() % 895)) * ((next_u64() & 1) ? -1 : 1);
        split_double(big, hi, lo);
        if (std::isfinite(hi)) return fail("sweep split of a value >= 2^128 is finite", big, hi);
    }
    {
        float hi, lo;
        split_double(INFINITY, hi, lo);
        if (!(std::isinf(hi) && hi > 0)) return fail("sweep split of +Inf", INFINITY, hi);
        split_double(-INFINITY, hi, lo);
        if (!(std::isinf(hi) && hi < 0)) return fail("sweep split of -Inf", -INFINITY, hi);
        split_double(NAN, hi, lo);
        if (std::isfinite(hi)) return fail("sweep split of NaN is finite", NAN, hi);
    }
    // Fast FP32 -> FP64 words: exact on normal values, +-2^-127 for zeros.
    for (int i = 0; i < 2000000; i++) {
        const uint32_t u = (uint32_t)next_u64();
        float f;
        std::memcpy(&f, &u, sizeof f);
        if (!std::isfinite(f) || (u & 0x7fffffffu) < 0x00800000u) continue;
        uint32_t hw, lw;
        f32_to_f64_words_fast(f, hw, lw);
        if (f64_of_words(hw, lw) != (double)f) return fail("f32_to_f64_words_fast", f, f64_of_words(hw, lw));
    }
    {
        uint32_t hw, lw;
        f32_to_f64_words_fast(0.0f, hw, lw);
        if (f64_of_words(hw, lw) != std::ldexp(1.0, -127)) return fail("fast conversion of +0", 0, 0);
        f32_to_f64_words_fast(-0.0f, hw, lw);
        if (f64_of_words(hw, lw) != -std::ldexp(1.0, -127)) return fail("fast conversion of -0", 0, 0);
    }
    // A renormalised pair (hi, lo) given as (hi, -lo) rounds once to FP64.
    for (int i = 0; i < 2000000; i++) {
        const float h = (float)std::ldexp(1.0 + unit(), -73 + (int)(next_u64() % 190)) * ((next_u64() & 1) ? -1.f : 1.f);
        float l = (float)(std::ldexp(unit() - 0.5, -24) * (double)h);
        if (next_u64() % 8 == 0) l = 0.0f;
        const f2 r = fast_two_sum(h, l);                                 // |lo| <= half an ulp of hi
        if (pair_to_f64(r.hi, -r.lo) != (double)r.hi + (double)r.lo) return fail("pair_to_f64", r.hi, r.lo);
    }
    if (pair_to_f64(0.0f, 0.0f) != 0.0) return fail("pair_to_f64 of an exact zero", 0, 0);
    // FP32 -> FP64 words: exact for normal values and zero; subnormals to zero.
    for (int i = 0; i < 2000000; i++) {
        const uint32_t u = (uint32_t)next_u64();
        float f;
        std::memcpy(&f, &u, sizeof f);
        if (!std::isfinite(f)) continue;
        uint32_t hw, lw;
        f32_to_f64_words(f, hw, lw);
        const double d = f64_of_words(hw, lw);
        const bool sub = (u & 0x7fffffffu) < 0x00800000u;
        if (sub ? (d != 0.0 || std::signbit(d) != std::signbit(f)) : d != (double)f)
            return fail("f32_to_f64_words", f, d);
    }
    std::printf("ok\n");
    return 0;
}
