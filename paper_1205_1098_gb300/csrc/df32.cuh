// Double-float arithmetic: a value held as an unevaluated sum hi + lo of two
// FP32 numbers (48 significant bits), for FP64 data on the FP32 pipe.
//
// Building blocks, each a published error-free transformation or a direct
// consequence of the FP64 format:
//   * split_f64: an FP64 number as hi + lo, from its bits with integer
//     operations only (no FP64 instruction): hi takes the sign, the exponent
//     and the top 23 fraction bits; lo the next 24 significant bits of the
//     remainder, truncated.  |x - (hi + lo)| <= 2^-47 |x|.  Exact when the
//     remainder has at most 24 significant bits (every FP32 value, every
//     integer below 2^48).  Requires the exponent in FP32's normal range with
//     room for a normal lo: 2^-74 <= |x| < 2^128, or x = 0 (`split_ok`).
//   * two_sum (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly.
//   * two_prod (via FMA; Ogita, Rump and Oishi, SISC 2005): p + e = a * b
//     exactly, unless underflow.
//   * df_mac: acc + a * b in double-float, the product's cross terms folded
//     into the low part and the sum renormalised with two_sum.
// Host and device: compiled by nvcc for kernels and by a C++ compiler for the
// CPU checks of these error bounds.
#pragma once
#include <cstdint>
#include <cstring>
#include <cmath>

#if defined(__CUDACC__)
#define DF_HD __host__ __device__ __forceinline__
#else
#define DF_HD inline
#endif

namespace bto {
namespace df {

struct f2 {
    float hi, lo;
};

DF_HD uint64_t bits_of(double x) {
    uint64_t u;
    std::memcpy(&u, &x, sizeof u);
    return u;
}

DF_HD float float_of(uint32_t u) {
    float f;
    std::memcpy(&f, &u, sizeof f);
    return f;
}

DF_HD int clz64(uint64_t v) {
#if defined(__CUDA_ARCH__)
    return __clzll((long long)v);
#else
    return v ? __builtin_clzll(v) : 64;
#endif
}

// True when split_f64 represents x to 2^-47 relative (or exactly, x = 0).
DF_HD bool split_ok(double x) {
    const int e = (int)((bits_of(x) >> 52) & 0x7ff);     // biased FP64 exponent
    return e == 0 ? (bits_of(x) << 1) == 0 : (e - 1023 >= -74 && e - 1023 <= 127);
}

// hi + lo from the bits of x (x finite, split_ok(x)).
DF_HD f2 split_f64(double x) {
    const uint64_t u = bits_of(x);
    const uint32_t sign = (uint32_t)(u >> 63) << 31;
    const int e = (int)((u >> 52) & 0x7ff);
    if (e == 0) return {float_of(sign), 0.0f};
    const int ue = e - 1023;                                  // unbiased exponent of x
    const uint64_t frac = u & ((1ull << 52) - 1);
    // hi: sign, exponent, top 23 fraction bits (truncated).
    const float hi = float_of(sign | ((uint32_t)(ue + 127) << 23) | (uint32_t)(frac >> 29));
    // Remainder: the low 29 fraction bits, worth rem * 2^(ue - 52).
    const uint64_t rem = frac & ((1ull << 29) - 1);
    if (rem == 0) return {hi, 0.0f};
    const int lead = 63 - clz64(rem);                          // position of its leading one
    const int le = ue - 52 + lead;                             // exponent of lo
    // lo: the leading one and the next 23 bits of the remainder, truncated.
    const uint32_t mant = lead >= 23 ? (uint32_t)(rem >> (lead - 23)) : (uint32_t)(rem << (23 - lead));
    const float lo = float_of(sign | ((uint32_t)(le + 127) << 23) | (mant & ((1u << 23) - 1)));
    return {hi, lo};
}

DF_HD f2 two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

DF_HD f2 fast_two_sum(float a, float b) {          // |a| >= |b|
    const float s = a + b;
    return {s, b - (s - a)};
}

DF_HD f2 two_prod(float a, float b) {
    const float p = a * b;
    return {p, std::fmaf(a, b, -p)};
}

// acc + a * b, with a and b double-floats.
DF_HD f2 df_mac(f2 acc, f2 a, f2 b) {
    const f2 p = two_prod(a.hi, b.hi);
    const float cross = std::fmaf(a.hi, b.lo, std::fmaf(a.lo, b.hi, p.lo));
    const f2 s = two_sum(acc.hi, p.hi);
    return fast_two_sum(s.hi, s.lo + (acc.lo + cross));
}

DF_HD double to_f64(f2 v) { return (double)v.hi + (double)v.lo; }

// ---------------------------------------------------------------- sweep split
// The split the double-float matrix sweeps use, from the two 32-bit words of
// an FP64 number (hw: sign, exponent, top 20 fraction bits; lw: low 32
// fraction bits), by integer operations and two FP32 operations:
//   hi: sign, exponent rebased to FP32 and clamped to [0, 255], fraction
//       bits 51..29 (truncated);
//   lo: fraction bits 28..6: the FP32 number with hi's sign and exponent
//       and those bits as its fraction, minus hi's sign and exponent alone
//       (exact), times 2^-23 (exact unless it underflows).
// For 2^-100 <= |x| < 2^128: |x - (hi + lo)| < 2^-46 |x| (47 significant
// bits kept), exact for FP32 values and integers below 2^47.  Zero gives
// hi = lo = 0 (signed as x).  Below 2^-127 the value is flushed: |hi| + |lo|
// < 2^-145.  At 2^128 and above, and for Inf and NaN, hi is Inf or NaN, so
// that anything computed from it is not finite and the sweeps' finiteness
// check sends the data to FP64.
constexpr uint32_t kSplitBias = 0x38000000u;      // (1023 - 127) << 20
constexpr uint32_t kSplitTop = 0x0ff00000u;       // FP32 exponent 255, pre-shift

DF_HD uint32_t float_bits(float f) {
    uint32_t u;
    std::memcpy(&u, &f, sizeof u);
    return u;
}

DF_HD void split_words(uint32_t hw, uint32_t lw, float& hi, float& lo) {
    const uint32_t ax = hw & 0x7fffffffu;
#if defined(__CUDA_ARCH__)
    const uint32_t t = min((uint32_t)__viaddmax_s32((int)ax, -(int)kSplitBias, 0), kSplitTop);
    const uint32_t hb = __funnelshift_l(lw, t, 3) | (hw & 0x80000000u);
#else
    const int32_t ti = (int32_t)ax - (int32_t)kSplitBias;
    const uint32_t t0 = ti > 0 ? (uint32_t)ti : 0u;
    const uint32_t t = t0 < kSplitTop ? t0 : kSplitTop;
    const uint32_t hb = ((t << 3) | (lw >> 29)) | (hw & 0x80000000u);
#endif
    const uint32_t base = hb & 0xff800000u;                      // sign and exponent of hi
    const uint32_t mx = base | ((lw >> 6) & 0x7fffffu);
    hi = float_of(hb);
    lo = (float_of(mx) - float_of(base)) * 0x1p-23f;
}

DF_HD void split_double(double x, float& hi, float& lo) {
    const uint64_t u = bits_of(x);
    split_words((uint32_t)(u >> 32), (uint32_t)u, hi, lo);
}

// An FP32 number as the two words of the equal FP64 number, by integer
// operations; subnormal FP32 inputs (below 2^-126) become signed zero.
DF_HD void f32_to_f64_words(float f, uint32_t& hw, uint32_t& lw) {
    const uint32_t u = float_bits(f), ax = u & 0x7fffffffu;
    hw = (ax >= 0x00800000u ? (ax >> 3) + kSplitBias : 0u) | (u & 0x80000000u);
    lw = ax >= 0x00800000u ? u << 29 : 0u;
}

// The same in four integer operations, exact for normal FP32 numbers; a
// signed zero becomes +-2^-127 and a subnormal a number of that order.
DF_HD void f32_to_f64_words_fast(float f, uint32_t& hw, uint32_t& lw) {
    const uint32_t u = float_bits(f);
    const uint32_t sx = (uint32_t)((int32_t)u >> 3);             // sign copied into bits 31..28
    hw = (sx & 0x8fffffffu) + kSplitBias;
    lw = u << 29;
}

DF_HD double f64_of_words(uint32_t hw, uint32_t lw) {
    const uint64_t u = ((uint64_t)hw << 32) | lw;
    double d;
    std::memcpy(&d, &u, sizeof d);
    return d;
}

}  // namespace df
}  // namespace bto

namespace bto {
namespace df {

// A double-float value hi + lo (|lo| <= half an FP32 ulp of hi), given as hi
// and nlo = -lo, rounded once to FP64: the FP64 sum of hi and -nlo, both
// converted by f32_to_f64_words_fast.  A zero nlo converts to +-2^-127,
// below half an FP64 ulp of any |hi| >= 2^-73; for hi = +0 (with nlo = +0,
// as the renormalisation yields for an exact zero sum) the two +2^-127 cancel
// exactly.  Callers keep |hi| >= 2^-73 or zero, or accept an absolute error
// of order 2^-126.
DF_HD double pair_to_f64(float hi, float nlo) {
    uint32_t h1, l1, h2, l2;
    f32_to_f64_words_fast(hi, h1, l1);
    f32_to_f64_words_fast(nlo, h2, l2);
    return f64_of_words(h1, l1) - f64_of_words(h2, l2);
}

}  // namespace df
}  // namespace bto
