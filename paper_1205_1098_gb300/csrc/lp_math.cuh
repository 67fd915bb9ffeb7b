// FP32 arithmetic helpers of the reduced-precision storage form.
#pragma once
#include <cuda_bf16.h>

namespace bto {
namespace lp {

// Knuth's TwoSum: s + e == a + b exactly, s = fl(a + b).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

template <typename TA> __device__ __forceinline__ float to_f(TA v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) {
    return __uint_as_float((unsigned)__bfloat16_as_ushort(v) << 16);
}
template <typename TA> __device__ __forceinline__ TA from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// Transposing butterfly over 16 column partials held by each of 32 lanes:
// lane l ends with the warp sum of column l mod 16 (v is destroyed).
__device__ __forceinline__ float butterfly16(float (&v)[16], int lane) {
#pragma unroll
    for (int half = 8; half >= 1; half >>= 1) {
        const bool upper = (lane & half) != 0;
#pragma unroll
        for (int k = 0; k < half; k++) {
            float send = upper ? v[k] : v[k + half];
            float keep = upper ? v[k + half] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, half);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
}

}  // namespace lp
}  // namespace bto
