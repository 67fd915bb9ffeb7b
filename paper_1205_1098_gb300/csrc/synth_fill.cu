// Device-side generation of the seeded synthetic inputs (not part of any
// Table I operation).  SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) used
// as a counter-based stream: element k of stream (seed, aid) is
//   fmix(key + (k + 1) * GAMMA),  key = fmix(seed * 2^32 + aid),
// where fmix is SplitMix64's output mix.  This is the same definition the
// host-side generator implements, so both sides see identical inputs.
#include "check.cuh"
#include <cuda_bf16.h>

namespace bto {
namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__device__ __host__ __forceinline__ uint64_t fmix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double gen_value(uint64_t key, uint64_t k, int kind) {
    const uint64_t r = fmix(key + (k + 1) * kGamma) >> 11;
    if (kind == 0) return 2.0 * ((double)r * 0x1.0p-53) - 1.0;
    return (double)(r % 17ull) - 8.0;
}

template <typename T>
__device__ __forceinline__ T convert(double v);
template <> __device__ __forceinline__ double convert<double>(double v) { return v; }
template <> __device__ __forceinline__ float convert<float>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ uint16_t convert<uint16_t>(double v) {
    return __bfloat16_as_ushort(__double2bfloat16(v));
}

template <typename T>
__global__ void fill_kernel(uint64_t key, int kind, int64_t m, int64_t n, const double* colscale,
                            T* out, int64_t ld) {
    const int64_t total = m * n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += stride) {
        const int64_t j = k / m, i = k - j * m;
        double v = gen_value(key, (uint64_t)k, kind);
        if (colscale) v = v * colscale[j];
        out[i + j * ld] = convert<T>(v);
    }
}

template <typename T>
bto_status fill(uint64_t seed, uint64_t aid, int kind, int64_t m, int64_t n, const double* colscale,
                T* out, int64_t ld, bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    if (kind != 0 && kind != 1) c.fail(3);
    c.size(4, m); c.size(5, n);
    if (!c.ok()) return c.finish();
    c.ptr(6, colscale, false);
    c.ptr(7, out, m > 0 && n > 0, sizeof(T));
    c.ld(8, ld, m);
    if (!c.ok()) return c.finish();
    if (m == 0 || n == 0) return BTO_OK;
    DeviceInfo d;
    if (!device_info(&d)) return BTO_ERR_CUDA;
    const uint64_t key = fmix((seed << 32) + aid);
    const int64_t blocks = std::min<int64_t>(ceil_div(m * n, 256), (int64_t)d.sms * 16);
    fill_kernel<T><<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(key, kind, m, n, colscale, out, ld);
    return launch_status();
}

}  // namespace
}  // namespace bto

extern "C" bto_status bto_fill_f64(uint64_t seed, uint64_t aid, int kind, int64_t m, int64_t n,
                                   const double* colscale, double* out, int64_t ld,
                                   bto_stream_t stream) {
    return bto::fill<double>(seed, aid, kind, m, n, colscale, out, ld, stream);
}
extern "C" bto_status bto_fill_f32(uint64_t seed, uint64_t aid, int kind, int64_t m, int64_t n,
                                   const double* colscale, float* out, int64_t ld,
                                   bto_stream_t stream) {
    return bto::fill<float>(seed, aid, kind, m, n, colscale, out, ld, stream);
}
extern "C" bto_status bto_fill_bf16(uint64_t seed, uint64_t aid, int kind, int64_t m, int64_t n,
                                    const double* colscale, uint16_t* out, int64_t ld,
                                    bto_stream_t stream) {
    return bto::fill<uint16_t>(seed, aid, kind, m, n, colscale, out, ld, stream);
}
