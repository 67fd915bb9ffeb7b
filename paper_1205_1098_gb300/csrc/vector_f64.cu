// Fused FP64 vector kernels of Table I: AXPYDOT, WAXPBY, VADD.
//
// Each is one pass over its vectors with 16-byte loads (when every operand
// is 16-byte aligned) in batches of four pairs per thread, so each thread
// keeps several loads in flight.  AXPYDOT forms z and the dot product z^T u
// in the same pass: z never has to be read back.  The dot is summed per
// thread in a fixed element order, then per block by a fixed butterfly and
// warp order, and the block partials are added in block order by a second
// one-block kernel, so the result is bitwise reproducible.
#include "check.cuh"

namespace bto {

namespace {

constexpr int kThreads = 256;
constexpr int kBatch = 4;

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        s = red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) s += red[w];
    }
    return s;
}

// mode 0: z = w - alpha v, partial of z^T u.   mode 1: partial of w^T u.
template <bool VEC2, int MODE>
__global__ void __launch_bounds__(kThreads) dot_partials_kernel(int64_t n, double alpha,
        const double* w, const double* __restrict__ v, const double* __restrict__ u,
        double* z, double* __restrict__ partials) {
    __shared__ double red[kThreads / 32];
    const int64_t tid = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    double acc = 0.0;
    if (VEC2) {
        const int64_t n2 = n / 2;
        const double2* w2 = reinterpret_cast<const double2*>(w);
        const double2* v2 = reinterpret_cast<const double2*>(v);
        const double2* u2 = reinterpret_cast<const double2*>(u);
        double2* z2 = reinterpret_cast<double2*>(z);
        int64_t i = tid;
        for (; i + (kBatch - 1) * stride < n2; i += kBatch * stride) {
            double2 a[kBatch], b[kBatch], c[kBatch];
#pragma unroll
            for (int k = 0; k < kBatch; k++) {
                a[k] = w2[i + k * stride];
                if (MODE == 0) b[k] = __ldg(v2 + i + k * stride);
                c[k] = __ldg(u2 + i + k * stride);
            }
#pragma unroll
            for (int k = 0; k < kBatch; k++) {
                if (MODE == 0) {
                    double2 zz = make_double2(fma(-alpha, b[k].x, a[k].x), fma(-alpha, b[k].y, a[k].y));
                    z2[i + k * stride] = zz;
                    acc = fma(zz.x, c[k].x, acc);
                    acc = fma(zz.y, c[k].y, acc);
                } else {
                    acc = fma(a[k].x, c[k].x, acc);
                    acc = fma(a[k].y, c[k].y, acc);
                }
            }
        }
        for (; i < n2; i += stride) {
            double2 a = w2[i], c = __ldg(u2 + i);
            if (MODE == 0) {
                double2 b = __ldg(v2 + i);
                double2 zz = make_double2(fma(-alpha, b.x, a.x), fma(-alpha, b.y, a.y));
                z2[i] = zz;
                acc = fma(zz.x, c.x, acc);
                acc = fma(zz.y, c.y, acc);
            } else {
                acc = fma(a.x, c.x, acc);
                acc = fma(a.y, c.y, acc);
            }
        }
        if ((n & 1) && tid == 0) {
            const int64_t e = n - 1;
            double zz = (MODE == 0) ? fma(-alpha, __ldg(v + e), w[e]) : w[e];
            if (MODE == 0) z[e] = zz;
            acc = fma(zz, __ldg(u + e), acc);
        }
    } else {
        for (int64_t i = tid; i < n; i += stride) {
            double zz = (MODE == 0) ? fma(-alpha, __ldg(v + i), w[i]) : w[i];
            if (MODE == 0) z[i] = zz;
            acc = fma(zz, __ldg(u + i), acc);
        }
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) dot_final_kernel(const double* __restrict__ partials,
                                                            int count, double* r) {
    __shared__ double red[kThreads / 32];
    double acc = 0.0;
    for (int k = threadIdx.x; k < count; k += kThreads) acc += partials[k];
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) *r = s;
}

// w = alpha x + beta y
template <bool VEC2>
__global__ void __launch_bounds__(kThreads) waxpby_kernel(int64_t n, double alpha,
        const double* __restrict__ x, double beta, const double* __restrict__ y, double* __restrict__ w) {
    const int64_t tid = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    if (VEC2) {
        const int64_t n2 = n / 2;
        const double2* x2 = reinterpret_cast<const double2*>(x);
        const double2* y2 = reinterpret_cast<const double2*>(y);
        double2* w2 = reinterpret_cast<double2*>(w);
        int64_t i = tid;
        for (; i + (kBatch - 1) * stride < n2; i += kBatch * stride) {
            double2 a[kBatch], b[kBatch];
#pragma unroll
            for (int k = 0; k < kBatch; k++) { a[k] = __ldg(x2 + i + k * stride); b[k] = __ldg(y2 + i + k * stride); }
#pragma unroll
            for (int k = 0; k < kBatch; k++)
                w2[i + k * stride] = make_double2(fma(alpha, a[k].x, beta * b[k].x), fma(alpha, a[k].y, beta * b[k].y));
        }
        for (; i < n2; i += stride) {
            double2 a = __ldg(x2 + i), b = __ldg(y2 + i);
            w2[i] = make_double2(fma(alpha, a.x, beta * b.x), fma(alpha, a.y, beta * b.y));
        }
        if ((n & 1) && tid == 0) w[n - 1] = fma(alpha, x[n - 1], beta * y[n - 1]);
    } else {
        for (int64_t i = tid; i < n; i += stride) w[i] = fma(alpha, x[i], beta * y[i]);
    }
}

// x = (w + y) + z
template <bool VEC2>
__global__ void __launch_bounds__(kThreads) vadd_kernel(int64_t n, const double* __restrict__ w,
        const double* __restrict__ y, const double* __restrict__ z, double* __restrict__ x) {
    const int64_t tid = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    if (VEC2) {
        const int64_t n2 = n / 2;
        const double2* w2 = reinterpret_cast<const double2*>(w);
        const double2* y2 = reinterpret_cast<const double2*>(y);
        const double2* z2 = reinterpret_cast<const double2*>(z);
        double2* x2 = reinterpret_cast<double2*>(x);
        int64_t i = tid;
        for (; i + (kBatch - 1) * stride < n2; i += kBatch * stride) {
            double2 a[kBatch], b[kBatch], c[kBatch];
#pragma unroll
            for (int k = 0; k < kBatch; k++) {
                a[k] = __ldg(w2 + i + k * stride); b[k] = __ldg(y2 + i + k * stride); c[k] = __ldg(z2 + i + k * stride);
            }
#pragma unroll
            for (int k = 0; k < kBatch; k++)
                x2[i + k * stride] = make_double2((a[k].x + b[k].x) + c[k].x, (a[k].y + b[k].y) + c[k].y);
        }
        for (; i < n2; i += stride) {
            double2 a = __ldg(w2 + i), b = __ldg(y2 + i), c = __ldg(z2 + i);
            x2[i] = make_double2((a.x + b.x) + c.x, (a.y + b.y) + c.y);
        }
        if ((n & 1) && tid == 0) x[n - 1] = (w[n - 1] + y[n - 1]) + z[n - 1];
    } else {
        for (int64_t i = tid; i < n; i += stride) x[i] = (w[i] + y[i]) + z[i];
    }
}

int elementwise_grid(int64_t n, int sms) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 8, ceil_div(n, kThreads)));
}

}  // namespace

int vector_grid(int sms) { return sms * 4; }

bto_status launch_dot_partials(int64_t n, double alpha, const double* w, const double* v,
                               const double* u, double* z, double* partials, int grid, int mode,
                               cudaStream_t st) {
    const bool vec2 = aligned16(w) && aligned16(u) && (mode == 1 || (aligned16(v) && aligned16(z)));
    if (mode == 0) {
        if (vec2) dot_partials_kernel<true, 0><<<grid, kThreads, 0, st>>>(n, alpha, w, v, u, z, partials);
        else dot_partials_kernel<false, 0><<<grid, kThreads, 0, st>>>(n, alpha, w, v, u, z, partials);
    } else {
        if (vec2) dot_partials_kernel<true, 1><<<grid, kThreads, 0, st>>>(n, alpha, w, v, u, z, partials);
        else dot_partials_kernel<false, 1><<<grid, kThreads, 0, st>>>(n, alpha, w, v, u, z, partials);
    }
    return launch_status();
}

bto_status launch_dot_final(const double* partials, int grid, double* r, cudaStream_t st) {
    dot_final_kernel<<<1, kThreads, 0, st>>>(partials, grid, r);
    return launch_status();
}

bto_status launch_waxpby(int64_t n, double alpha, const double* x, double beta, const double* y,
                         double* w, int sms, cudaStream_t st) {
    if (n == 0) return BTO_OK;
    const int g = elementwise_grid(n, sms);
    if (aligned16(x) && aligned16(y) && aligned16(w))
        waxpby_kernel<true><<<g, kThreads, 0, st>>>(n, alpha, x, beta, y, w);
    else
        waxpby_kernel<false><<<g, kThreads, 0, st>>>(n, alpha, x, beta, y, w);
    return launch_status();
}

bto_status launch_vadd(int64_t n, const double* w, const double* y, const double* z, double* x,
                       int sms, cudaStream_t st) {
    if (n == 0) return BTO_OK;
    const int g = elementwise_grid(n, sms);
    if (aligned16(w) && aligned16(y) && aligned16(z) && aligned16(x))
        vadd_kernel<true><<<g, kThreads, 0, st>>>(n, w, y, z, x);
    else
        vadd_kernel<false><<<g, kThreads, 0, st>>>(n, w, y, z, x);
    return launch_status();
}

}  // namespace bto

using namespace bto;

extern "C" bto_status bto_axpydot(int64_t n, double alpha, const double* w, const double* v,
                                  const double* u, double* z, double* r, void* ws,
                                  size_t ws_bytes, bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    c.size(1, n);
    if (!c.ok()) return c.finish();
    c.ptr(3, w, n > 0); c.ptr(4, v, n > 0); c.ptr(5, u, n > 0); c.ptr(6, z, n > 0); c.ptr(7, r, true);
    if (z != w) c.disjoint(6, z, vbytes(n), w, vbytes(n));
    c.disjoint(6, z, vbytes(n), v, vbytes(n)); c.disjoint(6, z, vbytes(n), u, vbytes(n));
    c.disjoint(7, r, 8, w, vbytes(n)); c.disjoint(7, r, 8, v, vbytes(n));
    c.disjoint(7, r, 8, u, vbytes(n)); c.disjoint(7, r, 8, z, vbytes(n));
    DeviceInfo d; WsLayout L;
    if (c.ok()) {
        if (!device_info(&d)) return BTO_ERR_CUDA;
        if (ws_layout(BTO_OP_AXPYDOT, BTO_FORM_FUSED, 0, n, BTO_F64, d, &L) != BTO_OK) return BTO_ERR_CUDA;
        c.ws(8, ws, ws_bytes, L);
    }
    if (!c.ok()) return c.finish();
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = vector_grid(d.sms);
    double* part = reinterpret_cast<double*>(static_cast<char*>(ws) + L.off[0]);
    bto_status e = launch_dot_partials(n, alpha, w, v, u, z, part, grid, 0, st);
    if (e != BTO_OK) return e;
    return launch_dot_final(part, grid, r, st);
}

extern "C" bto_status bto_waxpby(int64_t n, double alpha, const double* x, double beta,
                                 const double* y, double* w, bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    c.size(1, n);
    if (!c.ok()) return c.finish();
    c.ptr(3, x, n > 0); c.ptr(5, y, n > 0); c.ptr(6, w, n > 0);
    c.disjoint(6, w, vbytes(n), x, vbytes(n)); c.disjoint(6, w, vbytes(n), y, vbytes(n));
    if (!c.ok()) return c.finish();
    DeviceInfo d;
    if (!device_info(&d)) return BTO_ERR_CUDA;
    return launch_waxpby(n, alpha, x, beta, y, w, d.sms, (cudaStream_t)stream);
}

extern "C" bto_status bto_vadd(int64_t n, const double* w, const double* y, const double* z,
                               double* x, bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    c.size(1, n);
    if (!c.ok()) return c.finish();
    c.ptr(2, w, n > 0); c.ptr(3, y, n > 0); c.ptr(4, z, n > 0); c.ptr(5, x, n > 0);
    c.disjoint(5, x, vbytes(n), w, vbytes(n)); c.disjoint(5, x, vbytes(n), y, vbytes(n));
    c.disjoint(5, x, vbytes(n), z, vbytes(n));
    if (!c.ok()) return c.finish();
    DeviceInfo d;
    if (!device_info(&d)) return BTO_ERR_CUDA;
    return launch_vadd(n, w, y, z, x, d.sms, (cudaStream_t)stream);
}
