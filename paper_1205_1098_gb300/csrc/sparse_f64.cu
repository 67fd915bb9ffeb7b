// Sparse (CSR) forms of BICGK and BATAX, FP64: the sparse matrix format the
// paper names as future work (Section VII), with the fusion its row-major
// BATAX shows (Fig. 1) carried to rows of a compressed matrix.
//
// A group of G lanes takes a row: the lanes stride over the row's stored
// entries, gather x (or p) by column index and sum the products in a fixed
// order (a per-lane chain, then a butterfly over the group), so the row
// result is bitwise reproducible.  The transposed product scatters each
// entry's contribution with an FP64 atomic add.  BICGK: q_i = sum a_ij p_j
// and s_j += a_ij r_i in the same sweep.  BATAX: t_i = sum a_ij x_j is
// complete inside the group after the butterfly (every lane holds it), so
// y_j += beta a_ij t_i follows over the same entries, which the group still
// holds in registers for rows of up to G * kHeld entries (longer rows re-read
// theirs from L1/L2): A is read from memory once and t never exists as a
// vector, the fusion of Section III that a dense column-major sweep cannot
// have without an exchange between blocks.
//
// Every index is checked before it is used: row pointers are clamped to
// [0, nnz] and entries with a column index outside [0, n) are skipped; either
// sets the status word at the start of the workspace to
// BTO_ERR_INVALID_VALUE, which bto_device_status reads.
#include "check.cuh"

namespace bto {
namespace {

constexpr int kSpThreads = 256;
constexpr int kHeld = 4;          // entries per lane kept in registers (BATAX)

enum SpMode { SP_BICGK = 0, SP_ATAX = 1 };

__global__ void __launch_bounds__(kSpThreads) sp_zero_kernel(double* s, int64_t n, int* status) {
    const int64_t stride = (int64_t)gridDim.x * kSpThreads;
    for (int64_t i = blockIdx.x * (int64_t)kSpThreads + threadIdx.x; i < n; i += stride) s[i] = 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *status = BTO_OK;
}

template <int G>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
    for (int off = G / 2; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// MODE SP_BICGK: q <- A p (out_row), s <- A^T r (out_col).
// MODE SP_ATAX:  out_col <- out_col + beta A^T (A x), with x in `xin`.
template <int MODE, int G>
__global__ void __launch_bounds__(kSpThreads) sp_kernel(int64_t m, int64_t n, int64_t nnz,
                                                        const int64_t* __restrict__ row_ptr,
                                                        const int32_t* __restrict__ col,
                                                        const double* __restrict__ val,
                                                        const double* __restrict__ xin,
                                                        const double* __restrict__ rin, double beta,
                                                        double* __restrict__ out_row, double* out_col,
                                                        int* status) {
    constexpr int kRowsPerWarp = 32 / G;
    const int lane = threadIdx.x & 31, l = lane % G;
    const int64_t warp = (blockIdx.x * (int64_t)kSpThreads + threadIdx.x) >> 5;
    const int64_t warps = (int64_t)gridDim.x * (kSpThreads / 32);
    bool bad = false;
    // Every lane of a warp runs the same iterations (the group sums shuffle
    // across the whole warp); lanes past the last row take an empty row.
    for (int64_t base = warp * kRowsPerWarp; base < m; base += warps * kRowsPerWarp) {
        const int64_t i = base + lane / G;
        const bool active = i < m;
        int64_t b = 0, e = 0;
        if (active) {
            b = __ldg(row_ptr + i);
            e = __ldg(row_ptr + i + 1);
            if (b < 0 || e < b || e > nnz) bad = true;
            b = b < 0 ? 0 : (b > nnz ? nnz : b);
            e = e < b ? b : (e > nnz ? nnz : e);
        }
        double acc = 0.0;
        if (MODE == SP_BICGK) {
            const double ri = active ? __ldg(rin + i) : 0.0;
            for (int64_t k = b + l; k < e; k += G) {
                const int c = __ldg(col + k);
                const double a = __ldg(val + k);
                if (c >= 0 && c < n) {
                    acc = fma(a, __ldg(xin + c), acc);
                    atomicAdd(out_col + c, a * ri);
                } else {
                    bad = true;
                }
            }
            acc = group_sum<G>(acc);
            if (active && l == 0) out_row[i] = acc;
        } else {
            // The lane's first kHeld entries stay in registers for the scatter.
            int hc[kHeld];
            double ha[kHeld];
#pragma unroll
            for (int h = 0; h < kHeld; h++) {
                const int64_t k = b + l + (int64_t)h * G;
                hc[h] = -1;
                ha[h] = 0.0;
                if (k < e) {
                    const int c = __ldg(col + k);
                    const double a = __ldg(val + k);
                    if (c >= 0 && c < n) {
                        acc = fma(a, __ldg(xin + c), acc);
                        hc[h] = c;
                        ha[h] = a;
                    } else {
                        bad = true;
                    }
                }
            }
            for (int64_t k = b + l + (int64_t)kHeld * G; k < e; k += G) {
                const int c = __ldg(col + k);
                if (c >= 0 && c < n) acc = fma(__ldg(val + k), __ldg(xin + c), acc);
                else bad = true;
            }
            const double t = beta * group_sum<G>(acc);     // every lane of the group holds beta t_i
#pragma unroll
            for (int h = 0; h < kHeld; h++)
                if (hc[h] >= 0) atomicAdd(out_col + hc[h], ha[h] * t);
            // Entries beyond the held ones are read again (from L1/L2).
            for (int64_t k = b + l + (int64_t)kHeld * G; k < e; k += G) {
                const int c = __ldg(col + k);
                if (c >= 0 && c < n) atomicAdd(out_col + c, __ldg(val + k) * t);
            }
        }
    }
    if (bad) *status = BTO_ERR_INVALID_VALUE;
}

// Lanes per row: the average row length rounded up to a power of two, 4..32.
int lanes_per_row(int64_t m, int64_t nnz) {
    const int64_t avg = m > 0 ? (nnz + m - 1) / m : 1;
    int g = 4;
    while (g < 32 && g < avg) g *= 2;
    return g;
}

template <int MODE>
bto_status launch_sp(int g, int grid, int64_t m, int64_t n, int64_t nnz, const int64_t* rp, const int32_t* col,
                     const double* val, const double* x, const double* r, double beta, double* orow,
                     double* ocol, int* status, cudaStream_t st) {
    switch (g) {
        case 4: sp_kernel<MODE, 4><<<grid, kSpThreads, 0, st>>>(m, n, nnz, rp, col, val, x, r, beta, orow, ocol, status); break;
        case 8: sp_kernel<MODE, 8><<<grid, kSpThreads, 0, st>>>(m, n, nnz, rp, col, val, x, r, beta, orow, ocol, status); break;
        case 16: sp_kernel<MODE, 16><<<grid, kSpThreads, 0, st>>>(m, n, nnz, rp, col, val, x, r, beta, orow, ocol, status); break;
        default: sp_kernel<MODE, 32><<<grid, kSpThreads, 0, st>>>(m, n, nnz, rp, col, val, x, r, beta, orow, ocol, status); break;
    }
    return launch_status();
}

// Shared checks of the CSR arguments (positions: m 1, n 2, nnz 3, row_ptr 4,
// col 5, val 6; vectors and outputs follow in each entry point).
void check_csr(Check& c, int64_t m, int64_t n, int64_t nnz, const int64_t* rp, const int32_t* col,
               const double* val) {
    c.size(1, m); c.size(2, n); c.size(3, nnz);
    if (n > INT32_MAX) c.fail(2);
    c.ptr(4, rp, m > 0);
    c.ptr(5, col, nnz > 0, 4);
    c.ptr(6, val, nnz > 0);
}

}  // namespace
}  // namespace bto

using namespace bto;

extern "C" bto_status bto_csr_bicgk(int64_t m, int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                                    const double* val, const double* p, const double* r, double* q, double* s,
                                    void* ws, size_t ws_bytes, bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    check_csr(c, m, n, nnz, row_ptr, col, val);
    if (!c.ok()) return c.finish();
    c.ptr(7, p, n > 0 && m > 0); c.ptr(8, r, m > 0 && n > 0); c.ptr(9, q, m > 0); c.ptr(10, s, n > 0);
    c.disjoint(9, q, vbytes(m), s, vbytes(n)); c.disjoint(9, q, vbytes(m), p, vbytes(n));
    c.disjoint(9, q, vbytes(m), r, vbytes(m)); c.disjoint(9, q, vbytes(m), val, vbytes(nnz));
    c.disjoint(10, s, vbytes(n), p, vbytes(n)); c.disjoint(10, s, vbytes(n), r, vbytes(m));
    c.disjoint(10, s, vbytes(n), val, vbytes(nnz));
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < WS_HEADER) c.fail(11, BTO_ERR_WORKSPACE);
    if (!c.ok()) return c.finish();
    DeviceInfo d;
    if (!device_info(&d)) return BTO_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    int* status = static_cast<int*>(ws);
    const int zgrid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kSpThreads), (int64_t)d.sms * 4));
    sp_zero_kernel<<<zgrid, kSpThreads, 0, st>>>(s, n, status);
    bto_status e = launch_status();
    if (e != BTO_OK || m == 0) return e;
    const int g = lanes_per_row(m, nnz);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(m * g, kSpThreads), (int64_t)d.sms * 8));
    return launch_sp<SP_BICGK>(g, grid, m, n, nnz, row_ptr, col, val, p, r, 0.0, q, s, status, st);
}

extern "C" bto_status bto_csr_atax(int64_t m, int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                                   const double* val, double beta, const double* x, double* y, void* ws,
                                   size_t ws_bytes, bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    check_csr(c, m, n, nnz, row_ptr, col, val);
    if (!c.ok()) return c.finish();
    c.ptr(8, x, n > 0 && m > 0); c.ptr(9, y, n > 0);
    c.disjoint(9, y, vbytes(n), x, vbytes(n)); c.disjoint(9, y, vbytes(n), val, vbytes(nnz));
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < WS_HEADER) c.fail(10, BTO_ERR_WORKSPACE);
    if (!c.ok()) return c.finish();
    DeviceInfo d;
    if (!device_info(&d)) return BTO_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    int* status = static_cast<int*>(ws);
    const int zgrid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kSpThreads), (int64_t)d.sms * 4));
    sp_zero_kernel<<<zgrid, kSpThreads, 0, st>>>(y, n, status);
    bto_status e = launch_status();
    if (e != BTO_OK || m == 0) return e;
    const int g = lanes_per_row(m, nnz);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(m * g, kSpThreads), (int64_t)d.sms * 8));
    return launch_sp<SP_ATAX>(g, grid, m, n, nnz, row_ptr, col, val, x, nullptr, beta, nullptr, y, status, st);
}
