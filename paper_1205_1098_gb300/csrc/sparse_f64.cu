// Sparse (CSR) forms of BICGK and BATAX, FP64: the sparse matrix format the
// paper names as future work (Section VII).
//
// The stored entries are split evenly, not the rows: a warp takes a unit of
// 256 consecutive entries and each lane 8 consecutive ones, so every lane is
// busy whatever the row lengths (with one lane group per row, short rows left
// lanes idle while their FP64 instructions still occupied the pipe).  A lane
// finds the row of its first entry by a binary search of the row pointers
// between the unit's first and last rows (found once per unit by a pre-pass),
// then walks its entries, closing rows as it passes their ends.  Per entry:
//   - one FMA into the running row sum (q = A p, or t = A x for BATAX),
//   - one product scattered into the column output with an FP64 atomic add
//     (s = A^T r; BATAX's y = beta A^T t in its second pass).
// Row sums: a row that begins and ends inside one lane's 8 entries is
// written by that lane.  A row that crosses lanes is summed by a segmented
// scan over the lanes (5 shuffle rounds, keyed by row), and closed by the
// lane where it ends.  A row that crosses units leaves the part in its own
// unit in the output, and each later unit's part in a carry slot; a fix-up
// kernel adds the carries in unit order.  Every row sum is therefore formed
// in a fixed order (bitwise reproducible); the column outputs are sums of
// atomic adds (reproducible to rounding only).
//
// BATAX runs the row pass (t in the workspace), the fix-up, then a second
// entry sweep that scatters beta t_i A(i, j): A is read twice.
//
// Every index is checked before use.  The pre-pass checks the row pointers
// (in [0, nnz], nondecreasing); if any is bad it sets the status word at the
// start of the workspace to BTO_ERR_INVALID_VALUE and the sweeps take a
// plain row-by-row path with clamped pointers instead.  Entries with a
// column index outside [0, n) are skipped on either path and set the same
// status.
#include "check.cuh"

namespace bto {
namespace {

constexpr int kSpThreads = 256;
constexpr int kE = 8;                  // entries per lane per unit
constexpr int kUnit = 32 * kE;         // entries per warp unit

enum SpMode { SP_BICGK = 0, SP_ROWS = 1, SP_SCATTER = 2 };

struct CsrArgs {
    int64_t m, n, nnz, units;
    const int64_t* rp;
    const int32_t* col;
    const double* val;
    const double* x;        // row-product vector (p or x), n
    const double* r;        // BICGK: r (m); SCATTER: t (m)
    double beta;            // SCATTER
    double* rows;           // row outputs (q or t), m
    double* cols;           // column outputs (s or y), n, zeroed by the pre-pass
    int64_t* ustart;        // [units + 1]: row holding each unit's first entry
    int64_t* crow;          // [units]: row carried into the unit from before it, or -1
    double* carry;          // [units]
    int* status;            // the workspace status word
    int* rpbad;             // set by the pre-pass when a row pointer is malformed
};

__device__ __forceinline__ int64_t rp_at(const CsrArgs& a, int64_t r) {
    const int64_t v = __ldg(a.rp + r);
    return v < 0 ? 0 : (v > a.nnz ? a.nnz : v);
}

// Pre-pass: zero the column outputs, check the row pointers, write zero to
// the trailing empty rows (those starting at nnz, which no unit visits), and
// find each unit's first row (the largest r < m with rp[r] <= unit start).
__global__ void __launch_bounds__(kSpThreads) csr_prepass(const CsrArgs a, bool row_out) {
    const int64_t stride = (int64_t)gridDim.x * kSpThreads;
    const int64_t t0 = (int64_t)blockIdx.x * kSpThreads + threadIdx.x;
    bool bad = false;
    for (int64_t j = t0; j < a.n; j += stride) a.cols[j] = 0.0;
    for (int64_t r = t0; r < a.m; r += stride) {
        const int64_t b = __ldg(a.rp + r), e = __ldg(a.rp + r + 1);
        if (b < 0 || e < b || e > a.nnz) bad = true;
        if (row_out && (b < 0 ? 0 : (b > a.nnz ? a.nnz : b)) >= a.nnz) a.rows[r] = 0.0;
    }
    for (int64_t u = t0; u < a.units; u += stride) {
        const int64_t K0 = u * kUnit;
        int64_t lo = 0, hi = a.m - 1;          // largest r in [0, m-1] with rp[r] <= K0
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo + 1) / 2;
            if (rp_at(a, mid) <= K0) lo = mid; else hi = mid - 1;
        }
        a.ustart[u] = lo;
    }
    if (t0 == 0) a.ustart[a.units] = a.m - 1;
    if (bad) {
        *a.status = BTO_ERR_INVALID_VALUE;
        *a.rpbad = 1;
    }
}

// The plain path for malformed row pointers: one warp per row, clamped
// bounds, lanes strided over the row, a butterfly sum.
template <int MODE>
__device__ void csr_rows_safe(const CsrArgs& a) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * kSpThreads + threadIdx.x) >> 5;
    const int64_t warps = (int64_t)gridDim.x * (kSpThreads / 32);
    bool bad = false;
    for (int64_t i = warp; i < a.m; i += warps) {
        int64_t b = rp_at(a, i), e = rp_at(a, i + 1);
        if (e < b) e = b;
        double acc = 0.0;
        const double ri = MODE == SP_BICGK ? __ldg(a.r + i) : (MODE == SP_SCATTER ? a.beta * __ldg(a.r + i) : 0.0);
        for (int64_t k = b + lane; k < e; k += 32) {
            const int c = __ldg(a.col + k);
            if (c < 0 || c >= a.n) { bad = true; continue; }
            const double v = __ldg(a.val + k);
            if (MODE != SP_SCATTER) acc = fma(v, __ldg(a.x + c), acc);
            if (MODE != SP_ROWS) atomicAdd(a.cols + c, v * ri);
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (MODE != SP_SCATTER && lane == 0) a.rows[i] = acc;
    }
    if (bad) *a.status = BTO_ERR_INVALID_VALUE;
}

template <int MODE>
__global__ void __launch_bounds__(kSpThreads, 3) csr_unit_kernel(const CsrArgs a) {
    if (*(volatile int*)a.rpbad != 0) {
        csr_rows_safe<MODE>(a);
        return;
    }
    constexpr bool ROWS = MODE != SP_SCATTER;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * kSpThreads + threadIdx.x) >> 5;
    const int64_t warps = (int64_t)gridDim.x * (kSpThreads / 32);
    const bool vec = ((reinterpret_cast<uintptr_t>(a.val) | reinterpret_cast<uintptr_t>(a.col)) & 15u) == 0;
    bool bad = false;

    for (int64_t u = warp; u < a.units; u += warps) {
        const int64_t K0 = u * kUnit;
        const int64_t K1 = (K0 + kUnit < a.nnz) ? K0 + kUnit : a.nnz;
        const int64_t ks = K0 + (int64_t)lane * kE;
        const int64_t ke = (ks + kE < K1) ? ks + kE : K1;
        const bool live = ks < K1;
        const int64_t Rlo = a.ustart[u], Rhi = a.ustart[u + 1];

        // Entries of the lane.
        double av[kE];
        int cv[kE];
        if (live && vec && ke - ks == kE) {
            const double2* v2 = reinterpret_cast<const double2*>(a.val + ks);
#pragma unroll
            for (int h = 0; h < kE / 2; h++) {
                const double2 t = __ldg(v2 + h);
                av[2 * h] = t.x; av[2 * h + 1] = t.y;
            }
            const int4* c4 = reinterpret_cast<const int4*>(a.col + ks);
#pragma unroll
            for (int h = 0; h < kE / 4; h++) {
                const int4 t = __ldg(c4 + h);
                cv[4 * h] = t.x; cv[4 * h + 1] = t.y; cv[4 * h + 2] = t.z; cv[4 * h + 3] = t.w;
            }
        } else {
#pragma unroll
            for (int e = 0; e < kE; e++) {
                const bool in = live && ks + e < ke;
                av[e] = in ? __ldg(a.val + ks + e) : 0.0;
                cv[e] = in ? __ldg(a.col + ks + e) : -1;
            }
        }

        // Row of every entry: r0 = largest r in [Rlo, Rhi] with rp[r] <= ks,
        // then advance past each row end (and the empty rows behind it).
        int64_t r0 = Rlo;
        int ridx[kE];
        int64_t rend = 0, rbeg0 = 0;
        bool end_closed = false;
        if (live) {
            int64_t lo = Rlo, hi = Rhi;
            while (lo < hi) {
                const int64_t mid = lo + (hi - lo + 1) / 2;
                if (rp_at(a, mid) <= ks) lo = mid; else hi = mid - 1;
            }
            r0 = lo;
            rbeg0 = rp_at(a, r0);
            rend = rp_at(a, r0 + 1);
            int cur = 0;
#pragma unroll
            for (int e = 0; e < kE; e++) {
                const int64_t k = ks + e;
                if (k < ke) {
                    while (k >= rend && r0 + cur < a.m - 1) {
                        cur++;
                        rend = rp_at(a, r0 + cur + 1);
                    }
                }
                ridx[e] = cur;
            }
            end_closed = rend == ke;
            // Empty rows that start exactly at ks (ahead of r0) belong to this lane.
            if (ROWS && rbeg0 == ks)
                for (int64_t rr = r0 - 1; rr >= 0 && rp_at(a, rr) == ks; rr--) a.rows[rr] = 0.0;
        } else {
#pragma unroll
            for (int e = 0; e < kE; e++) ridx[e] = 0;
        }
        const bool first_before = live && rbeg0 < ks;   // first row began in an earlier lane or unit

        // Gathers, issued before the arithmetic.
        double xv[kE];
#pragma unroll
        for (int e = 0; e < kE; e++) {
            const int c = cv[e];
            const bool ok = c >= 0 && c < a.n;
            if (ks + e < ke && live && !ok) bad = true;
            if (MODE != SP_SCATTER) xv[e] = (ok && live && ks + e < ke) ? __ldg(a.x + c) : 0.0;
        }

        // Walk: row sums and the scatter.
        double acc = 0.0, h = 0.0;
        int64_t hk = -1;
        int cur = 0;
        double rcur = 0.0;
        if (live && MODE != SP_ROWS) {
            rcur = __ldg(a.r + r0);
            if (MODE == SP_SCATTER) rcur *= a.beta;
        }
#pragma unroll
        for (int e = 0; e < kE; e++) {
            if (!live || ks + e >= ke) continue;
            while (ridx[e] > cur) {            // close rows ending before entry e
                if (ROWS) {
                    if (cur == 0 && first_before) { h = acc; hk = r0; }
                    else a.rows[r0 + cur] = acc;
                }
                acc = 0.0;
                cur++;
                if (MODE != SP_ROWS) {
                    rcur = __ldg(a.r + r0 + cur);
                    if (MODE == SP_SCATTER) rcur *= a.beta;
                }
            }
            const int c = cv[e];
            if (c >= 0 && c < a.n) {
                if (ROWS) acc = fma(av[e], xv[e], acc);
                if (MODE != SP_ROWS) atomicAdd(a.cols + c, av[e] * rcur);
            }
        }
        if (!ROWS) continue;

        // The row open at the lane's end (if it does not end there).
        int64_t key = -1;
        double v = 0.0;
        if (live) {
            if (end_closed) {
                if (cur == 0 && first_before) { h = acc; hk = r0; }
                else a.rows[r0 + cur] = acc;
            } else {
                key = r0 + cur;
                v = acc;
            }
        } else {
            key = -2;
        }
        // Segmented inclusive scan of the open parts over the lanes, keyed
        // by row (equal keys are adjacent lanes).
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const double uv = __shfl_up_sync(0xffffffffu, v, d);
            const int64_t uk = __shfl_up_sync(0xffffffffu, key, d);
            if (lane >= d && uk == key) v += uv;
        }
        const double pv = __shfl_up_sync(0xffffffffu, v, 1);
        const int64_t pk = __shfl_up_sync(0xffffffffu, key, 1);
        const int64_t crow = (__shfl_sync(0xffffffffu, (int)first_before, 0) != 0) ? Rlo : -1;
        if (lane == 0) a.crow[u] = crow;
        if (hk >= 0) {
            const double tot = (lane > 0 && pk == hk) ? pv + h : h;
            if (hk == crow) a.carry[u] = tot;
            else a.rows[hk] = tot;
        }
        if (live && ke == K1 && key >= 0) {    // the unit's last lane: a row still open
            if (key == crow) a.carry[u] = v;
            else a.rows[key] = v;
        }
    }
    if (bad) *a.status = BTO_ERR_INVALID_VALUE;
}

// Adds each unit's carry to the row it belongs to, in unit order (the first
// unit of a run of equal carry rows adds the whole run).
__global__ void __launch_bounds__(kSpThreads) csr_fixup(const CsrArgs a) {
    if (*(volatile int*)a.rpbad != 0) return;
    const int64_t u = (int64_t)blockIdx.x * kSpThreads + threadIdx.x;
    if (u >= a.units) return;
    const int64_t cr = a.crow[u];
    if (cr < 0 || (u > 0 && a.crow[u - 1] == cr)) return;
    double sum = a.carry[u];
    for (int64_t w = u + 1; w < a.units && a.crow[w] == cr; w++) sum += a.carry[w];
    a.rows[cr] += sum;
}

struct CsrWs {
    size_t ustart = 0, crow = 0, carry = 0, t = 0, total = 0;
};

CsrWs csr_ws(int64_t m, int64_t nnz, bool atax) {
    CsrWs w;
    const int64_t units = ceil_div(nnz, kUnit);
    size_t off = WS_HEADER;
    w.ustart = off; off += round_up((units + 1) * 8, 256);
    w.crow = off;   off += round_up(units * 8, 256);
    w.carry = off;  off += round_up(units * 8, 256);
    if (atax) { w.t = off; off += round_up(m * 8, 256); }
    w.total = off;
    return w;
}

int sp_grid(const DeviceInfo& d, int64_t work_warps) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(work_warps, kSpThreads / 32), (int64_t)d.sms * 8));
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

bto_status csr_launch(int mode, CsrArgs a, const DeviceInfo& d, cudaStream_t st) {
    const int g = sp_grid(d, std::max<int64_t>(a.units, 1));
    if (mode == SP_BICGK) csr_unit_kernel<SP_BICGK><<<g, kSpThreads, 0, st>>>(a);
    else if (mode == SP_ROWS) csr_unit_kernel<SP_ROWS><<<g, kSpThreads, 0, st>>>(a);
    else csr_unit_kernel<SP_SCATTER><<<g, kSpThreads, 0, st>>>(a);
    bto_status e = launch_status();
    if (e != BTO_OK || mode == SP_SCATTER || a.units == 0) return e;
    csr_fixup<<<(int)ceil_div(a.units, kSpThreads), kSpThreads, 0, st>>>(a);
    return launch_status();
}

bto_status csr_prepare(CsrArgs& a, void* ws, bool row_out, const DeviceInfo& d, cudaStream_t st) {
    if (cudaMemsetAsync(ws, 0, 16, st) != cudaSuccess) return BTO_ERR_CUDA;   // status and row-pointer flag
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(
        ceil_div(std::max<int64_t>(std::max(a.m, a.n), a.units + 1), kSpThreads), (int64_t)d.sms * 8));
    csr_prepass<<<g, kSpThreads, 0, st>>>(a, row_out);
    return launch_status();
}

}  // namespace
}  // namespace bto

using namespace bto;

extern "C" bto_status bto_csr_workspace_bytes(int op, int64_t m, int64_t n, int64_t nnz, size_t* bytes) {
    clear_invalid_arg();
    Check c;
    if (op != BTO_OP_BICGK && op != BTO_OP_ATAX) c.fail(1);
    c.size(2, m); c.size(3, n); c.size(4, nnz);
    c.ptr(5, bytes, true, 1);
    if (!c.ok()) return c.finish();
    *bytes = csr_ws(m, nnz, op == BTO_OP_ATAX).total;
    return BTO_OK;
}

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
    const CsrWs W = csr_ws(m, nnz, false);
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < W.total) c.fail(11, BTO_ERR_WORKSPACE);
    if (!c.ok()) return c.finish();
    DeviceInfo d;
    if (!device_info(&d)) return BTO_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    char* w = static_cast<char*>(ws);
    CsrArgs a;
    a.m = m; a.n = n; a.nnz = m > 0 ? nnz : 0; a.units = m > 0 ? ceil_div(nnz, kUnit) : 0;
    a.rp = row_ptr; a.col = col; a.val = val; a.x = p; a.r = r; a.beta = 1.0;
    a.rows = q; a.cols = s;
    a.ustart = reinterpret_cast<int64_t*>(w + W.ustart);
    a.crow = reinterpret_cast<int64_t*>(w + W.crow);
    a.carry = reinterpret_cast<double*>(w + W.carry);
    a.status = static_cast<int*>(ws);
    a.rpbad = reinterpret_cast<int*>(w + 8);
    bto_status e = csr_prepare(a, ws, true, d, st);
    if (e != BTO_OK || m == 0) return e;
    return csr_launch(SP_BICGK, a, d, st);
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
    const CsrWs W = csr_ws(m, nnz, true);
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < W.total) c.fail(10, BTO_ERR_WORKSPACE);
    if (!c.ok()) return c.finish();
    DeviceInfo d;
    if (!device_info(&d)) return BTO_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    char* w = static_cast<char*>(ws);
    CsrArgs a;
    a.m = m; a.n = n; a.nnz = m > 0 ? nnz : 0; a.units = m > 0 ? ceil_div(nnz, kUnit) : 0;
    a.rp = row_ptr; a.col = col; a.val = val; a.x = x; a.beta = beta;
    a.rows = reinterpret_cast<double*>(w + W.t); a.cols = y;
    a.ustart = reinterpret_cast<int64_t*>(w + W.ustart);
    a.crow = reinterpret_cast<int64_t*>(w + W.crow);
    a.carry = reinterpret_cast<double*>(w + W.carry);
    a.status = static_cast<int*>(ws);
    a.rpbad = reinterpret_cast<int*>(w + 8);
    bto_status e = csr_prepare(a, ws, true, d, st);
    if (e != BTO_OK || m == 0) return e;
    // t = A x (rows), then y = beta A^T t (scatter, reading t).
    if ((e = csr_launch(SP_ROWS, a, d, st)) != BTO_OK) return e;
    a.r = a.rows;
    return csr_launch(SP_SCATTER, a, d, st);
}
