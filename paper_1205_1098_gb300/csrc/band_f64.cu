// BICGK and BATAX on banded and triangular matrices, the structured formats
// the paper plans beside sparse ones (Section VII).
//
// A is m x n with A(i, j) = 0 outside j - ku <= i <= j + kl.  The sweep
// works in band coordinates: band row rho = i - j + ku (0 <= rho <= kl + ku)
// and column j, so that every storage kind addresses a column as one
// contiguous run of rho:
//   full storage   A(i, j) = A[j*ld + i]           -> A[j*(ld+1) - ku + rho]
//   band storage   A(i, j) = A[j*ld + ku + i - j]  -> A[j*ld + rho]
//   packed upper   column j holds rows 0..j after j(j+1)/2 entries
//   packed lower   column j holds rows j..n-1 after j*n - j(j-1)/2 entries
// A tile is RT band rows x 128 columns; warp w of the 8 takes 16 consecutive
// columns, lane l band rows rho0 + 32k + l (k < RT/32).  Per column the lane
//   - adds A(i, j) r_i into the column's partial (r_i read from a shared
//     window of r, since i moves with j at fixed rho),
//   - adds A(i, j) p_j into its warp's shared window of row partials (row i
//     sits at window slot rho - rho0 + j - jw, so successive columns of one
//     lane walk down the window; a warp barrier orders them).
// Only entries inside the band enter the sums: a slot of 32 band rows that
// misses a column's band is skipped by the whole warp, and within a slot the
// lanes outside it neither load nor add.  The 16 column partials of a warp
// meet in the transposing butterfly; the 8 warp windows are added in warp
// order into the tile's row partials.  Blocks take tiles from an atomic
// counter and skip the tiles that hold no entry.  Two combine kernels add
// the partials of every output in a fixed order (band-row tiles ascending,
// then column tiles), so results are bitwise reproducible.
//
// Arithmetic is FP64 FMA: two per stored entry, the FP64 pipe is the bound
// (HBM would allow about three times the rate).
#include "internal.cuh"
#include "check.cuh"
#include <algorithm>

namespace bto {

namespace {

constexpr int kBWarps = 8;
constexpr int kBThreads = kBWarps * 32;
constexpr int kBCols = 16;                    // columns per warp per tile
constexpr int kCT = kBWarps * kBCols;         // 128 columns per tile
constexpr size_t kCounterOff = 64;            // tile counters in the workspace header

enum BandMode { BM_QS = 0, BM_Q = 1, BM_S = 2 };

// Geometry of one structured operand (host-computed, passed by value).
struct BandGeom {
    int storage = 0, unit = 0;
    int64_t m = 0, n = 0, kl = 0, ku = 0, ld = 0;
    int64_t rho_a = 0;     // first band row holding an entry
    int64_t rho_b = -1;    // last band row holding an entry
    int64_t ncols = 0;     // columns holding an entry: min(n, ku + m)
    int rt = 32;           // band rows per tile
    int64_t ntr = 0, ncb = 0;
    int64_t lq = 0;        // stride of a tile's row partials (its window spans rt + 127 rows)
};

struct BandArgs {
    BandGeom g;
    const double* A;
    const double* p;       // row-product vector (n)
    const double* r;       // column-product vector (m)
    double* qpart;         // [ntr * ncb][lq] row partials
    double* spart;         // [ntr][n] column partials
    unsigned long long* counter;
};

// Band rows of column j that hold entries: [vlo, vhi] (empty when vlo > vhi).
__host__ __device__ __forceinline__ int64_t band_vlo(const BandGeom& g, int64_t j) {
    return g.ku - j > 0 ? g.ku - j : 0;
}
__host__ __device__ __forceinline__ int64_t band_vhi(const BandGeom& g, int64_t j) {
    const int64_t a = g.kl + g.ku, b = g.ku - j + g.m - 1;
    return a < b ? a : b;
}

// Element offset of band row 0 of column j (A(i, j) at offset + rho).
__device__ __forceinline__ int64_t col_rho_base(const BandGeom& g, int64_t j) {
    switch (g.storage) {
        case BTO_STORE_FULL: return j * (g.ld + 1) - g.ku;
        case BTO_STORE_BAND: return j * g.ld;
        default:
            if (g.kl == 0) return j * (j + 1) / 2 + j - g.ku;           // packed upper
            return j * g.n - j * (j + 1) / 2 + j - g.ku;               // packed lower
    }
}

// Does tile (tr, cb) hold an entry?  The band rows of consecutive columns
// are overlapping intervals moving down, so the rows of the tile's columns
// form one interval [vlo(last column), vhi(first column)].
__host__ __device__ __forceinline__ bool tile_nonempty(const BandGeom& g, int64_t tr, int64_t cb) {
    const int64_t j0 = cb * kCT;
    int64_t jl = j0 + kCT;
    if (jl > g.ncols) jl = g.ncols;
    jl -= 1;
    if (j0 > jl) return false;
    const int64_t rho0 = g.rho_a + tr * g.rt;
    return rho0 <= band_vhi(g, j0) && rho0 + g.rt - 1 >= band_vlo(g, jl);
}

__device__ __forceinline__ int64_t floor_div(int64_t a, int64_t b) {
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}

template <int MODE, int RPL>
__global__ void __launch_bounds__(kBThreads, (MODE == BM_QS && RPL == 8) ? 2 : 3) band_kernel(const BandArgs a) {
    constexpr bool HQ = MODE != BM_S, HS = MODE != BM_Q;
    constexpr int RT = 32 * RPL;
    constexpr int QW = RT + kBCols;           // a warp's row-partial window
    __shared__ double rw[RT + kCT];           // r_i for the tile's rows
    __shared__ double qw[kBWarps][QW];
    __shared__ long long tile_s;
    const BandGeom& g = a.g;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = g.ntr * g.ncb;

    for (;;) {
        if (threadIdx.x == 0) {
            // Claim tiles until one holds an entry (or none are left).
            long long t;
            do {
                t = (long long)atomicAdd(a.counter, 1ull);
            } while (t < ntiles && !tile_nonempty(g, t / g.ncb, t % g.ncb));
            tile_s = t;
        }
        __syncthreads();
        const long long t = tile_s;
        if (t >= ntiles) break;
        const int64_t tr = t / g.ncb, cb = t % g.ncb;
        const int64_t rho0 = g.rho_a + tr * RT;
        const int64_t j0 = cb * kCT;
        const int64_t ib = rho0 + j0 - g.ku;  // row of window slot 0

        if (HS) {
            for (int x = threadIdx.x; x < RT + kCT; x += kBThreads) {
                const int64_t i = ib + x;
                rw[x] = (i >= 0 && i < g.m) ? __ldg(a.r + i) : 0.0;
            }
        }
        if (HQ) {
            for (int x = threadIdx.x; x < kBWarps * QW; x += kBThreads) (&qw[0][0])[x] = 0.0;
        }
        __syncthreads();

        const int64_t jw = j0 + warp * kBCols;
        double sl[kBCols];
        // The next column's entries are loaded before the current column's
        // arithmetic (two register buffers taking turns).
        double av[2][RPL];
        bool ok[2][RPL];
        auto fetch = [&](int jj, double (&v)[RPL], bool (&f)[RPL]) {
            const int64_t j = jw + jj;
#pragma unroll
            for (int k = 0; k < RPL; k++) { v[k] = 0.0; f[k] = false; }
            if (j >= g.ncols) return;
            const int64_t vlo = band_vlo(g, j) - rho0, vhi = band_vhi(g, j) - rho0;
            const double* col = a.A + col_rho_base(g, j) + rho0;
            const int64_t diag = g.unit ? g.ku - rho0 : -1;
#pragma unroll
            for (int k = 0; k < RPL; k++) {
                const int rr = 32 * k + lane;
                if (32 * k <= vhi && 32 * k + 31 >= vlo) {        // warp-uniform
                    f[k] = rr >= vlo && rr <= vhi;
                    if (f[k]) v[k] = (rr == diag) ? 1.0 : __ldg(col + rr);
                }
            }
        };
        fetch(0, av[0], ok[0]);
#pragma unroll
        for (int jj = 0; jj < kBCols; jj++) {
            const int cur = jj & 1;
            if (jj + 1 < kBCols) fetch(jj + 1, av[cur ^ 1], ok[cur ^ 1]);
            const int64_t j = jw + jj;
            double sacc = 0.0;
            if (j < g.ncols) {
                const double pj = HQ ? __ldg(a.p + j) : 0.0;
                const int off = (int)(j - j0);
#pragma unroll
                for (int k = 0; k < RPL; k++) {
                    if (ok[cur][k]) {
                        const int rr = 32 * k + lane;
                        if (HQ) qw[warp][rr + jj] = fma(av[cur][k], pj, qw[warp][rr + jj]);
                        if (HS) sacc = fma(av[cur][k], rw[rr + off], sacc);
                    }
                }
            }
            sl[jj] = sacc;
            if (HQ) __syncwarp();
        }
        if (HS) {
            const double cs = transpose_reduce16(sl, lane);
            if (lane < kBCols && jw + lane < g.n) a.spart[tr * g.n + jw + lane] = cs;
        }
        __syncthreads();
        if (HQ) {
            double* out = a.qpart + t * g.lq;
            for (int x = threadIdx.x; x < RT + kCT - 1; x += kBThreads) {
                double acc = 0.0;
#pragma unroll
                for (int w = 0; w < kBWarps; w++) {
                    const int u = x - w * kBCols;
                    if (u >= 0 && u < QW) acc += qw[w][u];
                }
                out[x] = acc;
            }
        }
        __syncthreads();
    }
}

// Row outputs: q_i = scale * (sum of the row partials of every tile whose
// window holds row i), tiles in (band-row tile, column tile) order.
__global__ void band_q_combine(const BandGeom g, const double* __restrict__ qpart, double* __restrict__ q) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.m) return;
    double acc = 0.0;
    if (g.n > 0 && g.rho_b >= g.rho_a) {
        // band rows of row i's entries
        const int64_t jhi = (i + g.ku < g.n - 1) ? i + g.ku : g.n - 1;
        const int64_t jlo = i - g.kl > 0 ? i - g.kl : 0;
        if (jlo <= jhi) {
            const int64_t rlo = i + g.ku - jhi, rhi = i + g.ku - jlo;
            const int64_t tlo = (rlo - g.rho_a) / g.rt, thi = (rhi - g.rho_a) / g.rt;
            const int64_t wq = g.rt + kCT - 1;          // rows a tile's window spans
            for (int64_t tr = tlo; tr <= thi && tr < g.ntr; tr++) {
                const int64_t rho0 = g.rho_a + tr * g.rt;
                int64_t c0 = floor_div(i + g.ku - rho0 - wq + 1 + kCT - 1, kCT);
                int64_t c1 = floor_div(i + g.ku - rho0, kCT);
                if (c0 < 0) c0 = 0;
                if (c1 > g.ncb - 1) c1 = g.ncb - 1;
                for (int64_t cb = c0; cb <= c1; cb++) {
                    if (!tile_nonempty(g, tr, cb)) continue;
                    const int64_t x = i - (rho0 + cb * kCT - g.ku);
                    if (x >= 0 && x < wq) acc += qpart[(tr * g.ncb + cb) * g.lq + x];
                }
            }
        }
    }
    q[i] = acc;
}

// Column outputs: s_j = (sum over the band-row tiles holding column j's
// entries, ascending) * beta (ATAX) or unscaled (BICGK).
template <bool SCALE>
__global__ void band_s_combine(const BandGeom g, const double* __restrict__ spart, double beta,
                               double* __restrict__ s) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.n) return;
    double acc = 0.0;
    if (j < g.ncols) {
        const int64_t tlo = (band_vlo(g, j) - g.rho_a) / g.rt, thi = (band_vhi(g, j) - g.rho_a) / g.rt;
        for (int64_t tr = tlo; tr <= thi; tr++) acc += spart[tr * g.n + j];
    }
    s[j] = SCALE ? acc * beta : acc;
}

int band_rpl(int64_t rows) {
    if (rows <= 32) return 1;
    if (rows <= 64) return 2;
    if (rows <= 128) return 4;
    return 8;
}

BandGeom make_geom(int storage, int64_t m, int64_t n, int64_t kl, int64_t ku, int unit, int64_t ld) {
    BandGeom g;
    g.storage = storage; g.unit = unit ? 1 : 0;
    g.m = m; g.n = n; g.kl = kl; g.ku = ku; g.ld = ld;
    if (m > 0 && n > 0) {
        g.rho_a = std::max<int64_t>(0, ku - (n - 1));
        g.rho_b = std::min<int64_t>(kl + ku, ku + m - 1);
        g.ncols = std::min<int64_t>(n, ku + m);
    }
    const int64_t rows = g.rho_b >= g.rho_a ? g.rho_b - g.rho_a + 1 : 0;
    g.rt = 32 * band_rpl(rows);
    g.ntr = ceil_div(rows, g.rt);
    g.ncb = rows > 0 ? ceil_div(g.ncols, kCT) : 0;
    g.lq = g.rt + kCT;
    return g;
}

struct BandWs {
    size_t qpart = 0, spart = 0, t = 0, total = 0;
};

BandWs band_ws(const BandGeom& g, bool atax) {
    BandWs w;
    size_t off = WS_HEADER;
    w.qpart = off;
    off += round_up((int64_t)(g.ntr * g.ncb * g.lq * (int64_t)sizeof(double)), 256);
    w.spart = off;
    off += round_up((int64_t)(g.ntr * g.n * (int64_t)sizeof(double)), 256);
    if (atax) {
        w.t = off;
        off += round_up(g.m * (int64_t)sizeof(double), 256);
    }
    w.total = off;
    return w;
}

template <int MODE>
bto_status launch_band(const BandArgs& a, int grid, cudaStream_t st) {
    switch (a.g.rt) {
        case 32: band_kernel<MODE, 1><<<grid, kBThreads, 0, st>>>(a); break;
        case 64: band_kernel<MODE, 2><<<grid, kBThreads, 0, st>>>(a); break;
        case 128: band_kernel<MODE, 4><<<grid, kBThreads, 0, st>>>(a); break;
        default: band_kernel<MODE, 8><<<grid, kBThreads, 0, st>>>(a); break;
    }
    return launch_status();
}

// Extent (bytes) of the stored operand.
size_t band_extent(int storage, int64_t m, int64_t n, int64_t kl, int64_t ku, int64_t ld) {
    if (m <= 0 || n <= 0) return 0;
    if (storage == BTO_STORE_FULL) return mat_extent_bytes(m, n, ld, 8);
    if (storage == BTO_STORE_BAND) return mat_extent_bytes(kl + ku + 1, n, ld, 8);
    return (size_t)(n * (n + 1) / 2) * 8;
}

// Shared checks (positions: storage 1, m 2, n 3, kl 4, ku 5, then A at apos
// and ld at apos + 1).
void check_band(Check& c, int storage, int64_t m, int64_t n, int64_t kl, int64_t ku, const double* A, int64_t ld,
                int apos) {
    if (storage < BTO_STORE_FULL || storage > BTO_STORE_PACKED) c.fail(1);
    c.size(2, m); c.size(3, n);
    if (m > INT32_MAX) c.fail(2);
    if (n > INT32_MAX) c.fail(3);
    if (kl < 0 || kl > (int64_t(1) << 40)) c.fail(4);
    if (ku < 0 || ku > (int64_t(1) << 40)) c.fail(5);
    if (!c.ok()) return;
    if (storage == BTO_STORE_PACKED) {
        const int64_t e = n > 0 ? n - 1 : 0;
        if (m != n) c.fail(2);
        else if (!((kl == 0 && ku == e) || (ku == 0 && kl == e))) c.fail(kl == 0 ? 5 : 4);
    } else if (storage == BTO_STORE_FULL) {
        c.ld(apos + 1, ld, m);
    } else if (ld < kl + ku + 1) {
        c.fail(apos + 1);
    }
    c.ptr(apos, A, m > 0 && n > 0);
}

bto_status band_run(int op, int storage, int64_t m, int64_t n, int64_t kl, int64_t ku, int unit, double beta,
                    const double* A, int64_t ld, const double* p, const double* r, double* q, double* s,
                    void* ws, size_t ws_bytes, int ws_pos, cudaStream_t st) {
    const bool atax = op == BTO_OP_ATAX;
    const BandGeom g = make_geom(storage, m, n, kl, ku, unit, ld);
    const BandWs W = band_ws(g, atax);
    Check c;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < W.total) c.fail(ws_pos, BTO_ERR_WORKSPACE);
    if (!c.ok()) return c.finish();
    DeviceInfo d;
    if (!device_info(&d)) return BTO_ERR_CUDA;
    char* w = static_cast<char*>(ws);
    // status word and the two tile counters
    if (cudaMemsetAsync(w, 0, 128, st) != cudaSuccess) return BTO_ERR_CUDA;
    auto* counters = reinterpret_cast<unsigned long long*>(w + kCounterOff);
    BandArgs a;
    a.g = g; a.A = A;
    a.qpart = reinterpret_cast<double*>(w + W.qpart);
    a.spart = reinterpret_cast<double*>(w + W.spart);
    const int64_t ntiles = g.ntr * g.ncb;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)d.sms * 3));
    const int cthreads = 256;
    bto_status e = BTO_OK;
    if (!atax) {
        a.p = p; a.r = r; a.counter = counters;
        if (ntiles > 0 && (e = launch_band<BM_QS>(a, grid, st)) != BTO_OK) return e;
        if (m > 0) band_q_combine<<<(int)ceil_div(m, cthreads), cthreads, 0, st>>>(g, a.qpart, q);
        if ((e = launch_status()) != BTO_OK) return e;
        if (n > 0) band_s_combine<false><<<(int)ceil_div(n, cthreads), cthreads, 0, st>>>(g, a.spart, 1.0, s);
        return launch_status();
    }
    // BATAX: t = A x (row partials, combined into the workspace), then
    // y = beta A^T t (column partials).  A is read twice.
    double* t = reinterpret_cast<double*>(w + W.t);
    a.p = p; a.r = nullptr; a.counter = counters;
    if (ntiles > 0 && (e = launch_band<BM_Q>(a, grid, st)) != BTO_OK) return e;
    if (m > 0) band_q_combine<<<(int)ceil_div(m, cthreads), cthreads, 0, st>>>(g, a.qpart, t);
    if ((e = launch_status()) != BTO_OK) return e;
    a.p = nullptr; a.r = t; a.counter = counters + 1;
    if (ntiles > 0 && (e = launch_band<BM_S>(a, grid, st)) != BTO_OK) return e;
    if (n > 0) band_s_combine<true><<<(int)ceil_div(n, cthreads), cthreads, 0, st>>>(g, a.spart, beta, s);
    return launch_status();
}

bool tri_args(int uplo, int unit, int packed, int64_t n, int* storage, int64_t* kl, int64_t* ku, Check& c) {
    if (uplo != BTO_UPPER && uplo != BTO_LOWER) c.fail(1);
    if (unit != 0 && unit != 1) c.fail(2);
    if (packed != 0 && packed != 1) c.fail(3);
    c.size(4, n);
    if (!c.ok()) return false;
    const int64_t e = n > 0 ? n - 1 : 0;
    *storage = packed ? BTO_STORE_PACKED : BTO_STORE_FULL;
    *kl = uplo == BTO_UPPER ? 0 : e;
    *ku = uplo == BTO_UPPER ? e : 0;
    return true;
}

}  // namespace
}  // namespace bto

using namespace bto;

extern "C" bto_status bto_band_workspace_bytes(int op, int64_t m, int64_t n, int64_t kl, int64_t ku,
                                               size_t* bytes) {
    clear_invalid_arg();
    Check c;
    if (op != BTO_OP_BICGK && op != BTO_OP_ATAX) c.fail(1);
    c.size(2, m); c.size(3, n);
    if (m > INT32_MAX) c.fail(2);
    if (n > INT32_MAX) c.fail(3);
    if (kl < 0 || kl > (int64_t(1) << 40)) c.fail(4);
    if (ku < 0 || ku > (int64_t(1) << 40)) c.fail(5);
    c.ptr(6, bytes, true, 1);
    if (!c.ok()) return c.finish();
    *bytes = band_ws(make_geom(BTO_STORE_FULL, m, n, kl, ku, 0, std::max<int64_t>(1, m)), op == BTO_OP_ATAX).total;
    return BTO_OK;
}

extern "C" bto_status bto_band_bicgk(int storage, int64_t m, int64_t n, int64_t kl, int64_t ku, int unit_diag,
                                     const double* A, int64_t ld, const double* p, const double* r, double* q,
                                     double* s, void* ws, size_t ws_bytes, bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    check_band(c, storage, m, n, kl, ku, A, ld, 7);
    if (unit_diag != 0 && unit_diag != 1) c.fail(6);
    if (!c.ok()) return c.finish();
    const size_t ab = band_extent(storage, m, n, kl, ku, ld);
    c.ptr(9, p, n > 0 && m > 0); c.ptr(10, r, m > 0 && n > 0); c.ptr(11, q, m > 0); c.ptr(12, s, n > 0);
    c.disjoint(11, q, vbytes(m), s, vbytes(n)); c.disjoint(11, q, vbytes(m), p, vbytes(n));
    c.disjoint(11, q, vbytes(m), r, vbytes(m)); c.disjoint(11, q, vbytes(m), A, ab);
    c.disjoint(12, s, vbytes(n), p, vbytes(n)); c.disjoint(12, s, vbytes(n), r, vbytes(m));
    c.disjoint(12, s, vbytes(n), A, ab);
    if (!c.ok()) return c.finish();
    return band_run(BTO_OP_BICGK, storage, m, n, kl, ku, unit_diag, 1.0, A, ld, p, r, q, s, ws, ws_bytes, 13,
                    (cudaStream_t)stream);
}

extern "C" bto_status bto_band_atax(int storage, int64_t m, int64_t n, int64_t kl, int64_t ku, int unit_diag,
                                    double beta, const double* A, int64_t ld, const double* x, double* y,
                                    void* ws, size_t ws_bytes, bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    check_band(c, storage, m, n, kl, ku, A, ld, 8);
    if (unit_diag != 0 && unit_diag != 1) c.fail(6);
    if (!c.ok()) return c.finish();
    // positions: beta 7, A 8, ld 9, x 10, y 11, ws 12
    const size_t ab = band_extent(storage, m, n, kl, ku, ld);
    c.ptr(10, x, n > 0 && m > 0); c.ptr(11, y, n > 0);
    c.disjoint(11, y, vbytes(n), x, vbytes(n)); c.disjoint(11, y, vbytes(n), A, ab);
    if (!c.ok()) return c.finish();
    return band_run(BTO_OP_ATAX, storage, m, n, kl, ku, unit_diag, beta, A, ld, x, nullptr, nullptr, y, ws,
                    ws_bytes, 12, (cudaStream_t)stream);
}

extern "C" bto_status bto_tri_workspace_bytes(int op, int uplo, int64_t n, size_t* bytes) {
    clear_invalid_arg();
    Check c;
    int storage;
    int64_t kl, ku;
    if (op != BTO_OP_BICGK && op != BTO_OP_ATAX) c.fail(1);
    if (uplo != BTO_UPPER && uplo != BTO_LOWER) c.fail(2);
    c.size(3, n);
    if (n > INT32_MAX) c.fail(3);
    c.ptr(4, bytes, true, 1);
    if (!c.ok()) return c.finish();
    Check c2;
    tri_args(uplo, 0, 0, n, &storage, &kl, &ku, c2);
    *bytes = band_ws(make_geom(BTO_STORE_FULL, n, n, kl, ku, 0, std::max<int64_t>(1, n)), op == BTO_OP_ATAX).total;
    return BTO_OK;
}

extern "C" bto_status bto_tri_bicgk(int uplo, int unit_diag, int packed, int64_t n, const double* A, int64_t lda,
                                    const double* p, const double* r, double* q, double* s, void* ws,
                                    size_t ws_bytes, bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    int storage;
    int64_t kl, ku;
    if (!tri_args(uplo, unit_diag, packed, n, &storage, &kl, &ku, c)) return c.finish();
    if (n > INT32_MAX) c.fail(4);
    if (!packed) c.ld(6, lda, n);
    c.ptr(5, A, n > 0);
    const size_t ab = band_extent(storage, n, n, kl, ku, lda);
    c.ptr(7, p, n > 0); c.ptr(8, r, n > 0); c.ptr(9, q, n > 0); c.ptr(10, s, n > 0);
    c.disjoint(9, q, vbytes(n), s, vbytes(n)); c.disjoint(9, q, vbytes(n), p, vbytes(n));
    c.disjoint(9, q, vbytes(n), r, vbytes(n)); c.disjoint(9, q, vbytes(n), A, ab);
    c.disjoint(10, s, vbytes(n), p, vbytes(n)); c.disjoint(10, s, vbytes(n), r, vbytes(n));
    c.disjoint(10, s, vbytes(n), A, ab);
    if (!c.ok()) return c.finish();
    return band_run(BTO_OP_BICGK, storage, n, n, kl, ku, unit_diag, 1.0, A, packed ? 1 : lda, p, r, q, s, ws,
                    ws_bytes, 11, (cudaStream_t)stream);
}

extern "C" bto_status bto_tri_atax(int uplo, int unit_diag, int packed, int64_t n, double beta, const double* A,
                                   int64_t lda, const double* x, double* y, void* ws, size_t ws_bytes,
                                   bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    int storage;
    int64_t kl, ku;
    if (!tri_args(uplo, unit_diag, packed, n, &storage, &kl, &ku, c)) return c.finish();
    if (n > INT32_MAX) c.fail(4);
    if (!packed) c.ld(7, lda, n);
    c.ptr(6, A, n > 0);
    const size_t ab = band_extent(storage, n, n, kl, ku, lda);
    c.ptr(8, x, n > 0); c.ptr(9, y, n > 0);
    c.disjoint(9, y, vbytes(n), x, vbytes(n)); c.disjoint(9, y, vbytes(n), A, ab);
    if (!c.ok()) return c.finish();
    return band_run(BTO_OP_ATAX, storage, n, n, kl, ku, unit_diag, beta, A, packed ? 1 : lda, x, nullptr, nullptr,
                    y, ws, ws_bytes, 10, (cudaStream_t)stream);
}
