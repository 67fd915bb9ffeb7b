// Panel engine: one pass over a column-major FP64 matrix that evaluates the
// fused statements of a Table I kernel tile by tile.
//
// The matrix is cut into NR row blocks x NC column panels (NR = 1 for wide
// matrices, so a panel spans every row).  A block of 8 warps takes a tile
// and walks it in row chunks of 2048 rows; within a chunk each lane owns 8
// rows of every column (four 16-byte loads per column in the aligned form),
// so a warp's loads of one column are 512 contiguous bytes.  For every
// column the lane
//   - adds A(i,j) * p_j into its row accumulators (the non-transposed
//     product, "A p": rows are independent, no reduction inside the tile),
//   - forms sum_i A(i,j) * r_i over its 8 rows (the transposed product,
//     "A^T r": a reduction over rows).
// After a group of 16 columns the 32 lanes hold 16 column partials each; a
// transposing butterfly (5 rounds of shuffles, 16 adds per lane) leaves lane
// l with the warp's sum for column l mod 16 of the group, so the transposed
// product costs one extra add per column per lane instead of a shuffle tree
// per column.  Loads of four columns are issued before any is consumed.  Warps then add their column sums into per-warp shared-memory
// rows, which the block sums in warp order at the end of the tile.
//
// This is the GPU form of the paper's fused partitioned loop nests
// (Section III-C fuse sets; Section III-D partition compatibility): both
// products read each A(i,j) once, and the "reduction at the parallel level"
// that a column partition of the non-transposed product introduces is a
// per-panel partial vector that a second kernel adds up in panel order.
// All sums run in a fixed order, so results are bitwise reproducible.
#include "internal.cuh"
#include <atomic>
#include <algorithm>

namespace bto {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kRPT = 8;                           // rows per lane per column
constexpr int kRowsPerWarp = 32 * kRPT;           // 256
constexpr int kChunk = kWarps * kRowsPerWarp;     // 2048 rows per chunk
constexpr int64_t kMaxPanel = 512;                // widest column panel
constexpr int kGroup = 16;                        // columns per transposing group
constexpr int kU = 4;                             // columns loaded before any is consumed

// Row offset (within a chunk) of the lane's k-th element.
template <int VEC>
__device__ __forceinline__ int row_of(int warp, int lane, int k) {
    if (VEC == 2) return warp * kRowsPerWarp + (k >> 1) * 64 + 2 * lane + (k & 1);
    return warp * kRowsPerWarp + k * 32 + lane;
}

// Loads the lane's 8 elements of one column segment; rows >= rend read as 0.
template <int VEC>
__device__ __forceinline__ void load_col(const double* __restrict__ col, int64_t R0, int64_t rend,
                                         int warp, int lane, double (&a)[kRPT]) {
    if (VEC == 2) {
#pragma unroll
        for (int h = 0; h < kRPT / 2; h++) {
            int64_t i = R0 + row_of<2>(warp, lane, 2 * h);
            if (i + 1 < rend) {
                double2 t = __ldg(reinterpret_cast<const double2*>(col + i));
                a[2 * h] = t.x; a[2 * h + 1] = t.y;
            } else if (i < rend) {
                a[2 * h] = __ldg(col + i); a[2 * h + 1] = 0.0;
            } else {
                a[2 * h] = 0.0; a[2 * h + 1] = 0.0;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < kRPT; k++) {
            int64_t i = R0 + row_of<1>(warp, lane, k);
            a[k] = (i < rend) ? __ldg(col + i) : 0.0;
        }
    }
}

// Plain (coherent) loads, for the GEMVER pass that may write B over A.
template <int VEC>
__device__ __forceinline__ void load_col_rw(const double* col, int64_t R0, int64_t rend,
                                            int warp, int lane, double (&a)[kRPT]) {
    if (VEC == 2) {
#pragma unroll
        for (int h = 0; h < kRPT / 2; h++) {
            int64_t i = R0 + row_of<2>(warp, lane, 2 * h);
            if (i + 1 < rend) {
                double2 t = *reinterpret_cast<const double2*>(col + i);
                a[2 * h] = t.x; a[2 * h + 1] = t.y;
            } else if (i < rend) {
                a[2 * h] = col[i]; a[2 * h + 1] = 0.0;
            } else {
                a[2 * h] = 0.0; a[2 * h + 1] = 0.0;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < kRPT; k++) {
            int64_t i = R0 + row_of<1>(warp, lane, k);
            a[k] = (i < rend) ? col[i] : 0.0;
        }
    }
}

template <int VEC>
__device__ __forceinline__ void store_col(double* col, int64_t R0, int64_t rend, int warp, int lane,
                                          const double (&b)[kRPT]) {
    if (VEC == 2) {
#pragma unroll
        for (int h = 0; h < kRPT / 2; h++) {
            int64_t i = R0 + row_of<2>(warp, lane, 2 * h);
            if (i + 1 < rend) {
                *reinterpret_cast<double2*>(col + i) = make_double2(b[2 * h], b[2 * h + 1]);
            } else if (i < rend) {
                col[i] = b[2 * h];
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < kRPT; k++) {
            int64_t i = R0 + row_of<1>(warp, lane, k);
            if (i < rend) col[i] = b[k];
        }
    }
}

template <int VEC>
__device__ __forceinline__ void load_vec_rows(const double* __restrict__ v, int64_t R0, int64_t rend,
                                              int warp, int lane, double (&o)[kRPT]) {
#pragma unroll
    for (int k = 0; k < kRPT; k++) {
        int64_t i = R0 + row_of<VEC>(warp, lane, k);
        o[k] = (i < rend) ? __ldg(v + i) : 0.0;
    }
}

template <int VEC>
__device__ __forceinline__ void store_vec_rows(double* v, int64_t R0, int64_t rend, int warp,
                                               int lane, const double (&o)[kRPT]) {
#pragma unroll
    for (int k = 0; k < kRPT; k++) {
        int64_t i = R0 + row_of<VEC>(warp, lane, k);
        if (i < rend) v[i] = o[k];
    }
}

// Balanced split of [0, n) into parts pieces; piece b starts at b*n/parts.
__device__ __host__ __forceinline__ int64_t split_at(int64_t n, int64_t parts, int64_t b) {
    return (n / parts) * b + ((n % parts) * b) / parts;   // floor(n*b/parts) without overflow
}
// Row blocks start on multiples of 64 rows so 16-byte row pairs stay aligned.
__device__ __host__ __forceinline__ int64_t row_split_at(int64_t m, int64_t parts, int64_t b) {
    if (b >= parts) return m;
    return (split_at(m, parts, b) / 64) * 64;
}

// Blocks per SM and columns loaded ahead.  Every mode runs two blocks per SM
// (128 registers), so one block's latency is covered by the other's FP64
// arithmetic; the two-product modes load one column ahead to fit, which
// measured faster than four columns ahead at one block per SM (GEMVER's
// first pass 2.20 -> 2.00 ms, BICGK 1.07 -> 0.98 ms, GESUMMV 1.13 -> 0.97 ms
// at n = 16384): with FP64 the bound, a second resident block hides more
// latency than loads issued early.  The q-only mode has its own loop (two
// buffers of two columns taking turns); three or four blocks per SM were
// slower for it.  The same loop for the s-only mode measured no faster than
// its four-column bursts; what raised that mode (77% -> 88% of the FP64
// peak) was walking column groups outside the row chunks (below).
template <int MODE>
struct BlocksPerSM { static constexpr int value = 2; };
template <int MODE>
struct ColsAhead { static constexpr int value = (MODE == PM_Q || MODE == PM_S) ? kU : 1; };

template <int MODE, int VEC>
__global__ void __launch_bounds__(kThreads, BlocksPerSM<MODE>::value) panel_kernel(const PanelArgs a) {
    constexpr bool HAS_Q = (MODE == PM_QS || MODE == PM_Q || MODE == PM_Q2 || MODE == PM_G1Q);
    constexpr bool HAS_S = (MODE == PM_QS || MODE == PM_S || MODE == PM_G1);
    constexpr bool GEN = (MODE == PM_G1 || MODE == PM_G1Q);   // forms and stores B
    constexpr bool COLS_OUTER = (MODE == PM_S);   // column sums alone (see below)
    extern __shared__ double sw[];   // [kWarps][TCmax] per-warp column sums
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t tcmax = (a.n + a.NC - 1) / a.NC;

    for (int64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int64_t tt = a.reverse ? (a.ntiles - 1 - t) : t;
        const int64_t cb = tt / a.NR, rb = tt % a.NR;
        const int64_t c0 = split_at(a.n, a.NC, cb), c1 = split_at(a.n, a.NC, cb + 1);
        const int64_t r0 = row_split_at(a.m, a.NR, rb), r1 = row_split_at(a.m, a.NR, rb + 1);
        const int ncols = (int)(c1 - c0);

        if (HAS_S) {
            for (int k = threadIdx.x; k < kWarps * tcmax; k += kThreads) sw[k] = 0.0;
            __syncthreads();
        }

        if (COLS_OUTER) {
            // Column groups outside the row chunks: each column's sum runs on
            // through every chunk of the row block, so the transposing
            // butterfly (one FP64 add per column and lane) runs once per group
            // and row block instead of once per chunk.  (GEMVER's first pass,
            // also column sums only, keeps the chunk-outer order: this one
            // would spill there.)
            for (int64_t g0 = c0; g0 < c1; g0 += kGroup) {
                const int nc = (int)((c1 - g0) < kGroup ? (c1 - g0) : kGroup);
                double sl[kGroup];
#pragma unroll
                for (int jj = 0; jj < kGroup; jj++) sl[jj] = 0.0;
#pragma unroll 1
                for (int64_t R0 = r0; R0 < r1; R0 += kChunk) {
                    double rv[kRPT];
                    load_vec_rows<VEC>(a.r, R0, r1, warp, lane, rv);
                    constexpr int KU = ColsAhead<MODE>::value;
#pragma unroll
                    for (int jb = 0; jb < kGroup; jb += KU) {
                        // Issue the loads of KU columns before consuming any of them.
                        double av[KU][kRPT];
#pragma unroll
                        for (int u = 0; u < KU; u++)
                            if (jb + u < nc) load_col<VEC>(a.A + (g0 + jb + u) * a.lda, R0, r1, warp, lane, av[u]);
#pragma unroll
                        for (int u = 0; u < KU; u++)
                            if (jb + u < nc) {
#pragma unroll
                                for (int k = 0; k < kRPT; k++) sl[jb + u] = fma(av[u][k], rv[k], sl[jb + u]);
                            }
                    }
                }
                const double cs = transpose_reduce16(sl, lane);
                if (lane < nc) sw[warp * tcmax + (g0 - c0) + lane] += cs;
            }
        } else
        for (int64_t R0 = r0; R0 < r1; R0 += kChunk) {
            double rv[kRPT], qacc[kRPT], qacc2[kRPT], u1r[kRPT], u2r[kRPT];
            if (HAS_S) load_vec_rows<VEC>(a.r, R0, r1, warp, lane, rv);
            if (GEN) {
                load_vec_rows<VEC>(a.u1, R0, r1, warp, lane, u1r);
                load_vec_rows<VEC>(a.u2, R0, r1, warp, lane, u2r);
            }
#pragma unroll
            for (int k = 0; k < kRPT; k++) { qacc[k] = 0.0; qacc2[k] = 0.0; }

            if (MODE == PM_Q) {
                // q alone: two buffers of two columns each take turns, the loads
                // of one issued before the other's FMAs, so each warp keeps loads
                // in flight while it computes (a burst of four columns followed by
                // their FMAs left the loads' latency exposed).  Columns are added
                // in the same order as before.
                double xa[2][kRPT], xb[2][kRPT], pa[2] = {0.0, 0.0}, pb[2] = {0.0, 0.0};
                auto fetch = [&](int64_t j, double (&x)[2][kRPT], double (&pv)[2]) {
#pragma unroll
                    for (int u = 0; u < 2; u++)
                        if (j + u < c1) {
                            load_col<VEC>(a.A + (j + u) * a.lda, R0, r1, warp, lane, x[u]);
                            pv[u] = __ldg(a.p + j + u);
                        }
                };
                auto use = [&](int64_t j, const double (&x)[2][kRPT], const double (&pv)[2]) {
#pragma unroll
                    for (int u = 0; u < 2; u++)
                        if (j + u < c1) {
#pragma unroll
                            for (int k = 0; k < kRPT; k++) qacc[k] = fma(x[u][k], pv[u], qacc[k]);
                        }
                };
                fetch(c0, xa, pa);
#pragma unroll 1
                for (int64_t j = c0; j < c1; j += 4) {
                    fetch(j + 2, xb, pb);
                    use(j, xa, pa);
                    fetch(j + 4, xa, pa);
                    use(j + 2, xb, pb);
                }
            } else if (MODE == PM_Q2) {
                // GESUMMV: one column of each matrix per step, two buffers taking
                // turns as in the q-only mode; columns in the same order.
                double ax[kRPT], bx[kRPT], ay[kRPT], by[kRPT], px = 0.0, py = 0.0;
                auto fetch2 = [&](int64_t j, double (&x)[kRPT], double (&y)[kRPT], double& pv) {
                    if (j < c1) {
                        load_col<VEC>(a.A + j * a.lda, R0, r1, warp, lane, x);
                        load_col<VEC>(a.B + j * a.ldb, R0, r1, warp, lane, y);
                        pv = __ldg(a.p + j);
                    }
                };
                auto use2 = [&](int64_t j, const double (&x)[kRPT], const double (&y)[kRPT], double pv) {
                    if (j < c1) {
#pragma unroll
                        for (int k = 0; k < kRPT; k++) {
                            qacc[k] = fma(x[k], pv, qacc[k]);
                            qacc2[k] = fma(y[k], pv, qacc2[k]);
                        }
                    }
                };
                fetch2(c0, ax, bx, px);
#pragma unroll 1
                for (int64_t j = c0; j < c1; j += 2) {
                    fetch2(j + 1, ay, by, py);
                    use2(j, ax, bx, px);
                    fetch2(j + 2, ax, bx, px);
                    use2(j + 1, ay, by, py);
                }
            } else
            for (int64_t g0 = c0; g0 < c1; g0 += kGroup) {
                const int nc = (int)((c1 - g0) < kGroup ? (c1 - g0) : kGroup);
                double sl[kGroup];
                constexpr int KU = ColsAhead<MODE>::value;
#pragma unroll
                for (int jb = 0; jb < kGroup; jb += KU) {
                    // Issue the loads of KU columns before consuming any of them.
                    double av[KU][kRPT], bv[KU][kRPT], pj[KU], v1j[KU], v2j[KU];
#pragma unroll
                    for (int u = 0; u < KU; u++) {
                        const int jj = jb + u;
                        if (jj < nc) {
                            const int64_t j = g0 + jj;
                            if (GEN) {
                                load_col_rw<VEC>(a.A + j * a.lda, R0, r1, warp, lane, av[u]);
                                v1j[u] = __ldg(a.v1 + j);
                                v2j[u] = __ldg(a.v2 + j);
                            } else {
                                load_col<VEC>(a.A + j * a.lda, R0, r1, warp, lane, av[u]);
                            }
                            if (MODE == PM_Q2) load_col<VEC>(a.B + j * a.ldb, R0, r1, warp, lane, bv[u]);
                            if (HAS_Q) pj[u] = __ldg(a.p + j);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < KU; u++) {
                        const int jj = jb + u;
                        if (jj < nc) {
                            const int64_t j = g0 + jj;
                            if (GEN) {
                                double b[kRPT];
#pragma unroll
                                for (int k = 0; k < kRPT; k++)
                                    b[k] = fma(u2r[k], v2j[u], fma(u1r[k], v1j[u], av[u][k]));
                                store_col<VEC>(a.Bout + j * a.ldb, R0, r1, warp, lane, b);
                                if (MODE == PM_G1) {
                                    double acc = b[0] * rv[0];
#pragma unroll
                                    for (int k = 1; k < kRPT; k++) acc = fma(b[k], rv[k], acc);
                                    sl[jj] = acc;
                                } else {
#pragma unroll
                                    for (int k = 0; k < kRPT; k++) qacc[k] = fma(b[k], pj[u], qacc[k]);
                                }
                            } else {
                                if (HAS_Q) {
#pragma unroll
                                    for (int k = 0; k < kRPT; k++) qacc[k] = fma(av[u][k], pj[u], qacc[k]);
                                }
                                if (MODE == PM_Q2) {
#pragma unroll
                                    for (int k = 0; k < kRPT; k++) qacc2[k] = fma(bv[u][k], pj[u], qacc2[k]);
                                }
                                if (HAS_S) {
                                    double acc = av[u][0] * rv[0];
#pragma unroll
                                    for (int k = 1; k < kRPT; k++) acc = fma(av[u][k], rv[k], acc);
                                    sl[jj] = acc;
                                }
                            }
                        } else if (HAS_S) {
                            sl[jj] = 0.0;
                        }
                    }
                }
                if (HAS_S) {
                    const double cs = transpose_reduce16(sl, lane);
                    if (lane < nc) sw[warp * tcmax + (g0 - c0) + lane] += cs;
                }
            }
            if (HAS_Q) {
                store_vec_rows<VEC>(a.qpart + cb * a.ldq, R0, r1, warp, lane, qacc);
                if (MODE == PM_Q2) store_vec_rows<VEC>(a.qpart2 + cb * a.ldq, R0, r1, warp, lane, qacc2);
            }
        }

        if (HAS_S) {
            __syncthreads();
            for (int k = threadIdx.x; k < ncols; k += kThreads) {
                double s = sw[k];
#pragma unroll
                for (int w = 1; w < kWarps; w++) s += sw[w * tcmax + k];
                a.spart[rb * a.lds + c0 + k] = s;
            }
            __syncthreads();
        }
    }
}

// Fixed-order combine of split partials.  A block handles 32 consecutive
// outputs; warp w adds the partials k = w, w + 8, w + 16, ... of output
// (block base + lane) with coalesced loads, then warp 0 adds the 8 warp
// sums in warp order.  The order depends only on K, so results are
// reproducible, and every load of a warp is one 256-byte segment.
constexpr int kCombWarps = 8;

__device__ __forceinline__ double strided_sum(const double* P, int64_t ld, int K, int w, int64_t i) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    int k = w;
    for (; k + 3 * kCombWarps < K; k += 4 * kCombWarps) {
#pragma unroll
        for (int u = 0; u < 4; u++) acc[u] += __ldg(P + (int64_t)(k + u * kCombWarps) * ld + i);
    }
    // At most three partials remain; unrolled so acc[] stays in registers.
#pragma unroll
    for (int u = 0; u < 3; u++)
        if (k + u * kCombWarps < K) acc[u] += __ldg(P + (int64_t)(k + u * kCombWarps) * ld + i);
    return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

__global__ void __launch_bounds__(kCombWarps * 32) combine_kernel(const CombineJob j0, const CombineJob j1, int njobs) {
    __shared__ double red[2][kCombWarps][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t blocks0 = (j0.len + 31) / 32;
    const int64_t nblk = blocks0 + (njobs > 1 ? (j1.len + 31) / 32 : 0);
    for (int64_t bI = blockIdx.x; bI < nblk; bI += gridDim.x) {
        const CombineJob& J = (bI < blocks0) ? j0 : j1;
        const int64_t i = ((bI < blocks0) ? bI : bI - blocks0) * 32 + lane;
        const bool ok = i < J.len;
        red[0][w][lane] = ok ? strided_sum(J.P1, J.ld1, J.K1, w, i) : 0.0;
        red[1][w][lane] = (ok && J.P2) ? strided_sum(J.P2, J.ld2, J.K2, w, i) : 0.0;
        __syncthreads();
        if (w == 0 && ok) {
            double s1 = red[0][0][lane];
#pragma unroll
            for (int q = 1; q < kCombWarps; q++) s1 += red[0][q][lane];
            double o = J.a1 * s1;
            if (J.P2) {
                double s2 = red[1][0][lane];
#pragma unroll
                for (int q = 1; q < kCombWarps; q++) s2 += red[1][q][lane];
                o = fma(J.a2, s2, o);
            }
            if (J.v) o = fma(J.b, J.v[i], o);
            J.out[i] = o;
        }
        __syncthreads();
    }
}

template <int MODE>
bto_status launch_mode(const PanelArgs& a, const PanelPlan& pl, bool vec2, cudaStream_t st) {
    const size_t smem = panel_smem_bytes(MODE, pl);
    const int grid = (int)std::min<int64_t>(pl.ntiles, (int64_t)pl.grid * BlocksPerSM<MODE>::value);
    if (vec2) {
        auto k = panel_kernel<MODE, 2>;
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return BTO_ERR_CUDA;
        k<<<grid, kThreads, smem, st>>>(a);
    } else {
        auto k = panel_kernel<MODE, 1>;
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return BTO_ERR_CUDA;
        k<<<grid, kThreads, smem, st>>>(a);
    }
    return launch_status();
}

}  // namespace

namespace {

// Schedule overrides, per (op, form): column panels and row blocks (0: the
// automatic choice).  Set from the host before the calls they affect.
constexpr int kSchedOps = BTO_OP_DGEMVT + 1;
std::atomic<int> g_sched[kSchedOps][2][2];

}  // namespace

PanelPlan panel_plan(int64_t m, int64_t n, int sms, int op, int form) {
    PanelPlan pl;
    pl.ldq = round_up(m > 0 ? m : 1, 32);
    pl.lds = round_up(n > 0 ? n : 1, 32);
    if (m <= 0 || n <= 0) return pl;
    const int64_t G = sms;
    int64_t NC = ceil_div(n, ceil_div(n, G));           // balanced panels, about G of them
    if (ceil_div(n, NC) > kMaxPanel) NC = ceil_div(n, kMaxPanel);
    // About two tiles per SM (so the two-blocks-per-SM modes fill the
    // machine).  Row blocks are at least one chunk (2048 rows: every warp of
    // the block has rows) unless m itself is shorter; a short matrix then has
    // about one tile per SM (n = 2048: 147 panels of 14 columns, one row
    // block).  Narrowing the panels to reach two tiles per SM was measured
    // and was slower there: GEMVER 69 -> 83 us with 187 panels, BICGK 41 ->
    // 49 us; 3 row blocks of 683 rows left five of the eight warps without
    // rows.
    int64_t NR = std::max<int64_t>(1, std::min<int64_t>(ceil_div(2 * G, NC), ceil_div(m, kChunk)));
    // Fused GEMVER: one chunk per row block (at n = 16384, 8 row blocks of
    // 2048 rows instead of 2), as the measured schedule search found best for
    // it (1.96 -> 1.92 ms); the other kernels' optima were within 1% of the
    // plan above.
    if (op == BTO_OP_GEMVER && form == BTO_FORM_FUSED) NR = std::max<int64_t>(NR, ceil_div(m, kChunk));
    // A schedule set with bto_schedule_set replaces the choices above.
    if (op >= 0 && op < kSchedOps && (form == BTO_FORM_FUSED || form == BTO_FORM_UNFUSED)) {
        const int hp = g_sched[op][form][0].load(std::memory_order_relaxed);
        const int hr = g_sched[op][form][1].load(std::memory_order_relaxed);
        if (hp > 0) {
            NC = std::min<int64_t>(hp, n);
            if (ceil_div(n, NC) > kMaxPanel) NC = ceil_div(n, kMaxPanel);
        }
        if (hr > 0) NR = std::min<int64_t>(hr, ceil_div(m, 64));
    }
    // Row blocks start on multiples of 64: drop blocks that would be empty.
    while (NR > 1 && row_split_at(m, NR, 1) == 0) NR--;
    pl.NR = (int)NR;
    pl.NC = (int)NC;
    pl.TCmax = ceil_div(n, NC);
    pl.ntiles = NR * NC;
    pl.grid = (int)G;   // times the blocks per SM of the mode, at launch
    return pl;
}

size_t panel_smem_bytes(int mode, const PanelPlan& pl) {
    const bool has_s = (mode == PM_QS || mode == PM_S || mode == PM_G1);
    return has_s ? (size_t)kWarps * (size_t)pl.TCmax * sizeof(double) : 0;
}

bto_status launch_panel(int mode, const PanelArgs& a, const PanelPlan& pl, cudaStream_t st) {
    if (pl.ntiles == 0) return BTO_OK;
    // 16-byte loads need 16-byte aligned columns: every matrix base and an
    // even leading dimension (rows pair up from even offsets).
    bool vec2 = aligned16(a.A) && (a.lda % 2 == 0);
    if (mode == PM_Q2) vec2 = vec2 && aligned16(a.B) && (a.ldb % 2 == 0);
    if (mode == PM_G1 || mode == PM_G1Q) vec2 = vec2 && aligned16(a.Bout) && (a.ldb % 2 == 0);
    switch (mode) {
        case PM_QS: return launch_mode<PM_QS>(a, pl, vec2, st);
        case PM_Q: return launch_mode<PM_Q>(a, pl, vec2, st);
        case PM_S: return launch_mode<PM_S>(a, pl, vec2, st);
        case PM_G1: return launch_mode<PM_G1>(a, pl, vec2, st);
        case PM_Q2: return launch_mode<PM_Q2>(a, pl, vec2, st);
        case PM_G1Q: return launch_mode<PM_G1Q>(a, pl, vec2, st);
    }
    return BTO_ERR_INVALID_VALUE;
}

bto_status launch_combine(const CombineJob* jobs, int njobs, cudaStream_t st) {
    int64_t blocks = 0;
    for (int i = 0; i < njobs; i++) blocks += ceil_div(jobs[i].len, 32);
    if (blocks == 0) return BTO_OK;
    DeviceInfo d;
    if (!device_info(&d)) return BTO_ERR_CUDA;
    blocks = std::min<int64_t>(blocks, (int64_t)d.sms * 8);
    CombineJob j1 = njobs > 1 ? jobs[1] : jobs[0];
    combine_kernel<<<(int)blocks, kCombWarps * 32, 0, st>>>(jobs[0], j1, njobs);
    return launch_status();
}

bool schedule_overridden(int op, int form) {
    if (op < BTO_OP_BICGK || op > BTO_OP_DGEMVT || form < BTO_FORM_FUSED || form > BTO_FORM_UNFUSED) return false;
    return g_sched[op][form][0].load(std::memory_order_relaxed) != 0 ||
           g_sched[op][form][1].load(std::memory_order_relaxed) != 0;
}

}  // namespace bto

using namespace bto;

extern "C" bto_status bto_schedule_set(int op, int form, int panels, int row_blocks) {
    clear_invalid_arg();
    if (op < BTO_OP_BICGK || op > BTO_OP_DGEMVT) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (form != BTO_FORM_FUSED && form != BTO_FORM_UNFUSED) { set_invalid_arg(2); return BTO_ERR_INVALID_VALUE; }
    if (panels < 0 || panels > (1 << 20)) { set_invalid_arg(3); return BTO_ERR_INVALID_VALUE; }
    if (row_blocks < 0 || row_blocks > (1 << 20)) { set_invalid_arg(4); return BTO_ERR_INVALID_VALUE; }
    g_sched[op][form][0].store(panels, std::memory_order_relaxed);
    g_sched[op][form][1].store(row_blocks, std::memory_order_relaxed);
    return BTO_OK;
}

extern "C" bto_status bto_panel_plan(int op, int form, int64_t m, int64_t n, int sms, int* row_blocks,
                                     int* panels) {
    clear_invalid_arg();
    if (op < BTO_OP_BICGK || op > BTO_OP_DGEMVT) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (form < BTO_FORM_FUSED || form > BTO_FORM_DF_UNFUSED) { set_invalid_arg(2); return BTO_ERR_INVALID_VALUE; }
    if (m < 0) { set_invalid_arg(3); return BTO_ERR_INVALID_VALUE; }
    if (n < 0) { set_invalid_arg(4); return BTO_ERR_INVALID_VALUE; }
    if (sms < 1 || sms > 4096) { set_invalid_arg(5); return BTO_ERR_INVALID_VALUE; }
    if (!row_blocks) { set_invalid_arg(6); return BTO_ERR_INVALID_VALUE; }
    if (!panels) { set_invalid_arg(7); return BTO_ERR_INVALID_VALUE; }
    const PanelPlan pl = form >= BTO_FORM_DF ? df_plan(m, n, sms) : panel_plan(m, n, sms, op, form);
    *row_blocks = pl.NR;
    *panels = pl.NC;
    return BTO_OK;
}

extern "C" bto_status bto_schedule_get(int op, int form, int* panels, int* row_blocks) {
    clear_invalid_arg();
    if (op < BTO_OP_BICGK || op > BTO_OP_DGEMVT) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (form != BTO_FORM_FUSED && form != BTO_FORM_UNFUSED) { set_invalid_arg(2); return BTO_ERR_INVALID_VALUE; }
    if (!panels) { set_invalid_arg(3); return BTO_ERR_INVALID_VALUE; }
    if (!row_blocks) { set_invalid_arg(4); return BTO_ERR_INVALID_VALUE; }
    *panels = g_sched[op][form][0].load(std::memory_order_relaxed);
    *row_blocks = g_sched[op][form][1].load(std::memory_order_relaxed);
    return BTO_OK;
}
