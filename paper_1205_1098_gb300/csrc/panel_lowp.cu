// Reduced-precision storage form of BICGK and GEMVER: A (and GEMVER's B)
// stored in FP32 or BF16, vectors in FP32, arithmetic in FP32 on the FP32
// pipes, accumulation compensated, FP64 only for the final combine.
//
// The matrix sweep is the FP64 panel schedule (tiles of NR row blocks x NC
// column panels, 8 warps, 8 rows per lane per column, 16-byte loads, four
// columns in flight) with FP32 arithmetic:
//   - A p: each lane adds a group of 16 columns into a plain FP32 FMA chain
//     per row, then folds the chain into a compensated (hi, lo) pair with
//     Knuth's TwoSum, so rounding error grows with the 16-term chains only.
//   - A^T r: each lane forms an 8-row FMA chain per column; a transposing
//     butterfly adds the 32 lanes; each warp folds its column sums into
//     (hi, lo) pairs in shared memory with TwoSum, row chunk after row chunk.
//   - At the end of a tile, the (hi, lo) pairs are stored as per-tile partials,
//     and the combine converts them and adds the partials of all tiles in FP64
//     in a fixed order, rounding once to the FP32 output.
// GEMVER's B is formed in FP32 and rounded to the storage type (round to
// nearest even); x and w are computed from the stored B, so the outputs are
// consistent with the B the caller receives.
#include "check.cuh"
#include "lp_math.cuh"

namespace bto {
namespace {

using namespace lp;

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kRPT = 8;
constexpr int kRowsPerWarp = 32 * kRPT;
constexpr int kChunk = kWarps * kRowsPerWarp;
constexpr int kGroup = 16;
constexpr int kU = 4;

// Row offset within a chunk of the lane's k-th element; V elements per
// 16-byte load (V = 1: scalar loads).
template <int V>
__device__ __forceinline__ int lrow(int warp, int lane, int k) {
    if (V == 1) return warp * kRowsPerWarp + k * 32 + lane;
    return warp * kRowsPerWarp + (k / V) * (32 * V) + lane * V + (k % V);
}

template <typename TA, int V, bool COHERENT>
__device__ __forceinline__ void lp_load_col(const TA* col, int64_t R0, int64_t rend, int warp, int lane,
                                            float (&a)[kRPT]) {
#pragma unroll
    for (int h = 0; h < kRPT / V; h++) {
        const int64_t i = R0 + lrow<V>(warp, lane, h * V);
        if (V > 1 && i + V <= rend) {
            uint4 t = COHERENT ? *reinterpret_cast<const uint4*>(col + i)
                               : __ldg(reinterpret_cast<const uint4*>(col + i));
            const TA* e = reinterpret_cast<const TA*>(&t);
#pragma unroll
            for (int q = 0; q < V; q++) a[h * V + q] = to_f<TA>(e[q]);
        } else {
#pragma unroll
            for (int q = 0; q < V; q++) a[h * V + q] = (i + q < rend) ? to_f<TA>(col[i + q]) : 0.0f;
        }
    }
}

template <typename TA, int V>
__device__ __forceinline__ void lp_store_col(TA* col, int64_t R0, int64_t rend, int warp, int lane,
                                             const TA (&b)[kRPT]) {
#pragma unroll
    for (int h = 0; h < kRPT / V; h++) {
        const int64_t i = R0 + lrow<V>(warp, lane, h * V);
        if (V > 1 && i + V <= rend) {
            uint4 t;
            TA* e = reinterpret_cast<TA*>(&t);
#pragma unroll
            for (int q = 0; q < V; q++) e[q] = b[h * V + q];
            *reinterpret_cast<uint4*>(col + i) = t;
        } else {
#pragma unroll
            for (int q = 0; q < V; q++)
                if (i + q < rend) col[i + q] = b[h * V + q];
        }
    }
}

template <int V>
__device__ __forceinline__ void lp_load_vec(const float* v, int64_t R0, int64_t rend, int warp, int lane,
                                            float (&o)[kRPT]) {
#pragma unroll
    for (int k = 0; k < kRPT; k++) {
        const int64_t i = R0 + lrow<V>(warp, lane, k);
        o[k] = (i < rend) ? __ldg(v + i) : 0.0f;
    }
}

template <typename TA, int MODE, int V>
__global__ void __launch_bounds__(kThreads, 1) lp_panel_kernel(const LpArgs a) {
    constexpr bool HAS_Q = (MODE == LP_QS || MODE == LP_Q);
    constexpr bool HAS_S = (MODE == LP_QS || MODE == LP_G1 || MODE == LP_S);
    extern __shared__ float sws[];   // [2][kWarps][tcmax]: hi, lo per warp and column
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t tcmax = a.tcmax;
    float* shi = sws;
    float* slo = sws + kWarps * tcmax;
    const TA* A = static_cast<const TA*>(a.A);
    TA* Bout = static_cast<TA*>(a.Bout);

    for (int64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int64_t tt = a.reverse ? (a.ntiles - 1 - t) : t;
        const int64_t cb = tt / a.NR, rb = tt % a.NR;
        const int64_t c0 = lp_col_at(a.n, a.NC, cb, a.cu), c1 = lp_col_at(a.n, a.NC, cb + 1, a.cu);
        const int64_t r0 = lp_row_at(a.m, a.NR, rb), r1 = lp_row_at(a.m, a.NR, rb + 1);
        const int ncols = (int)(c1 - c0);
        if (HAS_S) {
            for (int k = threadIdx.x; k < 2 * kWarps * tcmax; k += kThreads) sws[k] = 0.0f;
            __syncthreads();
        }
        for (int64_t R0 = r0; R0 < r1; R0 += kChunk) {
            float rv[kRPT], u1r[kRPT], u2r[kRPT], qhi[kRPT], qlo[kRPT];
            if (HAS_S) lp_load_vec<V>(a.r, R0, r1, warp, lane, rv);
            if (MODE == LP_G1) {
                lp_load_vec<V>(a.u1, R0, r1, warp, lane, u1r);
                lp_load_vec<V>(a.u2, R0, r1, warp, lane, u2r);
            }
#pragma unroll
            for (int k = 0; k < kRPT; k++) { qhi[k] = 0.0f; qlo[k] = 0.0f; }
            for (int64_t g0 = c0; g0 < c1; g0 += kGroup) {
                const int nc = (int)((c1 - g0) < kGroup ? (c1 - g0) : kGroup);
                float sl[kGroup], qt[kRPT];
#pragma unroll
                for (int k = 0; k < kRPT; k++) qt[k] = 0.0f;
#pragma unroll
                for (int jb = 0; jb < kGroup; jb += kU) {
                    float av[kU][kRPT], pj[kU], v1j[kU], v2j[kU];
#pragma unroll
                    for (int u = 0; u < kU; u++) {
                        const int jj = jb + u;
                        if (jj < nc) {
                            const int64_t j = g0 + jj;
                            lp_load_col<TA, V, MODE == LP_G1>(A + j * a.lda, R0, r1, warp, lane, av[u]);
                            if (HAS_Q) pj[u] = __ldg(a.p + j);
                            if (MODE == LP_G1) { v1j[u] = __ldg(a.v1 + j); v2j[u] = __ldg(a.v2 + j); }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kU; u++) {
                        const int jj = jb + u;
                        if (jj < nc) {
                            if (MODE == LP_G1) {
                                const int64_t j = g0 + jj;
                                TA bq[kRPT];
                                float bf[kRPT];
#pragma unroll
                                for (int k = 0; k < kRPT; k++) {
                                    bq[k] = from_f<TA>(fmaf(u2r[k], v2j[u], fmaf(u1r[k], v1j[u], av[u][k])));
                                    bf[k] = to_f<TA>(bq[k]);
                                }
                                lp_store_col<TA, V>(Bout + j * a.ldb, R0, r1, warp, lane, bq);
                                float acc = bf[0] * rv[0];
#pragma unroll
                                for (int k = 1; k < kRPT; k++) acc = fmaf(bf[k], rv[k], acc);
                                sl[jj] = acc;
                            } else {
                                if (HAS_Q) {
#pragma unroll
                                    for (int k = 0; k < kRPT; k++) qt[k] = fmaf(av[u][k], pj[u], qt[k]);
                                }
                                if (HAS_S) {
                                    float acc = av[u][0] * rv[0];
#pragma unroll
                                    for (int k = 1; k < kRPT; k++) acc = fmaf(av[u][k], rv[k], acc);
                                    sl[jj] = acc;
                                }
                            }
                        } else if (HAS_S) {
                            sl[jj] = 0.0f;
                        }
                    }
                }
                if (HAS_Q) {
#pragma unroll
                    for (int k = 0; k < kRPT; k++) {
                        float s, e;
                        two_sum(qhi[k], qt[k], s, e);
                        qhi[k] = s;
                        qlo[k] += e;
                    }
                }
                if (HAS_S) {
                    const float cs = butterfly16(sl, lane);
                    if (lane < nc) {
                        const int64_t o = warp * tcmax + (g0 - c0) + lane;
                        float s, e;
                        two_sum(shi[o], cs, s, e);
                        shi[o] = s;
                        slo[o] += e;
                    }
                }
            }
            if (HAS_Q) {
                float2* qp = reinterpret_cast<float2*>(a.qpart) + cb * a.ldq;
#pragma unroll
                for (int k = 0; k < kRPT; k++) {
                    const int64_t i = R0 + lrow<V>(warp, lane, k);
                    if (i < r1) qp[i] = make_float2(qhi[k], qlo[k]);
                }
            }
        }
        if (HAS_S) {
            __syncthreads();
            for (int k = threadIdx.x; k < ncols; k += kThreads) {
                float hs = shi[k], ls = slo[k];
#pragma unroll
                for (int w = 1; w < kWarps; w++) {
                    float s2, e2;
                    two_sum(hs, shi[w * tcmax + k], s2, e2);
                    hs = s2;
                    ls += e2 + slo[w * tcmax + k];
                }
                reinterpret_cast<float2*>(a.spart)[rb * a.lds + c0 + k] = make_float2(hs, ls);
            }
            __syncthreads();
        }
    }
}

// out[i] = (float)(a1 * sum_k P[k*ld + i] + b * v[i]).  Each partial is a
// compensated (hi, lo) FP32 pair; the pairs are converted and added in FP64
// in a fixed order (8 warps over the partials of 32 outputs, merged in warp
// order), and the result is rounded once to FP32.
// A second set of partials P2 (K2 of them, scaled by a2) may be added:
// out = a1 sum P + a2 sum P2 (GESUMMV's two products), each sum formed as
// above and the two scaled sums added in FP64 before the one rounding.
constexpr int kCW = 8;
__global__ void __launch_bounds__(kCW * 32) lp_combine_kernel(float* out, int64_t len, const double* P,
                                                             int64_t ld, int K, double a1, const float* v,
                                                             double b, const double* P2, int K2, double a2) {
    __shared__ double red[2][kCW][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nblk = (len + 31) / 32;
    for (int64_t bI = blockIdx.x; bI < nblk; bI += gridDim.x) {
        const int64_t i = bI * 32 + lane;
        double acc = 0.0, acc2 = 0.0;
        if (i < len) {
            for (int k = w; k < K; k += kCW) {
                const float2 h = __ldg(reinterpret_cast<const float2*>(P) + (int64_t)k * ld + i);
                acc += (double)h.x + (double)h.y;
            }
            for (int k = w; k < K2; k += kCW) {
                const float2 h = __ldg(reinterpret_cast<const float2*>(P2) + (int64_t)k * ld + i);
                acc2 += (double)h.x + (double)h.y;
            }
        }
        red[0][w][lane] = acc;
        red[1][w][lane] = acc2;
        __syncthreads();
        if (w == 0 && i < len) {
            double s = red[0][0][lane], s2 = red[1][0][lane];
#pragma unroll
            for (int q = 1; q < kCW; q++) { s += red[0][q][lane]; s2 += red[1][q][lane]; }
            double o = a1 * s;
            if (K2 > 0) o = fma(a2, s2, o);
            if (v) o = fma(b, (double)v[i], o);
            out[i] = (float)o;
        }
        __syncthreads();
    }
}

bto_status lp_combine(float* out, int64_t len, const double* P, int64_t ld, int K, double a1,
                      const float* v, double b, int sms, cudaStream_t st, const double* P2 = nullptr,
                      int K2 = 0, double a2 = 0.0) {
    if (len <= 0) return BTO_OK;
    const int64_t blocks = std::min<int64_t>(ceil_div(len, 32), (int64_t)sms * 8);
    lp_combine_kernel<<<(int)blocks, kCW * 32, 0, st>>>(out, len, P, ld, K, a1, v, b, P2, K2, a2);
    return launch_status();
}

template <typename TA, int MODE>
bto_status lp_launch_t(const LpArgs& a, const PanelPlan& pl, bool vec, cudaStream_t st) {
    constexpr int V = 16 / sizeof(TA);
    const size_t smem = (MODE == LP_Q) ? 0 : (size_t)2 * kWarps * a.tcmax * sizeof(float);
    const int grid = (int)std::min<int64_t>(pl.ntiles, (int64_t)pl.grid);
    if (vec) {
        auto k = lp_panel_kernel<TA, MODE, V>;
        if (smem > 48 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return BTO_ERR_CUDA;
        k<<<grid, kThreads, smem, st>>>(a);
    } else {
        auto k = lp_panel_kernel<TA, MODE, 1>;
        if (smem > 48 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return BTO_ERR_CUDA;
        k<<<grid, kThreads, smem, st>>>(a);
    }
    return launch_status();
}

bto_status lp_launch(int a_type, int mode, const LpArgs& a, const PanelPlan& pl, cudaStream_t st) {
    if (pl.ntiles == 0) return BTO_OK;
    bto_status tst;
    if (lp_tma_launch(a_type, mode, a, (int)std::min<int64_t>(pl.ntiles, pl.grid), pl.bps, st, &tst)) return tst;
    const size_t es = a_type == BTO_F32 ? 4 : 2;
    const int64_t V = 16 / (int64_t)es;
    bool vec = aligned16(a.A) && (a.lda % V == 0);
    if (mode == LP_G1) vec = vec && aligned16(a.Bout) && (a.ldb % V == 0);
    if (a_type == BTO_F32) {
        switch (mode) {
            case LP_QS: return lp_launch_t<float, LP_QS>(a, pl, vec, st);
            case LP_Q: return lp_launch_t<float, LP_Q>(a, pl, vec, st);
            case LP_G1: return lp_launch_t<float, LP_G1>(a, pl, vec, st);
            case LP_S: return lp_launch_t<float, LP_S>(a, pl, vec, st);
        }
    } else {
        switch (mode) {
            case LP_QS: return lp_launch_t<__nv_bfloat16, LP_QS>(a, pl, vec, st);
            case LP_Q: return lp_launch_t<__nv_bfloat16, LP_Q>(a, pl, vec, st);
            case LP_G1: return lp_launch_t<__nv_bfloat16, LP_G1>(a, pl, vec, st);
            case LP_S: return lp_launch_t<__nv_bfloat16, LP_S>(a, pl, vec, st);
        }
    }
    return BTO_ERR_INVALID_VALUE;
}

inline size_t fbytes(int64_t len) { return len > 0 ? (size_t)len * sizeof(float) : 0; }

}  // namespace
}  // namespace bto

using namespace bto;

extern "C" bto_status bto_bicgk_ex(int64_t m, int64_t n, int a_type, const void* A, int64_t lda,
                                   const float* p, const float* r, float* q, float* s, void* ws,
                                   size_t ws_bytes, bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    c.size(1, m); c.size(2, n);
    if (a_type != BTO_F32 && a_type != BTO_BF16) c.fail(3);
    if (!c.ok()) return c.finish();
    const size_t es = a_type == BTO_F32 ? 4 : 2;
    const size_t Ab = mat_extent_bytes(m, n, lda, es);
    c.ptr(4, A, m > 0 && n > 0, es); c.ld(5, lda, m);
    c.ptr(6, p, n > 0, 4); c.ptr(7, r, m > 0, 4); c.ptr(8, q, m > 0, 4); c.ptr(9, s, n > 0, 4);
    c.disjoint(8, q, fbytes(m), A, Ab); c.disjoint(8, q, fbytes(m), p, fbytes(n));
    c.disjoint(8, q, fbytes(m), r, fbytes(m)); c.disjoint(8, q, fbytes(m), s, fbytes(n));
    c.disjoint(9, s, fbytes(n), A, Ab); c.disjoint(9, s, fbytes(n), p, fbytes(n));
    c.disjoint(9, s, fbytes(n), r, fbytes(m));
    DeviceInfo d; WsLayout L;
    if (c.ok()) {
        if (!device_info(&d)) return BTO_ERR_CUDA;
        if (ws_layout(BTO_OP_BICGK, BTO_FORM_FUSED, m, n, a_type, d, &L) != BTO_OK) return BTO_ERR_CUDA;
        c.ws(10, ws, ws_bytes, L);
    }
    if (!c.ok()) return c.finish();
    cudaStream_t st = (cudaStream_t)stream;
    const PanelPlan pl = lp_plan(m, n, d.sms, a_type, lp_blocks_per_sm(BTO_OP_BICGK, a_type),
                                 lp_tma_ok(a_type, A, lda, m, n));
    char* w = static_cast<char*>(ws);
    if (cudaMemsetAsync(w, 0, sizeof(int), st) != cudaSuccess) return BTO_ERR_CUDA;
    LpArgs a{};
    a.m = m; a.n = n; a.A = A; a.lda = lda; a.p = p; a.r = r;
    a.tcmax = pl.TCmax; a.cu = lp_col_unit(a_type); a.status = reinterpret_cast<int*>(w);
    a.qpart = reinterpret_cast<double*>(w + L.off[0]); a.spart = reinterpret_cast<double*>(w + L.off[1]);
    a.ldq = pl.ldq; a.lds = pl.lds; a.NR = pl.NR; a.NC = pl.NC; a.ntiles = pl.ntiles;
    bto_status e = lp_launch(a_type, LP_QS, a, pl, st);
    if (e != BTO_OK) return e;
    if ((e = lp_combine(q, m, a.qpart, pl.ldq, pl.NC, 1.0, nullptr, 0.0, d.sms, st)) != BTO_OK) return e;
    return lp_combine(s, n, a.spart, pl.lds, pl.NR, 1.0, nullptr, 0.0, d.sms, st);
}

extern "C" bto_status bto_gemver_ex(int64_t m, int64_t n, float alpha, float beta, int a_type,
                                    const void* A, int64_t lda, const float* u1, const float* v1,
                                    const float* u2, const float* v2, const float* y, const float* z,
                                    void* B, int64_t ldb, float* x, float* w, void* ws, size_t ws_bytes,
                                    bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    c.size(1, m); c.size(2, n);
    if (a_type != BTO_F32 && a_type != BTO_BF16) c.fail(5);
    if (!c.ok()) return c.finish();
    const size_t es = a_type == BTO_F32 ? 4 : 2;
    const size_t Ab = mat_extent_bytes(m, n, lda, es), Bb = mat_extent_bytes(m, n, ldb, es);
    c.ptr(6, A, m > 0 && n > 0, es); c.ld(7, lda, m);
    c.ptr(8, u1, m > 0, 4); c.ptr(9, v1, n > 0, 4); c.ptr(10, u2, m > 0, 4); c.ptr(11, v2, n > 0, 4);
    c.ptr(12, y, m > 0, 4); c.ptr(13, z, n > 0, 4);
    c.ptr(14, B, m > 0 && n > 0, es); c.ld(15, ldb, m);
    c.ptr(16, x, n > 0, 4); c.ptr(17, w, m > 0, 4);
    const void* ins[6] = {u1, v1, u2, v2, y, z};
    const size_t inb[6] = {fbytes(m), fbytes(n), fbytes(m), fbytes(n), fbytes(m), fbytes(n)};
    if (!(B == A && ldb == lda)) c.disjoint(14, B, Bb, A, Ab);
    for (int k = 0; k < 6; k++) c.disjoint(14, B, Bb, ins[k], inb[k]);
    c.disjoint(16, x, fbytes(n), A, Ab); c.disjoint(16, x, fbytes(n), B, Bb);
    for (int k = 0; k < 5; k++) c.disjoint(16, x, fbytes(n), ins[k], inb[k]);
    if (x != z) c.disjoint(16, x, fbytes(n), z, fbytes(n));
    c.disjoint(17, w, fbytes(m), A, Ab); c.disjoint(17, w, fbytes(m), B, Bb);
    for (int k = 0; k < 6; k++) c.disjoint(17, w, fbytes(m), ins[k], inb[k]);
    c.disjoint(17, w, fbytes(m), x, fbytes(n));
    DeviceInfo d; WsLayout L;
    if (c.ok()) {
        if (!device_info(&d)) return BTO_ERR_CUDA;
        if (ws_layout(BTO_OP_GEMVER, BTO_FORM_FUSED, m, n, a_type, d, &L) != BTO_OK) return BTO_ERR_CUDA;
        c.ws(18, ws, ws_bytes, L);
    }
    if (!c.ok()) return c.finish();
    cudaStream_t st = (cudaStream_t)stream;
    // Both passes take the TMA path only when A and B both suit it.
    const PanelPlan pl = lp_plan(m, n, d.sms, a_type, 1,
                                 lp_tma_ok(a_type, A, lda, m, n) && lp_tma_ok(a_type, B, ldb, m, n));
    char* wk = static_cast<char*>(ws);
    if (cudaMemsetAsync(wk, 0, sizeof(int), st) != cudaSuccess) return BTO_ERR_CUDA;
    LpArgs a{};
    a.m = m; a.n = n; a.A = A; a.lda = lda; a.Bout = B; a.ldb = ldb;
    a.tcmax = pl.TCmax; a.cu = lp_col_unit(a_type); a.status = reinterpret_cast<int*>(wk);
    a.u1 = u1; a.v1 = v1; a.u2 = u2; a.v2 = v2; a.r = y;
    a.qpart = reinterpret_cast<double*>(wk + L.off[0]); a.spart = reinterpret_cast<double*>(wk + L.off[1]);
    a.ldq = pl.ldq; a.lds = pl.lds; a.NR = pl.NR; a.NC = pl.NC; a.ntiles = pl.ntiles;
    bto_status e = lp_launch(a_type, LP_G1, a, pl, st);                              // B, B^T y
    if (e != BTO_OK) return e;
    if ((e = lp_combine(x, n, a.spart, pl.lds, pl.NR, (double)beta, z, 1.0, d.sms, st)) != BTO_OK) return e;
    LpArgs b{};
    b.m = m; b.n = n; b.A = B; b.lda = ldb; b.p = x;
    b.qpart = a.qpart; b.ldq = pl.ldq; b.lds = pl.lds; b.NR = pl.NR; b.NC = pl.NC;
    b.ntiles = pl.ntiles; b.reverse = 1; b.tcmax = pl.TCmax; b.cu = a.cu; b.status = a.status;
    if ((e = lp_launch(a_type, LP_Q, b, pl, st)) != BTO_OK) return e;               // B x
    return lp_combine(w, m, b.qpart, pl.ldq, pl.NC, (double)alpha, nullptr, 0.0, d.sms, st);
}

// ATAX / BATAX (Table I; Section II, Fig. 1) in the reduced-precision storage
// form: t = A x by the q-only sweep and its combine (t in FP32 in the
// workspace), then y = beta A^T t by the s-only sweep, tiles in reverse order
// so that the first tiles of the second sweep find the last ones of the
// first in L2.  A is read twice; the FP64 form's single-read group-band
// kernel trades that read for an exchange between blocks, which pays off
// only where arithmetic, not bandwidth, is the bound.
extern "C" bto_status bto_atax_ex(int64_t m, int64_t n, float beta, int a_type, const void* A, int64_t lda,
                                  const float* x, float* y, void* ws, size_t ws_bytes, bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    c.size(1, m); c.size(2, n);
    if (a_type != BTO_F32 && a_type != BTO_BF16) c.fail(4);
    if (!c.ok()) return c.finish();
    const size_t es = a_type == BTO_F32 ? 4 : 2;
    const size_t Ab = mat_extent_bytes(m, n, lda, es);
    c.ptr(5, A, m > 0 && n > 0, es); c.ld(6, lda, m);
    c.ptr(7, x, n > 0, 4); c.ptr(8, y, n > 0, 4);
    c.disjoint(8, y, fbytes(n), A, Ab); c.disjoint(8, y, fbytes(n), x, fbytes(n));
    DeviceInfo d; WsLayout L;
    if (c.ok()) {
        if (!device_info(&d)) return BTO_ERR_CUDA;
        if (ws_layout(BTO_OP_ATAX, BTO_FORM_FUSED, m, n, a_type, d, &L) != BTO_OK) return BTO_ERR_CUDA;
        c.ws(9, ws, ws_bytes, L);
    }
    if (!c.ok()) return c.finish();
    cudaStream_t st = (cudaStream_t)stream;
    const PanelPlan pl = lp_plan(m, n, d.sms, a_type, lp_blocks_per_sm(BTO_OP_ATAX, a_type),
                                 lp_tma_ok(a_type, A, lda, m, n));
    char* w = static_cast<char*>(ws);
    if (cudaMemsetAsync(w, 0, sizeof(int), st) != cudaSuccess) return BTO_ERR_CUDA;
    if (n == 0) return BTO_OK;
    float* t = reinterpret_cast<float*>(w + L.off[0]);
    LpArgs a{};
    a.m = m; a.n = n; a.A = A; a.lda = lda; a.p = x;
    a.tcmax = pl.TCmax; a.cu = lp_col_unit(a_type); a.status = reinterpret_cast<int*>(w);
    a.qpart = reinterpret_cast<double*>(w + L.off[1]); a.spart = reinterpret_cast<double*>(w + L.off[2]);
    a.ldq = pl.ldq; a.lds = pl.lds; a.NR = pl.NR; a.NC = pl.NC; a.ntiles = pl.ntiles;
    bto_status e = lp_launch(a_type, LP_Q, a, pl, st);                               // A x
    if (e != BTO_OK) return e;
    if ((e = lp_combine(t, m, a.qpart, pl.ldq, pl.NC, 1.0, nullptr, 0.0, d.sms, st)) != BTO_OK) return e;
    a.p = nullptr; a.r = t; a.reverse = 1;
    if ((e = lp_launch(a_type, LP_S, a, pl, st)) != BTO_OK) return e;                // A^T t
    return lp_combine(y, n, a.spart, pl.lds, pl.NR, (double)beta, nullptr, 0.0, d.sms, st);
}

// GESUMMV (Table I) in the reduced-precision storage form: a q-only sweep
// over each matrix, then one combine forms alpha (A x) + beta (B x) in FP64
// from both sets of partials and rounds once.
extern "C" bto_status bto_gesummv_ex(int64_t m, int64_t n, float alpha, float beta, int a_type, const void* A,
                                     int64_t lda, const void* B, int64_t ldb, const float* x, float* y,
                                     void* ws, size_t ws_bytes, bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    c.size(1, m); c.size(2, n);
    if (a_type != BTO_F32 && a_type != BTO_BF16) c.fail(5);
    if (!c.ok()) return c.finish();
    const size_t es = a_type == BTO_F32 ? 4 : 2;
    const size_t Ab = mat_extent_bytes(m, n, lda, es), Bb = mat_extent_bytes(m, n, ldb, es);
    c.ptr(6, A, m > 0 && n > 0, es); c.ld(7, lda, m);
    c.ptr(8, B, m > 0 && n > 0, es); c.ld(9, ldb, m);
    c.ptr(10, x, n > 0, 4); c.ptr(11, y, m > 0, 4);
    c.disjoint(11, y, fbytes(m), A, Ab); c.disjoint(11, y, fbytes(m), B, Bb);
    c.disjoint(11, y, fbytes(m), x, fbytes(n));
    DeviceInfo d; WsLayout L;
    if (c.ok()) {
        if (!device_info(&d)) return BTO_ERR_CUDA;
        if (ws_layout(BTO_OP_GESUMMV, BTO_FORM_FUSED, m, n, a_type, d, &L) != BTO_OK) return BTO_ERR_CUDA;
        c.ws(12, ws, ws_bytes, L);
    }
    if (!c.ok()) return c.finish();
    cudaStream_t st = (cudaStream_t)stream;
    const PanelPlan pl = lp_plan(m, n, d.sms, a_type, lp_blocks_per_sm(BTO_OP_GESUMMV, a_type),
                                 lp_tma_ok(a_type, A, lda, m, n) && lp_tma_ok(a_type, B, ldb, m, n));
    char* w = static_cast<char*>(ws);
    if (cudaMemsetAsync(w, 0, sizeof(int), st) != cudaSuccess) return BTO_ERR_CUDA;
    LpArgs a{};
    a.m = m; a.n = n; a.A = A; a.lda = lda; a.p = x;
    a.tcmax = pl.TCmax; a.cu = lp_col_unit(a_type); a.status = reinterpret_cast<int*>(w);
    a.qpart = reinterpret_cast<double*>(w + L.off[0]);
    a.ldq = pl.ldq; a.lds = pl.lds; a.NR = pl.NR; a.NC = pl.NC; a.ntiles = pl.ntiles;
    bto_status e = lp_launch(a_type, LP_Q, a, pl, st);                               // A x
    if (e != BTO_OK) return e;
    LpArgs b = a;
    b.A = B; b.lda = ldb; b.qpart = reinterpret_cast<double*>(w + L.off[1]); b.reverse = 1;
    if ((e = lp_launch(a_type, LP_Q, b, pl, st)) != BTO_OK) return e;                // B x
    return lp_combine(y, m, a.qpart, pl.ldq, pl.NC, (double)alpha, nullptr, 0.0, d.sms, st, b.qpart, pl.NC,
                      (double)beta);
}
