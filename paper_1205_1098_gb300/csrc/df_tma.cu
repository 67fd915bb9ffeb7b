// Double-float sweeps of the FP64 matrix sequences: BICGK's two products,
// the single products of DGEMV, DGEMVT and ATAX, GEMVER's first pass, and
// GESUMMV's two matrices.
//
// GB300's FP64 unit issues two FMAs per clock per SM (1/64 of FP32), so a
// sweep that spends one or two FP64 FMAs per 8-byte matrix element is bound
// by that unit at a third to a half of HBM bandwidth.  These sweeps keep the
// FP64 data and the FP64 results but do the arithmetic on the FP32 pipes in
// double-float form (a value held as an unevaluated sum hi + lo of two FP32
// numbers):
//   - each FP64 element is split into hi + lo with integer operations only
//     (FP64 <-> FP32 conversions issue at the FP64 unit's rate): 47 of its 53
//     significant bits, exactly (df32.cuh, checked on the host);
//   - a product a v is the exact TwoProduct of the hi parts (FMA) plus the
//     cross terms a_hi v_lo + a_lo v_hi; the a_lo v_lo term (below 2^-47 of
//     the product) is dropped;
//   - sums are compensated: Knuth's TwoSum carries each rounding error of the
//     running sum into a low-order accumulator (the cascaded summation of
//     Ogita, Rump and Oishi), two rows per packed FP32 instruction;
//   - each 256-row chunk's sums become FP64 and add into FP64 partials, which
//     the panel engine's fixed-order FP64 combine reduces over the tiles.
// Error: each product keeps a relative error below 2^-45 and each
// compensated sum an error of order 2^-47 times its sum of magnitudes, so
// results stay within about 1e-14 normwise of exact FP64 arithmetic on
// ordinary data (the FP64 form's contract is 1e-12).  FP32's exponent range
// adds an underflow term: an element below 2^-127 in magnitude counts as
// zero, and products below about 2^-100 lose low-order bits, each an absolute
// error below 2^-126 times the other factor.
//
// Data movement: the matrix streams through shared memory as 256 x 16 boxes
// of FP64 (32 KB) copied by the tensor memory accelerator into a five-stage
// ring, fed by one producer warp; eight consumer warps take two columns of
// each box, lane l holding rows 2l and 2l + 1 of each 64-row quarter (one
// 16-byte shared-memory read per row pair).  A p accumulates per row in
// registers across the tile's columns; A^T r forms an 8-row partial per
// lane and column, then an 8-column transposing butterfly adds the 32
// lanes.  Row vectors of the next chunk are copied into shared memory
// asynchronously while the current chunk runs.
//
// Out of range.  An element of 2^128 or more in magnitude, Inf or NaN splits
// into a non-finite hi part, and a product or sum beyond FP32's range
// overflows, so either makes the chunk's results non-finite.  Chunk results
// are checked for finiteness; a 256-row chunk of a tile that fails is
// recomputed in FP64 from the matrix in global memory, so those inputs get
// plain FP64 semantics.  GEMVER's first pass forms B with two FP64 FMAs per
// element (the FP64 form's formula: its B, bit for bit), which leaves one
// FP64 instruction stream beside the FP32 work of the sums; B's column sums
// are double-float, and a chunk whose sums fail the check is recomputed in
// FP64 from the stored B.
//
// Every mbarrier wait is bounded by %globaltimer (2 s) and a shared abort
// flag; on expiry the block records BTO_ERR_TIMEOUT in the status word and
// the producer waits, again bounded, for the copies it issued.
#include "check.cuh"
#include "df32.cuh"
#include "tma.cuh"

namespace bto {
namespace {

constexpr int kCW = 8;                        // consumer warps
constexpr int kCT = kCW * 32;                 // consumer threads
constexpr int kThreadsT = kCT + 32;           // + one producer warp
constexpr int kBoxR = 256;                    // rows per stage (one chunk)
constexpr int kBoxC = 16;                     // columns per stage
constexpr int kStages = 5;
constexpr size_t kStageBytes = (size_t)kBoxR * kBoxC * sizeof(double);   // 32 KB
constexpr int kGS = 4;                        // stages per butterfly group (8 columns per warp)
constexpr int kMaxRowVecs = 3;                // u1, u2, y in GEMVER's first pass
constexpr int kMaxPanel = 1024;               // widest column panel (shared-memory vectors)
constexpr unsigned long long kWaitNs = 2000000000ull;

using df::split_words;

// ---------------------------------------------------------------- packed FP32
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// b - a, rounded once.
__device__ __forceinline__ float2 rsub2(float2 a, float2 b) { return __ffma2_rn(a, f2(-1.0f, -1.0f), b); }

// Knuth's TwoSum of S and P = -Pn: s + e == S - Pn exactly, s = fl(S - Pn).
__device__ __forceinline__ void two_sum_n(float2 S, float2 Pn, float2& s, float2& e) {
    s = rsub2(Pn, S);
    const float2 bb = rsub2(S, s);       // s - S
    const float2 t = rsub2(bb, s);       // s - bb
    const float2 e1 = rsub2(t, S);       // S - t
    const float2 e2n = add2(Pn, bb);     // -(P - bb)
    e = rsub2(e2n, e1);                  // e1 + (P - bb)
}
// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
    s = add2(a, b);
    const float2 bb = rsub2(a, s);       // s - a
    const float2 t = rsub2(bb, s);       // s - bb
    e = add2(rsub2(t, a), rsub2(bb, b)); // (a - t) + (b - bb)
}
__device__ __forceinline__ void two_sum1(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// Double-float add without renormalisation: (rh, rl) ~ (ah + al) + (bh + bl).
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& rh, float& rl) {
    float s, e;
    two_sum1(ah, bh, s, e);
    rh = s;
    rl = (al + bl) + e;
}

// Splits the two FP64 values of d (two rows) into packed hi and lo parts.
__device__ __forceinline__ void split_pair(double2 d, float2& H, float2& L) {
    split_words((uint32_t)__double2hiint(d.x), (uint32_t)__double2loint(d.x), H.x, L.x);
    split_words((uint32_t)__double2hiint(d.y), (uint32_t)__double2loint(d.y), H.y, L.y);
}
__device__ __forceinline__ void split_vec(double v, float& h, float& l) {
    split_words((uint32_t)__double2hiint(v), (uint32_t)__double2loint(v), h, l);
}

// Transposing butterfly over 8 column partials (hi, lo) per lane: lane l
// ends with the double-float sum over the 32 lanes of column l & 7.
__device__ __forceinline__ void butterfly8(float (&h)[8], float (&l)[8], int lane, float& oh, float& ol) {
#pragma unroll
    for (int half = 4; half >= 1; half >>= 1) {
        const bool upper = (lane & half) != 0;
#pragma unroll
        for (int k = 0; k < half; k++) {
            const float sh = upper ? h[k] : h[k + half], sl = upper ? l[k] : l[k + half];
            const float kh = upper ? h[k + half] : h[k], kl = upper ? l[k + half] : l[k];
            const float rh = __shfl_xor_sync(0xffffffffu, sh, half);
            const float rl = __shfl_xor_sync(0xffffffffu, sl, half);
            df_add(kh, kl, rh, rl, h[k], l[k]);
        }
    }
    float vh = h[0], vl = l[0];
#pragma unroll
    for (int d = 8; d <= 16; d <<= 1) {
        const float rh = __shfl_xor_sync(0xffffffffu, vh, d);
        const float rl = __shfl_xor_sync(0xffffffffu, vl, d);
        df_add(vh, vl, rh, rl, vh, vl);
    }
    oh = vh;
    ol = vl;
}

// Sum over the lane's 8 rows of a * v for one column: a as packed row pairs
// (AH, AL), v as packed row pairs (VH, its negation NVH, VL).  Returns the
// double-float sum (sh, sl).
__device__ __forceinline__ void col_partial(const float2 (&AH)[4], const float2 (&AL)[4], const float2 (&VH)[4],
                                            const float2 (&NVH)[4], const float2 (&VL)[4], float& sh, float& sl) {
    float2 Pn[4], Lx[4];
#pragma unroll
    for (int h = 0; h < 4; h++) {
        Pn[h] = mul2(AH[h], NVH[h]);                          // -(a_hi v_hi)
        const float2 E = fma2(AH[h], VH[h], Pn[h]);           // its rounding error, exact
        Lx[h] = fma2(AL[h], VH[h], fma2(AH[h], VL[h], E));    // + cross terms
    }
    float2 s01, e01, s23, e23, s, e;
    two_sum2(Pn[0], Pn[1], s01, e01);
    two_sum2(Pn[2], Pn[3], s23, e23);
    two_sum2(s01, s23, s, e);                                 // s + e + e01 + e23 = -(sum of hi products)
    float2 lo = add2(add2(Lx[0], Lx[1]), add2(Lx[2], Lx[3]));
    lo = rsub2(add2(add2(e01, e23), e), lo);
    float th, te;
    two_sum1(s.x, s.y, th, te);
    sh = -th;
    sl = (lo.x + lo.y) - te;
}

// Shared-memory plan of one block.
struct DfSmem {
    static size_t bytes(int64_t tcmax) {
        return kStages * kStageBytes + 2 * kStages * sizeof(uint64_t)   // ring, full, empty
               + (size_t)kCW * kBoxR * sizeof(float2)                      // q reduction (hi, lo)
               + (size_t)2 * kMaxRowVecs * kBoxR * sizeof(double)          // row vectors, two chunks
               + (size_t)tcmax * sizeof(double)                            // FP64 column sums of the tile
               + (size_t)6 * tcmax * sizeof(float);                        // chunk sums, p / v1, v2 parts
    }
};

template <int MODE>
__global__ void __launch_bounds__(kThreadsT, 1) df_kernel(const __grid_constant__ CUtensorMap tmA,
                                                          const __grid_constant__ CUtensorMap tmB, const DfArgs a) {
    constexpr bool HAS_Q = MODE == DF_QS || MODE == DF_Q || MODE == DF_Q2;
    constexpr bool HAS_S = MODE == DF_QS || MODE == DF_S || MODE == DF_G1;
    constexpr int SPU = MODE == DF_Q2 ? 2 : 1;              // stages per 16-column unit
    constexpr int NRV = MODE == DF_G1 ? 3 : (HAS_S ? 1 : 0);  // row vectors staged per chunk
    extern __shared__ __align__(1024) unsigned char smem[];
    double* ring = reinterpret_cast<double*>(smem);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
    uint64_t* empty = full + kStages;
    float2* qred = reinterpret_cast<float2*>(empty + kStages);               // [kCW][kBoxR]
    double* rowv = reinterpret_cast<double*>(qred + kCW * kBoxR);            // [2][kMaxRowVecs][kBoxR]
    double* sacc = rowv + 2 * kMaxRowVecs * kBoxR;                           // [tcmax]
    float* csh = reinterpret_cast<float*>(sacc + a.tcmax);                   // [tcmax] chunk column sums
    float* csl = csh + a.tcmax;
    float* vph = csl + a.tcmax;                                              // p (or v1) hi, lo
    float* vpl = vph + a.tcmax;
    float* v2h = vpl + a.tcmax;                                              // v2 hi, lo (GEMVER)
    float* v2l = v2h + a.tcmax;
    __shared__ int s_abort_;
    __shared__ int s_bad[2];
    volatile int* s_abort_p = &s_abort_;
    volatile int* s_badp = s_bad;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;

    if (tid == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kCW);
        }
        *s_abort_p = 0;
        s_badp[0] = s_badp[1] = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == kCW) {
        // ---------------- producer
        if (lane == 0) {
            long long g = 0;
            bool stop = false;       // testing only: see DfArgs::stall_block
            for (int64_t t = blockIdx.x; t < a.ntiles && !*s_abort_p && !stop; t += gridDim.x) {
                const int64_t tt = a.reverse ? (a.ntiles - 1 - t) : t;
                const int64_t cb = tt / a.NR, rb = tt % a.NR;
                const int64_t c0 = lp_col_at(a.n, a.NC, cb, kBoxC), c1 = lp_col_at(a.n, a.NC, cb + 1, kBoxC);
                const int64_t r0 = lp_row_at(a.m, a.NR, rb), r1 = lp_row_at(a.m, a.NR, rb + 1);
                for (int64_t R0 = r0; R0 < r1 && !*s_abort_p && !stop; R0 += kBoxR) {
                    for (int64_t cs = c0; cs < c1 && !*s_abort_p && !stop; cs += kBoxC) {
                        for (int u = 0; u < SPU; u++, g++) {
                            if ((int)blockIdx.x == a.stall_block && g >= kStages) {
                                stop = true;
                                break;
                            }
                            const int slot = (int)(g % kStages);
                            if (g >= kStages &&
                                !mbar_wait_bounded(&empty[slot], (uint32_t)(((g / kStages) - 1) & 1), a.wait_ns, s_abort_p)) {
                                atomicExch(a.status, (int)BTO_ERR_TIMEOUT);
                                *s_abort_p = 1;
                                break;
                            }
                            mbar_arrive_expect_tx(&full[slot], (uint32_t)kStageBytes);
                            tma_load_2d(ring + (size_t)slot * kBoxR * kBoxC, u ? &tmB : &tmA, (int)R0, (int)cs,
                                        &full[slot]);
                        }
                    }
                }
            }
            if (*s_abort_p || stop) {
                // Wait (bounded) for the copies this thread issued before leaving.
                const long long first = g > kStages ? g - kStages : 0;
                for (long long h = first; h < g; h++) mbar_wait_timed(&full[(int)(h % kStages)], (uint32_t)((h / kStages) & 1), kWaitNs);
            }
        }
        return;
    }

    // ---------------- consumers
    int slot = 0;            // ring slot of the next stage
    uint32_t ph = 0;         // parity of its use
    long long chunk = 0;     // chunks processed by this block (flag parity)
    for (int64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int64_t tt = a.reverse ? (a.ntiles - 1 - t) : t;
        const int64_t cb = tt / a.NR, rb = tt % a.NR;
        const int64_t c0 = lp_col_at(a.n, a.NC, cb, kBoxC), c1 = lp_col_at(a.n, a.NC, cb + 1, kBoxC);
        const int64_t r0 = lp_row_at(a.m, a.NR, rb), r1 = lp_row_at(a.m, a.NR, rb + 1);
        const int ncols = (int)(c1 - c0);
        const int ncols_u = (ncols + kBoxC - 1) / kBoxC * kBoxC;

        // Column vectors of the tile, split once (zero beyond the matrix);
        // GEMVER's v1 and v2 stay FP64 (B is formed with FP64 FMAs), in the
        // space of the split parts.
        double* v1d = reinterpret_cast<double*>(vph);
        double* v2d = reinterpret_cast<double*>(v2h);
        for (int k = tid; k < ncols_u; k += kCT) {
            if (HAS_S) sacc[k] = 0.0;
            if (HAS_Q) {
                const double v = k < ncols ? __ldg(a.p + c0 + k) : 0.0;
                split_vec(v, vph[k], vpl[k]);
            }
            if (MODE == DF_G1) {
                v1d[k] = k < ncols ? __ldg(a.v1 + c0 + k) : 0.0;
                v2d[k] = k < ncols ? __ldg(a.v2 + c0 + k) : 0.0;
            }
        }
        // Row vectors of the tile's first chunk.
        auto stage_rows = [&](int64_t R, int buf) {
            if (NRV == 0) return;
            const int64_t i = R + tid;
#pragma unroll
            for (int v = 0; v < NRV; v++) {
                const double* src = v == 0 ? (MODE == DF_G1 ? a.u1 : a.r) : (v == 1 ? a.u2 : a.r);
                double* dst = rowv + ((size_t)buf * kMaxRowVecs + v) * kBoxR + tid;
                if (i < r1) {
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src + i) : "memory");
                } else {
                    *dst = 0.0;
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        stage_rows(r0, 0);
        named_bar(1, kCT);

        int rbuf = 0;
        for (int64_t R0 = r0; R0 < r1; R0 += kBoxR, chunk++, rbuf ^= 1) {
            asm volatile("cp.async.wait_all;" ::: "memory");
            named_bar(1, kCT);
            if (R0 + kBoxR < r1) stage_rows(R0 + kBoxR, rbuf ^ 1);

            // The lane's rows: pair h holds rows R0 + 64h + 2 lane + {0, 1}.
            float2 RH[4], NRH[4], RL[4];         // r (or y) parts
            double2 U1[4], U2[4];                // GEMVER's u1, u2 (FP64)
            const double* rv = rowv + (size_t)rbuf * kMaxRowVecs * kBoxR;
#pragma unroll
            for (int h = 0; h < 4; h++) {
                const int row = 64 * h + 2 * lane;
                if (HAS_S) {
                    const int vi = MODE == DF_G1 ? 2 : 0;
                    float hx, lx, hy, ly;
                    split_vec(rv[vi * kBoxR + row], hx, lx);
                    split_vec(rv[vi * kBoxR + row + 1], hy, ly);
                    RH[h] = f2(hx, hy); NRH[h] = f2(-hx, -hy); RL[h] = f2(lx, ly);
                }
                if (MODE == DF_G1) {
                    U1[h] = make_double2(rv[row], rv[row + 1]);
                    U2[h] = make_double2(rv[kBoxR + row], rv[kBoxR + row + 1]);
                }
            }
            float2 QH[4], QL[4], QH2[4], QL2[4];
#pragma unroll
            for (int h = 0; h < 4; h++) {
                QH[h] = f2(0.f, 0.f); QL[h] = f2(0.f, 0.f); QH2[h] = f2(0.f, 0.f); QL2[h] = f2(0.f, 0.f);
            }

            for (int64_t gbase = c0; gbase < c1; gbase += (int64_t)kGS * kBoxC) {
                float sh[8], sl[8];
#pragma unroll
                for (int k = 0; k < 8; k++) { sh[k] = 0.f; sl[k] = 0.f; }
#pragma unroll
                for (int gs = 0; gs < kGS; gs++) {
                    const int64_t cs = gbase + (int64_t)gs * kBoxC;
                    if (cs < c1) {
#pragma unroll
                        for (int u = 0; u < SPU; u++) {
                            // A stage that completed holds valid data even after an
                            // abort; once the producer has stopped, the wait sees the
                            // abort flag on its first spin and returns false.
                            const bool have = mbar_wait_bounded(&full[slot], ph, a.wait_ns, s_abort_p);
                            if (!have) {
                                if (lane == 0) atomicExch(a.status, (int)BTO_ERR_TIMEOUT);
                                *s_abort_p = 1;
                            }
                            const double* buf = ring + (size_t)slot * kBoxR * kBoxC;
                            const int lc0 = (int)(cs - c0);
#pragma unroll
                            for (int cc = 0; cc < 2; cc++) {
                                const int c = 2 * warp + cc, lc = lc0 + c;
                                if (!have) continue;
                                const double2* col = reinterpret_cast<const double2*>(buf + c * kBoxR);
                                double2 D[4];
                                float2 AH[4], AL[4];
#pragma unroll
                                for (int h = 0; h < 4; h++) {
                                    D[h] = col[h * 32 + lane];
                                    if (MODE != DF_G1) split_pair(D[h], AH[h], AL[h]);
                                }
                                if (HAS_Q) {
                                    const float p_h = vph[lc], p_l = vpl[lc];
                                    const float2 PH = f2(p_h, p_h), NPH = f2(-p_h, -p_h), PL = f2(p_l, p_l);
#pragma unroll
                                    for (int h = 0; h < 4; h++) {
                                        const float2 Pn = mul2(AH[h], NPH);
                                        const float2 E = fma2(AH[h], PH, Pn);
                                        float2 s, e;
                                        // A's columns take turns between two accumulator
                                        // sets (B's in GESUMMV), so consecutive updates of
                                        // a row are independent.
                                        if (MODE == DF_Q2 ? u == 0 : cc == 0) {
                                            two_sum_n(QH[h], Pn, s, e);
                                            QH[h] = s;
                                            QL[h] = fma2(AL[h], PH, fma2(AH[h], PL, add2(QL[h], add2(E, e))));
                                        } else {
                                            two_sum_n(QH2[h], Pn, s, e);
                                            QH2[h] = s;
                                            QL2[h] = fma2(AL[h], PH, fma2(AH[h], PL, add2(QL2[h], add2(E, e))));
                                        }
                                    }
                                }
                                if (MODE == DF_QS || MODE == DF_S)
                                    col_partial(AH, AL, RH, NRH, RL, sh[2 * gs + cc], sl[2 * gs + cc]);
                                if (MODE == DF_G1) {
                                    // B = (A + u1 v1^T) + u2 v2^T with two FP64 FMAs per
                                    // element (the FP64 form's formula, so the same bits),
                                    // stored, then split for the double-float column sum.
                                    const double v1j = v1d[lc], v2j = v2d[lc];
                                    const int64_t col_g = cs + c;
                                    double* bcol = a.Bout + col_g * a.ldbo;
                                    float2 BH[4], BL[4];
#pragma unroll
                                    for (int h = 0; h < 4; h++) {
                                        const int64_t i0 = R0 + 64 * h + 2 * lane;
                                        const double b0 = fma(U2[h].x, v2j, fma(U1[h].x, v1j, D[h].x));
                                        const double b1 = fma(U2[h].y, v2j, fma(U1[h].y, v1j, D[h].y));
                                        if (col_g < c1) {
                                            if (i0 + 1 < r1) {
                                                *reinterpret_cast<double2*>(bcol + i0) = make_double2(b0, b1);
                                            } else if (i0 < r1) {
                                                bcol[i0] = b0;
                                            }
                                        }
                                        split_pair(make_double2(b0, b1), BH[h], BL[h]);
                                    }
                                    col_partial(BH, BL, RH, NRH, RL, sh[2 * gs + cc], sl[2 * gs + cc]);
                                }
                            }
                            __syncwarp();
                            if (lane == 0 && have) mbar_arrive(&empty[slot]);
                            if (++slot == kStages) { slot = 0; ph ^= 1u; }
                        }
                    }
                }
                if (HAS_S) {
                    float oh, ol;
                    butterfly8(sh, sl, lane, oh, ol);
                    if (lane < 8) {
                        const int64_t col = gbase + (int64_t)(lane >> 1) * kBoxC + 2 * warp + (lane & 1);
                        if (col < c1) {
                            csh[col - c0] = oh;
                            csl[col - c0] = ol;
                        }
                    }
                }
            }

            // ---- chunk end: rows of q, check, write or recompute in FP64
            const int fl = (int)(chunk & 1);
            double qv = 0.0, qv2 = 0.0;
            if (MODE == DF_QS || MODE == DF_Q) {
#pragma unroll
                for (int h = 0; h < 4; h++) {
                    float2 s, e;
                    two_sum2(QH[h], QH2[h], s, e);
                    QH[h] = s;
                    QL[h] = add2(add2(QL[h], QL2[h]), e);
                }
            }
#pragma unroll
            for (int pass = 0; pass < (MODE == DF_Q2 ? 2 : (HAS_Q ? 1 : 0)); pass++) {
                if (pass == 1) named_bar(1, kCT);
#pragma unroll
                for (int h = 0; h < 4; h++) {
                    const float2 hh = pass ? QH2[h] : QH[h], ll = pass ? QL2[h] : QL[h];
                    qred[warp * kBoxR + 64 * h + 2 * lane] = f2(hh.x, ll.x);
                    qred[warp * kBoxR + 64 * h + 2 * lane + 1] = f2(hh.y, ll.y);
                }
                named_bar(1, kCT);
                float2 acc = qred[tid];
#pragma unroll
                for (int w = 1; w < kCW; w++) {
                    const float2 v = qred[w * kBoxR + tid];
                    float s, e;
                    two_sum1(acc.x, v.x, s, e);
                    acc.x = s;
                    acc.y += v.y + e;
                }
                const double v = (double)acc.x + (double)acc.y;
                if (!isfinite(v)) s_badp[fl] = 1;
                if (pass == 0) qv = v; else qv2 = v;
            }
            if (HAS_S) {
                if (!HAS_Q) named_bar(1, kCT);
                for (int k = tid; k < ncols; k += kCT)
                    if (!isfinite(csh[k]) || !isfinite(csl[k])) s_badp[fl] = 1;
            }
            named_bar(1, kCT);
            const bool bad = s_badp[fl] != 0;
            if (tid == 0) s_badp[fl ^ 1] = 0;
            const int64_t i = R0 + tid;
            if (!bad) {
                if (HAS_Q && i < r1) a.qpart[cb * a.ldq + i] = qv;
                if (MODE == DF_Q2 && i < r1) a.qpart2[cb * a.ldq + i] = qv2;
                if (HAS_S)
                    for (int k = tid; k < ncols; k += kCT) sacc[k] += (double)csh[k] + (double)csl[k];
            } else {
                // FP64 recomputation of this chunk of the tile, fixed order.
                if (HAS_Q && i < r1) {
                    double acc = 0.0, acc2 = 0.0;
                    for (int64_t j = c0; j < c1; j++) {
                        const double pj = __ldg(a.p + j);
                        acc = fma(__ldg(a.A + i + j * a.lda), pj, acc);
                        if (MODE == DF_Q2) acc2 = fma(__ldg(a.B + i + j * a.ldb), pj, acc2);
                    }
                    a.qpart[cb * a.ldq + i] = acc;
                    if (MODE == DF_Q2) a.qpart2[cb * a.ldq + i] = acc2;
                }
                if (HAS_S) {
                    const double* M = MODE == DF_G1 ? a.Bout : a.A;
                    const int64_t ld = MODE == DF_G1 ? a.ldbo : a.lda;
                    const int64_t rend = R0 + kBoxR < r1 ? R0 + kBoxR : r1;
                    for (int64_t j = c0 + warp; j < c1; j += kCW) {
                        double acc = 0.0;
                        for (int64_t ii = R0 + lane; ii < rend; ii += 32)
                            acc = fma(MODE == DF_G1 ? M[ii + j * ld] : __ldg(M + ii + j * ld), __ldg(a.r + ii), acc);
#pragma unroll
                        for (int d = 16; d >= 1; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
                        if (lane == 0) sacc[j - c0] += acc;
                    }
                }
            }
            named_bar(1, kCT);
        }
        if (HAS_S)
            for (int k = tid; k < ncols; k += kCT) a.spart[rb * a.lds + c0 + k] = sacc[k];
        named_bar(1, kCT);
    }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

template <int MODE>
bto_status launch_t(const CUtensorMap& ma, const CUtensorMap& mb, const DfArgs& a, int grid, cudaStream_t st) {
    auto k = df_kernel<MODE>;
    const size_t smem = DfSmem::bytes(a.tcmax);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return BTO_ERR_CUDA;
    k<<<grid, kThreadsT, smem, st>>>(ma, mb, a);
    return launch_status();
}

}  // namespace

PanelPlan df_plan(int64_t m, int64_t n, int sms) {
    PanelPlan pl;
    pl.bps = 1;
    pl.ldq = round_up(m > 0 ? m : 1, 32);
    pl.lds = round_up(n > 0 ? n : 1, 32);
    if (m <= 0 || n <= 0) return pl;
    const int64_t G = sms, cu = kBoxC;
    const int64_t cunits = ceil_div(n, cu), runits = ceil_div(m, kBoxR);
    // NR row blocks x NC column panels, panels no wider than kMaxPanel columns
    // (their vectors live in shared memory).  With at most one tile per
    // block, take the split with the least busiest-block work (widest panel x
    // tallest row block, in 256 x 16 units) times one plus the bytes of FP64
    // partials written and read again (NC x m and NR x n) over the matrix
    // bytes.  Wider matrices than one tile per block allows take panels of
    // kMaxPanel columns, several per block.
    const int64_t wmax = kMaxPanel / kBoxC;
    const double abytes = 8.0 * (double)m * (double)n;
    int64_t bestNR = 0, bestNC = 0;
    double best = 0.0;
    for (int64_t NR = 1; NR <= std::min<int64_t>(G, runits); NR++) {
        const int64_t NC = std::min<int64_t>(cunits, G / NR);
        if (NC < 1) break;
        const int64_t wu = ceil_div(cunits, NC), hc = ceil_div(runits, NR);
        if (wu > wmax) continue;
        const double pbytes = 2.0 * 8.0 * ((double)NC * (double)m + (double)NR * (double)n);
        const double cost = (double)(wu * hc) * (1.0 + pbytes / abytes);
        if (bestNR == 0 || cost < best) { best = cost; bestNR = NR; bestNC = NC; }
    }
    if (bestNR == 0) {
        bestNC = std::max<int64_t>(std::min<int64_t>(G, cunits), ceil_div(cunits, wmax));
        bestNR = std::max<int64_t>(1, std::min<int64_t>(G / bestNC, runits));
    }
    pl.NC = (int)bestNC;
    pl.NR = (int)bestNR;
    pl.TCmax = ceil_div(cunits, bestNC) * cu;
    pl.ntiles = bestNR * bestNC;
    pl.grid = (int)std::min<int64_t>(G, pl.ntiles);
    return pl;
}

bto_status df_ws_layout(int op, int form, int64_t m, int64_t n, const DeviceInfo& d, WsLayout* out) {
    if (op < BTO_OP_BICGK || op > BTO_OP_DGEMVT) return BTO_ERR_UNSUPPORTED;
    // The FP64 form the call runs when the layout does not suit the copies.
    WsLayout F;
    bto_status e = ws_layout(op, form == BTO_FORM_DF ? BTO_FORM_FUSED : BTO_FORM_UNFUSED, m, n, BTO_F64, d, &F);
    if (e != BTO_OK) return e;
    const PanelPlan pl = df_plan(m, n, d.sms);
    const size_t qp = (size_t)pl.NC * pl.ldq * sizeof(double);
    const size_t sp = (size_t)pl.NR * pl.lds * sizeof(double);
    WsLayout L;
    size_t cur = WS_HEADER;
    auto region = [&](size_t bytes) {
        const size_t at = cur;
        cur += round_up((int64_t)bytes, 256);
        return at;
    };
    switch (op) {
        case BTO_OP_BICGK:
        case BTO_OP_GEMVER:
        case BTO_OP_DGEMVT:
            L.off[0] = region(qp);
            L.off[1] = region(sp);
            break;
        case BTO_OP_DGEMV:
            L.off[0] = region(qp);
            break;
        case BTO_OP_GESUMMV:
            L.off[0] = region(qp);
            L.off[1] = region(qp);
            break;
        case BTO_OP_ATAX:
            L.off[0] = region((size_t)std::max<int64_t>(m, 1) * sizeof(double));   // t = A x
            L.off[1] = region(qp);
            L.off[2] = region(sp);
            break;
    }
    L.total = std::max(cur, F.total);
    *out = L;
    return BTO_OK;
}

DfArgs df_args(int64_t m, int64_t n, const double* A, int64_t lda, const PanelPlan& pl, void* ws) {
    DfArgs a{};
    a.m = m; a.n = n; a.A = A; a.lda = lda;
    a.ldq = pl.ldq; a.lds = pl.lds; a.tcmax = pl.TCmax;
    a.NR = pl.NR; a.NC = pl.NC; a.ntiles = pl.ntiles;
    a.status = static_cast<int*>(ws);
    a.wait_ns = kWaitNs;
    a.stall_block = -1;
    return a;
}

bto_status df_gemv_n(int64_t m, int64_t n, double alpha, const double* A, int64_t lda, const double* v,
                     double beta, const double* y, double* out, double* qpart, const PanelPlan& pl, void* ws,
                     int reverse, cudaStream_t st) {
    if (m <= 0) return BTO_OK;
    DfArgs a = df_args(m, n, A, lda, pl, ws);
    a.p = v; a.qpart = qpart; a.reverse = reverse;
    bto_status e = df_launch(DF_Q, a, pl, st);
    if (e != BTO_OK) return e;
    CombineJob j = {out, m, qpart, pl.ldq, n > 0 ? pl.NC : 0, alpha, nullptr, 0, 0, 0.0, y, beta};
    return launch_combine(&j, 1, st);
}

bto_status df_gemv_t(int64_t m, int64_t n, double alpha, const double* A, int64_t lda, const double* v,
                     double beta, const double* y, double* out, double* spart, const PanelPlan& pl, void* ws,
                     int reverse, cudaStream_t st) {
    if (n <= 0) return BTO_OK;
    DfArgs a = df_args(m, n, A, lda, pl, ws);
    a.r = v; a.spart = spart; a.reverse = reverse;
    bto_status e = df_launch(DF_S, a, pl, st);
    if (e != BTO_OK) return e;
    CombineJob j = {out, n, spart, pl.lds, m > 0 ? pl.NR : 0, alpha, nullptr, 0, 0, 0.0, y, beta};
    return launch_combine(&j, 1, st);
}

bool df_layout_ok(int mode, const DfArgs& a) {
    if (a.m <= 0 || a.n <= 0 || a.m > INT32_MAX || a.n > INT32_MAX) return false;
    auto mat_ok = [](const void* p, int64_t ld) { return aligned16(p) && ld % 2 == 0; };
    if (!mat_ok(a.A, a.lda)) return false;
    if (mode == DF_Q2 && !mat_ok(a.B, a.ldb)) return false;
    if (mode == DF_G1 && !mat_ok(a.Bout, a.ldbo)) return false;
    return true;
}

bto_status df_launch(int mode, const DfArgs& a, const PanelPlan& pl, cudaStream_t st) {
    if (pl.ntiles == 0) return BTO_OK;
    if (!df_layout_ok(mode, a) || a.tcmax > kMaxPanel) return BTO_ERR_INVALID_VALUE;
    CUtensorMap ma, mb;
    if (!encode_tmap_2d(&ma, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, a.A, a.m, a.n, a.lda, kBoxR, kBoxC))
        return BTO_ERR_CUDA;
    mb = ma;
    if (mode == DF_Q2 &&
        !encode_tmap_2d(&mb, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, a.B, a.m, a.n, a.ldb, kBoxR, kBoxC))
        return BTO_ERR_CUDA;
    const int grid = pl.grid;
    switch (mode) {
        case DF_QS: return launch_t<DF_QS>(ma, mb, a, grid, st);
        case DF_Q: return launch_t<DF_Q>(ma, mb, a, grid, st);
        case DF_S: return launch_t<DF_S>(ma, mb, a, grid, st);
        case DF_G1: return launch_t<DF_G1>(ma, mb, a, grid, st);
        case DF_Q2: return launch_t<DF_Q2>(ma, mb, a, grid, st);
    }
    return BTO_ERR_INVALID_VALUE;
}

}  // namespace bto
