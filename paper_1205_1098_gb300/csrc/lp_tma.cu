// TMA-fed sweep of the reduced-precision storage form (BICGK, both GEMVER
// passes, and the q-only and s-only sweeps that ATAX and GESUMMV are made of,
// with the matrices in FP32/BF16).
//
// Each stage is a 256-row x 16-column box of the matrix, copied by the tensor
// memory accelerator (cp.async.bulk.tensor) into a ring of shared-memory
// buffers.  One producer warp issues the copies; eight consumer warps take
// two columns of the stage each, with lane l holding 8 rows (one 16-byte
// shared-memory read per column for BF16, two for FP32).  Buffers are handed
// back and forth with mbarriers (a "full" barrier completed by the copy's
// transaction bytes, an "empty" barrier that the eight consumer warps arrive
// on), so 6-8 stages of the matrix are in flight per SM without holding any
// registers.  The arithmetic is that of the load-instruction sweep:
//   A p   : FP32 FMA chains over 16 columns per row, folded into TwoSum pairs;
//   A^T r : per column two 4-row FMA chains (even and odd rows), a 16-column
//           transposing butterfly across the warp, folded into TwoSum pairs
//           in shared memory;
// FMAs on pairs of rows use the packed FP32 instructions (__ffma2_rn).
// tiles end in (hi, lo) FP32 pairs that a fixed-order FP64 combine adds.
// Every mbarrier wait is bounded by %globaltimer (2 s) and by a shared abort
// flag: on expiry the block records BTO_ERR_TIMEOUT in the status word,
// skips the remaining waits (so every warp still reaches every named
// barrier), and the producer waits, again with a bound, for the copies it
// issued before the block exits.
#include "check.cuh"
#include "lp_math.cuh"
#include "tma.cuh"
#include <mutex>

namespace bto {
namespace {

using namespace lp;

constexpr int kConsumerWarps = 8;
constexpr int kConsumers = kConsumerWarps * 32;
constexpr int kThreadsT = kConsumers + 32;       // + one producer warp
constexpr int kBoxR = 256;                        // rows per stage
constexpr int kRPT = 8;                           // rows per lane
constexpr unsigned long long kWaitNs = 2000000000ull;

// A stage is one 16 KB box: 256 rows x 32 columns of BF16 or 256 x 16 of
// FP32 (the copy engine's cost grows with the number of boxes, so boxes are
// as large as the panel unit allows); each consumer warp takes CPW = BoxC / 8
// of its columns.  Twelve stages keep 192 KB of the matrix in flight per SM.
template <typename TA> struct Cfg {
    static constexpr int BoxC = sizeof(TA) == 2 ? 32 : 16;
    static constexpr int CPW = BoxC / kConsumerWarps;
    static constexpr int GroupStages = 16 / CPW;        // stages per 16-column butterfly group
    static constexpr int S = 12;
};

template <typename TA>
constexpr size_t stage_bytes() { return (size_t)kBoxR * Cfg<TA>::BoxC * sizeof(TA); }

// Ring depth for BPS blocks per SM: twelve stages at one block, five each at
// two (the plan decides; see lp_blocks_per_sm).  With BF16 the consumers have
// twice the elements per byte of FP32 and wait on shuffle and FMA chains; a
// second block per SM covers those waits (BF16 BICGK 0.568 -> 0.514 ms at
// n = 32768).
template <typename TA, int BPS> struct LpStages {
    static constexpr int value = BPS == 2 ? 5 : Cfg<TA>::S;
};

// nvec column vectors of the tile: s (hi, lo) and p, plus v1 and v2 in
// GEMVER's first pass (5); 3 otherwise.
template <typename TA, int BPS>
size_t tma_smem(int64_t tcmax, int nvec) {
    return LpStages<TA, BPS>::value * stage_bytes<TA>()     // ring
           + 2 * LpStages<TA, BPS>::value * sizeof(uint64_t)   // full, empty
           + 2 * kConsumerWarps * kBoxR * sizeof(float)      // q reduction (hi, lo)
           + (size_t)nvec * (size_t)tcmax * sizeof(float) + 128;
}
constexpr int lp_nvec(int mode) { return mode == LP_G1 ? 5 : 3; }

template <typename TA>
constexpr int box_cols() { return Cfg<TA>::BoxC; }

// Row (within the stage) of lane's k-th element: V = 16 / sizeof(TA) rows
// per 16-byte read.
template <int V>
__device__ __forceinline__ int trow(int lane, int k) { return (k / V) * (32 * V) + lane * V + (k % V); }

// sum_k a[k] r[k] over a lane's 8 rows as two interleaved FMA chains (even
// and odd rows) in packed FP32 instructions, added at the end.
__device__ __forceinline__ float dot8(const float (&a)[kRPT], const float (&r)[kRPT]) {
    float2 acc = __fmul2_rn(make_float2(a[0], a[1]), make_float2(r[0], r[1]));
#pragma unroll
    for (int k = 2; k < kRPT; k += 2) acc = __ffma2_rn(make_float2(a[k], a[k + 1]), make_float2(r[k], r[k + 1]), acc);
    return acc.x + acc.y;
}

// The V values of a 16-byte shared-memory read as FP32: one bit operation
// per BF16 value (the high half of a 32-bit word is already an FP32 bit
// pattern; the low half is shifted up).
template <typename TA>
__device__ __forceinline__ void unpack16(const uint4& raw, float* out) {
    const unsigned w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int k = 0; k < 4; k++) {
        if (sizeof(TA) == 4) {
            out[k] = __uint_as_float(w[k]);
        } else {
            out[2 * k] = __uint_as_float(w[k] << 16);
            out[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
        }
    }
}

template <typename TA, int MODE, int BPS>
__global__ void __launch_bounds__(kThreadsT, BPS) lp_tma_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                const LpArgs a) {
    constexpr int V = 16 / sizeof(TA);
    constexpr int S = LpStages<TA, BPS>::value;
    constexpr int kBoxC = Cfg<TA>::BoxC;
    constexpr int CPW = Cfg<TA>::CPW;
    constexpr bool HAS_Q = (MODE == LP_QS || MODE == LP_Q);
    constexpr bool HAS_S = (MODE == LP_QS || MODE == LP_G1 || MODE == LP_S);
    extern __shared__ __align__(1024) unsigned char smem[];
    TA* ring = reinterpret_cast<TA*>(smem);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * stage_bytes<TA>());
    uint64_t* empty = full + S;
    float* qred = reinterpret_cast<float*>(empty + S);          // [2][8][256]
    float* shi = qred + 2 * kConsumerWarps * kBoxR;               // [tcmax]
    float* slo = shi + a.tcmax;
    float* sp = slo + a.tcmax;                                    // p, v1, v2 of the tile
    float* sv1 = sp + a.tcmax;
    float* sv2 = sv1 + a.tcmax;
    __shared__ int s_abort_;
    volatile int* s_abort_p = &s_abort_;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        *s_abort_p = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == kConsumerWarps) {
        // ---------------- producer
        if (lane == 0) {
            long long g = 0;
            for (int64_t t = blockIdx.x; t < a.ntiles && !*s_abort_p; t += gridDim.x) {
                const int64_t tt = a.reverse ? (a.ntiles - 1 - t) : t;
                const int64_t cb = tt / a.NR, rb = tt % a.NR;
                const int64_t c0 = lp_col_at(a.n, a.NC, cb, kBoxC), c1 = lp_col_at(a.n, a.NC, cb + 1, kBoxC);
                const int64_t r0 = lp_row_at(a.m, a.NR, rb), r1 = lp_row_at(a.m, a.NR, rb + 1);
                for (int64_t R0 = r0; R0 < r1 && !*s_abort_p; R0 += kBoxR) {
                    for (int64_t cs = c0; cs < c1; cs += kBoxC, g++) {
                        const int slot = (int)(g % S);
                        if (g >= S && !mbar_wait_bounded(&empty[slot], (uint32_t)(((g / S) - 1) & 1), kWaitNs, s_abort_p)) {
                            atomicExch(a.status, (int)BTO_ERR_TIMEOUT);
                            *s_abort_p = 1;
                            break;
                        }
                        mbar_arrive_expect_tx(&full[slot], (uint32_t)stage_bytes<TA>());
                        tma_load_2d(ring + (size_t)slot * kBoxR * kBoxC, &tmA, (int)R0, (int)cs, &full[slot]);
                    }
                }
            }
            if (*s_abort_p) {
                // Wait (bounded) for the copies this thread issued before leaving.
                const long long first = g > S ? g - S : 0;
                for (long long h = first; h < g; h++) {
                    const int slot = (int)(h % S);
                    const unsigned long long t0 = global_ns();
                    while (!mbar_try_wait(&full[slot], (uint32_t)((h / S) & 1)) && global_ns() - t0 < kWaitNs) {
                    }
                }
            }
        }
        return;
    }

    // ---------------- consumers
    TA* Bout = static_cast<TA*>(a.Bout);
    int slot = 0;            // ring slot of the next stage
    uint32_t ph = 0;         // parity of its use (stage index / S, mod 2)
    for (int64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int64_t tt = a.reverse ? (a.ntiles - 1 - t) : t;
        const int64_t cb = tt / a.NR, rb = tt % a.NR;
        const int64_t c0 = lp_col_at(a.n, a.NC, cb, kBoxC), c1 = lp_col_at(a.n, a.NC, cb + 1, kBoxC);
        const int64_t r0 = lp_row_at(a.m, a.NR, rb), r1 = lp_row_at(a.m, a.NR, rb + 1);
        const int ncols = (int)(c1 - c0);
        for (int k = threadIdx.x; k < ncols; k += kConsumers) {
            shi[k] = 0.0f; slo[k] = 0.0f;
            if (HAS_Q) sp[k] = __ldg(a.p + c0 + k);
            if (MODE == LP_G1) { sv1[k] = __ldg(a.v1 + c0 + k); sv2[k] = __ldg(a.v2 + c0 + k); }
        }
        named_bar(1, kConsumers);
        // Row vectors of the next chunk are loaded one chunk ahead, so their
        // latency overlaps the current chunk's stages.
        float rvn[kRPT], u1n[kRPT], u2n[kRPT];
        auto load_rows = [&](int64_t R) {
#pragma unroll
            for (int k = 0; k < kRPT; k++) {
                const int64_t i = R + trow<V>(lane, k);
                rvn[k] = (HAS_S && i < r1) ? __ldg(a.r + i) : 0.0f;
                u1n[k] = (MODE == LP_G1 && i < r1) ? __ldg(a.u1 + i) : 0.0f;
                u2n[k] = (MODE == LP_G1 && i < r1) ? __ldg(a.u2 + i) : 0.0f;
            }
        };
        load_rows(r0);
        for (int64_t R0 = r0; R0 < r1; R0 += kBoxR) {
            float rv[kRPT], u1r[kRPT], u2r[kRPT], qhi[kRPT], qlo[kRPT], qt[kRPT], sl[16];
#pragma unroll
            for (int k = 0; k < kRPT; k++) {
                rv[k] = rvn[k]; u1r[k] = u1n[k]; u2r[k] = u2n[k];
                qhi[k] = 0.0f; qlo[k] = 0.0f; qt[k] = 0.0f;
            }
            if (R0 + kBoxR < r1) load_rows(R0 + kBoxR);
#pragma unroll
            for (int k = 0; k < 16; k++) sl[k] = 0.0f;
            // Butterfly groups of GroupStages stages; the stage loop is unrolled so
            // that sl[] is indexed by constants (and stays in registers).
            constexpr int GS = Cfg<TA>::GroupStages;
            for (int64_t gbase = c0; gbase < c1; gbase += (int64_t)GS * kBoxC) {
#pragma unroll
            for (int gs = 0; gs < GS; gs++) {
              const int64_t cs = gbase + (int64_t)gs * kBoxC;
              if (cs < c1) {
                bool have = true;
                if (!*s_abort_p && !mbar_wait_bounded(&full[slot], ph, kWaitNs, s_abort_p)) {
                    if (lane == 0) atomicExch(a.status, (int)BTO_ERR_TIMEOUT);
                    *s_abort_p = 1;
                }
                if (*s_abort_p) have = false;
                const TA* buf = ring + (size_t)slot * kBoxR * kBoxC;
                const int lc0 = (int)(cs - c0);      // tile-local column of the stage's first column
#pragma unroll
                for (int cc = 0; cc < CPW; cc++) {
                    const int c = CPW * warp + cc;
                    const int lc = lc0 + c;
                    if (have && lc < ncols) {
                        const int64_t col = c0 + lc;
                        float av[kRPT];
#pragma unroll
                        for (int h = 0; h < kRPT / V; h++)
                            unpack16<TA>(*reinterpret_cast<const uint4*>(buf + c * kBoxR + h * 32 * V + lane * V), av + h * V);
                        if (MODE == LP_G1) {
                            const float v1j = sv1[lc], v2j = sv2[lc];
                            TA bq[kRPT];
                            float bf[kRPT];
                            unsigned bw[kRPT / 2];     // BF16: the rounded pairs as stored
#pragma unroll
                            for (int k = 0; k < kRPT; k += 2) {
                                // Two rows per packed FMA; per element the same two FMAs as before.
                                const float2 t = __ffma2_rn(make_float2(u2r[k], u2r[k + 1]), make_float2(v2j, v2j),
                                                            __ffma2_rn(make_float2(u1r[k], u1r[k + 1]),
                                                                       make_float2(v1j, v1j),
                                                                       make_float2(av[k], av[k + 1])));
                                if constexpr (sizeof(TA) == 2) {
                                    // One conversion rounds both rows (nearest even, as the
                                    // single-value form); the word is what is stored, and its
                                    // halves widen back with one bit operation each.
                                    const __nv_bfloat162 b2 = __float22bfloat162_rn(t);
                                    const unsigned w = *reinterpret_cast<const unsigned*>(&b2);
                                    bw[k / 2] = w;
                                    bf[k] = __uint_as_float(w << 16);
                                    bf[k + 1] = __uint_as_float(w & 0xFFFF0000u);
                                } else {
                                    bq[k] = from_f<TA>(t.x);
                                    bq[k + 1] = from_f<TA>(t.y);
                                    bf[k] = to_f<TA>(bq[k]);
                                    bf[k + 1] = to_f<TA>(bq[k + 1]);
                                }
                            }
                            TA* bcol = Bout + col * a.ldb;
#pragma unroll
                            for (int h = 0; h < kRPT / V; h++) {
                                const int64_t i = R0 + h * 32 * V + lane * V;
                                if (i + V <= r1) {   // B and ldb are 16-byte aligned on this path
                                    uint4 raw;
                                    if constexpr (sizeof(TA) == 2) {
                                        raw = make_uint4(bw[4 * h], bw[4 * h + 1], bw[4 * h + 2], bw[4 * h + 3]);
                                    } else {
                                        TA* e = reinterpret_cast<TA*>(&raw);
#pragma unroll
                                        for (int q = 0; q < V; q++) e[q] = bq[h * V + q];
                                    }
                                    *reinterpret_cast<uint4*>(bcol + i) = raw;
                                } else {
#pragma unroll
                                    for (int q = 0; q < V; q++) {
                                        if (i + q < r1) {
                                            if constexpr (sizeof(TA) == 2) {
                                                const unsigned w = bw[(h * V + q) / 2];
                                                const unsigned short bits = (unsigned short)(((h * V + q) & 1) ? (w >> 16) : (w & 0xFFFFu));
                                                bcol[i + q] = __ushort_as_bfloat16(bits);
                                            } else {
                                                bcol[i + q] = bq[h * V + q];
                                            }
                                        }
                                    }
                                }
                            }
                            sl[CPW * gs + cc] = dot8(bf, rv);
                        } else {
                            if (HAS_Q) {
                                const float pj = sp[lc];
#pragma unroll
                                for (int k = 0; k < kRPT; k += 2) {
                                    const float2 t = __ffma2_rn(make_float2(av[k], av[k + 1]), make_float2(pj, pj),
                                                                make_float2(qt[k], qt[k + 1]));
                                    qt[k] = t.x;
                                    qt[k + 1] = t.y;
                                }
                            }
                            if (HAS_S) sl[CPW * gs + cc] = dot8(av, rv);
                        }
                    }
                }
                __syncwarp();
                if (lane == 0 && have) mbar_arrive(&empty[slot]);
                if (++slot == S) { slot = 0; ph ^= 1u; }
              }
            }
                    if (HAS_Q) {
#pragma unroll
                        for (int k = 0; k < kRPT; k++) {
                            float s, e;
                            two_sum(qhi[k], qt[k], s, e);
                            qhi[k] = s; qlo[k] += e; qt[k] = 0.0f;
                        }
                    }
                    if (HAS_S) {
                        const float v = butterfly16(sl, lane);
                        if (lane < 16) {
                            const int64_t col = gbase + (int64_t)(lane / CPW) * kBoxC + CPW * warp + (lane % CPW);
                            if (col < c1) {
                                float s, e;
                                two_sum(shi[col - c0], v, s, e);
                                shi[col - c0] = s;
                                slo[col - c0] += e;
                            }
                        }
#pragma unroll
                        for (int k = 0; k < 16; k++) sl[k] = 0.0f;
                    }
            }
            if (HAS_Q) {
                // Add the eight warps' row sums (each warp saw other columns).
#pragma unroll
                for (int k = 0; k < kRPT; k++) {
                    qred[warp * kBoxR + trow<V>(lane, k)] = qhi[k];
                    qred[(kConsumerWarps + warp) * kBoxR + trow<V>(lane, k)] = qlo[k];
                }
                named_bar(1, kConsumers);
                const int64_t i = R0 + threadIdx.x;
                if (i < r1) {
                    // Compensated FP32: TwoSum over the warps' hi parts, lo parts added;
                    // the pair goes to the combine, which converts and adds in FP64.
                    float hs = qred[threadIdx.x], ls = qred[kConsumerWarps * kBoxR + threadIdx.x];
#pragma unroll
                    for (int w = 1; w < kConsumerWarps; w++) {
                        float s2, e2;
                        two_sum(hs, qred[w * kBoxR + threadIdx.x], s2, e2);
                        hs = s2;
                        ls += e2 + qred[(kConsumerWarps + w) * kBoxR + threadIdx.x];
                    }
                    reinterpret_cast<float2*>(a.qpart)[cb * a.ldq + i] = make_float2(hs, ls);
                }
                named_bar(1, kConsumers);
            }
        }
        named_bar(1, kConsumers);
        if (HAS_S)
            for (int k = threadIdx.x; k < ncols; k += kConsumers)
                reinterpret_cast<float2*>(a.spart)[rb * a.lds + c0 + k] = make_float2(shi[k], slo[k]);
        named_bar(1, kConsumers);
    }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
    static std::once_flag once;
    static EncodeFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

template <typename TA, int MODE, int BPS>
bto_status launch_t(const CUtensorMap& map, const LpArgs& a, int grid, cudaStream_t st) {
    auto k = lp_tma_kernel<TA, MODE, BPS>;
    const size_t smem = tma_smem<TA, BPS>(a.tcmax, lp_nvec(MODE));
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return BTO_ERR_CUDA;
    k<<<grid, kThreadsT, smem, st>>>(map, a);
    return launch_status();
}

}  // namespace

bool encode_tmap_2d(CUtensorMap* map, CUtensorMapDataType dtype, size_t esize, const void* base,
                    int64_t rows, int64_t cols, int64_t ld, uint32_t box_rows, uint32_t box_cols,
                    CUtensorMapSwizzle swizzle) {
    EncodeFn fn = encode_fn();
    if (!fn || rows <= 0 || cols <= 0) return false;
    if (!aligned16(base) || ((size_t)ld * esize) % 16 != 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * esize};
    const cuuint32_t box[2] = {box_rows, box_cols};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, dtype, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool lp_tma_ok(int a_type, const void* A, int64_t lda, int64_t m, int64_t n) {
    const size_t es = a_type == BTO_F32 ? 4 : 2;
    return m <= INT32_MAX && n <= INT32_MAX && aligned16(A) && ((size_t)lda * es) % 16 == 0;
}

PanelPlan lp_plan(int64_t m, int64_t n, int sms, int a_type, int bps, bool balanced) {
    PanelPlan pl;
    pl.bps = bps;
    pl.ldq = round_up(m > 0 ? m : 1, 32);
    pl.lds = round_up(n > 0 ? n : 1, 32);
    if (m <= 0 || n <= 0) return pl;
    const int64_t G = (int64_t)sms * bps, cu = lp_col_unit(a_type);
    const int64_t cunits = ceil_div(n, cu), runits = ceil_div(m, kBoxR);
    if (!balanced) {
        // The load-instruction kernel (operands the tensor memory accelerator
        // cannot copy): one panel per block, row blocks only to fill the
        // grid.  Its per-warp column partials live in shared memory for the
        // whole panel, so the wide panels below cost it occupancy (GEMVER
        // with an unaligned B measured 1.6 to 3.6 times slower with them).
        const int64_t NC = std::min<int64_t>(G, cunits);
        const int64_t NR = std::max<int64_t>(1, std::min<int64_t>(G / NC, runits));
        pl.NC = (int)NC;
        pl.NR = (int)NR;
        pl.TCmax = ceil_div(cunits, NC) * cu;
        pl.ntiles = NR * NC;
        pl.grid = (int)G;
        return pl;
    }
    // TMA-fed sweeps.  At most one tile per block: NR row blocks x NC column panels with
    // NR NC <= G.  The busiest block does (widest panel) x (tallest row
    // block) units of 256 rows x cu columns; column panels leave NC x m row
    // partials and row blocks NR x n column partials (FP32 pairs) that are
    // written and read again.  Take the split with the least of
    //   busiest block's units x (1 + partial bytes / matrix bytes)
    // among those whose panel vectors fit the block's shared memory (one
    // block per SM: 227 KB and GEMVER's five vectors; two: 113 KB each and
    // three).  With one row block the panels of 1024 BF16 units over 304
    // blocks were 3 or 4 units wide: a quarter of the blocks worked 19% longer
    // than the mean.
    const bool bf = a_type == BTO_BF16;
    auto fits = [&](int64_t tc) {
        const size_t smem = bf ? (bps == 2 ? tma_smem<__nv_bfloat16, 2>(tc, 3) : tma_smem<__nv_bfloat16, 1>(tc, 5))
                               : (bps == 2 ? tma_smem<float, 2>(tc, 3) : tma_smem<float, 1>(tc, 5));
        return smem <= (bps == 2 ? (size_t)115712 : (size_t)232448);
    };
    const double abytes = (double)m * (double)n * (bf ? 2.0 : 4.0);
    int64_t bestNR = 0, bestNC = 0;
    double best = 0.0;
    for (int64_t NR = 1; NR <= std::min<int64_t>(G, runits); NR++) {
        const int64_t NC = std::min<int64_t>(cunits, G / NR);
        if (NC < 1) break;
        const int64_t wu = ceil_div(cunits, NC), hc = ceil_div(runits, NR);
        if (!fits(wu * cu)) continue;
        const double pbytes = 2.0 * 8.0 * ((double)NC * (double)m + (double)NR * (double)n);
        const double cost = (double)(wu * hc) * (1.0 + pbytes / abytes);
        if (bestNR == 0 || cost < best) { best = cost; bestNR = NR; bestNC = NC; }
    }
    if (bestNR == 0) {          // no split fits (not reached for n >= 1): one row block
        bestNC = std::min<int64_t>(G, cunits);
        bestNR = std::max<int64_t>(1, std::min<int64_t>(G / bestNC, runits));
    }
    pl.NC = (int)bestNC;
    pl.NR = (int)bestNR;
    pl.TCmax = ceil_div(cunits, bestNC) * cu;
    pl.ntiles = bestNR * bestNC;
    pl.grid = (int)G;
    return pl;
}

bool lp_tma_launch(int a_type, int mode, const LpArgs& a, int grid, int bps, cudaStream_t st, bto_status* out) {
    const size_t es = a_type == BTO_F32 ? 4 : 2;
    const void* base = a.A;
    CUtensorMap map;
    const CUtensorMapDataType dt = a_type == BTO_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    // In place (B == A) the B stores of one stage must not overwrite elements
    // a later stage still has to copy: each element is copied once, before it
    // is stored, so this holds; the copies of a stage complete before its
    // consumers run.
    if (a.m > INT32_MAX || a.n > INT32_MAX) return false;
    // The B stores are 16-byte vector stores: B and its columns must be aligned.
    if (mode == LP_G1 && !(aligned16(a.Bout) && ((size_t)a.ldb * es) % 16 == 0)) return false;
    const uint32_t bc = a_type == BTO_F32 ? box_cols<float>() : box_cols<__nv_bfloat16>();
    if (!encode_tmap_2d(&map, dt, es, base, a.m, a.n, a.lda, kBoxR, bc)) return false;
    if (a_type == BTO_F32 && bps == 2 && mode == LP_QS) {
        *out = launch_t<float, LP_QS, 2>(map, a, grid, st);
        return true;
    } else if (a_type == BTO_F32) {
        switch (mode) {
            case LP_QS: *out = launch_t<float, LP_QS, 1>(map, a, grid, st); return true;
            case LP_Q: *out = launch_t<float, LP_Q, 1>(map, a, grid, st); return true;
            case LP_G1: *out = launch_t<float, LP_G1, 1>(map, a, grid, st); return true;
            case LP_S: *out = launch_t<float, LP_S, 1>(map, a, grid, st); return true;
        }
    } else if (bps == 2) {
        switch (mode) {   // GEMVER's first pass (LP_G1) is planned for one block per SM
            case LP_QS: *out = launch_t<__nv_bfloat16, LP_QS, 2>(map, a, grid, st); return true;
            case LP_Q: *out = launch_t<__nv_bfloat16, LP_Q, 2>(map, a, grid, st); return true;
            case LP_S: *out = launch_t<__nv_bfloat16, LP_S, 2>(map, a, grid, st); return true;
        }
    } else {
        switch (mode) {
            case LP_QS: *out = launch_t<__nv_bfloat16, LP_QS, 1>(map, a, grid, st); return true;
            case LP_Q: *out = launch_t<__nv_bfloat16, LP_Q, 1>(map, a, grid, st); return true;
            case LP_G1: *out = launch_t<__nv_bfloat16, LP_G1, 1>(map, a, grid, st); return true;
            case LP_S: *out = launch_t<__nv_bfloat16, LP_S, 1>(map, a, grid, st); return true;
        }
    }
    return false;
}

}  // namespace bto
