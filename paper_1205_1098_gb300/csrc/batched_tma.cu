// TMA path of the batched form: the instances whose matrices suit the tensor
// memory accelerator (16-byte aligned bases, leading dimensions a multiple of
// 16 bytes) run through the reduced-precision sweep, as work items that flow
// through one copy ring per SM.
//
//   - Host: one tensor map per matrix (in the workspace); each instance is cut
//     into tiles of at most 512 columns (whole TMA box widths) by at most 2048
//     rows (whole 256-row boxes); the tiles become items, sorted by
//     decreasing size and dealt to the blocks round-robin, so every block
//     knows its sequence without communication.
//   - Stage one (one persistent launch per storage type): a producer warp
//     issues cp.async.bulk.tensor copies of 256-row boxes of the items, in
//     order, into a 12-stage ring; eight consumer warps run the sweep's
//     arithmetic on them (BICGK's q and s, GEMVER's B and B^T y, ATAX's A x,
//     GESUMMV's A x and B x as two items) and leave per-tile (hi, lo) partials.
//     The ring runs across item boundaries: the next item's copies are in
//     flight while the consumers finish the current one.
//   - A combine launch adds each output's partials in FP64 in a fixed order
//     (q, s, GEMVER's x, ATAX's t, GESUMMV's y).
//   - Stage two (same kernel): GEMVER's w = alpha B x over the stored B and
//     ATAX's y = beta A^T t, then a second combine.
// Kernel boundaries order the stages, so no item waits for another.  Every
// mbarrier wait is bounded (about 2 s of %globaltimer) and sets the status
// word on expiry; the producer then drains its own copies (bounded).
#include "check.cuh"
#include "lp_math.cuh"
#include "tma.cuh"
#include <algorithm>
#include <queue>
#include <cstring>
#include <vector>

namespace bto {
namespace {

using namespace lp;

constexpr int kCW = 8;                          // consumer warps
constexpr int kConsumers = kCW * 32;
constexpr int kThreadsT = kConsumers + 32;      // + one producer warp
constexpr int kBoxR = 256;                      // rows per box
constexpr int kRPT = 8;                         // rows per lane
constexpr int kStagesT = 12;                    // ring stages (16 KB each)
constexpr int kMaxTw = 512;                     // widest tile (columns)
constexpr int kRowsPerTile = 2048;              // tallest tile (rows)
constexpr unsigned long long kWaitNs = 2000000000ull;
constexpr double kItemCost = 40000.0;           // an item's fixed work, in matrix elements
constexpr double kChunkCost = 2500.0;           // a 256-row chunk's reductions, in matrix elements

template <typename TA> struct Cfg {
    static constexpr int BoxC = sizeof(TA) == 2 ? 32 : 16;   // 16 KB boxes
    static constexpr int CPW = BoxC / kCW;                     // columns per consumer warp per stage
    static constexpr int GroupStages = 16 / CPW;               // stages per 16-column butterfly group
};

template <typename TA>
constexpr size_t stage_bytes() { return (size_t)kBoxR * Cfg<TA>::BoxC * sizeof(TA); }

template <typename TA>
constexpr size_t bt_smem() {
    return 1024 + kStagesT * stage_bytes<TA>() + 2 * kStagesT * sizeof(uint64_t) +
           2 * kCW * kBoxR * sizeof(float) + 8 * kMaxTw * sizeof(float);
}

}  // namespace

// Device records (written by the host into the workspace image).  BtInst
// takes the tensor maps' alignment; its region starts on 256 bytes.
struct BtInst {
    CUtensorMap mapA;          // A (m x n)
    CUtensorMap mapB;          // GEMVER: its B (read by stage two); GESUMMV: the second matrix
    const float* u1; const float* v1; const float* u2; const float* v2;   // GEMVER
    void* Bout;                // GEMVER's B (written by stage one)
    int64_t ldb;
};
static_assert(alignof(BtInst) >= 64 && sizeof(BtInst) % 64 == 0, "tensor maps need 64-byte alignment");

struct BtItem {
    const float* p;            // column-indexed vector (q modes)
    const float* r;            // row-indexed vector (s modes; GEMVER's first pass: y)
    float2* qdst;              // this tile's q partial, indexed by absolute row
    float2* sdst;              // this tile's s partial, indexed by absolute column
    int32_t inst, mode, matB, pad;
    int32_t r0, r1, c0, c1;
};

struct BtComb {
    float* out;
    const float2* P;           // K partials of len values, ld apart
    const float2* P2;          // K2 more (GESUMMV's B x), or NULL
    const float* v;            // added vector (GEMVER's z), or NULL
    int64_t len, ld;
    int32_t K, K2;
    double a1, a2, b;
};

struct BtChunk { int32_t job, start; };   // 256 consecutive outputs of one combine job

struct BtHeader {
    int32_t ninst, pad;
    uint32_t bar_count, bar_gen;   // the one-launch form's grid barrier (zero when uploaded)
    int32_t nitems[2][2];      // [stage][FP32, BF16]
    int32_t ncomb[2];
    int32_t nchunk[2];
    int64_t off_inst;
    int64_t off_items[2][2];
    int64_t off_comb[2];
    int64_t off_chunk[2];
};

namespace {

// The workspace's second 8 bytes hold the offset of the BtHeader (0: no TMA path).
__device__ __forceinline__ const BtHeader* bt_header(const char* ws) {
    const int64_t off = *reinterpret_cast<const int64_t*>(ws + 8);
    return off ? reinterpret_cast<const BtHeader*>(ws + off) : nullptr;
}

template <int V>
__device__ __forceinline__ int trow(int lane, int k) { return (k / V) * (32 * V) + lane * V + (k % V); }

__device__ __forceinline__ float dot8(const float (&a)[kRPT], const float (&r)[kRPT]) {
    float2 acc = __fmul2_rn(make_float2(a[0], a[1]), make_float2(r[0], r[1]));
#pragma unroll
    for (int k = 2; k < kRPT; k += 2) acc = __ffma2_rn(make_float2(a[k], a[k + 1]), make_float2(r[k], r[k + 1]), acc);
    return acc.x + acc.y;
}

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

struct Smem {
    unsigned char* ring;
    uint64_t* full;
    uint64_t* empty;
    float* qred;               // [2][8][256]
    float* shi; float* slo;    // [kMaxTw]
    float* sp; float* sv1; float* sv2;   // the current item's column vectors (one of two buffers)
};

__device__ __forceinline__ void cp4(float* dst, const float* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// Issues (cp.async, 4 bytes each) the copies of an item's column vectors into
// the buffer at vb ([3][kMaxTw]: p, v1, v2) and commits them as one group.
__device__ __forceinline__ void fetch_vectors(const BtItem& it, const BtInst& in, float* vb) {
    const int ncols = it.c1 - it.c0;
    const bool q = it.mode == LP_QS || it.mode == LP_Q, g1 = it.mode == LP_G1;
    for (int k = threadIdx.x; k < ncols; k += kConsumers) {
        if (q) cp4(vb + k, it.p + it.c0 + k);
        if (g1) { cp4(vb + kMaxTw + k, in.v1 + it.c0 + k); cp4(vb + 2 * kMaxTw + k, in.v2 + it.c0 + k); }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// One item on the consumer warps: the tile's stages in ring order, the
// arithmetic of the reduced-precision sweep, and the tile's partials.
template <typename TA, int MODE>
__device__ __forceinline__ void consume(const BtItem& it, const BtInst& in, const Smem& sm, int& slot, uint32_t& ph,
                                        volatile int* abortp, int* status) {
    constexpr int V = 16 / sizeof(TA);
    constexpr int S = kStagesT;
    constexpr int kBoxC = Cfg<TA>::BoxC;
    constexpr int CPW = Cfg<TA>::CPW;
    constexpr bool HAS_Q = (MODE == LP_QS || MODE == LP_Q);
    constexpr bool HAS_S = (MODE == LP_QS || MODE == LP_G1 || MODE == LP_S);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t c0 = it.c0, c1 = it.c1, r0 = it.r0, r1 = it.r1;
    const int ncols = (int)(c1 - c0);
    TA* ring = reinterpret_cast<TA*>(sm.ring);
    // The column vectors were copied during the previous item (fetch_vectors);
    // the barrier makes every thread's copies visible.
    for (int k = threadIdx.x; k < ncols; k += kConsumers) { sm.shi[k] = 0.0f; sm.slo[k] = 0.0f; }
    named_bar(1, kConsumers);
    TA* Bout = static_cast<TA*>(in.Bout);
    for (int64_t R0 = r0; R0 < r1; R0 += kBoxR) {
        float rv[kRPT], u1r[kRPT], u2r[kRPT], qhi[kRPT], qlo[kRPT], qt[kRPT], sl[16];
#pragma unroll
        for (int k = 0; k < kRPT; k++) {
            const int64_t i = R0 + trow<V>(lane, k);
            rv[k] = (HAS_S && i < r1) ? __ldg(it.r + i) : 0.0f;
            u1r[k] = (MODE == LP_G1 && i < r1) ? __ldg(in.u1 + i) : 0.0f;
            u2r[k] = (MODE == LP_G1 && i < r1) ? __ldg(in.u2 + i) : 0.0f;
            qhi[k] = 0.0f; qlo[k] = 0.0f; qt[k] = 0.0f;
        }
#pragma unroll
        for (int k = 0; k < 16; k++) sl[k] = 0.0f;
        constexpr int GS = Cfg<TA>::GroupStages;
        for (int64_t gbase = c0; gbase < c1; gbase += (int64_t)GS * kBoxC) {
#pragma unroll
            for (int gs = 0; gs < GS; gs++) {
                const int64_t cs = gbase + (int64_t)gs * kBoxC;
                if (cs < c1) {
                    // A stage that completed holds valid data even after an abort; once
                    // the producer has stopped, the wait sees the flag on its first spin.
                    const bool have = mbar_wait_bounded(&sm.full[slot], ph, kWaitNs, abortp);
                    if (!have) {
                        if (lane == 0) atomicExch(status, (int)BTO_ERR_TIMEOUT);
                        *abortp = 1;
                    }
                    const TA* buf = ring + (size_t)slot * kBoxR * kBoxC;
                    const int lc0 = (int)(cs - c0);
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
                                const float v1j = sm.sv1[lc], v2j = sm.sv2[lc];
                                TA bq[kRPT];
                                float bf[kRPT];
                                unsigned bw[kRPT / 2];     // BF16: the rounded pairs as stored
#pragma unroll
                                for (int k = 0; k < kRPT; k += 2) {
                                    const float2 t = __ffma2_rn(make_float2(u2r[k], u2r[k + 1]), make_float2(v2j, v2j),
                                                                __ffma2_rn(make_float2(u1r[k], u1r[k + 1]),
                                                                           make_float2(v1j, v1j),
                                                                           make_float2(av[k], av[k + 1])));
                                    if constexpr (sizeof(TA) == 2) {
                                        // One conversion rounds both rows (nearest even).
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
                                TA* bcol = Bout + col * in.ldb;
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
                                                    bcol[i + q] = __ushort_as_bfloat16(
                                                        (unsigned short)(((h * V + q) & 1) ? (w >> 16) : (w & 0xFFFFu)));
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
                                    const float pj = sm.sp[lc];
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
                    if (lane == 0 && have) mbar_arrive(&sm.empty[slot]);
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
                        two_sum(sm.shi[col - c0], v, s, e);
                        sm.shi[col - c0] = s;
                        sm.slo[col - c0] += e;
                    }
                }
#pragma unroll
                for (int k = 0; k < 16; k++) sl[k] = 0.0f;
            }
        }
        if (HAS_Q) {
#pragma unroll
            for (int k = 0; k < kRPT; k++) {
                sm.qred[warp * kBoxR + trow<V>(lane, k)] = qhi[k];
                sm.qred[(kCW + warp) * kBoxR + trow<V>(lane, k)] = qlo[k];
            }
            named_bar(1, kConsumers);
            const int64_t i = R0 + threadIdx.x;
            if (i < r1) {
                float hs = sm.qred[threadIdx.x], ls = sm.qred[kCW * kBoxR + threadIdx.x];
#pragma unroll
                for (int w = 1; w < kCW; w++) {
                    float s2, e2;
                    two_sum(hs, sm.qred[w * kBoxR + threadIdx.x], s2, e2);
                    hs = s2;
                    ls += e2 + sm.qred[(kCW + w) * kBoxR + threadIdx.x];
                }
                it.qdst[i] = make_float2(hs, ls);
            }
            named_bar(1, kConsumers);
        }
    }
    named_bar(1, kConsumers);
    if (HAS_S)
        for (int k = threadIdx.x; k < ncols; k += kConsumers) it.sdst[c0 + k] = make_float2(sm.shi[k], sm.slo[k]);
    named_bar(1, kConsumers);
}

// Shared memory of the sweep (bt_smem<TA>() bytes), carved once per block.
template <typename TA>
__device__ __forceinline__ Smem carve(unsigned char* smraw) {
    Smem sm;
    sm.ring = reinterpret_cast<unsigned char*>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    sm.full = reinterpret_cast<uint64_t*>(sm.ring + kStagesT * stage_bytes<TA>());
    sm.empty = sm.full + kStagesT;
    sm.qred = reinterpret_cast<float*>(sm.empty + kStagesT);
    sm.shi = sm.qred + 2 * kCW * kBoxR;
    sm.slo = sm.shi + kMaxTw;
    return sm;
}

// One stage's sweep over this block's items of storage type TA: the producer
// warp copies their boxes through the ring, the consumer warps run them.  The
// ring's position (g for the producer, slot and ph for the consumers) carries
// over from one call to the next.
template <typename TA>
__device__ __forceinline__ void sweep_stage(char* ws, const BtHeader* bh, int stage, const Smem& sm0,
                                            volatile int* abortp, long long& g, int& slot, uint32_t& ph) {
    constexpr int T = sizeof(TA) == 2 ? 1 : 0;
    const int nitems = bh->nitems[stage][T];
    if ((int)blockIdx.x >= nitems) return;
    const BtItem* items = reinterpret_cast<const BtItem*>(ws + bh->off_items[stage][T]);
    const BtInst* insts = reinterpret_cast<const BtInst*>(ws + bh->off_inst);
    int* status = reinterpret_cast<int*>(ws);
    constexpr int S = kStagesT;
    constexpr int kBoxC = Cfg<TA>::BoxC;
    Smem sm = sm0;
    float* vbuf = sm.slo + kMaxTw;      // [2][3][kMaxTw]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == kCW) {
        // ---------------- producer: every box of this block's items, in order
        if (lane == 0) {
            TA* ring = reinterpret_cast<TA*>(sm.ring);
            const long long g0 = g;
            for (int t = blockIdx.x; t < nitems && !*abortp; t += gridDim.x) {
                const BtItem it = items[t];
                const CUtensorMap* map = it.matB ? &insts[it.inst].mapB : &insts[it.inst].mapA;
                for (int R0 = it.r0; R0 < it.r1 && !*abortp; R0 += kBoxR) {
                    for (int cs = it.c0; cs < it.c1; cs += kBoxC, g++) {
                        const int slot_ = (int)(g % S);
                        if (g >= S && !mbar_wait_bounded(&sm.empty[slot_], (uint32_t)(((g / S) - 1) & 1), kWaitNs, abortp)) {
                            atomicExch(status, (int)BTO_ERR_TIMEOUT);
                            *abortp = 1;
                            break;
                        }
                        mbar_arrive_expect_tx(&sm.full[slot_], (uint32_t)stage_bytes<TA>());
                        tma_load_2d(ring + (size_t)slot_ * kBoxR * kBoxC, map, R0, cs, &sm.full[slot_]);
                    }
                }
            }
            if (*abortp) {
                // Wait (bounded) for the copies this thread issued before leaving.
                const long long first = g - S > g0 ? g - S : g0;
                for (long long h = first; h < g; h++) {
                    const int slot_ = (int)(h % S);
                    mbar_wait_timed(&sm.full[slot_], (uint32_t)((h / S) & 1), kWaitNs);
                }
            }
        }
        return;
    }

    // ---------------- consumers
    // Column vectors go through two buffers: the next item's are copied
    // (cp.async) while this item runs.
    int buf = 0;
    {
        const BtItem first = items[blockIdx.x];
        fetch_vectors(first, insts[first.inst], vbuf);
    }
    for (int t = blockIdx.x; t < nitems; t += gridDim.x, buf ^= 1) {
        const BtItem it = items[t];
        const BtInst& in = insts[it.inst];
        const int tn = t + gridDim.x;
        float* nb = vbuf + (buf ^ 1) * 3 * kMaxTw;
        if (tn < nitems) {
            const BtItem nx = items[tn];
            fetch_vectors(nx, insts[nx.inst], nb);
        } else {
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        asm volatile("cp.async.wait_group 1;" ::: "memory");   // this item's copies are in
        if (it.mode < 0) continue;                               // a slot the plan left empty
        sm.sp = vbuf + buf * 3 * kMaxTw;
        sm.sv1 = sm.sp + kMaxTw;
        sm.sv2 = sm.sv1 + kMaxTw;
        switch (it.mode) {
            case LP_QS: consume<TA, LP_QS>(it, in, sm, slot, ph, abortp, status); break;
            case LP_Q: consume<TA, LP_Q>(it, in, sm, slot, ph, abortp, status); break;
            case LP_G1: consume<TA, LP_G1>(it, in, sm, slot, ph, abortp, status); break;
            default: consume<TA, LP_S>(it, in, sm, slot, ph, abortp, status); break;
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

template <typename TA>
__device__ __forceinline__ void init_ring(const Smem& sm, volatile int* abortp) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStagesT; s++) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], kCW);
        }
        *abortp = 0;
        fence_mbar_init();
    }
    __syncthreads();
}

template <typename TA>
__global__ void __launch_bounds__(kThreadsT, 1) bt_sweep(char* ws, int stage) {
    const BtHeader* bh = bt_header(ws);
    if (!bh) return;
    constexpr int T = sizeof(TA) == 2 ? 1 : 0;
    if ((int)blockIdx.x >= bh->nitems[stage][T]) return;
    extern __shared__ unsigned char smraw[];
    const Smem sm = carve<TA>(smraw);
    __shared__ int s_abort_;
    volatile int* abortp = &s_abort_;
    init_ring<TA>(sm, abortp);
    long long g = 0;
    int slot = 0;
    uint32_t ph = 0;
    sweep_stage<TA>(ws, bh, stage, sm, abortp, g, slot, ph);
}

// out[i] = a1 sum_k P[k][i] + a2 sum_k P2[k][i] + b v[i], each partial a
// (hi, lo) pair converted to FP64, partials added in k order, one rounding.
// A block takes one chunk of 256 outputs of one job (a flat list built by the
// host), one output per thread, and loads an output's partials four at a
// time before adding them, so the loads overlap instead of forming a chain
// of round trips.
__device__ __forceinline__ double sum_partials(const float2* P, int64_t ld, int K, int64_t i) {
    double s = 0.0;
    int k = 0;
    for (; k + 4 <= K; k += 4) {
        float2 h[4];
#pragma unroll
        for (int u = 0; u < 4; u++) h[u] = __ldcg(P + (int64_t)(k + u) * ld + i);
#pragma unroll
        for (int u = 0; u < 4; u++) s += (double)h[u].x + (double)h[u].y;
    }
    for (; k < K; k++) {
        const float2 h = __ldcg(P + (int64_t)k * ld + i);
        s += (double)h.x + (double)h.y;
    }
    return s;
}

// One stage's combine, chunks dealt over the grid, one output per thread of
// the block's first 256 threads (out[i] = a1 sum_k P[k][i] + a2 sum_k P2[k][i]
// + b v[i], as described above).
__device__ __forceinline__ void combine_stage(const char* ws, const BtHeader* bh, int stage) {
    if (threadIdx.x >= 256) return;
    const int nch = bh->nchunk[stage];
    const BtComb* jobs = reinterpret_cast<const BtComb*>(ws + bh->off_comb[stage]);
    const BtChunk* chunks = reinterpret_cast<const BtChunk*>(ws + bh->off_chunk[stage]);
    for (int ci = blockIdx.x; ci < nch; ci += gridDim.x) {
        const BtChunk ch = chunks[ci];
        const BtComb& c = jobs[ch.job];
        const int64_t i = (int64_t)ch.start + threadIdx.x;
        if (i < c.len) {
            const double s = sum_partials(c.P, c.ld, c.K, i);
            double o = c.a1 * s;
            if (c.K2 > 0) o = fma(c.a2, sum_partials(c.P2, c.ld, c.K2, i), o);
            if (c.v) o = fma(c.b, (double)__ldcg(c.v + i), o);
            c.out[i] = (float)o;
        }
    }
}

__global__ void __launch_bounds__(256) bt_combine(const char* ws, int stage) {
    const BtHeader* bh = bt_header(ws);
    if (!bh) return;
    combine_stage(ws, bh, stage);
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barrier of the one-launch form, bounded (about two seconds of
// %globaltimer, then BTO_ERR_TIMEOUT in the status word and false).  It resets
// itself: a block reads the generation before it arrives; the last of the
// grid to arrive zeroes the count and then advances the generation, which
// releases the others.  Nothing has to be cleared between runs.
__device__ __forceinline__ bool grid_sync(BtHeader* bh, int* status, int stall_block, unsigned long long limit_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned gen0 = ld_acquire_gpu(&bh->bar_gen);
        __threadfence();
        // (stall_block: fault injection for tests, a block that never arrives.)
        const unsigned arrived = (int)blockIdx.x == stall_block ? 0u : atomicAdd(&bh->bar_count, 1u);
        if ((int)blockIdx.x != stall_block && arrived == gridDim.x - 1) {
            *reinterpret_cast<volatile unsigned*>(&bh->bar_count) = 0u;
            __threadfence();
            st_release_gpu(&bh->bar_gen, gen0 + 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (ld_acquire_gpu(&bh->bar_gen) == gen0) {
                if (global_ns() - t0 > limit_ns) {
                    atomicExch(status, (int)BTO_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// The whole batch in one cooperative launch, when every instance takes the
// TMA path with storage type TA: stage one's sweep, a grid barrier, its
// combine, a barrier, stage two's sweep, a barrier, its combine.  The copy
// ring runs on across the stages.  The status word is cleared by block 0 at
// the start (a timeout needs seconds of waiting, so no block can have set it).
template <typename TA>
__global__ void __launch_bounds__(kThreadsT, 1) bt_fused(char* ws, int stall_block, unsigned long long limit_ns) {
    BtHeader* bh = const_cast<BtHeader*>(bt_header(ws));
    if (!bh) return;
    int* status = reinterpret_cast<int*>(ws);
    if (blockIdx.x == 0 && threadIdx.x == 0) *status = BTO_OK;
    extern __shared__ unsigned char smraw[];
    const Smem sm = carve<TA>(smraw);
    __shared__ int s_abort_;
    volatile int* abortp = &s_abort_;
    init_ring<TA>(sm, abortp);
    long long g = 0;
    int slot = 0;
    uint32_t ph = 0;
#pragma unroll 1
    for (int stage = 0; stage < 2; stage++) {
        sweep_stage<TA>(ws, bh, stage, sm, abortp, g, slot, ph);
        if (!grid_sync(bh, status, stall_block, limit_ns)) return;
        combine_stage(ws, bh, stage);
        if (stage == 0 && !grid_sync(bh, status, stall_block, limit_ns)) return;
    }
}

}  // namespace

// ------------------------------------------------------------------ host plan

struct BtPlan {
    int tile_cols = 0;
    std::vector<BtInst> inst;
    // Records with workspace offsets in place of pointers into the workspace
    // (qdst, sdst, P, P2, and ATAX's t as p or r or out); resolved when written.
    struct ItemRec { BtItem it; int64_t q_off, s_off, t_off; double cost; int type, stage; };
    struct CombRec { BtComb c; int64_t p_off, p2_off, t_out_off; int stage; };
    std::vector<ItemRec> items;
    std::vector<CombRec> combs;
    int64_t q_elems = 0, s_elems = 0, t_elems = 0;   // float2, float2, float
    // Layout (set by bt_plan_layout).
    int64_t off_hdr = 0, off_inst = 0, off_items[2][2] = {{0, 0}, {0, 0}}, off_comb[2] = {0, 0}, off_chunk[2] = {0, 0};
    std::vector<BtChunk> chunks[2];
    int64_t off_q = 0, off_s = 0, off_t = 0;
    int32_t nitems[2][2] = {{0, 0}, {0, 0}}, ncomb[2] = {0, 0}, nchunk[2] = {0, 0};
};

BtPlan* bt_plan_create() { return new BtPlan(); }
void bt_plan_destroy(BtPlan* p) { delete p; }

void bt_plan_reset(BtPlan* P, int tile_cols) {
    P->tile_cols = tile_cols;
    P->inst.clear();
    P->items.clear();
    P->combs.clear();
    P->q_elems = P->s_elems = P->t_elems = 0;
}

bool bt_plan_empty(const BtPlan* P) { return P->inst.empty(); }

bool bt_plan_add(BtPlan* P, const bto_batch_desc& d) {
    const int op = d.op;
    if (op != BTO_OP_BICGK && op != BTO_OP_GEMVER && op != BTO_OP_ATAX && op != BTO_OP_GESUMMV) return false;
    if (d.a_type != BTO_F32 && d.a_type != BTO_BF16) return false;
    if (d.m <= 0 || d.n <= 0 || d.m > INT32_MAX || d.n > INT32_MAX) return false;
    const size_t es = d.a_type == BTO_BF16 ? 2 : 4;
    const bool twomat = op == BTO_OP_GEMVER || op == BTO_OP_GESUMMV;
    if (!aligned16(d.A) || ((size_t)d.lda * es) % 16 != 0) return false;
    if (twomat && (!aligned16(d.B) || ((size_t)d.ldb * es) % 16 != 0)) return false;
    const int type = d.a_type == BTO_BF16 ? 1 : 0;
    const CUtensorMapDataType dt = type ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const int64_t cu = type ? 32 : 16;   // box width
    BtInst ti;
    std::memset(&ti, 0, sizeof(ti));
    if (!encode_tmap_2d(&ti.mapA, dt, es, d.A, d.m, d.n, d.lda, kBoxR, (uint32_t)cu)) return false;
    if (twomat && !encode_tmap_2d(&ti.mapB, dt, es, d.B, d.m, d.n, d.ldb, kBoxR, (uint32_t)cu)) return false;
    if (op == BTO_OP_GEMVER) {
        ti.u1 = d.in[0]; ti.v1 = d.in[1]; ti.u2 = d.in[2]; ti.v2 = d.in[3];
        ti.Bout = d.B; ti.ldb = d.ldb;
    }
    const int32_t idx = (int32_t)P->inst.size();
    P->inst.push_back(ti);

    const int64_t m = d.m, n = d.n;
    const int64_t tw = std::max<int64_t>(cu, std::min<int64_t>(kMaxTw, P->tile_cols) / cu * cu);
    const int64_t NC = ceil_div(n, tw), NR = ceil_div(m, kRowsPerTile);
    const int64_t nq = (op == BTO_OP_GESUMMV ? 2 : 1) * NC;
    const int64_t q_off = P->q_elems, s_off = P->s_elems, t_off = P->t_elems;
    P->q_elems += nq * m;                                         // q partials (GEMVER: stage two's w)
    if (op == BTO_OP_BICGK || op == BTO_OP_GEMVER || op == BTO_OP_ATAX) P->s_elems += NR * n;
    if (op == BTO_OP_ATAX) P->t_elems += round_up(m, 64);

    auto item = [&](int stage, int mode, int matB, int64_t rb, int64_t cb, int64_t qrow, const float* p,
                    const float* r, bool p_is_t, bool r_is_t, double w) {
        BtPlan::ItemRec rec{};
        rec.it.inst = idx; rec.it.mode = mode; rec.it.matB = matB;
        rec.it.r0 = (int32_t)lp_row_at(m, NR, rb); rec.it.r1 = (int32_t)lp_row_at(m, NR, rb + 1);
        rec.it.c0 = (int32_t)lp_col_at(n, NC, cb, cu); rec.it.c1 = (int32_t)lp_col_at(n, NC, cb + 1, cu);
        rec.it.p = p; rec.it.r = r;
        rec.q_off = qrow >= 0 ? q_off + qrow * m : -1;
        rec.s_off = (mode == LP_QS || mode == LP_G1 || mode == LP_S) ? s_off + rb * n : -1;
        rec.t_off = (p_is_t || r_is_t) ? t_off : -1;
        if (p_is_t) rec.it.p = nullptr;
        if (r_is_t) rec.it.r = nullptr;
        // Elements streamed (weighted: GEMVER's first pass also writes B), plus
        // each item's fixed work (its vectors, partial writes) and each
        // 256-row chunk's reductions, in the same units.
        rec.cost = w * (double)(rec.it.r1 - rec.it.r0) * (double)(rec.it.c1 - rec.it.c0) + kItemCost +
                   kChunkCost * (double)ceil_div(rec.it.r1 - rec.it.r0, kBoxR);
        rec.type = type;
        rec.stage = stage;
        if (rec.it.r1 > rec.it.r0 && rec.it.c1 > rec.it.c0) P->items.push_back(rec);
    };
    for (int64_t rb = 0; rb < NR; rb++)
        for (int64_t cb = 0; cb < NC; cb++) {
            switch (op) {
                case BTO_OP_BICGK: item(0, LP_QS, 0, rb, cb, cb, d.in[0], d.in[1], false, false, 1.0); break;
                case BTO_OP_GEMVER:
                    item(0, LP_G1, 0, rb, cb, -1, nullptr, d.in[4], false, false, 2.0);
                    item(1, LP_Q, 1, rb, cb, cb, d.out[0], nullptr, false, false, 1.0);
                    break;
                case BTO_OP_ATAX:
                    item(0, LP_Q, 0, rb, cb, cb, d.in[0], nullptr, false, false, 1.0);
                    item(1, LP_S, 0, rb, cb, -1, nullptr, nullptr, false, true, 1.0);
                    break;
                default:
                    item(0, LP_Q, 0, rb, cb, cb, d.in[0], nullptr, false, false, 1.0);
                    item(0, LP_Q, 1, rb, cb, NC + cb, d.in[0], nullptr, false, false, 1.0);
                    break;
            }
        }
    auto comb = [&](int stage, float* out, int64_t len, int64_t p_off, int64_t ld, int K, double a1,
                    int64_t p2_off, int K2, double a2, const float* v, double b, bool out_is_t) {
        BtPlan::CombRec rec{};
        rec.c.out = out; rec.c.len = len; rec.c.ld = ld; rec.c.K = K; rec.c.K2 = K2;
        rec.c.a1 = a1; rec.c.a2 = a2; rec.c.v = v; rec.c.b = b;
        rec.p_off = p_off; rec.p2_off = p2_off; rec.t_out_off = out_is_t ? t_off : -1;
        rec.stage = stage;
        P->combs.push_back(rec);
    };
    switch (op) {
        case BTO_OP_BICGK:
            comb(0, d.out[0], m, q_off, m, (int)NC, 1.0, -1, 0, 0.0, nullptr, 0.0, false);            // q
            comb(0, d.out[1], n, -s_off - 1, n, (int)NR, 1.0, -1, 0, 0.0, nullptr, 0.0, false);       // s
            break;
        case BTO_OP_GEMVER:
            comb(0, d.out[0], n, -s_off - 1, n, (int)NR, (double)d.beta, -1, 0, 0.0, d.in[5], 1.0, false);   // x
            comb(1, d.out[1], m, q_off, m, (int)NC, (double)d.alpha, -1, 0, 0.0, nullptr, 0.0, false);      // w
            break;
        case BTO_OP_ATAX:
            comb(0, nullptr, m, q_off, m, (int)NC, 1.0, -1, 0, 0.0, nullptr, 0.0, true);              // t
            comb(1, d.out[0], n, -s_off - 1, n, (int)NR, (double)d.beta, -1, 0, 0.0, nullptr, 0.0, false);  // y
            break;
        default:
            comb(0, d.out[0], m, q_off, m, (int)NC, (double)d.alpha, q_off + NC * m, (int)NC, (double)d.beta,
                 nullptr, 0.0, false);                                                                   // y
            break;
    }
    return true;
}

// Assigns the regions of the plan's records (part of the uploaded image) from
// `cur` on and returns the new end; sorts the items (stage, storage type,
// decreasing size), orders each group for a grid of G blocks and counts them.
// Longest-processing-time assignment (Graham): items 0..count-1, in
// decreasing cost, each to the least loaded of G blocks, ties to the lower
// block; lists[b] receives block b's items in order.
static void lpt_assign(const double* cost, size_t count, int G, std::vector<std::vector<size_t>>& lists) {
    lists.assign((size_t)G, {});
    using Load = std::pair<double, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> least;
    for (int b = 0; b < G; b++) least.push(Load(0.0, b));
    for (size_t k = 0; k < count; k++) {
        const Load l = least.top();
        least.pop();
        lists[(size_t)l.second].push_back(k);
        least.push(Load(l.first + cost[k], l.second));
    }
}

void lpt_blocks(const double* cost, int64_t count, int G, int32_t* block) {
    std::vector<std::vector<size_t>> lists;
    lpt_assign(cost, (size_t)count, G, lists);
    for (int b = 0; b < G; b++)
        for (size_t k : lists[(size_t)b]) block[k] = b;
}

int64_t bt_plan_layout_records(BtPlan* P, int64_t cur, int G) {
    auto region = [&](int64_t bytes) { const int64_t at = cur; cur += round_up(std::max<int64_t>(bytes, 1), 256); return at; };
    // Items sorted by stage, storage type, then decreasing cost (ties: order of addition).
    std::stable_sort(P->items.begin(), P->items.end(), [](const BtPlan::ItemRec& a, const BtPlan::ItemRec& b) {
        if (a.stage != b.stage) return a.stage < b.stage;
        if (a.type != b.type) return a.type < b.type;
        return a.cost > b.cost;
    });
    // Block b of the sweep takes slots b, b + G, b + 2G, ... of its group.  A
    // group of more than G items is assigned longest-processing-time first
    // (each item, in decreasing cost, to the least loaded block; ties to the
    // lower block) and laid out so that the walk gives every block its list;
    // slots past the end of a shorter list hold a no-op item (mode -1).
    if (G > 0) {
        std::vector<BtPlan::ItemRec> out;
        out.reserve(P->items.size());
        size_t i = 0;
        while (i < P->items.size()) {
            size_t j = i;
            while (j < P->items.size() && P->items[j].stage == P->items[i].stage && P->items[j].type == P->items[i].type) j++;
            if ((int64_t)(j - i) <= G) {
                out.insert(out.end(), P->items.begin() + i, P->items.begin() + j);
            } else {
                std::vector<double> cost(j - i);
                for (size_t k = i; k < j; k++) cost[k - i] = P->items[k].cost;
                std::vector<std::vector<size_t>> lists;
                lpt_assign(cost.data(), cost.size(), G, lists);
                size_t K = 0;
                for (const auto& l : lists) K = std::max(K, l.size());
                BtPlan::ItemRec pad{};
                pad.it.mode = -1;
                pad.q_off = pad.s_off = pad.t_off = -1;
                pad.stage = P->items[i].stage;
                pad.type = P->items[i].type;
                for (size_t k = 0; k < K; k++)
                    for (int b = 0; b < G; b++) out.push_back(k < lists[b].size() ? P->items[i + lists[b][k]] : pad);
            }
            i = j;
        }
        P->items.swap(out);
    }
    for (int s = 0; s < 2; s++) {
        for (int t = 0; t < 2; t++) P->nitems[s][t] = 0;
        P->ncomb[s] = 0;
    }
    for (const auto& r : P->items) P->nitems[r.stage][r.type]++;
    std::stable_sort(P->combs.begin(), P->combs.end(),
                     [](const BtPlan::CombRec& a, const BtPlan::CombRec& b) { return a.stage < b.stage; });
    for (int s = 0; s < 2; s++) P->chunks[s].clear();
    for (const auto& c : P->combs) {
        const int32_t j = P->ncomb[c.stage]++;
        for (int64_t st = 0; st < c.c.len; st += 256) P->chunks[c.stage].push_back(BtChunk{j, (int32_t)st});
    }
    for (int s = 0; s < 2; s++) P->nchunk[s] = (int32_t)P->chunks[s].size();
    P->off_hdr = region(sizeof(BtHeader));
    P->off_inst = region((int64_t)(P->inst.size() * sizeof(BtInst)));
    for (int s = 0; s < 2; s++)
        for (int t = 0; t < 2; t++) P->off_items[s][t] = region((int64_t)P->nitems[s][t] * (int64_t)sizeof(BtItem));
    for (int s = 0; s < 2; s++) P->off_comb[s] = region((int64_t)P->ncomb[s] * (int64_t)sizeof(BtComb));
    for (int s = 0; s < 2; s++) P->off_chunk[s] = region((int64_t)P->nchunk[s] * (int64_t)sizeof(BtChunk));
    return cur;
}

// Assigns the device-only partial arrays (q, s, ATAX's t) from `cur` on.
int64_t bt_plan_layout_partials(BtPlan* P, int64_t cur) {
    auto region = [&](int64_t bytes) { const int64_t at = cur; cur += round_up(std::max<int64_t>(bytes, 1), 256); return at; };
    P->off_q = region(P->q_elems * (int64_t)sizeof(float2));
    P->off_s = region(P->s_elems * (int64_t)sizeof(float2));
    P->off_t = region(P->t_elems * (int64_t)sizeof(float));
    return cur;
}

// Writes the plan's records into the host image of a workspace whose device
// address is `ws` (pointers into the workspace are resolved against it), and
// the BtHeader's offset into the image's bytes 8..15.
void bt_plan_write(const BtPlan* P, char* img, char* ws) {
    if (P->inst.empty()) return;   // bytes 8..15 stay 0: no TMA path
    *reinterpret_cast<int64_t*>(img + 8) = P->off_hdr;
    BtHeader h{};
    h.ninst = (int32_t)P->inst.size();
    h.off_inst = P->off_inst;
    for (int s = 0; s < 2; s++) {
        for (int t = 0; t < 2; t++) { h.nitems[s][t] = P->nitems[s][t]; h.off_items[s][t] = P->off_items[s][t]; }
        h.ncomb[s] = P->ncomb[s];
        h.off_comb[s] = P->off_comb[s];
        h.nchunk[s] = P->nchunk[s];
        h.off_chunk[s] = P->off_chunk[s];
        if (!P->chunks[s].empty())
            std::memcpy(img + P->off_chunk[s], P->chunks[s].data(), P->chunks[s].size() * sizeof(BtChunk));
    }
    std::memcpy(img + P->off_hdr, &h, sizeof(h));
    if (!P->inst.empty()) std::memcpy(img + P->off_inst, P->inst.data(), P->inst.size() * sizeof(BtInst));
    float2* q = reinterpret_cast<float2*>(ws + P->off_q);
    float2* s = reinterpret_cast<float2*>(ws + P->off_s);
    float* t = reinterpret_cast<float*>(ws + P->off_t);
    int64_t pos[2][2] = {{0, 0}, {0, 0}};
    for (const auto& r : P->items) {
        BtItem it = r.it;
        if (r.q_off >= 0) it.qdst = q + r.q_off;
        if (r.s_off >= 0) it.sdst = s + r.s_off;
        if (r.t_off >= 0) {
            if (it.mode == LP_S) it.r = t + r.t_off;
            else it.p = t + r.t_off;
        }
        std::memcpy(img + P->off_items[r.stage][r.type] + pos[r.stage][r.type]++ * sizeof(BtItem), &it, sizeof(it));
    }
    int64_t cpos[2] = {0, 0};
    for (const auto& r : P->combs) {
        BtComb c = r.c;
        // p_off >= 0: a q offset; p_off < 0: an s offset (encoded as -off - 1).
        c.P = r.p_off >= 0 ? q + r.p_off : s + (-r.p_off - 1);
        c.P2 = r.p2_off >= 0 ? q + r.p2_off : nullptr;
        if (r.t_out_off >= 0) c.out = t + r.t_out_off;
        std::memcpy(img + P->off_comb[r.stage] + cpos[r.stage]++ * sizeof(BtComb), &c, sizeof(c));
    }
}

namespace {

template <typename TA>
bool bt_setup() {
    static int done = 0;
    if (!done) {
        if (cudaFuncSetAttribute(bt_sweep<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt_smem<TA>()) !=
                cudaSuccess ||
            cudaFuncSetAttribute(bt_fused<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt_smem<TA>()) !=
                cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        done = 1;
    }
    return true;
}

}  // namespace

// The one-launch form applies when every item has storage type 0 (FP32) or
// every item type 1 (BF16): returns that type, or -1.
int bt_fused_type(const BtPlan* P) {
    const bool f32 = P->nitems[0][0] + P->nitems[1][0] > 0, bf16 = P->nitems[0][1] + P->nitems[1][1] > 0;
    if (f32 == bf16) return -1;
    return f32 ? 0 : 1;
}

// Launches bt_fused<type> cooperatively (one block per SM).
bto_status bt_launch_fused(char* ws, int type, cudaStream_t st, int stall_block, unsigned long long limit_ns) {
    DeviceInfo dinf;
    if (!device_info(&dinf) || !dinf.coop) return BTO_ERR_CUDA;
    if (!bt_setup<float>() || !bt_setup<__nv_bfloat16>()) return BTO_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(dinf.sms);
    cfg.blockDim = dim3(kThreadsT);
    cfg.dynamicSmemBytes = type ? bt_smem<__nv_bfloat16>() : bt_smem<float>();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = type ? cudaLaunchKernelEx(&cfg, bt_fused<__nv_bfloat16>, ws, stall_block, limit_ns)
                               : cudaLaunchKernelEx(&cfg, bt_fused<float>, ws, stall_block, limit_ns);
    return e == cudaSuccess ? BTO_OK : BTO_ERR_CUDA;
}

// Launches the TMA path: stage one (both storage types), its combine, stage
// two, its combine.  With the host plan, only the launches that have work,
// each grid at most its items; without (P == NULL: a prepared workspace, as
// bto_batch_run replays it), every launch, sized to the GPU, reading its
// counts from the workspace.
bto_status bt_launch(char* ws, const BtPlan* P, cudaStream_t st) {
    DeviceInfo dinf;
    if (!device_info(&dinf)) return BTO_ERR_CUDA;
    if (!bt_setup<float>() || !bt_setup<__nv_bfloat16>()) return BTO_ERR_CUDA;
    for (int stage = 0; stage < 2; stage++) {
        for (int t = 0; t < 2; t++) {
            const int n = P ? P->nitems[stage][t] : dinf.sms;
            if (n == 0) continue;
            const int grid = std::min(n, dinf.sms);
            if (t == 0) bt_sweep<float><<<grid, kThreadsT, bt_smem<float>(), st>>>(ws, stage);
            else bt_sweep<__nv_bfloat16><<<grid, kThreadsT, bt_smem<__nv_bfloat16>(), st>>>(ws, stage);
        }
        const int nc = P ? P->nchunk[stage] : dinf.sms * 8;
        if (nc > 0) bt_combine<<<std::min(nc, dinf.sms * 8), 256, 0, st>>>(ws, stage);
    }
    return launch_status();
}

}  // namespace bto
