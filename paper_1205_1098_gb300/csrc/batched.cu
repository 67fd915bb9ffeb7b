// Batched form: many independent, uneven BICGK, GEMVER, ATAX and GESUMMV
// instances (matrices in FP32 or BF16, vectors in FP32) in one persistent
// launch.  The serving loop drives it too.
//
// bto_batch_prepare builds a work list on the host and uploads it into the
// caller's workspace.  Stage-one items: (instance, column panel) for BICGK,
// GEMVER's first pass and GESUMMV; (instance, 256-row block) for ATAX's t = A x.
// Stage-two items: (instance, 256-row block) for GEMVER's w = alpha B x and
// (instance, column panel) for ATAX's y = beta A^T t.  Stage-one items come
// first, largest estimated cost first (longest-processing-time order), then
// the stage-two items.  bto_batch_run launches a persistent grid whose blocks
// pull items from a device counter, so the load balances itself and the
// launch contains no host synchronisation (it can be captured into a graph).
//
// Per item the arithmetic is that of the reduced-precision form: warps own
// 16-column groups, lanes own 8 rows (16-byte loads), FP32 FMA chains folded
// into TwoSum (hi, lo) pairs, a transposing butterfly for column sums.  An
// instance split into P column panels (BICGK's q, GESUMMV's y) leaves P
// row-partial vectors; the panel that finishes last (per-instance counter)
// adds them in panel order in FP64.  A stage-two item waits, bounded by
// %globaltimer, until every stage-one item of its instance has published
// (release/acquire on the counter); the wait always ends because all those
// items were taken earlier by resident blocks.  Results do not depend on
// which block runs an item, so an instance gives the same bits alone or in a
// batch planned with the same panel width.
#include "check.cuh"
#include "lp_math.cuh"
#include <algorithm>
#include <mutex>
#include <unordered_map>
#include <cstring>
#include <vector>

namespace bto {
namespace {

using namespace lp;

constexpr int kThreads = 256;
constexpr int kWarps = 8;
constexpr int kRows = 256;                 // rows per chunk: 32 lanes x 8 rows
constexpr unsigned long long kWaitNs = 2000000000ull;

enum ItemKind { IT_BICGK = 0, IT_GEMVER1 = 1, IT_GEMVER2 = 2, IT_ATAX1 = 3, IT_ATAX2 = 4, IT_GESUMMV = 5 };

struct Item { int32_t inst, kind, lo, hi; };

struct InstInfo {
    int32_t stage1;        // stage-one items of the instance (what stage two waits for)
    int32_t vec;           // 16-byte loads allowed (matrices and leading dimensions aligned)
    int64_t qoff;          // BICGK/GESUMMV: offset (float2) of the panel partials, -1 if one panel
    int64_t toff;          // ATAX: offset (float) of t
};

constexpr int kQueues = 4;   // (FP32, BF16) x (BICGK/GEMVER, ATAX/GESUMMV)

struct Header {
    int32_t count, nitems, tile_cols, pad0;
    int32_t qstart[kQueues + 1];                 // items of queue q: [qstart[q], qstart[q+1])
    int32_t pad1[3];
    int64_t off_desc, off_info, off_items, off_counters, off_qpart, off_t;
    int64_t counters_bytes, total;
};

constexpr size_t kHeaderOff = 64;    // the status word is the first int of the workspace

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Lane's k-th row within a 256-row chunk: FP32 as two groups of four
// consecutive rows, BF16 as eight consecutive rows (one 16-byte load).
template <typename TA>
__device__ __forceinline__ int brow(int lane, int k) {
    if (sizeof(TA) == 2) return lane * 8 + k;
    return (k >> 2) * 128 + lane * 4 + (k & 3);
}

// Element q of a 16-byte vector, as FP32, using register operations only.
template <typename TA>
__device__ __forceinline__ float unpack(const uint4& t, int q) {
    const unsigned w = q < (sizeof(TA) == 2 ? 2 : 1) ? t.x
                     : q < (sizeof(TA) == 2 ? 4 : 2) ? t.y
                     : q < (sizeof(TA) == 2 ? 6 : 3) ? t.z : t.w;
    if (sizeof(TA) == 4) return __uint_as_float(w);
    return __uint_as_float((q & 1) ? (w & 0xFFFF0000u) : (w << 16));
}

template <typename TA>
__device__ __forceinline__ unsigned bits_of(TA v);
template <> __device__ __forceinline__ unsigned bits_of<float>(float v) { return __float_as_uint(v); }
template <> __device__ __forceinline__ unsigned bits_of<__nv_bfloat16>(__nv_bfloat16 v) {
    return (unsigned)__bfloat16_as_ushort(v);
}

template <typename TA, bool COHERENT>
__device__ __forceinline__ void load8(const TA* col, int64_t R0, int64_t m, int lane, bool vec, float (&a)[8]) {
    constexpr int V = 16 / sizeof(TA);
#pragma unroll
    for (int h = 0; h < 8 / V; h++) {
        const int64_t i = R0 + brow<TA>(lane, h * V);
        if (vec && i + V <= m) {
            const uint4 t = COHERENT ? __ldcg(reinterpret_cast<const uint4*>(col + i))
                                     : __ldg(reinterpret_cast<const uint4*>(col + i));
#pragma unroll
            for (int q = 0; q < V; q++) a[h * V + q] = unpack<TA>(t, q);
        } else {
#pragma unroll
            for (int q = 0; q < V; q++) {
                float v = 0.0f;
                if (i + q < m) {
                    if (sizeof(TA) == 2) {
                        const unsigned short b = COHERENT ? __ldcg(reinterpret_cast<const unsigned short*>(col + i + q))
                                                          : __ldg(reinterpret_cast<const unsigned short*>(col + i + q));
                        v = __uint_as_float((unsigned)b << 16);
                    } else {
                        v = COHERENT ? __ldcg(reinterpret_cast<const float*>(col + i + q))
                                     : __ldg(reinterpret_cast<const float*>(col + i + q));
                    }
                }
                a[h * V + q] = v;
            }
        }
    }
}

template <typename TA>
__device__ __forceinline__ void store8(TA* col, int64_t R0, int64_t m, int lane, bool vec, const TA (&b)[8]) {
    constexpr int V = 16 / sizeof(TA);
#pragma unroll
    for (int h = 0; h < 8 / V; h++) {
        const int64_t i = R0 + brow<TA>(lane, h * V);
        if (vec && i + V <= m) {
            uint4 t;
            if (sizeof(TA) == 4) {
                t.x = bits_of<TA>(b[h * V]); t.y = bits_of<TA>(b[h * V + 1]);
                t.z = bits_of<TA>(b[h * V + 2]); t.w = bits_of<TA>(b[h * V + 3]);
            } else {
                t.x = bits_of<TA>(b[0]) | (bits_of<TA>(b[1]) << 16);
                t.y = bits_of<TA>(b[2]) | (bits_of<TA>(b[3]) << 16);
                t.z = bits_of<TA>(b[4]) | (bits_of<TA>(b[5]) << 16);
                t.w = bits_of<TA>(b[6]) | (bits_of<TA>(b[7]) << 16);
            }
            *reinterpret_cast<uint4*>(col + i) = t;
        } else {
#pragma unroll
            for (int q = 0; q < V; q++) if (i + q < m) col[i + q] = b[h * V + q];
        }
    }
}

// ---------------------------------------------------------------- copy ring
// Matrices whose columns allow 16-byte copies stream through a per-warp ring
// of kStages batches in shared memory, filled with cp.async kStages - 1
// batches ahead of use (about 12 KB in flight per warp instead of the 4 KB a
// register prefetch can hold).  A batch is up to kBatchCols column slots of
// one 256-row chunk.  Each lane copies, and later reads, only its own rows
// of every slot (the chunks brow() gives it), so a lane's own
// cp.async.wait_group orders its copies before its reads: no barrier is
// needed.  Rows past m are zero-filled by the copy.
constexpr int kStages = 4;
constexpr int kBatchCols = 4;
constexpr int kMaxTile = 1024;     // widest column panel (tile_cols)

template <typename TA>
constexpr int ring_elems() { return kStages * kBatchCols * kRows; }

__device__ __forceinline__ void cp16_zfill(void* dst, const void* src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                 ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_ring() { asm volatile("cp.async.wait_group %0;" ::"n"(kStages - 2) : "memory"); }

// The lane's 8 rows of column `col` (chunk rows R0 .. R0+255) into a 256-row slot.
template <typename TA>
__device__ __forceinline__ void cp_col(TA* slot, const TA* col, int64_t R0, int64_t m, int lane) {
    constexpr int V = 16 / sizeof(TA);
#pragma unroll
    for (int h = 0; h < 8 / V; h++) {
        const int r = brow<TA>(lane, h * V);
        const int64_t i = R0 + r;
        const int64_t left = m - i;
        const int valid = left <= 0 ? 0 : (left >= V ? V : (int)left);
        cp16_zfill(slot + r, valid > 0 ? (const void*)(col + i) : (const void*)col, valid * (int)sizeof(TA));
    }
}

// The lane's 8 rows of a slot, as FP32.
template <typename TA>
__device__ __forceinline__ void read_col(const TA* slot, int lane, float (&a)[8]) {
    constexpr int V = 16 / sizeof(TA);
#pragma unroll
    for (int h = 0; h < 8 / V; h++) {
        const uint4 t = *reinterpret_cast<const uint4*>(slot + brow<TA>(lane, h * V));
#pragma unroll
        for (int q = 0; q < V; q++) a[h * V + q] = unpack<TA>(t, q);
    }
}

template <typename TA, bool COHERENT>
__device__ __forceinline__ void load_rows(const float* v, int64_t R0, int64_t m, int lane, float (&o)[8]) {
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const int64_t i = R0 + brow<TA>(lane, k);
        o[k] = (i < m) ? (COHERENT ? __ldcg(v + i) : __ldg(v + i)) : 0.0f;
    }
}

// Adds the warps' (hi, lo) row partials (red: [2][kWarps][kRows]) in warp
// order with TwoSum; thread t handles row t.
__device__ __forceinline__ void warp_rows_sum(const float* red, int t, float& hs, float& ls) {
    hs = red[t];
    ls = red[kWarps * kRows + t];
#pragma unroll
    for (int w = 1; w < kWarps; w++) {
        float s2, e2;
        two_sum(hs, red[w * kRows + t], s2, e2);
        hs = s2;
        ls += e2 + red[(kWarps + w) * kRows + t];
    }
}

template <typename TA>
__device__ __forceinline__ void stash_rows(float* red, int warp, int lane, const float (&hi)[8], const float (&lo)[8]) {
#pragma unroll
    for (int k = 0; k < 8; k++) {
        red[warp * kRows + brow<TA>(lane, k)] = hi[k];
        red[(kWarps + warp) * kRows + brow<TA>(lane, k)] = lo[k];
    }
}

// t[k] += a[k] * x for a lane's 8 rows, two rows per packed FP32 FMA.
__device__ __forceinline__ void fma8(const float (&a)[8], float x, float (&t)[8]) {
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
        const float2 r = __ffma2_rn(make_float2(a[k], a[k + 1]), make_float2(x, x), make_float2(t[k], t[k + 1]));
        t[k] = r.x;
        t[k + 1] = r.y;
    }
}

// sum_k a[k] r[k] over a lane's 8 rows: two interleaved chains (even and odd
// rows) in packed FP32 instructions, added at the end.
__device__ __forceinline__ float dot8(const float (&a)[8], const float (&r)[8]) {
    float2 acc = __fmul2_rn(make_float2(a[0], a[1]), make_float2(r[0], r[1]));
#pragma unroll
    for (int k = 2; k < 8; k += 2) acc = __ffma2_rn(make_float2(a[k], a[k + 1]), make_float2(r[k], r[k + 1]), acc);
    return acc.x + acc.y;
}

__device__ __forceinline__ void fold(float (&hi)[8], float (&lo)[8], float (&t)[8]) {
#pragma unroll
    for (int k = 0; k < 8; k++) {
        float s2, e2;
        two_sum(hi[k], t[k], s2, e2);
        hi[k] = s2; lo[k] += e2; t[k] = 0.0f;
    }
}

// Column-panel item over all rows of instance d, columns [c0, c1).
//   IT_BICGK   : s for the panel's columns, q row partials.
//   IT_GEMVER1 : B = A + u1 v1^T + u2 v2^T for the panel, x for its columns.
//   IT_ATAX2   : y = beta A^T t for the panel's columns (t from the workspace).
//   IT_GESUMMV : row partials of A x and B x.
template <int KIND, typename TA>
__device__ __forceinline__ void panel_item(const bto_batch_desc& d, const InstInfo& info, int panel, int64_t c0, int64_t c1,
                           float* red, float* red2, float* shi, float* slo, float2* qpart, const float* tbuf,
                           TA* ring) {
    constexpr bool HAS_Q = (KIND == IT_BICGK || KIND == IT_GESUMMV);
    constexpr bool HAS_S = (KIND == IT_BICGK || KIND == IT_GEMVER1 || KIND == IT_ATAX2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m = d.m, ncols = c1 - c0;
    const bool vec = info.vec != 0;
    const TA* A = static_cast<const TA*>(d.A);
    const TA* B2 = static_cast<const TA*>(d.B);      // GESUMMV's second matrix
    TA* Bo = static_cast<TA*>(d.B);                  // GEMVER's output
    const float* xin = d.in[0];
    for (int k = threadIdx.x; k < ncols; k += kThreads) { shi[k] = 0.0f; slo[k] = 0.0f; }
    __syncthreads();
    // Columns loaded ahead of use: four (two for GESUMMV, which loads two matrices).
    constexpr int KU = KIND == IT_GESUMMV ? 2 : 4;
    constexpr int GB = 16 / KU;                 // batches per 16-column butterfly group
    // Columns are dealt to the warps in batches of KU: warp w takes batches
    // w, w + 8, w + 16, ... of the panel, so the warps' shares differ by at
    // most one batch (whole 16-column groups left warps idle on narrow panels).
    const int nbt = (int)((ncols + KU - 1) / KU);
    const int nbw = nbt > warp ? (nbt - warp + kWarps - 1) / kWarps : 0;
    // Copy-ring schedule: batch = (chunk, this warp's batch t), in loop order.
    const int nbat = vec ? (int)((m + kRows - 1) / kRows) * nbw : 0;
    int bi = 0, iss = 0, ic = 0, it = 0;
    auto issue = [&]() {
        if (iss < nbat) {
            const int64_t R0i = (int64_t)ic * kRows, cbi = c0 + (int64_t)KU * (warp + kWarps * it);
            const int nci = (int)((c1 - cbi) < KU ? (c1 - cbi) : KU);
            TA* st = ring + (iss % kStages) * (kBatchCols * kRows);
#pragma unroll
            for (int u = 0; u < KU; u++) {
                if (u < nci) {
                    cp_col<TA>(st + u * kRows, A + (cbi + u) * d.lda, R0i, m, lane);
                    if (KIND == IT_GESUMMV) cp_col<TA>(st + (KU + u) * kRows, B2 + (cbi + u) * d.ldb, R0i, m, lane);
                }
            }
            if (++it == nbw) { it = 0; ++ic; }
        }
        cp_commit();
        iss++;
    };
    if (vec)
        for (int k = 0; k < kStages - 1; k++) issue();
    for (int64_t R0 = 0; R0 < m; R0 += kRows) {
        float rv[8], u1r[8], u2r[8], qhi[8], qlo[8], q2hi[8], q2lo[8];
        if (KIND == IT_BICGK) load_rows<TA, false>(d.in[1], R0, m, lane, rv);
        if (KIND == IT_GEMVER1) {
            load_rows<TA, false>(d.in[4], R0, m, lane, rv);
            load_rows<TA, false>(d.in[0], R0, m, lane, u1r);
            load_rows<TA, false>(d.in[2], R0, m, lane, u2r);
        }
        if (KIND == IT_ATAX2) load_rows<TA, true>(tbuf + info.toff, R0, m, lane, rv);
#pragma unroll
        for (int k = 0; k < 8; k++) { qhi[k] = 0.0f; qlo[k] = 0.0f; q2hi[k] = 0.0f; q2lo[k] = 0.0f; }
        for (int t0 = 0; t0 < nbw; t0 += GB) {
            float sl[16], qt[8], q2t[8];
#pragma unroll
            for (int k = 0; k < 8; k++) { qt[k] = 0.0f; q2t[k] = 0.0f; }
#pragma unroll
            for (int tt = 0; tt < GB; tt++) {
                const int t = t0 + tt;
                if (t >= nbw) {
                    if (HAS_S) {
#pragma unroll
                        for (int u = 0; u < KU; u++) sl[KU * tt + u] = 0.0f;
                    }
                    continue;
                }
                const int64_t cb = c0 + (int64_t)KU * (warp + kWarps * t);
                const int nc = (int)((c1 - cb) < KU ? (c1 - cb) : KU);
                float av[KU][8], bv[KU][8];
                if (vec) {
                    // Batch bi is in the ring once at most kStages - 2 newer batches are pending.
                    cp_wait_ring();
                    const TA* st = ring + (bi % kStages) * (kBatchCols * kRows);
#pragma unroll
                    for (int u = 0; u < KU; u++)
                        if (u < nc) {
                            read_col<TA>(st + u * kRows, lane, av[u]);
                            if (KIND == IT_GESUMMV) read_col<TA>(st + (KU + u) * kRows, lane, bv[u]);
                        }
                    bi++;
                    issue();     // refills the slot of batch bi - 1, read in the previous step
                } else {
#pragma unroll
                    for (int u = 0; u < KU; u++)
                        if (u < nc) {
                            load8<TA, false>(A + (cb + u) * d.lda, R0, m, lane, vec, av[u]);
                            if (KIND == IT_GESUMMV) load8<TA, false>(B2 + (cb + u) * d.ldb, R0, m, lane, vec, bv[u]);
                        }
                }
#pragma unroll
                for (int u = 0; u < KU; u++) {
                    const int jj = KU * tt + u;
                    if (u < nc) {
                        const int64_t j = cb + u;
                        if (HAS_Q) {
                            const float pj = __ldg(xin + j);
                            fma8(av[u], pj, qt);
                            if (KIND == IT_GESUMMV) fma8(bv[u], pj, q2t);
                        }
                        if (KIND == IT_GEMVER1) {
                            const float v1j = __ldg(d.in[1] + j), v2j = __ldg(d.in[3] + j);
                            TA bq[8];
#pragma unroll
                            for (int k = 0; k < 8; k += 2) {
                                // Two rows per packed FMA; per element the same two FMAs.
                                const float2 t2 = __ffma2_rn(make_float2(u2r[k], u2r[k + 1]), make_float2(v2j, v2j),
                                                             __ffma2_rn(make_float2(u1r[k], u1r[k + 1]),
                                                                        make_float2(v1j, v1j),
                                                                        make_float2(av[u][k], av[u][k + 1])));
                                bq[k] = from_f<TA>(t2.x);
                                bq[k + 1] = from_f<TA>(t2.y);
                                av[u][k] = to_f<TA>(bq[k]);     // x uses the stored B
                                av[u][k + 1] = to_f<TA>(bq[k + 1]);
                            }
                            store8<TA>(Bo + j * d.ldb, R0, m, lane, vec, bq);
                        }
                        if (HAS_S) sl[jj] = dot8(av[u], rv);
                    } else if (HAS_S) {
                        sl[jj] = 0.0f;
                    }
                }
            }
            if (HAS_Q) fold(qhi, qlo, qt);
            if (KIND == IT_GESUMMV) fold(q2hi, q2lo, q2t);
            if (HAS_S) {
                // Lane l < 16 holds slot l of the group: batch t0 + l / KU, column l % KU of it.
                const float cs = butterfly16(sl, lane);
                const int t = t0 + lane / KU;
                if (lane < 16 && t < nbw) {
                    const int64_t o = (int64_t)KU * (warp + kWarps * t) + lane % KU;
                    if (o < ncols) {
                        float s2, e2;
                        two_sum(shi[o], cs, s2, e2);
                        shi[o] = s2; slo[o] += e2;
                    }
                }
            }
        }
        if (HAS_Q) {
            stash_rows<TA>(red, warp, lane, qhi, qlo);
            if (KIND == IT_GESUMMV) stash_rows<TA>(red2, warp, lane, q2hi, q2lo);
            __syncthreads();
            const int64_t i = R0 + threadIdx.x;
            if (i < m) {
                float hs, ls;
                warp_rows_sum(red, threadIdx.x, hs, ls);
                if (KIND == IT_BICGK) {
                    if (info.qoff < 0) d.out[0][i] = (float)((double)hs + (double)ls);
                    else qpart[info.qoff + (int64_t)panel * m + i] = make_float2(hs, ls);
                } else {
                    float h2, l2;
                    warp_rows_sum(red2, threadIdx.x, h2, l2);
                    if (info.qoff < 0) {
                        d.out[0][i] = (float)fma((double)d.alpha, (double)hs + (double)ls,
                                                 (double)d.beta * ((double)h2 + (double)l2));
                    } else {
                        qpart[info.qoff + ((int64_t)panel * 2) * m + i] = make_float2(hs, ls);
                        qpart[info.qoff + ((int64_t)panel * 2 + 1) * m + i] = make_float2(h2, l2);
                    }
                }
            }
            __syncthreads();
        }
    }
    __syncthreads();
    if (HAS_S) {
        for (int k = threadIdx.x; k < ncols; k += kThreads) {
            const double s = (double)shi[k] + (double)slo[k];
            if (KIND == IT_BICGK) d.out[1][c0 + k] = (float)s;
            else if (KIND == IT_GEMVER1) d.out[0][c0 + k] = (float)fma((double)d.beta, s, (double)__ldg(d.in[5] + c0 + k));
            else d.out[0][c0 + k] = (float)((double)d.beta * s);
        }
    }
}

// Row-block item over all columns, rows [R0, R0 + 256): out = scale * M v.
//   IT_GEMVER2 : w = alpha B x (B and x written by stage one: coherent loads).
//   IT_ATAX1   : t = A x into the workspace.
template <int KIND, typename TA>
__device__ __forceinline__ void row_item(const bto_batch_desc& d, const InstInfo& info, int64_t R0, float* red, float* tbuf,
                                         TA* ring) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m = d.m, n = d.n;
    const bool vec = info.vec != 0;
    const TA* M = static_cast<const TA*>(KIND == IT_GEMVER2 ? d.B : d.A);
    const int64_t ld = KIND == IT_GEMVER2 ? d.ldb : d.lda;
    const float* v = KIND == IT_GEMVER2 ? d.out[0] : d.in[0];
    float qhi[8], qlo[8], qt[8];
#pragma unroll
    for (int k = 0; k < 8; k++) { qhi[k] = 0.0f; qlo[k] = 0.0f; qt[k] = 0.0f; }
    // Columns are dealt to the warps in batches of 4 (warp w takes batches
    // w, w + 8, ...); the copy ring follows the same order (see cp_col).
    // cp.async.cg reads through L2, so GEMVER's B written by stage one is seen.
    const int nbt = (int)((n + 3) / 4);
    const int nbw = nbt > warp ? (nbt - warp + kWarps - 1) / kWarps : 0;
    const int nbat = vec ? nbw : 0;
    int bi = 0, iss = 0;
    auto issue = [&]() {
        if (iss < nbat) {
            const int64_t cbi = 4 * (int64_t)(warp + kWarps * iss);
            const int nci = (int)((n - cbi) < 4 ? (n - cbi) : 4);
            TA* st = ring + (iss % kStages) * (kBatchCols * kRows);
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (u < nci) cp_col<TA>(st + u * kRows, M + (cbi + u) * ld, R0, m, lane);
        }
        cp_commit();
        iss++;
    };
    if (vec)
        for (int k = 0; k < kStages - 1; k++) issue();
    for (int t = 0; t < nbw; t++) {
        const int64_t cb = 4 * (int64_t)(warp + kWarps * t);
        const int nc = (int)((n - cb) < 4 ? (n - cb) : 4);
        float av[4][8], xj[4];
        if (vec) {
            cp_wait_ring();
            const TA* st = ring + (bi % kStages) * (kBatchCols * kRows);
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (u < nc) {
                    read_col<TA>(st + u * kRows, lane, av[u]);
                    xj[u] = KIND == IT_GEMVER2 ? __ldcg(v + cb + u) : __ldg(v + cb + u);
                }
            bi++;
            issue();
        } else {
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (u < nc) {
                    load8<TA, KIND == IT_GEMVER2>(M + (cb + u) * ld, R0, m, lane, vec, av[u]);
                    xj[u] = KIND == IT_GEMVER2 ? __ldcg(v + cb + u) : __ldg(v + cb + u);
                }
        }
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (u < nc) fma8(av[u], xj[u], qt);
        if ((t & 3) == 3 || t + 1 == nbw) fold(qhi, qlo, qt);   // every 16 columns, as the panel sweep
    }
    stash_rows<TA>(red, warp, lane, qhi, qlo);
    __syncthreads();
    const int64_t i = R0 + threadIdx.x;
    if (i < m) {
        float hs, ls;
        warp_rows_sum(red, threadIdx.x, hs, ls);
        if (KIND == IT_GEMVER2) d.out[1][i] = (float)((double)d.alpha * ((double)hs + (double)ls));
        else tbuf[info.toff + i] = (float)((double)hs + (double)ls);
    }
    __syncthreads();
}

// Item families, each run by its own kernel so that one family's register
// needs do not burden the other's: 0 = BICGK and GEMVER, 1 = ATAX and GESUMMV.
__host__ __device__ inline int family_of(int kind) {
    return (kind == IT_BICGK || kind == IT_GEMVER1 || kind == IT_GEMVER2) ? 0 : 1;
}

template <typename TA, int FAM>
__device__ void run_item(const Item& item, const bto_batch_desc& d, const InstInfo& info, int tile_cols,
                         float* red, float* red2, float* shi, float* slo, float2* qpart, float* tbuf, TA* ring) {
    const int panel = tile_cols ? (int)(item.lo / tile_cols) : 0;
    if (FAM == 0) {
        switch (item.kind) {
            case IT_BICGK: panel_item<IT_BICGK, TA>(d, info, panel, item.lo, item.hi, red, red2, shi, slo, qpart, tbuf, ring); break;
            case IT_GEMVER1: panel_item<IT_GEMVER1, TA>(d, info, panel, item.lo, item.hi, red, red2, shi, slo, qpart, tbuf, ring); break;
            case IT_GEMVER2: row_item<IT_GEMVER2, TA>(d, info, item.lo, red, tbuf, ring); break;
        }
    } else {
        switch (item.kind) {
            case IT_ATAX2: panel_item<IT_ATAX2, TA>(d, info, panel, item.lo, item.hi, red, red2, shi, slo, qpart, tbuf, ring); break;
            case IT_GESUMMV: panel_item<IT_GESUMMV, TA>(d, info, panel, item.lo, item.hi, red, red2, shi, slo, qpart, tbuf, ring); break;
            case IT_ATAX1: row_item<IT_ATAX1, TA>(d, info, item.lo, red, tbuf, ring); break;
        }
    }
}

template <typename TA, int FAM>
__global__ void __launch_bounds__(kThreads, 1) batch_kernel(char* ws) {
    const Header* h = reinterpret_cast<const Header*>(ws + kHeaderOff);
    const bto_batch_desc* descs = reinterpret_cast<const bto_batch_desc*>(ws + h->off_desc);
    const InstInfo* infos = reinterpret_cast<const InstInfo*>(ws + h->off_info);
    constexpr int Q = (sizeof(TA) == 2 ? 2 : 0) + FAM;   // this kernel's queue (storage type, family)
    const Item* items = reinterpret_cast<const Item*>(ws + h->off_items) + h->qstart[Q];
    unsigned* counters = reinterpret_cast<unsigned*>(ws + h->off_counters);   // [0..3] queues, [4+i] instances
    float2* qpart = reinterpret_cast<float2*>(ws + h->off_qpart);
    float* tbuf = reinterpret_cast<float*>(ws + h->off_t);
    int* status = reinterpret_cast<int*>(ws);
    extern __shared__ float sm[];   // red [2][8][256], red2 [2][8][256], s (hi, lo) [2][tile_cols]
    float* red = sm;
    float* red2 = sm + 2 * kWarps * kRows;
    float* shi = red2 + 2 * kWarps * kRows;
    float* slo = shi + h->tile_cols;
    // This warp's copy ring, after the fixed regions (16-byte aligned).
    TA* ring = reinterpret_cast<TA*>(sm + 4 * kWarps * kRows + 2 * kMaxTile) + (threadIdx.x >> 5) * ring_elems<TA>();
    __shared__ int s_item, s_ok, s_last;
    const int nitems = h->qstart[Q + 1] - h->qstart[Q];
    while (true) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counters + Q, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        const Item item = items[it];
        const bto_batch_desc d = descs[item.inst];
        const InstInfo info = infos[item.inst];
        const bool stage2 = item.kind == IT_GEMVER2 || item.kind == IT_ATAX2;
        if (stage2) {
            if (threadIdx.x == 0) {
                const unsigned long long t0 = gtimer();
                int ok = 1;
                while (ld_acquire_u32(counters + kQueues + item.inst) < (unsigned)info.stage1) {
                    if (gtimer() - t0 > kWaitNs) { ok = 0; atomicExch(status, (int)BTO_ERR_TIMEOUT); break; }
                    __nanosleep(100);
                }
                s_ok = ok;
            }
            __syncthreads();
        }
        if (!stage2 || s_ok) run_item<TA, FAM>(item, d, info, h->tile_cols, red, red2, shi, slo, qpart, tbuf, ring);
        if (stage2) continue;
        // Publish this stage-one item (release); the last panel of a split
        // BICGK or GESUMMV adds the row partials in panel order.
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned old = atomicAdd(counters + kQueues + item.inst, 1u);
            s_last = ((item.kind == IT_BICGK || item.kind == IT_GESUMMV) && info.qoff >= 0 &&
                      old == (unsigned)(info.stage1 - 1));
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            const int P = info.stage1;   // panels of this split instance
            for (int64_t i = threadIdx.x; i < d.m; i += kThreads) {
                if (item.kind == IT_BICGK) {
                    double s = 0.0;
                    for (int p = 0; p < P; p++) {
                        const float2 v = __ldcg(qpart + info.qoff + (int64_t)p * d.m + i);
                        s += (double)v.x + (double)v.y;
                    }
                    d.out[0][i] = (float)s;
                } else {
                    double sa = 0.0, sb = 0.0;
                    for (int p = 0; p < P; p++) {
                        const float2 va = __ldcg(qpart + info.qoff + ((int64_t)p * 2) * d.m + i);
                        const float2 vb = __ldcg(qpart + info.qoff + ((int64_t)p * 2 + 1) * d.m + i);
                        sa += (double)va.x + (double)va.y;
                        sb += (double)vb.x + (double)vb.y;
                    }
                    d.out[0][i] = (float)fma((double)d.alpha, sa, (double)d.beta * sb);
                }
            }
        }
    }
}

// Clears the status word and the counters recorded in the plan's header.
__global__ void batch_reset_kernel(char* ws) {
    const Header* h = reinterpret_cast<const Header*>(ws + kHeaderOff);
    unsigned* c = reinterpret_cast<unsigned*>(ws + h->off_counters);
    const int64_t nc = h->counters_bytes / (int64_t)sizeof(unsigned);
    for (int64_t i = threadIdx.x; i < nc; i += blockDim.x) c[i] = 0u;
    if (threadIdx.x == 0) *reinterpret_cast<int*>(ws) = 0;
}

constexpr size_t kSmemBytes = (4 * kWarps * kRows + 2 * kMaxTile) * sizeof(float) +
                              (size_t)kWarps * ring_elems<float>() * sizeof(float);

struct Plan {
    Header h{};
    std::vector<bto_batch_desc> descs;
    std::vector<InstInfo> info;
    std::vector<Item> items;
    BtPlan* bt;                 // instances on the TMA path
    Plan() : bt(bt_plan_create()) {}
    ~Plan() { bt_plan_destroy(bt); }
    Plan(const Plan&) = delete;
    Plan& operator=(const Plan&) = delete;
};

int64_t esize(int a_type) { return a_type == BTO_BF16 ? 2 : 4; }

bool valid_desc(const bto_batch_desc& d) {
    const int op = d.op;
    if (op != BTO_OP_BICGK && op != BTO_OP_GEMVER && op != BTO_OP_ATAX && op != BTO_OP_GESUMMV) return false;
    if (d.a_type != BTO_F32 && d.a_type != BTO_BF16) return false;
    if (d.m < 0 || d.n < 0 || d.m > INT32_MAX || d.n > INT32_MAX) return false;
    if (d.lda < std::max<int64_t>(1, d.m)) return false;
    const bool mat = d.m > 0 && d.n > 0;
    if (mat && (!d.A || reinterpret_cast<uintptr_t>(d.A) % esize(d.a_type))) return false;
    if ((op == BTO_OP_GEMVER || op == BTO_OP_GESUMMV) &&
        (d.ldb < std::max<int64_t>(1, d.m) || (mat && !d.B))) return false;
    // Input and output vector lengths per op.
    int64_t in_len[6] = {0, 0, 0, 0, 0, 0}, out_len[2] = {0, 0};
    if (op == BTO_OP_BICGK) { in_len[0] = d.n; in_len[1] = d.m; out_len[0] = d.m; out_len[1] = d.n; }
    if (op == BTO_OP_GEMVER) {
        for (int k = 0; k < 6; k++) in_len[k] = (k % 2 == 0) ? d.m : d.n;
        out_len[0] = d.n; out_len[1] = d.m;
    }
    if (op == BTO_OP_ATAX) { in_len[0] = d.n; out_len[0] = d.n; }
    if (op == BTO_OP_GESUMMV) { in_len[0] = d.n; out_len[0] = d.m; }
    for (int k = 0; k < 6; k++) if (in_len[k] > 0 && !d.in[k]) return false;
    for (int k = 0; k < 2; k++) if (out_len[k] > 0 && !d.out[k]) return false;
    return true;
}

bool make_plan(int count, const bto_batch_desc* descs, int tile_cols, Plan* P, int* bad_desc) {
    P->descs.assign(descs, descs + count);
    P->info.resize(count);
    P->items.clear();
    bt_plan_reset(P->bt, tile_cols);
    std::vector<std::pair<double, Item>> first, second;
    int64_t qsize = 0, tsize = 0;
    for (int i = 0; i < count; i++) {
        const bto_batch_desc& d = descs[i];
        if (!valid_desc(d)) { *bad_desc = i; return false; }
        const int op = d.op;
        const int64_t m = d.m, n = d.n, es = esize(d.a_type), V = 16 / es;
        InstInfo& inf = P->info[i];
        inf.vec = aligned16(d.A) && d.lda % V == 0 &&
                  ((op != BTO_OP_GEMVER && op != BTO_OP_GESUMMV) || (aligned16(d.B) && d.ldb % V == 0));
        inf.qoff = -1;
        inf.toff = -1;
        inf.stage1 = 0;
        // Instances whose matrices suit the TMA go through the sweep path.
        if (bt_plan_add(P->bt, d)) continue;
        const int64_t panels = n > 0 ? ceil_div(n, tile_cols) : 0;
        const int64_t rblocks = m > 0 ? ceil_div(m, kRows) : 0;
        auto push = [&](std::vector<std::pair<double, Item>>& v, int kind, int64_t lo, int64_t hi, double cost) {
            v.push_back({cost, Item{i, kind, (int32_t)lo, (int32_t)hi}});
        };
        const double mm = (double)m;
        if (op == BTO_OP_BICGK || op == BTO_OP_GESUMMV) {
            const int kind = op == BTO_OP_BICGK ? IT_BICGK : IT_GESUMMV;
            const double w = op == BTO_OP_GESUMMV ? 2.0 : 1.0;
            if (panels == 0) {
                if (m > 0) push(first, kind, 0, 0, 0.0);     // writes the empty sums
                inf.stage1 = m > 0 ? 1 : 0;
            } else {
                for (int64_t c = 0; c < n; c += tile_cols)
                    push(first, kind, c, std::min<int64_t>(n, c + tile_cols), w * mm * (double)(std::min<int64_t>(n, c + tile_cols) - c));
                inf.stage1 = (int32_t)panels;
                if (panels > 1 && m > 0) { inf.qoff = qsize; qsize += panels * m * (op == BTO_OP_GESUMMV ? 2 : 1); }
            }
        } else if (op == BTO_OP_GEMVER) {
            for (int64_t c = 0; c < n; c += tile_cols)
                push(first, IT_GEMVER1, c, std::min<int64_t>(n, c + tile_cols), 2.0 * mm * (double)(std::min<int64_t>(n, c + tile_cols) - c));
            inf.stage1 = (int32_t)panels;
            for (int64_t r = 0; r < m; r += kRows)
                push(second, IT_GEMVER2, r, std::min<int64_t>(m, r + kRows), (double)(std::min<int64_t>(m, r + kRows) - r) * (double)n);
        } else {   // ATAX: t = A x by row blocks, then y = beta A^T t by panels
            for (int64_t r = 0; r < m; r += kRows)
                push(first, IT_ATAX1, r, std::min<int64_t>(m, r + kRows), (double)(std::min<int64_t>(m, r + kRows) - r) * (double)n);
            inf.stage1 = (int32_t)rblocks;
            if (m > 0) { inf.toff = tsize; tsize += round_up(m, 64); }
            for (int64_t c = 0; c < n; c += tile_cols)
                push(second, IT_ATAX2, c, std::min<int64_t>(n, c + tile_cols), mm * (double)(std::min<int64_t>(n, c + tile_cols) - c));
        }
    }
    auto by_cost = [](const std::pair<double, Item>& a, const std::pair<double, Item>& b) {
        if (a.first != b.first) return a.first > b.first;
        if (a.second.inst != b.second.inst) return a.second.inst < b.second.inst;
        return a.second.lo < b.second.lo;
    };
    std::stable_sort(first.begin(), first.end(), by_cost);
    std::stable_sort(second.begin(), second.end(), by_cost);
    // Four queues, one per (storage type, item family), each run by its own
    // kernel; within a queue, stage one before stage two.
    Header& H = P->h;
    for (int q = 0; q < kQueues; q++) {
        const int want_t = q < 2 ? BTO_F32 : BTO_BF16, want_f = q % 2;
        H.qstart[q] = (int32_t)P->items.size();
        for (auto* v : {&first, &second})
            for (auto& e : *v)
                if (descs[e.second.inst].a_type == want_t && family_of(e.second.kind) == want_f)
                    P->items.push_back(e.second);
    }
    H.qstart[kQueues] = (int32_t)P->items.size();
    H.count = count;
    H.nitems = (int32_t)P->items.size();
    H.tile_cols = tile_cols;
    size_t cur = 256;
    auto region = [&](size_t bytes) { size_t at = cur; cur += round_up((int64_t)bytes, 256); return at; };
    H.off_desc = region((size_t)count * sizeof(bto_batch_desc));
    H.off_info = region((size_t)count * sizeof(InstInfo));
    H.off_items = region(P->items.size() * sizeof(Item));
    if (!bt_plan_empty(P->bt)) {
        // The TMA sweep runs one block per SM (bt_launch): its items are
        // ordered for that grid.
        DeviceInfo dinf;
        const int G = device_info(&dinf) ? dinf.sms : 0;
        cur = (size_t)bt_plan_layout_records(P->bt, (int64_t)cur, G);
    }
    H.counters_bytes = (int64_t)(count + kQueues) * sizeof(unsigned);
    H.off_counters = region((size_t)H.counters_bytes);
    H.off_qpart = region((size_t)std::max<int64_t>(qsize, 1) * sizeof(float2));
    H.off_t = region((size_t)std::max<int64_t>(tsize, 1) * sizeof(float));
    if (!bt_plan_empty(P->bt)) cur = (size_t)bt_plan_layout_partials(P->bt, (int64_t)cur);
    H.total = cur;
    return true;
}

bool check_tile(int tile_cols) { return tile_cols >= 16 && tile_cols <= kMaxTile && tile_cols % 16 == 0; }

// Resident blocks per SM of the persistent kernels (set up once).
int batch_occupancy() {
    static int occ = 0;
    if (occ == 0) {
        int o = 0;
        if (cudaFuncSetAttribute(batch_kernel<float, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) != cudaSuccess ||
            cudaFuncSetAttribute(batch_kernel<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) != cudaSuccess ||
            cudaFuncSetAttribute(batch_kernel<__nv_bfloat16, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) != cudaSuccess ||
            cudaFuncSetAttribute(batch_kernel<__nv_bfloat16, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, batch_kernel<float, 0>, kThreads, kSmemBytes) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        occ = std::max(o, 1);
    }
    return occ;
}

// The plan's device image: status word, header, descriptors, instance
// records, items and, when `counters`, the zeroed counters (which then need
// no reset kernel).
size_t image_bytes(const Plan& P, bool counters) {
    return (size_t)P.h.off_counters + (counters ? (size_t)P.h.counters_bytes : 0);
}

void write_image(const Plan& P, char* img, bool counters, char* ws) {
    std::memset(img, 0, image_bytes(P, counters));
    bt_plan_write(P.bt, img, ws);
    std::memcpy(img + kHeaderOff, &P.h, sizeof(Header));
    const size_t count = P.descs.size();
    if (count) std::memcpy(img + P.h.off_desc, P.descs.data(), count * sizeof(bto_batch_desc));
    if (count) std::memcpy(img + P.h.off_info, P.info.data(), P.info.size() * sizeof(InstInfo));
    if (!P.items.empty()) std::memcpy(img + P.h.off_items, P.items.data(), P.items.size() * sizeof(Item));
}

// The one-launch form (bt_fused) runs a prepared workspace when every instance
// takes the TMA path with one storage type and the device launches
// cooperatively: its storage type, or -1.
int fused_type(const Plan& P) {
    if (!P.items.empty() || bt_plan_empty(P.bt)) return -1;
    DeviceInfo dinf;
    if (!device_info(&dinf) || !dinf.coop) return -1;
    return bt_fused_type(P.bt);
}

// Workspaces prepared for the one-launch form, with their storage type, so
// that bto_batch_run (which sees only the workspace) takes it.
std::mutex g_fused_mu;
std::unordered_map<const void*, int> g_fused_ws;

void note_fused(const void* ws, int type) {
    std::lock_guard<std::mutex> lock(g_fused_mu);
    if (type >= 0) g_fused_ws[ws] = type;
    else g_fused_ws.erase(ws);
}

int fused_of(const void* ws) {
    std::lock_guard<std::mutex> lock(g_fused_mu);
    const auto it = g_fused_ws.find(ws);
    return it == g_fused_ws.end() ? -1 : it->second;
}

bto_status submit_plan(const Plan& P, void* ws, size_t ws_bytes, void* staging, size_t staging_bytes,
                       cudaStream_t st, bool allow_fused) {
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < (size_t)P.h.total) return BTO_ERR_WORKSPACE;
    DeviceInfo dinf;
    if (!device_info(&dinf)) return BTO_ERR_CUDA;
    const int occ = batch_occupancy();
    if (occ == 0) return BTO_ERR_CUDA;
    const size_t nb = image_bytes(P, true);
    if (staging && staging_bytes >= nb) {
        // Pinned staging that the caller keeps until the stream has passed
        // this copy: no host wait.
        write_image(P, static_cast<char*>(staging), true, static_cast<char*>(ws));
        if (cudaMemcpyAsync(ws, staging, nb, cudaMemcpyHostToDevice, st) != cudaSuccess) return BTO_ERR_CUDA;
    } else {
        std::vector<char> img(nb);
        write_image(P, img.data(), true, static_cast<char*>(ws));
        if (cudaMemcpyAsync(ws, img.data(), nb, cudaMemcpyHostToDevice, st) != cudaSuccess) return BTO_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return BTO_ERR_CUDA;
    }
    char* w = static_cast<char*>(ws);
    // The workspace now holds this plan: a later bto_batch_run takes its form.
    const int ft = allow_fused ? fused_type(P) : -1;
    note_fused(ws, ft);
    if (ft >= 0) return bt_launch_fused(w, ft, st);
    // Only the queues that hold items, each grid no larger than its items:
    // a small batch leaves the other SMs to work on other streams.

    const int64_t full = (int64_t)dinf.sms * occ;
    for (int q = 0; q < kQueues; q++) {
        const int64_t ni = P.h.qstart[q + 1] - P.h.qstart[q];
        if (ni == 0) continue;
        const int grid = (int)std::min<int64_t>(full, ni);
        switch (q) {
            case 0: batch_kernel<float, 0><<<grid, kThreads, kSmemBytes, st>>>(w); break;
            case 1: batch_kernel<float, 1><<<grid, kThreads, kSmemBytes, st>>>(w); break;
            case 2: batch_kernel<__nv_bfloat16, 0><<<grid, kThreads, kSmemBytes, st>>>(w); break;
            default: batch_kernel<__nv_bfloat16, 1><<<grid, kThreads, kSmemBytes, st>>>(w); break;
        }
    }
    const bto_status e = launch_status();
    if (e != BTO_OK || bt_plan_empty(P.bt)) return e;
    return bt_launch(w, P.bt, st);
}

}  // namespace

struct BatchPlan {
    Plan p;
};

BatchPlan* batch_plan_create() { return new BatchPlan(); }
void batch_plan_destroy(BatchPlan* b) { delete b; }

bool batch_plan_build(BatchPlan* b, int count, const bto_batch_desc* descs, int tile_cols, size_t* ws_bytes) {
    int bad = -1;
    if (count < 0 || (count > 0 && !descs) || !check_tile(tile_cols)) return false;
    if (!make_plan(count, descs, tile_cols, &b->p, &bad)) return false;
    *ws_bytes = (size_t)b->p.h.total;
    return true;
}

size_t batch_plan_image_bytes(const BatchPlan* b) { return image_bytes(b->p, true); }

bto_status batch_plan_submit(const BatchPlan* b, void* ws, size_t ws_bytes, void* staging, size_t staging_bytes,
                             cudaStream_t st) {
    // The serving loop: its slots run side by side, so no cooperative launch
    // that would hold every SM.
    return submit_plan(b->p, ws, ws_bytes, staging, staging_bytes, st, false);
}

}  // namespace bto

using namespace bto;

// Testing (declared in bto.h's testing section): the batched sweep's
// assignment of a list of items to the blocks of a grid, on the host.
extern "C" bto_status bto_debug_lpt(int64_t count, const double* cost, int grid, int32_t* block) {
    clear_invalid_arg();
    if (count < 0) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (count > 0 && !cost) { set_invalid_arg(2); return BTO_ERR_INVALID_VALUE; }
    for (int64_t k = 0; k < count; k++)
        if (!(cost[k] >= 0.0) || (k > 0 && cost[k] > cost[k - 1])) { set_invalid_arg(2); return BTO_ERR_INVALID_VALUE; }
    if (grid < 1 || grid > 65536) { set_invalid_arg(3); return BTO_ERR_INVALID_VALUE; }
    if (count > 0 && !block) { set_invalid_arg(4); return BTO_ERR_INVALID_VALUE; }
    if (count > 0) lpt_blocks(cost, count, grid, block);
    return BTO_OK;
}

extern "C" bto_status bto_batch_workspace_bytes(int count, const bto_batch_desc* descs, int tile_cols,
                                                size_t* bytes) {
    clear_invalid_arg();
    if (count < 0) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (count > 0 && !descs) { set_invalid_arg(2); return BTO_ERR_INVALID_VALUE; }
    if (tile_cols == 0) tile_cols = 128;
    if (!check_tile(tile_cols)) { set_invalid_arg(3); return BTO_ERR_INVALID_VALUE; }
    if (!bytes) { set_invalid_arg(4); return BTO_ERR_INVALID_VALUE; }
    Plan P;
    int bad = -1;
    if (!make_plan(count, descs, tile_cols, &P, &bad)) { set_invalid_arg(2); return BTO_ERR_INVALID_VALUE; }
    *bytes = (size_t)P.h.total;
    return BTO_OK;
}

extern "C" bto_status bto_batch_prepare(int count, const bto_batch_desc* descs, int tile_cols, void* ws,
                                        size_t ws_bytes, bto_stream_t stream) {
    clear_invalid_arg();
    if (count < 0) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (count > 0 && !descs) { set_invalid_arg(2); return BTO_ERR_INVALID_VALUE; }
    if (tile_cols == 0) tile_cols = 128;
    if (!check_tile(tile_cols)) { set_invalid_arg(3); return BTO_ERR_INVALID_VALUE; }
    Plan P;
    int bad = -1;
    if (!make_plan(count, descs, tile_cols, &P, &bad)) { set_invalid_arg(2); return BTO_ERR_INVALID_VALUE; }
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < (size_t)P.h.total) {
        set_invalid_arg(4);
        return BTO_ERR_WORKSPACE;
    }
    // Stage the plan in one host image and copy it with one transfer; the
    // counters are reset by bto_batch_run's first kernel.
    std::vector<char> img(image_bytes(P, false));
    write_image(P, img.data(), false, static_cast<char*>(ws));
    if (cudaMemcpyAsync(ws, img.data(), img.size(), cudaMemcpyHostToDevice, (cudaStream_t)stream) != cudaSuccess)
        return BTO_ERR_CUDA;
    // The host image is released on return: wait for the copy to leave it.
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return BTO_ERR_CUDA;
    note_fused(ws, fused_type(P));
    return BTO_OK;
}

extern "C" bto_status bto_batch_run(void* ws, size_t ws_bytes, bto_stream_t stream) {
    clear_invalid_arg();
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u)) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (ws_bytes < 1024) { set_invalid_arg(2); return BTO_ERR_WORKSPACE; }
    DeviceInfo dinf;
    if (!device_info(&dinf)) return BTO_ERR_CUDA;
    const int occ = batch_occupancy();
    if (occ == 0) return BTO_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    char* w = static_cast<char*>(ws);
    // A workspace prepared for the one-launch form: that launch alone.
    const int ft = fused_of(ws);
    if (ft >= 0) return bt_launch_fused(w, ft, st);
    const int grid = dinf.sms * occ;
    batch_reset_kernel<<<1, 256, 0, st>>>(w);
    if (cudaGetLastError() != cudaSuccess) return BTO_ERR_CUDA;
    // One kernel per queue, in order; a kernel whose queue is empty exits at once.
    batch_kernel<float, 0><<<grid, kThreads, kSmemBytes, st>>>(w);
    batch_kernel<float, 1><<<grid, kThreads, kSmemBytes, st>>>(w);
    batch_kernel<__nv_bfloat16, 0><<<grid, kThreads, kSmemBytes, st>>>(w);
    batch_kernel<__nv_bfloat16, 1><<<grid, kThreads, kSmemBytes, st>>>(w);
    const bto_status e = launch_status();
    if (e != BTO_OK) return e;
    // The TMA path's kernels read their counts from the workspace (none: they return at once).
    return bt_launch(w, nullptr, st);
}

// Fault injection for tests (bto.h's testing section): the one-launch form
// of a prepared workspace with block `stall_block` never arriving at the grid
// barriers, so that every wait expires after `timeout_ms`.
extern "C" bto_status bto_debug_batch_stall(void* ws, size_t ws_bytes, int stall_block, int timeout_ms,
                                            bto_stream_t stream) {
    clear_invalid_arg();
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u)) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (ws_bytes < 1024) { set_invalid_arg(2); return BTO_ERR_WORKSPACE; }
    if (timeout_ms < 1 || timeout_ms > 10000) { set_invalid_arg(4); return BTO_ERR_INVALID_VALUE; }
    const int ft = fused_of(ws);
    if (ft < 0) return BTO_ERR_UNSUPPORTED;
    return bt_launch_fused(static_cast<char*>(ws), ft, (cudaStream_t)stream, stall_block,
                           (unsigned long long)timeout_ms * 1000000ull);
}

extern "C" bto_status bto_batch_one_launch(const void* ws, int* one) {
    clear_invalid_arg();
    if (!ws) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (!one) { set_invalid_arg(2); return BTO_ERR_INVALID_VALUE; }
    *one = fused_of(ws) >= 0 ? 1 : 0;
    return BTO_OK;
}

extern "C" bto_status bto_batch_submit(int count, const bto_batch_desc* descs, int tile_cols, void* ws,
                                       size_t ws_bytes, void* staging, size_t staging_bytes,
                                       bto_stream_t stream) {
    clear_invalid_arg();
    if (count < 0) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (count > 0 && !descs) { set_invalid_arg(2); return BTO_ERR_INVALID_VALUE; }
    if (tile_cols == 0) tile_cols = 128;
    if (!check_tile(tile_cols)) { set_invalid_arg(3); return BTO_ERR_INVALID_VALUE; }
    Plan P;
    int bad = -1;
    if (!make_plan(count, descs, tile_cols, &P, &bad)) { set_invalid_arg(2); return BTO_ERR_INVALID_VALUE; }
    const bto_status e = submit_plan(P, ws, ws_bytes, staging, staging_bytes, (cudaStream_t)stream, true);
    if (e == BTO_ERR_WORKSPACE) set_invalid_arg(4);
    return e;
}
