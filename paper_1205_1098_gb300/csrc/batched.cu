// Batched form: many independent, uneven BICGK and GEMVER instances (FP32
// storage) in one persistent launch.
//
// bto_batch_prepare builds a work list on the host and uploads it into the
// caller's workspace: one item per (instance, column panel) for BICGK and for
// GEMVER's first pass, one item per (instance, 256-row block) for GEMVER's
// second pass.  First-pass-like items come first, largest estimated cost
// first (longest-processing-time order), then the second-pass items.
// bto_batch_run launches a persistent grid (as many blocks as are resident)
// whose blocks pull items from a device counter, so the load balances itself
// and the launch contains no host synchronisation (it can be captured into a
// CUDA graph).
//
// Per item the arithmetic is that of the reduced-precision form: warps own
// 16-column groups, lanes own 8 rows (two 16-byte loads per column), FP32
// FMA chains folded into TwoSum (hi, lo) pairs, a transposing butterfly for
// column sums.  A BICGK instance split into P panels leaves P row-partial
// vectors; the panel that finishes last (per-instance counter) adds them in
// panel order in FP64.  A GEMVER second-pass item waits, bounded by
// %globaltimer, until every first-pass panel of its instance has published
// (release/acquire on the counter); the wait always ends because all those
// items were taken earlier by resident blocks.  Results do not depend on
// which block runs an item, so an instance gives the same bits alone or in a
// batch with the same panel width.
#include "check.cuh"
#include "lp_math.cuh"
#include <algorithm>
#include <cstring>
#include <vector>

namespace bto {
namespace {

using namespace lp;

constexpr int kThreads = 256;
constexpr int kWarps = 8;
constexpr int kRows = 256;                 // rows per chunk: 32 lanes x 8 rows
constexpr unsigned long long kWaitNs = 2000000000ull;

enum ItemKind { IT_BICGK = 0, IT_GEMVER1 = 1, IT_GEMVER2 = 2 };

struct Item { int32_t inst, kind, lo, hi; };

struct InstInfo {
    int32_t panels;        // first-pass panels of the instance
    int32_t vec;           // 16-byte loads allowed (A, B and their leading dimensions aligned)
    int64_t qoff;          // BICGK: offset (in float2) of its panel partials, -1 if one panel
};

struct Header {
    int32_t count, nitems, tile_cols, pad;
    int64_t off_desc, off_info, off_items, off_counters, off_qpart;
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

// Lane's k-th row within a 256-row chunk: two groups of four consecutive rows.
__device__ __forceinline__ int brow(int lane, int k) { return (k >> 2) * 128 + lane * 4 + (k & 3); }

template <bool COHERENT>
__device__ __forceinline__ void load8(const float* col, int64_t R0, int64_t m, int lane, bool vec, float (&a)[8]) {
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int64_t i = R0 + h * 128 + lane * 4;
        if (vec && i + 4 <= m) {
            const float4 t = COHERENT ? __ldcg(reinterpret_cast<const float4*>(col + i))
                                      : __ldg(reinterpret_cast<const float4*>(col + i));
            a[4 * h] = t.x; a[4 * h + 1] = t.y; a[4 * h + 2] = t.z; a[4 * h + 3] = t.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; e++) a[4 * h + e] = (i + e < m) ? (COHERENT ? __ldcg(col + i + e) : __ldg(col + i + e)) : 0.0f;
        }
    }
}

__device__ __forceinline__ void load_rows(const float* v, int64_t R0, int64_t m, int lane, float (&o)[8]) {
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const int64_t i = R0 + brow(lane, k);
        o[k] = (i < m) ? __ldg(v + i) : 0.0f;
    }
}

// Adds the warps' (hi, lo) row partials of one chunk (red: [2][kWarps][kRows])
// in warp order with TwoSum; thread t handles row t.
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

// First-pass item: columns [c0, c1) of instance d over all its rows.
// BICGK: s complete for the panel's columns, q partial (or complete).
// GEMVER: B = A + u1 v1^T + u2 v2^T for the panel, x complete for its columns.
template <int KIND>
__device__ void first_pass(const bto_batch_desc& d, const InstInfo& info, int panel, int64_t c0, int64_t c1,
                           float* red, float* shi, float* slo, float2* qpart) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m = d.m, ncols = c1 - c0;
    const bool vec = info.vec != 0;
    for (int k = threadIdx.x; k < ncols; k += kThreads) { shi[k] = 0.0f; slo[k] = 0.0f; }
    __syncthreads();
    const float* rvec = (KIND == IT_BICGK) ? d.in[1] : d.in[4];        // r, or GEMVER's y
    for (int64_t R0 = 0; R0 < m; R0 += kRows) {
        float rv[8], u1r[8], u2r[8], qhi[8], qlo[8];
        load_rows(rvec, R0, m, lane, rv);
        if (KIND == IT_GEMVER1) { load_rows(d.in[0], R0, m, lane, u1r); load_rows(d.in[2], R0, m, lane, u2r); }
#pragma unroll
        for (int k = 0; k < 8; k++) { qhi[k] = 0.0f; qlo[k] = 0.0f; }
        for (int64_t g0 = c0 + 16 * warp; g0 < c1; g0 += 16 * kWarps) {
            const int nc = (int)((c1 - g0) < 16 ? (c1 - g0) : 16);
            float sl[16], qt[8];
#pragma unroll
            for (int k = 0; k < 8; k++) qt[k] = 0.0f;
#pragma unroll
            for (int jb = 0; jb < 16; jb += 4) {
                float av[4][8];
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (jb + u < nc) load8<false>(d.A + (g0 + jb + u) * d.lda, R0, m, lane, vec, av[u]);
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int jj = jb + u;
                    if (jj < nc) {
                        const int64_t j = g0 + jj;
                        if (KIND == IT_BICGK) {
                            const float pj = __ldg(d.in[0] + j);
#pragma unroll
                            for (int k = 0; k < 8; k++) qt[k] = fmaf(av[u][k], pj, qt[k]);
                            float acc = av[u][0] * rv[0];
#pragma unroll
                            for (int k = 1; k < 8; k++) acc = fmaf(av[u][k], rv[k], acc);
                            sl[jj] = acc;
                        } else {
                            const float v1j = __ldg(d.in[1] + j), v2j = __ldg(d.in[3] + j);
                            float b[8];
#pragma unroll
                            for (int k = 0; k < 8; k++) b[k] = fmaf(u2r[k], v2j, fmaf(u1r[k], v1j, av[u][k]));
                            float* bc = d.B + j * d.ldb;
#pragma unroll
                            for (int h = 0; h < 2; h++) {
                                const int64_t i = R0 + h * 128 + lane * 4;
                                if (vec && i + 4 <= m) {
                                    *reinterpret_cast<float4*>(bc + i) = make_float4(b[4 * h], b[4 * h + 1], b[4 * h + 2], b[4 * h + 3]);
                                } else {
#pragma unroll
                                    for (int e = 0; e < 4; e++) if (i + e < m) bc[i + e] = b[4 * h + e];
                                }
                            }
                            float acc = b[0] * rv[0];
#pragma unroll
                            for (int k = 1; k < 8; k++) acc = fmaf(b[k], rv[k], acc);
                            sl[jj] = acc;
                        }
                    } else {
                        sl[jj] = 0.0f;
                    }
                }
            }
            if (KIND == IT_BICGK) {
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    float s2, e2;
                    two_sum(qhi[k], qt[k], s2, e2);
                    qhi[k] = s2; qlo[k] += e2;
                }
            }
            const float cs = butterfly16(sl, lane);
            if (lane < nc) {
                const int64_t o = g0 + lane - c0;
                float s2, e2;
                two_sum(shi[o], cs, s2, e2);
                shi[o] = s2; slo[o] += e2;
            }
        }
        if (KIND == IT_BICGK) {
#pragma unroll
            for (int k = 0; k < 8; k++) {
                red[warp * kRows + brow(lane, k)] = qhi[k];
                red[(kWarps + warp) * kRows + brow(lane, k)] = qlo[k];
            }
            __syncthreads();
            const int64_t i = R0 + threadIdx.x;
            if (i < m) {
                float hs, ls;
                warp_rows_sum(red, threadIdx.x, hs, ls);
                if (info.qoff < 0) d.out[0][i] = (float)((double)hs + (double)ls);
                else qpart[info.qoff + (int64_t)panel * m + i] = make_float2(hs, ls);
            }
            __syncthreads();
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < ncols; k += kThreads) {
        const double s = (double)shi[k] + (double)slo[k];
        if (KIND == IT_BICGK) d.out[1][c0 + k] = (float)s;
        else d.out[0][c0 + k] = (float)fma((double)d.beta, s, (double)__ldg(d.in[5] + c0 + k));
    }
}

// GEMVER second pass: w = alpha B x for rows [r0, r1) (r1 - r0 <= 256), all columns.
__device__ void gemver_second(const bto_batch_desc& d, const InstInfo& info, int64_t R0, float* red) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m = d.m, n = d.n;
    const bool vec = info.vec != 0;
    float qhi[8], qlo[8];
#pragma unroll
    for (int k = 0; k < 8; k++) { qhi[k] = 0.0f; qlo[k] = 0.0f; }
    for (int64_t g0 = 16 * warp; g0 < n; g0 += 16 * kWarps) {
        const int nc = (int)((n - g0) < 16 ? (n - g0) : 16);
        float qt[8];
#pragma unroll
        for (int k = 0; k < 8; k++) qt[k] = 0.0f;
#pragma unroll
        for (int jb = 0; jb < 16; jb += 4) {
            float av[4][8], xj[4];
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (jb + u < nc) {
                    load8<true>(d.B + (g0 + jb + u) * d.ldb, R0, m, lane, vec, av[u]);
                    xj[u] = __ldcg(d.out[0] + g0 + jb + u);
                }
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (jb + u < nc) {
#pragma unroll
                    for (int k = 0; k < 8; k++) qt[k] = fmaf(av[u][k], xj[u], qt[k]);
                }
        }
#pragma unroll
        for (int k = 0; k < 8; k++) {
            float s2, e2;
            two_sum(qhi[k], qt[k], s2, e2);
            qhi[k] = s2; qlo[k] += e2;
        }
    }
#pragma unroll
    for (int k = 0; k < 8; k++) {
        red[warp * kRows + brow(lane, k)] = qhi[k];
        red[(kWarps + warp) * kRows + brow(lane, k)] = qlo[k];
    }
    __syncthreads();
    const int64_t i = R0 + threadIdx.x;
    if (i < m) {
        float hs, ls;
        warp_rows_sum(red, threadIdx.x, hs, ls);
        d.out[1][i] = (float)((double)d.alpha * ((double)hs + (double)ls));
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads, 1) batch_kernel(char* ws) {
    const Header* h = reinterpret_cast<const Header*>(ws + kHeaderOff);
    const bto_batch_desc* descs = reinterpret_cast<const bto_batch_desc*>(ws + h->off_desc);
    const InstInfo* infos = reinterpret_cast<const InstInfo*>(ws + h->off_info);
    const Item* items = reinterpret_cast<const Item*>(ws + h->off_items);
    unsigned* counters = reinterpret_cast<unsigned*>(ws + h->off_counters);   // [0] queue, [1+i] instance
    float2* qpart = reinterpret_cast<float2*>(ws + h->off_qpart);
    int* status = reinterpret_cast<int*>(ws);
    __shared__ float red[2 * kWarps * kRows];
    extern __shared__ float sacc[];   // [2][tile_cols]
    float* shi = sacc;
    float* slo = sacc + h->tile_cols;
    __shared__ int s_item, s_ok, s_last;
    const int nitems = h->nitems;
    while (true) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counters, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        const Item item = items[it];
        const bto_batch_desc d = descs[item.inst];
        const InstInfo info = infos[item.inst];
        if (item.kind == IT_GEMVER2) {
            if (threadIdx.x == 0) {
                const unsigned long long t0 = gtimer();
                int ok = 1;
                while (ld_acquire_u32(counters + 1 + item.inst) < (unsigned)info.panels) {
                    if (gtimer() - t0 > kWaitNs) { ok = 0; atomicExch(status, (int)BTO_ERR_TIMEOUT); break; }
                    __nanosleep(100);
                }
                s_ok = ok;
            }
            __syncthreads();
            if (s_ok) gemver_second(d, info, item.lo, red);
            continue;
        }
        const int64_t c0 = item.lo, c1 = item.hi;
        const int panel = (int)(c0 / h->tile_cols);
        if (item.kind == IT_BICGK) first_pass<IT_BICGK>(d, info, panel, c0, c1, red, shi, slo, qpart);
        else first_pass<IT_GEMVER1>(d, info, panel, c0, c1, red, shi, slo, qpart);
        // Publish this panel (release); the last BICGK panel adds the row partials.
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned old = atomicAdd(counters + 1 + item.inst, 1u);
            s_last = (item.kind == IT_BICGK && info.qoff >= 0 && old == (unsigned)(info.panels - 1));
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            for (int64_t i = threadIdx.x; i < d.m; i += kThreads) {
                double s = 0.0;
                for (int p = 0; p < info.panels; p++) {
                    const float2 v = __ldcg(qpart + info.qoff + (int64_t)p * d.m + i);
                    s += (double)v.x + (double)v.y;
                }
                d.out[0][i] = (float)s;
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

constexpr size_t kSaccBytes = 2 * 1024 * sizeof(float);   // s (hi, lo) for panels up to 1024 columns

struct Plan {
    Header h{};
    std::vector<InstInfo> info;
    std::vector<Item> items;
};

bool make_plan(int count, const bto_batch_desc* descs, int tile_cols, Plan* P, int* bad_desc) {
    P->info.resize(count);
    std::vector<std::pair<double, Item>> first, second;
    int64_t qsize = 0;
    for (int i = 0; i < count; i++) {
        const bto_batch_desc& d = descs[i];
        const bool bicgk = d.op == BTO_OP_BICGK, gemver = d.op == BTO_OP_GEMVER;
        bool ok = (bicgk || gemver) && d.m >= 0 && d.n >= 0 && d.lda >= std::max<int64_t>(1, d.m);
        if (ok && d.m > 0 && d.n > 0) ok = d.A != nullptr;
        if (ok && gemver) ok = d.ldb >= std::max<int64_t>(1, d.m) && (d.m == 0 || d.n == 0 || d.B);
        const int nin = bicgk ? 2 : 6;
        for (int k = 0; ok && k < nin; k++) {
            // BICGK: p (n), r (m).  GEMVER: u1 (m), v1 (n), u2 (m), v2 (n), y (m), z (n).
            const int64_t len = bicgk ? (k == 0 ? d.n : d.m) : (k % 2 == 0 ? d.m : d.n);
            if (len > 0 && !d.in[k]) ok = false;
        }
        for (int k = 0; ok && k < 2; k++) {
            const int64_t len = bicgk ? (k == 0 ? d.m : d.n) : (k == 0 ? d.n : d.m);
            if (len > 0 && !d.out[k]) ok = false;
        }
        if (!ok) { *bad_desc = i; return false; }
        InstInfo& inf = P->info[i];
        const int64_t panels = d.n > 0 ? ceil_div(d.n, tile_cols) : 0;
        inf.panels = (int32_t)panels;
        inf.vec = aligned16(d.A) && d.lda % 4 == 0 && (!gemver || (aligned16(d.B) && d.ldb % 4 == 0));
        inf.qoff = -1;
        if (bicgk && panels > 1 && d.m > 0) { inf.qoff = qsize; qsize += panels * d.m; }
        if (d.n == 0 || d.m == 0) {
            // Degenerate instance: one first-pass item still writes the empty sums.
            if (d.n > 0) {
                for (int64_t c = 0; c < d.n; c += tile_cols)
                    first.push_back({0.0, Item{i, bicgk ? IT_BICGK : IT_GEMVER1, (int32_t)c,
                                               (int32_t)std::min<int64_t>(d.n, c + tile_cols)}});
            } else if (d.m > 0) {
                inf.panels = 0;
                if (bicgk) first.push_back({0.0, Item{i, IT_BICGK, 0, 0}});
            }
            if (gemver && d.m > 0)
                for (int64_t r = 0; r < d.m; r += kRows)
                    second.push_back({0.0, Item{i, IT_GEMVER2, (int32_t)r, (int32_t)std::min<int64_t>(d.m, r + kRows)}});
            continue;
        }
        for (int64_t c = 0; c < d.n; c += tile_cols) {
            const int64_t c1 = std::min<int64_t>(d.n, c + tile_cols);
            const double cost = (double)d.m * (double)(c1 - c) * (gemver ? 2.0 : 1.0);
            first.push_back({cost, Item{i, bicgk ? IT_BICGK : IT_GEMVER1, (int32_t)c, (int32_t)c1}});
        }
        if (gemver)
            for (int64_t r = 0; r < d.m; r += kRows) {
                const int64_t r1 = std::min<int64_t>(d.m, r + kRows);
                second.push_back({(double)(r1 - r) * (double)d.n, Item{i, IT_GEMVER2, (int32_t)r, (int32_t)r1}});
            }
    }
    auto by_cost = [](const std::pair<double, Item>& a, const std::pair<double, Item>& b) {
        if (a.first != b.first) return a.first > b.first;
        if (a.second.inst != b.second.inst) return a.second.inst < b.second.inst;
        return a.second.lo < b.second.lo;
    };
    std::stable_sort(first.begin(), first.end(), by_cost);
    std::stable_sort(second.begin(), second.end(), by_cost);
    for (auto& e : first) P->items.push_back(e.second);
    for (auto& e : second) P->items.push_back(e.second);
    Header& H = P->h;
    H.count = count;
    H.nitems = (int32_t)P->items.size();
    H.tile_cols = tile_cols;
    size_t cur = 256;
    auto region = [&](size_t bytes) { size_t at = cur; cur += round_up((int64_t)bytes, 256); return at; };
    H.off_desc = region((size_t)count * sizeof(bto_batch_desc));
    H.off_info = region((size_t)count * sizeof(InstInfo));
    H.off_items = region(P->items.size() * sizeof(Item));
    H.counters_bytes = (int64_t)(count + 1) * sizeof(unsigned);
    H.off_counters = region((size_t)H.counters_bytes);
    H.off_qpart = region((size_t)std::max<int64_t>(qsize, 1) * sizeof(float2));
    H.total = cur;
    return true;
}

bool check_tile(int tile_cols) { return tile_cols >= 16 && tile_cols <= 1024 && tile_cols % 16 == 0; }

}  // namespace
}  // namespace bto

using namespace bto;

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
    // Stage the plan in one host image and copy it with one transfer.
    std::vector<char> img((size_t)P.h.off_counters, 0);
    std::memcpy(img.data() + kHeaderOff, &P.h, sizeof(Header));
    if (count) std::memcpy(img.data() + P.h.off_desc, descs, (size_t)count * sizeof(bto_batch_desc));
    if (count) std::memcpy(img.data() + P.h.off_info, P.info.data(), P.info.size() * sizeof(InstInfo));
    if (!P.items.empty()) std::memcpy(img.data() + P.h.off_items, P.items.data(), P.items.size() * sizeof(Item));
    if (cudaMemcpyAsync(ws, img.data(), img.size(), cudaMemcpyHostToDevice, (cudaStream_t)stream) != cudaSuccess)
        return BTO_ERR_CUDA;
    // The host image is released on return: wait for the copy to leave it.
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return BTO_ERR_CUDA;
    return BTO_OK;
}

extern "C" bto_status bto_batch_run(void* ws, size_t ws_bytes, bto_stream_t stream) {
    clear_invalid_arg();
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u)) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (ws_bytes < 1024) { set_invalid_arg(2); return BTO_ERR_WORKSPACE; }
    DeviceInfo dinf;
    if (!device_info(&dinf)) return BTO_ERR_CUDA;
    static int occ = 0;
    if (occ == 0 &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel, kThreads, kSaccBytes) != cudaSuccess)
        return BTO_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    char* w = static_cast<char*>(ws);
    batch_reset_kernel<<<1, 256, 0, st>>>(w);
    if (cudaGetLastError() != cudaSuccess) return BTO_ERR_CUDA;
    batch_kernel<<<dinf.sms * std::max(occ, 1), kThreads, kSaccBytes, st>>>(w);
    return launch_status();
}
