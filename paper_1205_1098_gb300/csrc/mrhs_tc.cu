// Multi-right-hand-side BICGK on the 5th-generation tensor cores:
//   Q <- A P,  S <- A^T R   (A m x n BF16, P n x k, R m x k BF16; Q, S FP32)
// With k right-hand sides the two products of the BiCGK kernel (Table 1) form
// a dense contraction (4mnk flops over 2mn bytes of A), so they run as
// tcgen05.mma (kind::f16: BF16 inputs, FP32 accumulation in tensor memory).
// As in the fused form, every tile of A is read from HBM once and feeds both
// products.
//
// Work decomposition.  Columns are cut into panels of 512 (four 128-column
// sub-panels), rows into 128-row tiles; a work unit is (panel, row tile), and
// units are numbered panel-major.  A persistent grid of G <= #SM blocks gives
// block b the contiguous units [b U / G, (b+1) U / G), so a block walks down
// one panel (or the end of one and the start of the next).  Per unit it
// processes four 128 x 128 A tiles (one per sub-panel):
//   S_c += A_tile^T R_tile   (A read K-major: K = rows)
//   Q   += A_tile P_c        (A read MN-major: K = columns)
// The four S_c (128 x k each) stay in tensor memory while the block stays in
// a panel (a "segment"); Q (128 x k, double-buffered when 6k <= 512 columns)
// is read out after each unit.  Per-unit Q partials and per-segment S
// partials go to the workspace; a combine kernel adds them in a fixed order
// (compensated FP32), so results are reproducible bit for bit.  A is loaded
// with an L2 evict-first policy so that the partials (tens of MB) stay in L2
// until the combine reads them; the combine then discards their lines from
// L2 so that they are not written back to HBM.
//
// Two main kernels compute the same MMAs in the same order (so the same
// bits):
//  * mrhs_tma_kernel, when A, P and R allow tensor maps (16-byte aligned
//    bases, leading dimensions multiples of 8): warp 0 issues TMA copies of
//    128-byte-swizzled tiles into an NS-stage ring, warp 1 issues the MMAs,
//    warps 2-5 read Q and S out of tensor memory; mbarriers connect them.
//  * mrhs_ldg_kernel otherwise: all threads copy 16-byte chunks with
//    cp.async into an unswizzled core-matrix layout, NS - 1 tiles ahead.
//
// Waits are bounded (%globaltimer, 1 s): on expiry the status word at the
// start of the workspace records BTO_ERR_TIMEOUT, later waits and MMAs are
// skipped, copies and MMAs in flight are drained (again bounded), and the
// block frees its tensor memory before it exits.
#include "check.cuh"
#include "tma.cuh"

namespace bto {
namespace {

constexpr int kTile = 128;                  // A tile: 128 rows x 128 columns
constexpr int kSub = 4;                     // sub-panels per panel
constexpr int kPanel = kTile * kSub;        // 512 columns
constexpr int kTileBytes = kTile * kTile * 2;
constexpr uint32_t kTmemCols = 512;
constexpr int kMaxStages = 4;
constexpr unsigned long long kWaitNs = 1000000000ull;

struct MrhsArgs {
    int64_t m, n; int k;
    const uint16_t* A; int64_t lda;
    const uint16_t* P; int64_t ldp;
    const uint16_t* R; int64_t ldr;
    float* qpart; float* spart;             // [NP][k][ldqp], [G+NP-1][k][512]
    int64_t ldqp;
    int64_t nrt, U; int G, NS;
    int* status;
};

// Shared-memory matrix descriptor: start address, leading byte offset,
// stride byte offset (16-byte units), descriptor version 1 at bit 46 and the
// layout (0 = no swizzle, 2 = 128-byte swizzle) at bit 61.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)layout << 61;
    return d;
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, A K-major
// (0) or MN-major (1), B K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t idesc(int N, int a_mn_major) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn_major << 15) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTile >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(dtm), "l"(ad), "l"(bd), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* slot) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(slot)), "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_free(uint32_t tm) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(kTmemCols));
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint64_t evict_first_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Tile bookkeeping shared by both kernels: tile t of a block is sub-panel
// c = t % 4 of its unit v = t / 4 (global unit u0 + v = panel * nrt + row
// tile).  The two divisions happen once per block; positions of later units
// follow by carrying, since 64-bit division is slow on the GPU.
struct Sched {
    int64_t u0, u1, nrt, p0, r0;
    __device__ Sched(const MrhsArgs& a) {
        u0 = (int64_t)blockIdx.x * a.U / a.G;
        u1 = ((int64_t)blockIdx.x + 1) * a.U / a.G;
        nrt = a.nrt;
        p0 = u0 / nrt;
        r0 = u0 - p0 * nrt;
    }
    __device__ int tiles() const { return (int)(u1 - u0) * kSub; }
    __device__ int units() const { return (int)(u1 - u0); }
    // Panel and row tile of unit v.
    __device__ void pos(int v, int64_t& p, int64_t& r) const {
        p = p0;
        r = r0 + v;
        while (r >= nrt) { r -= nrt; p++; }
    }
    __device__ bool seg_first(int v) const { int64_t p, r; pos(v, p, r); return v == 0 || r == 0; }
    __device__ bool seg_last(int v) const { int64_t p, r; pos(v, p, r); return u0 + v + 1 == u1 || r == nrt - 1; }
    __device__ int64_t panel(int v) const { int64_t p, r; pos(v, p, r); return p; }
    __device__ int64_t row_tile(int v) const { int64_t p, r; pos(v, p, r); return r; }
};

// Q of unit v (one tensor-memory lane per row) -> qpart[p][j][row]; the
// calling warp reads lanes 32 * quarter .. + 31, columns j0 .. in steps of jstep.
__device__ __forceinline__ void store_q(const MrhsArgs& a, const Sched& sc, int v, uint32_t tq, int quarter,
                                        int lane, int jfirst, int jstep) {
    const int64_t p = sc.panel(v), row = sc.row_tile(v) * kTile + quarter * 32 + lane;
    const uint32_t t = tq + ((uint32_t)(quarter * 32) << 16);
    for (int j0 = jfirst; j0 < a.k; j0 += jstep) {
        uint32_t x[16];
        tmem_ld16(t + (uint32_t)j0, x);
        if (row < a.m) {
            float* q = a.qpart + (p * a.k + j0) * a.ldqp + row;
#pragma unroll
            for (int j = 0; j < 16; j++) q[j * a.ldqp] = __uint_as_float(x[j]);
        }
    }
}

// The four S_c of the segment ending at unit v -> spart[slot b + p][j][c * 128 + lane row].
__device__ __forceinline__ void store_s(const MrhsArgs& a, const Sched& sc, int v, uint32_t tm, int quarter,
                                        int lane, int jfirst, int jstep) {
    const int64_t p = sc.panel(v);
    float* base = a.spart + ((int64_t)blockIdx.x + p) * a.k * kPanel;
    for (int c = 0; c < kSub; c++) {
        const int cc = c * kTile + quarter * 32 + lane;
        const bool ok = p * kPanel + cc < a.n;
        for (int j0 = jfirst; j0 < a.k; j0 += jstep) {
            uint32_t x[16];
            tmem_ld16(tm + (uint32_t)(c * a.k + j0) + ((uint32_t)(quarter * 32) << 16), x);
            if (ok) {
#pragma unroll
                for (int j = 0; j < 16; j++) base[(int64_t)(j0 + j) * kPanel + cc] = __uint_as_float(x[j]);
            }
        }
    }
}

__device__ __forceinline__ void set_abort(volatile int* abortp, int* status) {
    if (!*abortp) {
        atomicExch(status, (int)BTO_ERR_TIMEOUT);
        *abortp = 1;
    }
}

// ===================================================================== TMA path
// Operand tiles in shared memory, 128-byte swizzled, as TMA writes them:
//   A tile: two boxes {64 rows, 128 columns}; each column is a 128-byte line
//           of 64 rows.  Read K-major (S: M = columns, K = rows): 32-byte
//           steps along K inside a line, box 1 at +16 KB; 8-line groups at
//           1024 bytes.  Read MN-major (Q: M = rows, K = columns): the two
//           64-row halves at 16 KB (leading offset), 8-column groups at 1024
//           bytes (stride offset), 2048 bytes per 16-column K step.
//   P_c, R: two boxes {64 K values, k right-hand sides}, K-major like A's
//           K-major reading (box 1 at + 128 k bytes).

constexpr int kTmaThreads = 192;            // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue

__global__ void __launch_bounds__(kTmaThreads, 1)
mrhs_tma_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mP,
                const __grid_constant__ CUtensorMap mR, const MrhsArgs a) {
    extern __shared__ uint8_t smraw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    const int k = a.k, NS = a.NS;
    const uint32_t bk = (uint32_t)kTile * k * 2;        // one 128 x k operand (two boxes)
    uint8_t* sP = base;                                   // [4][bk]
    uint8_t* sR = sP + 4 * bk;                            // [2][bk]
    uint8_t* sA = sR + 2 * bk;                            // [NS][32 KB]
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], qfull[2], qempty[2], sfull, sempty;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    volatile int* abortp = &s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Sched sc(a);
    const int T = sc.tiles(), V = sc.units();
    const bool qdb = 6 * k <= (int)kTmemCols;

    if (threadIdx.x == 0) {
        // This call's status starts at BTO_OK (a timeout needs a second of waiting).
        if (blockIdx.x == 0) *a.status = BTO_OK;
        // The combine may be scheduled now; it waits for this grid to finish.
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        for (int s = 0; s < NS; s++) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int b = 0; b < 2; b++) { mbar_init(&qfull[b], 1); mbar_init(&qempty[b], 4); }
        mbar_init(&sfull, 1);
        mbar_init(&sempty, 4);
        *abortp = 0;
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(&s_tmem);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = s_tmem;

    if (warp == 0) {
        if (lane == 0) {
            // Producer: TMA copies of tile t into stage t % NS once the MMAs of
            // tile t - NS (the stage's previous user) completed.
            const uint64_t pol = evict_first_policy();
            int issued = 0, s = 0;
            uint32_t ph = 0;                       // (t / NS) & 1
            for (int t = 0; t < T && !*abortp; t++, s = (s + 1 == NS) ? (ph ^= 1u, 0) : s + 1) {
                const int v = t / kSub, c = t % kSub;
                if (t >= NS && !mbar_wait_bounded(&empty[s], ph ^ 1u, kWaitNs, abortp)) {
                    set_abort(abortp, a.status);
                    break;
                }
                int64_t p, r;
                sc.pos(v, p, r);
                const bool sf = v == 0 || r == 0;
                const int R0 = (int)(r * kTile);
                const int C0 = (int)(p * kPanel + c * kTile);
                mbar_arrive_expect_tx(&full[s], (uint32_t)kTileBytes + (c == 0 ? bk : 0u) + (sf ? bk : 0u));
                uint8_t* dA = sA + s * kTileBytes;
                tma_load_2d_hint(dA, &mA, R0, C0, &full[s], pol);
                tma_load_2d_hint(dA + kTileBytes / 2, &mA, R0 + 64, C0, &full[s], pol);
                if (c == 0) {
                    // R rows of this unit; the buffer's previous user (unit v - 2) is done.
                    uint8_t* dR = sR + (v & 1) * bk;
                    tma_load_2d(dR, &mR, R0, 0, &full[s]);
                    tma_load_2d(dR + bk / 2, &mR, R0 + 64, 0, &full[s]);
                }
                if (sf) {
                    // P rows of sub-panel c at a segment start; its previous
                    // user, tile t - 4, is done since NS <= 4.
                    uint8_t* dP = sP + c * bk;
                    tma_load_2d(dP, &mP, C0, 0, &full[s]);
                    tma_load_2d(dP + bk / 2, &mP, C0 + 64, 0, &full[s]);
                }
                issued = t + 1;
            }
            // Drain: copies in flight complete before the block exits.
            for (int t = issued > NS ? issued - NS : 0; t < issued; t++)
                mbar_wait_timed(&full[t % NS], (uint32_t)((t / NS) & 1), kWaitNs);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idS = idesc(k, 0), idQ = idesc(k, 1);
            int seg = 0, issued = 0, s = 0;
            uint32_t ph = 0;                       // (t / NS) & 1
            for (int t = 0; t < T && !*abortp; t++, s = (s + 1 == NS) ? (ph ^= 1u, 0) : s + 1) {
                const int v = t / kSub, c = t % kSub;
                int64_t p, r;
                sc.pos(v, p, r);
                const bool sf = v == 0 || r == 0;
                const bool sl = v + 1 == V || r == sc.nrt - 1;
                const int qb = qdb ? (v & 1) : 0, nq = qdb ? (v >> 1) : v;
                bool ok = mbar_wait_bounded(&full[s], ph, kWaitNs, abortp);
                if (ok && c == 0 && nq >= 1) ok = mbar_wait_bounded(&qempty[qb], (uint32_t)((nq - 1) & 1), kWaitNs, abortp);
                if (ok && c == 0 && sf && seg >= 1) ok = mbar_wait_bounded(&sempty, (uint32_t)((seg - 1) & 1), kWaitNs, abortp);
                if (!ok) { set_abort(abortp, a.status); break; }
                tc_fence_after();
                const uint32_t aA = smem_u32(sA + s * kTileBytes);
                const uint32_t aR = smem_u32(sR + (v & 1) * bk);
                const uint32_t aP = smem_u32(sP + c * bk);
                const uint32_t tS = tm + (uint32_t)(c * k), tQ = tm + (uint32_t)(kSub * k + qb * k);
                // The descriptors of the eight K steps differ only in the start
                // address (bits 0-13, in 16-byte units; shared-memory addresses
                // stay below 2^18, so the field never carries): form each base
                // once and add the steps' offsets.
                const uint64_t dS0 = sdesc(aA, 16, 1024, 2), dQ0 = sdesc(aA, kTileBytes / 2, 1024, 2);
                const uint64_t dR0 = sdesc(aR, 16, 1024, 2), dP0 = sdesc(aP, 16, 1024, 2);
                const uint64_t bh = (uint64_t)(bk / 2) >> 4;
#pragma unroll
                for (int ks = 0; ks < kTile / 16; ks++) {
                    const uint64_t oA = (uint64_t)(((ks >> 2) * (kTileBytes / 2) + (ks & 3) * 32) >> 4);
                    const uint64_t oB = (uint64_t)(ks >> 2) * bh + (uint64_t)((ks & 3) * 2);
                    mma(tS, dS0 + oA, dR0 + oB, idS, (!sf || ks > 0) ? 1u : 0u);
                    mma(tQ, dQ0 + (uint64_t)(ks * 128), dP0 + oB, idQ, (c > 0 || ks > 0) ? 1u : 0u);
                }
                mma_commit(&empty[s]);
                if (c == kSub - 1) mma_commit(&qfull[qb]);
                if (c == kSub - 1 && sl) { mma_commit(&sfull); seg++; }
                issued = t + 1;
            }
            // Drain: the last MMAs complete before tensor memory is freed.
            if (issued > 0) mbar_wait_timed(&empty[(issued - 1) % NS], (uint32_t)(((issued - 1) / NS) & 1), kWaitNs);
        }
    } else {
        // Epilogue warps 2-5: tensor-memory lanes 32 * (warp % 4) ..
        const int quarter = warp & 3;
        int seg = 0;
        for (int v = 0; v < V && !*abortp; v++) {
            const int qb = qdb ? (v & 1) : 0, nq = qdb ? (v >> 1) : v;
            if (!mbar_wait_bounded(&qfull[qb], (uint32_t)(nq & 1), kWaitNs, abortp)) { set_abort(abortp, a.status); break; }
            tc_fence_after();
            store_q(a, sc, v, tm + (uint32_t)(kSub * k + qb * k), quarter, lane, 0, 16);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&qempty[qb]);
            if (sc.seg_last(v)) {
                if (!mbar_wait_bounded(&sfull, (uint32_t)(seg & 1), kWaitNs, abortp)) { set_abort(abortp, a.status); break; }
                tc_fence_after();
                store_s(a, sc, v, tm, quarter, lane, 0, 16);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sempty);
                seg++;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        tmem_free(tm);
    }
}

// ===================================================================== cp.async path
constexpr int kLdgThreads = 256;

__device__ __forceinline__ void cp16(uint32_t dst, const uint16_t* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp16_hint(uint32_t dst, const uint16_t* src, uint64_t pol) {
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void cp_wait_pending(int pending) {
    if (pending <= 0) cp_wait<0>();
    else if (pending == 1) cp_wait<1>();
    else cp_wait<2>();
}

// One 16-byte chunk of 8 consecutive BF16 values src[0..valid) (zeros past
// `valid`) into shared memory at `dst`; cp.async when whole and aligned.
__device__ __forceinline__ void chunk(uint16_t* dst, const uint16_t* src, int valid, bool hint, uint64_t pol) {
    if (valid == 8 && (reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
        if (hint) cp16_hint(smem_u32(dst), src, pol);
        else cp16(smem_u32(dst), src);
    } else {
        uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
        for (int e = 0; e < 8; e++)
            if (e < valid) w[e >> 1] |= (uint32_t)src[e] << (16 * (e & 1));
        *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Unswizzled core-matrix layout (128 along K): the chunk of 8 consecutive K
// values of line j (a column of A, or a right-hand side) in K-group g sits at
// ((j / 8) * 16 + g) * 128 + (j % 8) * 16 bytes.  Thread ids map j % 8
// fastest, so eight consecutive threads fill one 128-byte row of shared
// memory.

// A tile rows [R0, R0+128) x columns [C0, C0+128).
__device__ __forceinline__ void load_a(uint16_t* dst, const MrhsArgs& a, int64_t R0, int64_t C0, uint64_t pol) {
#pragma unroll 2
    for (int id = threadIdx.x; id < 16 * kTile; id += kLdgThreads) {
        const int jl = id & 7, g = (id >> 3) & 15, jg = id >> 7;
        const int64_t col = C0 + jg * 8 + jl, row = R0 + 8 * g;
        int valid = 0;
        if (col < a.n && row < a.m) valid = a.m - row < 8 ? (int)(a.m - row) : 8;
        chunk(dst + ((jg * 16 + g) * 128 + jl * 16) / 2, valid > 0 ? a.A + col * a.lda + row : a.A, valid, true, pol);
    }
}

// 128 (K) x k operand from column-major X: K rows [K0, K0+128) of the k columns.
__device__ __forceinline__ void load_k(uint16_t* dst, const uint16_t* X, int64_t ldx, int64_t K0, int64_t Klim, int k) {
    for (int id = threadIdx.x; id < 16 * k; id += kLdgThreads) {
        const int jl = id & 7, g = (id >> 3) & 15, jg = id >> 7;
        const int64_t kk = K0 + 8 * g;
        int valid = 0;
        if (kk < Klim) valid = Klim - kk < 8 ? (int)(Klim - kk) : 8;
        chunk(dst + ((jg * 16 + g) * 128 + jl * 16) / 2, valid > 0 ? X + (int64_t)(jg * 8 + jl) * ldx + kk : X,
              valid, false, 0);
    }
}

__global__ void __launch_bounds__(kLdgThreads, 1) mrhs_ldg_kernel(const MrhsArgs a) {
    extern __shared__ __align__(1024) uint16_t sm[];
    const int k = a.k, NS = a.NS;
    uint16_t* sP = sm;                                  // [4][128 x k]
    uint16_t* sR = sP + kSub * kTile * k;               // [2][128 x k]
    uint16_t* sA = sR + 2 * kTile * k;                  // [NS][128 x 128]
    __shared__ __align__(8) uint64_t bars[kMaxStages];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    volatile int* abortp = &s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quarter = warp & 3, half = warp >> 2;
    const uint64_t pol = evict_first_policy();
    const Sched sc(a);
    const int T = sc.tiles();
    const bool qdb = 6 * k <= (int)kTmemCols;

    if (threadIdx.x == 0) {
        if (blockIdx.x == 0) *a.status = BTO_OK;
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        for (int s = 0; s < NS; s++) mbar_init(&bars[s], 1);
        *abortp = 0;
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&s_tmem);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = s_tmem;
    const uint32_t idS = idesc(k, 0), idQ = idesc(k, 1);

    // Loads of tile t (A, plus R / P when its unit / segment starts) as one group.
    auto load_tile = [&](int t) {
        if (t < T) {
            const int v = t / kSub, c = t % kSub;
            const int64_t R0 = sc.row_tile(v) * kTile, C0 = sc.panel(v) * kPanel + c * kTile;
            load_a(sA + (t % NS) * (kTile * kTile), a, R0, C0, pol);
            if (c == 0) load_k(sR + (v & 1) * (kTile * k), a.R, a.ldr, R0, a.m, k);
            if (sc.seg_first(v)) load_k(sP + c * (kTile * k), a.P, a.ldp, C0, a.n, k);
        }
        cp_commit();
    };
    auto wait_tile = [&](int t) {
        if (*abortp) return;
        if (!mbar_wait_bounded(&bars[t % NS], (uint32_t)((t / NS) & 1), kWaitNs, abortp)) set_abort(abortp, a.status);
    };
    auto qaddr = [&](int v) { return tm + (uint32_t)(kSub * k + ((qdb && (v & 1)) ? k : 0)); };

    int issued = 0;
    for (int t = 0; t < NS - 1; t++) load_tile(t);
    for (int t = 0; t < T; t++) {
        const int v = t / kSub, c = t % kSub;
        const bool sf = sc.seg_first(v);
        const bool unit_last = c == kSub - 1;
        const bool seg_last = unit_last && sc.seg_last(v);
        const bool sync_read = seg_last || (unit_last && !qdb);
        // Tile t's group has landed once at most NS-2 newer groups are pending.
        cp_wait_pending(NS - 2);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0 && !*abortp) {
            tc_fence_after();
            const uint32_t aA = smem_u32(sA + (t % NS) * (kTile * kTile));
            const uint32_t aR = smem_u32(sR + (v & 1) * (kTile * k));
            const uint32_t aP = smem_u32(sP + c * (kTile * k));
            const uint32_t tS = tm + (uint32_t)(c * k);
#pragma unroll
            for (int ks = 0; ks < kTile / 16; ks++) {
                mma(tS, sdesc(aA + ks * 256, 128, 2048, 0), sdesc(aR + ks * 256, 128, 2048, 0), idS,
                    (!sf || ks > 0) ? 1u : 0u);
                mma(qaddr(v), sdesc(aA + ks * 4096, 2048, 128, 0), sdesc(aP + ks * 256, 128, 2048, 0), idQ,
                    (c > 0 || ks > 0) ? 1u : 0u);
            }
            mma_commit(&bars[t % NS]);
        }
        issued = t + 1;
        // The stage refilled next was read by tile t-1.
        if (t > 0) wait_tile(t - 1);
        load_tile(t + NS - 1);
        if (qdb && c == 0 && t > 0 && !sf) {
            // Unit v-1 ended at tile t-1 inside its segment: its Q buffer is
            // read out while tile t's MMAs (into the other buffer) run.
            tc_fence_after();
            store_q(a, sc, v - 1, qaddr(v - 1), quarter, lane, half * 16, 32);
        }
        if (sync_read) {
            wait_tile(t);
            tc_fence_after();
            store_q(a, sc, v, qaddr(v), quarter, lane, half * 16, 32);
            if (seg_last) store_s(a, sc, v, tm, quarter, lane, half * 16, 32);
        }
        tc_fence_before();
        if (sync_read) __syncthreads();
    }
    cp_wait<0>();
    if (*abortp && threadIdx.x == 0 && issued > 0)
        mbar_wait_timed(&bars[(issued - 1) % NS], (uint32_t)(((issued - 1) / NS) & 1), kWaitNs);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_free(tm);
}

// ===================================================================== combine
// Fixed-order compensated FP32 sums (TwoSum), four consecutive outputs per
// thread (float4 loads), 512 outputs per block, blockIdx.y = right-hand side j:
//   Q[i + j ldq] = sum_p qpart[p][j][i]                 (p = 0 .. NP-1)
//   S[c + j lds] = sum_b spart[b + p][j][c mod 512]    (b over the blocks of panel p = c / 512)
// Blocks 0 .. ceil(m/512)-1 produce Q, the rest S (one panel per block).
// After reading, the block discards the partials' 128-byte lines from L2.
constexpr int kCombThreads = 128;
constexpr int kCombSpan = 4 * kCombThreads;             // 512 outputs per block

__device__ __forceinline__ void two_sum_acc(float& s, float& e, float x) {
    const float t = s + x, bp = t - s;
    e += (s - (t - bp)) + (x - bp);
    s = t;
}
__device__ __forceinline__ void two_sum_acc4(float4& s, float4& e, const float4 x) {
    two_sum_acc(s.x, e.x, x.x);
    two_sum_acc(s.y, e.y, x.y);
    two_sum_acc(s.z, e.z, x.z);
    two_sum_acc(s.w, e.w, x.w);
}

__global__ void __launch_bounds__(kCombThreads)
mrhs_combine(const float* __restrict__ qpart, const float* __restrict__ spart, int64_t m, int64_t n, int k,
             int NP, int64_t ldqp, int64_t nrt, int64_t U, int G, int qblocks, float* Q, int64_t ldq, float* S,
             int64_t lds) {
    // Launched as a programmatic dependent of the main kernel: wait until it
    // has finished and its partials are visible.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int j = blockIdx.y;
    const bool isq = (int)blockIdx.x < qblocks;
    const int64_t e0 = (int64_t)(isq ? blockIdx.x : blockIdx.x - qblocks) * kCombSpan;
    const int64_t len = isq ? m : n;
    const float* base;          // this block's slice of the first partial
    int64_t stride;             // distance between consecutive partials
    int cnt;
    if (isq) {
        base = qpart + (int64_t)j * ldqp + e0;
        stride = (int64_t)k * ldqp;
        cnt = NP;
    } else {
        const int64_t p = e0 / kPanel;
        const int64_t blo = ((p * nrt + 1) * G - 1) / U, bhi = (((p + 1) * nrt) * G - 1) / U;
        base = spart + ((blo + p) * k + j) * kPanel;
        stride = (int64_t)k * kPanel;
        cnt = (int)(bhi - blo + 1);
    }
    const int64_t e = e0 + 4 * threadIdx.x;
    if (e < len) {
        const float* src = base + 4 * threadIdx.x;
        float4 sm = make_float4(0.f, 0.f, 0.f, 0.f), er = sm;
        int i = 0;
        for (; i + 4 <= cnt; i += 4) {
            const float4 x0 = *reinterpret_cast<const float4*>(src + (i + 0) * stride);
            const float4 x1 = *reinterpret_cast<const float4*>(src + (i + 1) * stride);
            const float4 x2 = *reinterpret_cast<const float4*>(src + (i + 2) * stride);
            const float4 x3 = *reinterpret_cast<const float4*>(src + (i + 3) * stride);
            two_sum_acc4(sm, er, x0);
            two_sum_acc4(sm, er, x1);
            two_sum_acc4(sm, er, x2);
            two_sum_acc4(sm, er, x3);
        }
        for (; i < cnt; i++) two_sum_acc4(sm, er, *reinterpret_cast<const float4*>(src + i * stride));
        float* dst = isq ? Q + e + (int64_t)j * ldq : S + e + (int64_t)j * lds;
        const float r[4] = {sm.x + er.x, sm.y + er.y, sm.z + er.z, sm.w + er.w};
#pragma unroll
        for (int q = 0; q < 4; q++)
            if (e + q < len) dst[q] = r[q];
    }
    __syncthreads();
    // Lines that start below len lie inside this block's rows of the partials.
    for (int l = threadIdx.x; l < cnt * (kCombSpan / 32); l += kCombThreads) {
        const int i = l / (kCombSpan / 32), w = l % (kCombSpan / 32);
        if (e0 + 32 * w >= len) continue;
        const float* line = base + i * stride + 32 * w;
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(line) : "memory");
    }
}

// ===================================================================== host
struct MrhsPlan {
    int NP = 0, G = 0, NS = 2, NS_tma = 2;
    int64_t nrt = 0, U = 0, ldqp = 0;
    size_t smem = 0, smem_tma = 0, q_bytes = 0, s_bytes = 0, ws = 0;
};

MrhsPlan mrhs_plan(int64_t m, int64_t n, int k, const DeviceInfo& d) {
    MrhsPlan p;
    p.ldqp = round_up(std::max<int64_t>(m, 1), 32);
    if (m > 0 && n > 0) {
        p.NP = (int)ceil_div(n, kPanel);
        p.nrt = ceil_div(m, kTile);
        p.U = p.NP * p.nrt;
        p.G = (int)std::min<int64_t>(d.sms, p.U);
    }
    const int64_t fixed = (int64_t)(kSub + 2) * kTile * k * 2;
    // Static shared memory and the 1024-byte alignment slack come off the top.
    const int64_t room = (int64_t)d.max_smem_optin - fixed - 2048;
    p.NS = p.NS_tma = (int)std::max<int64_t>(2, std::min<int64_t>(kMaxStages, room / kTileBytes));
    p.smem = (size_t)fixed + (size_t)p.NS * kTileBytes;
    p.smem_tma = p.smem + 1024;
    p.q_bytes = round_up((int64_t)p.NP * k * p.ldqp * 4, 256);
    p.s_bytes = p.NP > 0 ? round_up((int64_t)(p.G + p.NP - 1) * k * kPanel * 4, 256) : 0;
    p.ws = 256 + p.q_bytes + p.s_bytes;
    return p;
}

bool valid_k(int64_t k) { return k >= 16 && k <= 96 && k % 16 == 0; }

// Tensor maps for A, P, R, when their layout allows (16-byte aligned bases,
// leading dimensions that are multiples of 8 elements, extents below 2^31).
bool tma_maps(const MrhsArgs& a, CUtensorMap* mA, CUtensorMap* mP, CUtensorMap* mR) {
    if (a.m > INT32_MAX || a.n > INT32_MAX) return false;
    const CUtensorMapDataType bf = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_128B;
    return encode_tmap_2d(mA, bf, 2, a.A, a.m, a.n, a.lda, 64, kTile, sw) &&
           encode_tmap_2d(mP, bf, 2, a.P, a.n, a.k, a.ldp, 64, (uint32_t)a.k, sw) &&
           encode_tmap_2d(mR, bf, 2, a.R, a.m, a.k, a.ldr, 64, (uint32_t)a.k, sw);
}

}  // namespace
}  // namespace bto

using namespace bto;

extern "C" bto_status bto_bicgk_mrhs_workspace_bytes(int64_t m, int64_t n, int64_t k, size_t* bytes) {
    clear_invalid_arg();
    if (m < 0) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (n < 0) { set_invalid_arg(2); return BTO_ERR_INVALID_VALUE; }
    if (!valid_k(k)) { set_invalid_arg(3); return BTO_ERR_INVALID_VALUE; }
    if (!bytes) { set_invalid_arg(4); return BTO_ERR_INVALID_VALUE; }
    DeviceInfo d;
    if (!device_info(&d)) return BTO_ERR_CUDA;
    *bytes = mrhs_plan(m, n, (int)k, d).ws;
    return BTO_OK;
}

extern "C" bto_status bto_bicgk_mrhs(int64_t m, int64_t n, int64_t k, const uint16_t* A, int64_t lda,
                                     const uint16_t* P, int64_t ldp, const uint16_t* R, int64_t ldr, float* Q,
                                     int64_t ldq, float* S, int64_t lds, void* ws, size_t ws_bytes,
                                     bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    c.size(1, m);
    c.size(2, n);
    if (!valid_k(k)) c.fail(3);
    if (!c.ok()) return c.finish();
    c.ptr(4, A, m > 0 && n > 0, 2); c.ld(5, lda, m);
    c.ptr(6, P, n > 0, 2); c.ld(7, ldp, n);
    c.ptr(8, R, m > 0, 2); c.ld(9, ldr, m);
    c.ptr(10, Q, m > 0, 4); c.ld(11, ldq, m);
    c.ptr(12, S, n > 0, 4); c.ld(13, lds, n);
    const size_t Ab = mat_extent_bytes(m, n, lda, 2), Pb = mat_extent_bytes(n, k, ldp, 2),
                 Rb = mat_extent_bytes(m, k, ldr, 2);
    const size_t Qb = mat_extent_bytes(m, k, ldq, 4), Sb = mat_extent_bytes(n, k, lds, 4);
    c.disjoint(10, Q, Qb, A, Ab); c.disjoint(10, Q, Qb, P, Pb); c.disjoint(10, Q, Qb, R, Rb);
    c.disjoint(10, Q, Qb, S, Sb);
    c.disjoint(12, S, Sb, A, Ab); c.disjoint(12, S, Sb, P, Pb); c.disjoint(12, S, Sb, R, Rb);
    if (!c.ok()) return c.finish();
    DeviceInfo d;
    if (!device_info(&d)) return BTO_ERR_CUDA;
    const MrhsPlan pl = mrhs_plan(m, n, (int)k, d);
    WsLayout L;
    L.total = pl.ws;
    c.ws(14, ws, ws_bytes, L);
    if (!c.ok()) return c.finish();
    cudaStream_t st = (cudaStream_t)stream;
    char* w = static_cast<char*>(ws);
    float* qpart = reinterpret_cast<float*>(w + 256);
    float* spart = reinterpret_cast<float*>(w + 256 + pl.q_bytes);
    if (pl.NP > 0) {
        MrhsArgs a{};
        a.m = m; a.n = n; a.k = (int)k;
        a.A = A; a.lda = lda; a.P = P; a.ldp = ldp; a.R = R; a.ldr = ldr;
        a.qpart = qpart; a.spart = spart; a.ldqp = pl.ldqp;
        a.nrt = pl.nrt; a.U = pl.U; a.G = pl.G;
        a.status = reinterpret_cast<int*>(w);
        CUtensorMap mA, mP, mR;
        if (tma_maps(a, &mA, &mP, &mR)) {
            a.NS = pl.NS_tma;
            if (cudaFuncSetAttribute(mrhs_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)pl.smem_tma) != cudaSuccess)
                return BTO_ERR_CUDA;
            mrhs_tma_kernel<<<pl.G, kTmaThreads, pl.smem_tma, st>>>(mA, mP, mR, a);
        } else {
            a.NS = pl.NS;
            if (cudaFuncSetAttribute(mrhs_ldg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem) !=
                cudaSuccess)
                return BTO_ERR_CUDA;
            mrhs_ldg_kernel<<<pl.G, kLdgThreads, pl.smem, st>>>(a);
        }
        if (cudaGetLastError() != cudaSuccess) return BTO_ERR_CUDA;
        const int qblocks = (int)ceil_div(m, kCombSpan), sblocks = (int)ceil_div(n, kCombSpan);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(qblocks + sblocks, (unsigned)k);
        cfg.blockDim = dim3(kCombThreads);
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaLaunchKernelEx(&cfg, mrhs_combine, (const float*)qpart, (const float*)spart, m, n, (int)k, pl.NP,
                               pl.ldqp, pl.nrt, pl.U, pl.G, qblocks, Q, ldq, S, lds) != cudaSuccess)
            return BTO_ERR_CUDA;
    } else {
        if (cudaMemsetAsync(w, 0, sizeof(int), st) != cudaSuccess) return BTO_ERR_CUDA;
        // An empty sum: Q = 0 (n = 0) and S = 0 (m = 0).
        for (int64_t j = 0; j < k; j++) {
            if (m > 0 && cudaMemsetAsync(Q + j * ldq, 0, (size_t)m * 4, st) != cudaSuccess) return BTO_ERR_CUDA;
            if (n > 0 && cudaMemsetAsync(S + j * lds, 0, (size_t)n * 4, st) != cudaSuccess) return BTO_ERR_CUDA;
        }
    }
    return launch_status();
}
