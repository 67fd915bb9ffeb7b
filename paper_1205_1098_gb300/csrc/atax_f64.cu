// ATAX / BATAX (Table I; Section II, Fig. 1): y <- beta A^T (A x), with the
// temporary t = A x contracted (it never reaches device memory as a vector)
// and A streamed from HBM once.
//
// The paper's Max-Fuse result for BATAX partitions the rows (p(i)), fuses
// the two row loops, and keeps the two inner column loops apart because t_i
// is complete only after its whole row has been summed (Section III-D,
// Section IV-A).  Here a row band plays the role of the fused row loop:
//
//   - The cooperative grid (two blocks per SM, so that one block's
//     arithmetic covers the other's barriers and waits) is cut into NG
//     groups of S blocks (S = 16 for n <= 65536).  Group g takes the 16-row bands
//     g, g + NG, g + 2 NG, ...; inside a group, block r owns a fixed slice
//     of about n / S columns.
//   - Pass 1 over band b (the first column loop): lane l of a warp owns the
//     row pair 2 (l mod 8), 2 (l mod 8) + 1 of the band and every fourth of
//     the warp's columns, so a warp load covers four whole 128-byte column
//     segments and each lane keeps two partial t_i; two exchanges across the
//     column lanes and the warps, in a fixed order, give the block's partial
//     of t_b.  FP64 arithmetic is the bound on this part (2 FMA per clock per
//     SM), so the mapping keeps the adds outside the FMAs to four per lane
//     per band.  The S partials meet in a
//     double-buffered slot in L2 behind per-block release flags, and every
//     block adds them in rank order, so all blocks hold the same t_b.
//   - Pass 2 over band b (the second column loop): y_j += sum_i A(i,j) t_i
//     for the block's columns (one thread per column, the FMAs chained onto
//     y_j), re-reading the band while it is still in L2
//     (two bands per group are in flight: about 80 MB at n = 16384), so HBM
//     sees A once.
//   - Pass 1 of band b+1 runs before the wait for t_b, so the exchange
//     latency is hidden behind a band's worth of arithmetic.
//   - Each group leaves a partial y over all n columns; a combine adds the NG
//     partials in group order and scales by beta.
//
// Every wait is bounded (about two seconds of %globaltimer, or the limit a
// test sets): on expiry the block writes BTO_ERR_TIMEOUT into the status
// word at the start of the workspace and returns, and the other blocks of
// its group then expire too; the host reads the word with bto_device_status.
#include "check.cuh"

namespace bto {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kTB = 16;                 // band height (rows) the plan uses
constexpr int kLook = 1;                // bands of lookahead the plan uses
constexpr int kBlocksPerSM = 2;         // two blocks per SM: one computes while the other waits
constexpr int kMinGroup = 16;           // blocks per group
constexpr int64_t kMaxSlice = 4096;     // widest column slice per block (x, y slices in shared memory)

struct AtaxArgs {
    int64_t m, n;
    const double* A; int64_t lda;
    const double* x;
    unsigned* flag;      // [G] bands published by each block (sequence number within its group)
    double* tslot;       // [NG][2 D][S][TB] block partials of t
    double* ypart;       // [NG][ldy] group partials of y
    int64_t ldy;
    int* status;
    int64_t nb;          // bands
    int S, NG;
    int64_t cmax;        // widest column slice
    int64_t stall_band;  // fault injection: this band's rank-0 partial is never published (-1: none)
    unsigned long long timeout_ns;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __host__ __forceinline__ int64_t split_at(int64_t n, int64_t parts, int64_t b) {
    return (n / parts) * b + ((n % parts) * b) / parts;
}

// The TB values of a column segment starting at row R0 (rows past m read as 0).
template <int TB, bool VEC2>
__device__ __forceinline__ void load_seg(const double* col, bool whole, int rows, double (&v)[TB]) {
    if (VEC2 && whole) {
#pragma unroll
        for (int i = 0; i < TB; i += 2) {
            const double2 t = __ldg(reinterpret_cast<const double2*>(col + i));
            v[i] = t.x;
            v[i + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < TB; i++) v[i] = i < rows ? __ldg(col + i) : 0.0;
    }
}

template <int TB, int D, bool VEC2>
__global__ void __launch_bounds__(kThreads, kBlocksPerSM) atax_kernel(const AtaxArgs a) {
    constexpr int NSL = 2 * D;               // partial slots per group (see publish)
    extern __shared__ double sm[];
    double* xs = sm;                         // [cmax] x over this block's columns
    double* ys = xs + a.cmax;                // [cmax] y accumulators
    __shared__ double red[kWarps][TB];
    __shared__ double tnext[TB], ts[TB];
    __shared__ double gbuf[kThreads];        // a round of gathered partials
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x / a.S, r = blockIdx.x % a.S;
    const int64_t c0 = split_at(a.n, a.S, r), c1 = split_at(a.n, a.S, r + 1);
    const int nc = (int)(c1 - c0);
    const int64_t Q = g < a.nb ? (a.nb - g + a.NG - 1) / a.NG : 0;   // bands of this group
    const bool vec_ok = VEC2;

    for (int jl = threadIdx.x; jl < nc; jl += kThreads) {
        xs[jl] = __ldg(a.x + c0 + jl);
        ys[jl] = 0.0;
    }
    if (threadIdx.x == 0) s_abort = 0;
    __syncthreads();

    // Pass 1 over the q-th band of the group: the block's partial t in tnext.
    auto pass1 = [&](int64_t q) {
        const int64_t R0 = (g + q * a.NG) * TB;
        const int rows = (int)(a.m - R0 < TB ? a.m - R0 : TB);
        const bool whole = rows == TB;
        constexpr int RP = TB / 2;              // row pairs per band = lanes per column
        constexpr int CPW = 32 / RP;            // columns a warp covers per load
        const int rp = lane % RP;
        const int i0 = 2 * rp;
        const int jb = warp * CPW + lane / RP;
        double t0 = 0.0, t1 = 0.0;
        // The two loops differ only in how a row pair is loaded; keeping the
        // test outside lets the eight-fold unrolled loads issue together.
        if (whole && vec_ok) {
#pragma unroll 8
            for (int jl = jb; jl < nc; jl += kWarps * CPW) {
                const double2 v = __ldg(reinterpret_cast<const double2*>(a.A + (c0 + jl) * a.lda + R0 + i0));
                const double xj = xs[jl];
                t0 = fma(v.x, xj, t0);
                t1 = fma(v.y, xj, t1);
            }
        } else {
#pragma unroll 4
            for (int jl = jb; jl < nc; jl += kWarps * CPW) {
                const double* col = a.A + (c0 + jl) * a.lda + R0 + i0;
                const double xj = xs[jl];
                t0 = fma(i0 < rows ? __ldg(col) : 0.0, xj, t0);
                t1 = fma(i0 + 1 < rows ? __ldg(col + 1) : 0.0, xj, t1);
            }
        }
#pragma unroll
        for (int h = RP; h < 32; h *= 2) {
            t0 += __shfl_xor_sync(0xffffffffu, t0, h);
            t1 += __shfl_xor_sync(0xffffffffu, t1, h);
        }
        if (lane < RP) { red[warp][i0] = t0; red[warp][i0 + 1] = t1; }
        __syncthreads();
        if (threadIdx.x < TB) {
            double t = red[0][threadIdx.x];
#pragma unroll
            for (int k = 1; k < kWarps; k++) t += red[k][threadIdx.x];
            tnext[threadIdx.x] = t;
        }
        __syncthreads();
    };
    // Publishes tnext as this block's partial of the group's q-th band.
    auto publish = [&](int64_t q) {
        double* slot = a.tslot + (((int64_t)g * NSL + q % NSL) * a.S + r) * TB;
        if (threadIdx.x < TB) slot[threadIdx.x] = tnext[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 0 && !(r == 0 && g + q * a.NG == a.stall_band)) {
            // The barrier orders the partial's stores (threads 0..TB-1) before
            // this release store, which is cumulative: a peer that acquires the
            // flag sees them.
            st_release(a.flag + blockIdx.x, (unsigned)(q + 1));
        }
    };
    // Waits for the group's S partials of its q-th band; ts = their sum in rank
    // order.  S threads poll the S flags at once, and all threads fetch the
    // partials in one round into shared memory (kThreads / TB ranks per
    // round): no chain of dependent L2 round trips.
    auto gather = [&](int64_t q) -> bool {
        if (threadIdx.x < a.S) {
            const unsigned* f = a.flag + (int64_t)g * a.S + threadIdx.x;
            const unsigned long long t0 = globaltimer();
            volatile int* abortp = &s_abort;
            while (ld_acquire(f) < (unsigned)(q + 1)) {
                if (*abortp) break;
                if (globaltimer() - t0 > a.timeout_ns) {
                    atomicExch(a.status, (int)BTO_ERR_TIMEOUT);
                    *abortp = 1;
                    break;
                }
                __nanosleep(32);
            }
        }
        __syncthreads();
        if (s_abort) return false;
        const double* slot = a.tslot + ((int64_t)g * NSL + q % NSL) * a.S * TB;
        constexpr int RPR = kThreads / TB;          // ranks per round
        double t = 0.0;
        for (int rr0 = 0; rr0 < a.S; rr0 += RPR) {
            const int rr = rr0 + threadIdx.x / TB;
            gbuf[threadIdx.x] = rr < a.S ? __ldcg(slot + (int64_t)rr * TB + threadIdx.x % TB) : 0.0;
            __syncthreads();
            if (threadIdx.x < TB) {
                const int nr = a.S - rr0 < RPR ? a.S - rr0 : RPR;
                for (int k = 0; k < nr; k++) t = (rr0 + k == 0) ? gbuf[threadIdx.x] : t + gbuf[k * TB + threadIdx.x];
            }
            __syncthreads();
        }
        if (threadIdx.x < TB) ts[threadIdx.x] = t;
        __syncthreads();
        return true;
    };
    // Pass 2 over the q-th band: y_j += sum_i A(i,j) t_i.
    auto pass2 = [&](int64_t q) {
        const int64_t R0 = (g + q * a.NG) * TB;
        const int rows = (int)(a.m - R0 < TB ? a.m - R0 : TB);
        const bool whole = rows == TB;
        double tr[TB];
#pragma unroll
        for (int i = 0; i < TB; i++) tr[i] = ts[i];
#pragma unroll 2
        for (int jl = threadIdx.x; jl < nc; jl += kThreads) {
            double v[TB];
            load_seg<TB, VEC2>(a.A + (c0 + jl) * a.lda + R0, whole && vec_ok, rows, v);
            double e = ys[jl];
#pragma unroll
            for (int i = 0; i < TB; i++) e = fma(v[i], tr[i], e);
            ys[jl] = e;
        }
    };

    // Pass 1 runs D bands ahead of the exchange.  The partial of band q + D
    // goes to slot (q + D) mod 2D, last used by band q - D: every peer read
    // that slot in its gather(q - D), before it published band q, and this
    // block has seen all peers publish band q (gather(q)) before it writes.
    for (int64_t q0 = 0; q0 < D && q0 < Q; q0++) {
        pass1(q0);
        publish(q0);
    }
    for (int64_t q = 0; q < Q; q++) {
        if (q + D < Q) pass1(q + D);
        if (!gather(q)) return;
        if (q + D < Q) publish(q + D);
        pass2(q);
    }
    __syncthreads();
    for (int jl = threadIdx.x; jl < nc; jl += kThreads) a.ypart[(int64_t)g * a.ldy + c0 + jl] = ys[jl];
}

size_t atax_smem(int64_t cmax) { return (size_t)2 * cmax * sizeof(double); }

template <bool VEC2>
void* atax_fn() { return (void*)atax_kernel<kTB, kLook, VEC2>; }

}  // namespace

AtaxPlan atax_plan(int64_t m, int64_t n, const DeviceInfo& d) {
    AtaxPlan p;
    p.G = d.sms;
    if (m <= 0 || n <= 0) { p.fused = true; return p; }
    if (!d.coop) return p;
    const int S = (int)std::max<int64_t>(kMinGroup, ceil_div(n, kMaxSlice));
    const int NG = d.sms * kBlocksPerSM / S;
    if (NG < 1) return p;
    const int64_t cmax = ceil_div(n, S);
    const size_t sz = atax_smem(cmax);
    void* fn = atax_fn<true>();
    int occ = 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sz) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, sz) != cudaSuccess) {
        cudaGetLastError();
        return p;
    }
    if (occ < kBlocksPerSM) return p;
    p.G = NG * S; p.S = S; p.NG = NG; p.cmax = cmax; p.TB = kTB; p.D = kLook; p.smem = sz;
    p.nb = ceil_div(m, kTB);
    p.ldy = round_up(n, 32);
    p.fused = true;
    return p;
}

}  // namespace bto

using namespace bto;

namespace {

bto_status atax_impl(int form, int64_t m, int64_t n, double beta, const double* A, int64_t lda,
                     const double* x, double* y, void* ws, size_t ws_bytes, int64_t stall_band,
                     unsigned long long timeout_ns, bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    c.size(1, m); c.size(2, n);
    if (!c.ok()) return c.finish();
    const size_t Ab = mat_extent_bytes(m, n, lda, 8);
    c.ptr(4, A, m > 0 && n > 0); c.ld(5, lda, m);
    c.ptr(6, x, n > 0); c.ptr(7, y, n > 0);
    c.disjoint(7, y, vbytes(n), A, Ab); c.disjoint(7, y, vbytes(n), x, vbytes(n));
    DeviceInfo d; WsLayout L;
    if (c.ok()) {
        if (!device_info(&d)) return BTO_ERR_CUDA;
        if (ws_layout(BTO_OP_ATAX, form, m, n, BTO_F64, d, &L) != BTO_OK) return BTO_ERR_CUDA;
        c.ws(8, ws, ws_bytes, L);
    }
    if (!c.ok()) return c.finish();
    cudaStream_t st = (cudaStream_t)stream;
    char* w = static_cast<char*>(ws);
    if (n == 0) return BTO_OK;
    if (form == BTO_FORM_DF) {
        // Double-float form: t = A x into the workspace, then y = beta A^T t
        // with the tiles in reverse (the last ones are still in L2).
        const PanelPlan dp = df_plan(m, n, d.sms);
        const DfArgs probe = df_args(m, n, A, lda, dp, ws);
        if (m > 0 && df_layout_ok(DF_Q, probe)) {
            if (cudaMemsetAsync(w, 0, sizeof(int), st) != cudaSuccess) return BTO_ERR_CUDA;
            double* t = reinterpret_cast<double*>(w + L.off[0]);
            bto_status e = df_gemv_n(m, n, 1.0, A, lda, x, 0.0, nullptr, t,
                                     reinterpret_cast<double*>(w + L.off[1]), dp, ws, 0, st);
            if (e != BTO_OK) return e;
            return df_gemv_t(m, n, beta, A, lda, t, 0.0, nullptr, y, reinterpret_cast<double*>(w + L.off[2]), dp,
                             ws, 1, st);
        }
        if (ws_layout(BTO_OP_ATAX, BTO_FORM_FUSED, m, n, BTO_F64, d, &L) != BTO_OK) return BTO_ERR_CUDA;
    }
    const AtaxPlan ap = atax_plan(m, n, d);
    // The status word reads BTO_OK after every form; the group-band kernel
    // clears it below together with its flags.
    if ((m == 0 || !ap.fused) && cudaMemsetAsync(w, 0, sizeof(int), st) != cudaSuccess) return BTO_ERR_CUDA;
    if (m == 0) {   // y = beta * (empty sum)
        CombineJob j = {y, n, nullptr, 0, 0, beta, nullptr, 0, 0, 0.0, nullptr, 0.0};
        return launch_combine(&j, 1, st);
    }
    if (!ap.fused) {
        // Slices too wide for shared memory: t = A x into the workspace, then
        // y = beta A^T t (A is read twice).
        const PanelPlan pl = panel_plan(m, n, d.sms, BTO_OP_ATAX, BTO_FORM_FUSED);
        double* t = reinterpret_cast<double*>(w + L.off[0]);
        PanelArgs a{};
        a.m = m; a.n = n; a.A = A; a.lda = lda; a.p = x;
        a.qpart = reinterpret_cast<double*>(w + L.off[1]);
        a.spart = reinterpret_cast<double*>(w + L.off[2]);
        a.ldq = pl.ldq; a.lds = pl.lds; a.NR = pl.NR; a.NC = pl.NC; a.ntiles = pl.ntiles;
        bto_status e = launch_panel(PM_Q, a, pl, st);
        if (e != BTO_OK) return e;
        CombineJob jt = {t, m, a.qpart, pl.ldq, pl.NC, 1.0, nullptr, 0, 0, 0.0, nullptr, 0.0};
        if ((e = launch_combine(&jt, 1, st)) != BTO_OK) return e;
        a.p = nullptr; a.r = t; a.reverse = 1;
        if ((e = launch_panel(PM_S, a, pl, st)) != BTO_OK) return e;
        CombineJob jy = {y, n, a.spart, pl.lds, pl.NR, beta, nullptr, 0, 0, 0.0, nullptr, 0.0};
        return launch_combine(&jy, 1, st);
    }
    // Zero the status word and the per-block flags.
    if (cudaMemsetAsync(w, 0, L.off[0] + (size_t)ap.G * sizeof(unsigned), st) != cudaSuccess)
        return BTO_ERR_CUDA;
    AtaxArgs a{};
    a.m = m; a.n = n; a.A = A; a.lda = lda; a.x = x;
    a.flag = reinterpret_cast<unsigned*>(w + L.off[0]);
    a.tslot = reinterpret_cast<double*>(w + L.off[1]);
    a.ypart = reinterpret_cast<double*>(w + L.off[2]);
    a.ldy = ap.ldy;
    a.status = reinterpret_cast<int*>(w);
    a.nb = ap.nb; a.S = ap.S; a.NG = ap.NG; a.cmax = ap.cmax;
    a.stall_band = stall_band; a.timeout_ns = timeout_ns;
    const bool vec2 = aligned16(A) && (lda % 2 == 0);
    void* fn = vec2 ? atax_fn<true>() : atax_fn<false>();
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ap.smem) != cudaSuccess)
        return BTO_ERR_CUDA;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, ap.smem) != cudaSuccess)
        return BTO_ERR_CUDA;
    if ((int64_t)occ * d.sms < ap.G) return BTO_ERR_UNSUPPORTED;   // cooperative grid must be co-resident
    void* args[] = {(void*)&a};
    if (cudaLaunchCooperativeKernel(fn, dim3(ap.G), dim3(kThreads), args, ap.smem, st) != cudaSuccess)
        return BTO_ERR_CUDA;
    // y = beta * (sum of the group partials, in group order).
    CombineJob jy = {y, n, a.ypart, ap.ldy, ap.NG, beta, nullptr, 0, 0, 0.0, nullptr, 0.0};
    return launch_combine(&jy, 1, st);
}

}  // namespace

extern "C" bto_status bto_atax(int64_t m, int64_t n, double beta, const double* A, int64_t lda,
                               const double* x, double* y, void* ws, size_t ws_bytes,
                               bto_stream_t stream) {
    return atax_impl(BTO_FORM_FUSED, m, n, beta, A, lda, x, y, ws, ws_bytes, -1, 2000000000ull, stream);
}

extern "C" bto_status bto_atax_df(int64_t m, int64_t n, double beta, const double* A, int64_t lda,
                                  const double* x, double* y, void* ws, size_t ws_bytes,
                                  bto_stream_t stream) {
    return atax_impl(BTO_FORM_DF, m, n, beta, A, lda, x, y, ws, ws_bytes, -1, 2000000000ull, stream);
}

// Fault injection for tests (declared in bto.h's testing section): band
// `stall_band`'s ready flag is never published, so every wait for it
// expires after `timeout_ms` and the status word reads BTO_ERR_TIMEOUT.
extern "C" bto_status bto_debug_atax_stall(int64_t m, int64_t n, double beta, const double* A,
                                           int64_t lda, const double* x, double* y, void* ws,
                                           size_t ws_bytes, int64_t stall_band, int timeout_ms,
                                           bto_stream_t stream) {
    if (timeout_ms < 1 || timeout_ms > 10000) { set_invalid_arg(11); return BTO_ERR_INVALID_VALUE; }
    return atax_impl(BTO_FORM_FUSED, m, n, beta, A, lda, x, y, ws, ws_bytes, stall_band,
                     (unsigned long long)timeout_ms * 1000000ull, stream);
}
