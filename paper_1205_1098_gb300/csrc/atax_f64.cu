// ATAX / BATAX (Table I; Section II, Fig. 1): y <- beta A^T (A x), with the
// temporary t = A x contracted and A read from device memory once.
//
// The paper's Max-Fuse result for BATAX partitions the rows (p(i)), fuses
// the two row loops, and keeps the two inner column loops apart because
// t_i is complete only after its whole row has been summed (Section III-D,
// Section IV-A).  On a GPU with column-major A the rows are the strided
// direction, so the schedule here is a wavefront over row bands:
//
//   - Block c of a cooperative grid (one block per SM) owns a fixed slice of
//     columns, and therefore owns y_j for those columns outright: no
//     cross-block reduction of y is ever needed.
//   - Rows are processed in bands of TB rows.  For band b every block loads
//     its TB x (slice) piece of A from device memory into shared memory
//     (512-byte column segments for TB = 64), forming on the way its partial
//     t over its columns.
//   - The partial t of band b goes to a per-band slot; the block that
//     arrives last (an atomic counter) adds the G partials in block order
//     and publishes the complete t_b with a release flag.
//   - Each block then sweeps its shared-memory copy of the band once more,
//     y_j += sum_i A(i,j) t_i, with threads owning columns.  The band copy
//     stays resident for nbuf-1 further bands, so the wait for t_b overlaps
//     the loading of the next bands.
//
// Every wait is bounded (about two seconds of %globaltimer, or the limit a
// test sets): on expiry the block writes BTO_ERR_TIMEOUT into the status
// word at the start of the workspace and returns, and every other wait then
// expires too; the host reads the word with bto_device_status.
#include "check.cuh"

namespace bto {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int64_t kMaxSlice = 512;        // widest column slice per block
constexpr int kYPerThread = kMaxSlice / kThreads;
constexpr int kBatch = 8;             // column segments in flight per warp in phase 1

struct AtaxArgs {
    int64_t m, n;
    const double* A; int64_t lda;
    const double* x;
    double* y;
    double beta;
    unsigned* cnt;       // [nb] arrivals
    unsigned* flag;      // [nb] band ready
    double* tpart;       // [nb][G][TB]
    double* tfull;       // [nb][TB]
    int* status;
    int64_t nb;
    int nbuf;
    int64_t cstride;     // shared-memory column stride (TB + 1)
    int64_t stall_band;  // fault injection: this band's flag is never published (-1: none)
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

template <int TB, bool VEC2>
__global__ void __launch_bounds__(kThreads, 1) atax_kernel(const AtaxArgs a) {
    constexpr int RPL = TB / 32;   // rows per lane in phase 1 (1 or 2)
    extern __shared__ double sm[];
    const int G = gridDim.x, c = blockIdx.x;
    const int64_t c0 = split_at(a.n, G, c), c1 = split_at(a.n, G, c + 1);
    const int nc = (int)(c1 - c0);
    const int64_t cmax = (a.n + G - 1) / G;
    double* bufs = sm;                                   // [nbuf][cmax][cstride]
    double* tred = bufs + (int64_t)a.nbuf * cmax * a.cstride;   // [kWarps][TB]
    double* ts = tred + kWarps * TB;                     // [TB]
    double* rsum = ts + TB;                              // [kThreads] last-arriver scratch
    __shared__ int s_last, s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    double yacc[kYPerThread];
#pragma unroll
    for (int k = 0; k < kYPerThread; k++) yacc[k] = 0.0;
    if (threadIdx.x == 0) s_abort = 0;
    __syncthreads();

    const int D = a.nbuf - 1;
    for (int64_t b = 0; b < a.nb + D; b++) {
        // ---------------- phase 1: load band b, partial t over this block's columns
        if (b < a.nb) {
            const int64_t R0 = b * TB, rend = min(a.m, R0 + TB);
            double* buf = bufs + (b % a.nbuf) * cmax * a.cstride;
            double tp[RPL];
#pragma unroll
            for (int k = 0; k < RPL; k++) tp[k] = 0.0;
            // Columns jl = warp + kWarps*u, in batches of kBatch per warp, so each
            // warp has kBatch column segments in flight before it consumes any.
            for (int jb = warp; jb < nc; jb += kWarps * kBatch) {
                double v[kBatch][RPL], xj[kBatch];
#pragma unroll
                for (int u = 0; u < kBatch; u++) {
                    const int jl = jb + u * kWarps;
                    xj[u] = 0.0;
#pragma unroll
                    for (int k = 0; k < RPL; k++) v[u][k] = 0.0;
                    if (jl < nc) {
                        const double* col = a.A + (c0 + jl) * a.lda;
                        xj[u] = __ldg(a.x + c0 + jl);
                        if (RPL == 2) {
                            const int64_t i = R0 + 2 * lane;
                            if (VEC2 && i + 1 < rend) {
                                double2 t = __ldg(reinterpret_cast<const double2*>(col + i));
                                v[u][0] = t.x; v[u][RPL - 1] = t.y;
                            } else {
                                if (i < rend) v[u][0] = __ldg(col + i);
                                if (i + 1 < rend) v[u][RPL - 1] = __ldg(col + i + 1);
                            }
                        } else {
                            const int64_t i = R0 + lane;
                            if (i < rend) v[u][0] = __ldg(col + i);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < kBatch; u++) {
                    const int jl = jb + u * kWarps;
                    if (jl < nc) {
#pragma unroll
                        for (int k = 0; k < RPL; k++) {
                            tp[k] = fma(v[u][k], xj[u], tp[k]);
                            buf[jl * a.cstride + RPL * lane + k] = v[u][k];
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < RPL; k++) tred[warp * TB + RPL * lane + k] = tp[k];
            __syncthreads();
            if (threadIdx.x < TB) {
                double s = tred[threadIdx.x];
#pragma unroll
                for (int w = 1; w < kWarps; w++) s += tred[w * TB + threadIdx.x];
                a.tpart[(b * G + c) * TB + threadIdx.x] = s;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                // The barrier orders the block's partial stores before this
                // fence; fence + atomic form the release of this band's partial.
                __threadfence();
                const unsigned old = atomicAdd(a.cnt + b, 1u);
                s_last = (old == (unsigned)(G - 1));
            }
            __syncthreads();
            if (s_last) {
                // Last arrival: t_b = sum over blocks in block order.  Threads
                // split the blocks into kThreads/TB strided groups; the group
                // sums are then added in group order.
                __threadfence();
                constexpr int P = kThreads / TB;
                const int row = threadIdx.x % TB, part = threadIdx.x / TB;
                // Eight independent accumulators keep eight loads in flight.
                double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
                int cc = part;
                for (; cc + 7 * P < G; cc += 8 * P) {
#pragma unroll
                    for (int u = 0; u < 8; u++) acc[u] += __ldcg(a.tpart + (b * G + cc + u * P) * TB + row);
                }
                for (int u = 0; cc < G; cc += P, u++) acc[u] += __ldcg(a.tpart + (b * G + cc) * TB + row);
                rsum[threadIdx.x] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
                __syncthreads();
                if (threadIdx.x < TB) {
                    double t = rsum[threadIdx.x];
#pragma unroll
                    for (int p = 1; p < P; p++) t += rsum[p * TB + threadIdx.x];
                    a.tfull[b * TB + threadIdx.x] = t;
                }
                __syncthreads();
                if (threadIdx.x == 0 && b != a.stall_band) {
                    __threadfence();
                    st_release(a.flag + b, 1u);
                }
            }
        }
        // ---------------- phase 2: y += A_band^T t_band for band b - D
        const int64_t bb = b - D;
        if (bb >= 0) {
            if (threadIdx.x == 0) {
                const unsigned long long t0 = globaltimer();
                while (ld_acquire(a.flag + bb) == 0u) {
                    if (globaltimer() - t0 > a.timeout_ns) {
                        atomicExch(a.status, (int)BTO_ERR_TIMEOUT);
                        s_abort = 1;
                        break;
                    }
                    __nanosleep(200);
                }
            }
            __syncthreads();
            if (s_abort) return;
            const int64_t R0 = bb * TB;
            if (threadIdx.x < TB)
                ts[threadIdx.x] = (R0 + threadIdx.x < a.m) ? __ldcg(a.tfull + bb * TB + threadIdx.x) : 0.0;
            __syncthreads();
            const double* buf = bufs + (bb % a.nbuf) * cmax * a.cstride;
#pragma unroll
            for (int k = 0; k < kYPerThread; k++) {
                const int jl = threadIdx.x + k * kThreads;
                if (jl < nc) {
                    // Two interleaved chains (even and odd rows), added in a fixed order.
                    double e0 = 0.0, e1 = 0.0;
                    const double* colbuf = buf + jl * a.cstride;
#pragma unroll 16
                    for (int i = 0; i < TB; i += 2) {
                        e0 = fma(colbuf[i], ts[i], e0);
                        e1 = fma(colbuf[i + 1], ts[i + 1], e1);
                    }
                    yacc[k] += e0 + e1;
                }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int k = 0; k < kYPerThread; k++) {
        const int jl = threadIdx.x + k * kThreads;
        if (jl < nc) a.y[c0 + jl] = a.beta * yacc[k];
    }
}

size_t atax_smem(int TB, int nbuf, int64_t cmax) {
    return ((size_t)nbuf * cmax * (TB + 1) + (size_t)kWarps * TB + TB + kThreads) * sizeof(double);
}

template <int TB, bool VEC2>
void* atax_fn() { return (void*)atax_kernel<TB, VEC2>; }

}  // namespace

AtaxPlan atax_plan(int64_t m, int64_t n, const DeviceInfo& d) {
    AtaxPlan p;
    p.G = d.sms;
    if (m <= 0 || n <= 0) { p.fused = true; return p; }
    if (!d.coop) return p;
    // One block per SM: more blocks per band multiply the partials the last
    // arrival must add, which costs more than the overlap they bring.
    const int cand[4][2] = {{64, 3}, {64, 2}, {32, 3}, {32, 2}};
    for (int per_sm = 1; per_sm >= 1; per_sm--) {
        const int64_t G = (int64_t)d.sms * per_sm;
        const int64_t cmax = ceil_div(n, G);
        if (cmax > kMaxSlice) continue;
        const size_t limit = ((size_t)d.max_smem_optin - 2048) / per_sm;
        for (auto& cd : cand) {
            const size_t sz = atax_smem(cd[0], cd[1], cmax);
            if (sz > limit) continue;
            void* fn = cd[0] == 64 ? atax_fn<64, true>() : atax_fn<32, false>();
            int occ = 0;
            if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sz) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, sz) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            if (occ < per_sm) continue;
            p.G = (int)G; p.cmax = cmax; p.TB = cd[0]; p.nbuf = cd[1]; p.smem = sz;
            p.nb = ceil_div(m, p.TB);
            p.fused = true;
            return p;
        }
    }
    return p;
}

}  // namespace bto

using namespace bto;

namespace {

bto_status atax_impl(int64_t m, int64_t n, double beta, const double* A, int64_t lda,
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
        if (ws_layout(BTO_OP_ATAX, BTO_FORM_FUSED, m, n, BTO_F64, d, &L) != BTO_OK) return BTO_ERR_CUDA;
        c.ws(8, ws, ws_bytes, L);
    }
    if (!c.ok()) return c.finish();
    cudaStream_t st = (cudaStream_t)stream;
    char* w = static_cast<char*>(ws);
    if (n == 0) return BTO_OK;
    if (m == 0) {   // y = beta * (empty sum)
        CombineJob j = {y, n, nullptr, 0, 0, beta, nullptr, 0, 0, 0.0, nullptr, 0.0};
        return launch_combine(&j, 1, st);
    }
    const AtaxPlan ap = atax_plan(m, n, d);
    if (!ap.fused) {
        // Slices too wide for shared memory: t = A x into the workspace, then
        // y = beta A^T t (A is read twice).
        const PanelPlan pl = panel_plan(m, n, d.sms);
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
    // Zero the status word, the counters and the flags.
    if (cudaMemsetAsync(w, 0, L.off[0] + 2 * ap.nb * sizeof(unsigned), st) != cudaSuccess)
        return BTO_ERR_CUDA;
    AtaxArgs a{};
    a.m = m; a.n = n; a.A = A; a.lda = lda; a.x = x; a.y = y; a.beta = beta;
    a.cnt = reinterpret_cast<unsigned*>(w + L.off[0]);
    a.flag = a.cnt + ap.nb;
    a.tpart = reinterpret_cast<double*>(w + L.off[1]);
    a.tfull = reinterpret_cast<double*>(w + L.off[2]);
    a.status = reinterpret_cast<int*>(w);
    a.nb = ap.nb; a.nbuf = ap.nbuf; a.cstride = ap.TB + 1;
    a.stall_band = stall_band; a.timeout_ns = timeout_ns;
    const bool vec2 = aligned16(A) && (lda % 2 == 0);
    void* fn = ap.TB == 64 ? (vec2 ? atax_fn<64, true>() : atax_fn<64, false>())
                           : atax_fn<32, false>();
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ap.smem) != cudaSuccess)
        return BTO_ERR_CUDA;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, ap.smem) != cudaSuccess)
        return BTO_ERR_CUDA;
    if ((int64_t)occ * d.sms < ap.G) return BTO_ERR_UNSUPPORTED;   // cooperative grid must be co-resident
    void* args[] = {(void*)&a};
    if (cudaLaunchCooperativeKernel(fn, dim3(ap.G), dim3(kThreads), args, ap.smem, st) != cudaSuccess)
        return BTO_ERR_CUDA;
    return BTO_OK;
}

}  // namespace

extern "C" bto_status bto_atax(int64_t m, int64_t n, double beta, const double* A, int64_t lda,
                               const double* x, double* y, void* ws, size_t ws_bytes,
                               bto_stream_t stream) {
    return atax_impl(m, n, beta, A, lda, x, y, ws, ws_bytes, -1, 2000000000ull, stream);
}

// Fault injection for tests (declared in bto.h's testing section): band
// `stall_band`'s ready flag is never published, so every wait for it
// expires after `timeout_ms` and the status word reads BTO_ERR_TIMEOUT.
extern "C" bto_status bto_debug_atax_stall(int64_t m, int64_t n, double beta, const double* A,
                                           int64_t lda, const double* x, double* y, void* ws,
                                           size_t ws_bytes, int64_t stall_band, int timeout_ms,
                                           bto_stream_t stream) {
    if (timeout_ms < 1 || timeout_ms > 10000) { set_invalid_arg(11); return BTO_ERR_INVALID_VALUE; }
    return atax_impl(m, n, beta, A, lda, x, y, ws, ws_bytes, stall_band,
                     (unsigned long long)timeout_ms * 1000000ull, stream);
}
