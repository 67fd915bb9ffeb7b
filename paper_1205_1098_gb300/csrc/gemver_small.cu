// GEMVER in one launch, for matrices small enough that B stays in L2
// (Table I's GEMVER; the n = 2048 configuration is 32 MiB of FP64).
//
// The two passes of the panel engine need four launches (pass 1, the
// combine of x, pass 2, the combine of w); at this size each launch's start
// and drain cost as much as its arithmetic.  Here one cooperative grid does
// both passes with one grid-wide barrier between them:
//   pass 1  a warp takes whole columns: B(:, j) = A(:, j) + u1 v1_j + u2 v2_j
//           (two FMAs per element, the panel engine's formula, so B is the
//           same bits), stored once, and x_j = beta (B(:, j)^T y) + z_j from
//           the same registers: a column's sum never leaves its warp, so x
//           needs no partials and no combine;
//   barrier every block has written its columns of B and x;
//   pass 2  a block takes 8 rows: w_i = alpha (B(i, :) x), with x staged in
//           shared memory, B read from L2 (it was just written), 32 column
//           groups per row added in a fixed order.
// B is formed in FP64 (two FMAs per element: at 4 FP64 FMAs per element the
// FP64 unit alone would need the whole time).  The two sums, B^T y and B x,
// run in double-float on the FP32 pipe: each FP64 value is split into hi +
// lo (47 bits, integer operations, df32.cuh), products are TwoProduct plus
// cross terms, sums are compensated with TwoSum; the result is within about
// 1e-14 of exact FP64 arithmetic and exact for integer data below 2^47.
// A sum whose operands leave [2^-40, 2^40] in magnitude (zero excepted),
// where FP32's exponent range would cost bits, is recomputed in FP64 from the
// stored B: a column of x by its warp, a block's 8 rows of w by the block.
// Every sum runs in a fixed order, so results are bitwise reproducible.
// The barrier's wait is bounded by %globaltimer; on expiry the block records
// BTO_ERR_TIMEOUT in the status word and returns without pass 2.
#include "check.cuh"
#include "df32.cuh"

namespace bto {
namespace {

constexpr int kGW = 8;                   // warps per block
constexpr int kGT = kGW * 32;
constexpr int kP2Rows = 8;               // rows per block step in pass 2
constexpr int kP2Groups = kGT / kP2Rows; // column groups per row
constexpr size_t kBarrierOff = 128;      // grid-barrier counter in the workspace header
constexpr unsigned long long kWaitNs = 2000000000ull;
constexpr size_t kSmemCap = 100 * 1024;  // dynamic shared memory per block (two blocks per SM)

struct GsArgs {
    int64_t m, n;
    double alpha, beta;
    const double* A; int64_t lda;
    const double* u1; const double* v1; const double* u2; const double* v2;
    const double* y; const double* z;
    double* B; int64_t ldb;
    double* x; double* w;
    unsigned* counter;
    int* status;
    int stall_block;                      // fault injection: this block never arrives (-1: none)
    unsigned long long timeout_ns;
};

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

// Outside the double-float range of the sums: 2^-40 <= |v| <= 2^40 or v = 0.
__device__ __forceinline__ bool df_out_of_range(uint32_t hw, uint32_t lw) {
    const uint32_t e = (hw >> 20) & 0x7ffu;
    return (e - 983u) > 80u && ((hw << 1) | lw) != 0u;
}

// (sh, sl) += (bh + bl) (vh + vl) in double-float.
__device__ __forceinline__ void df_mac1(float& sh, float& sl, float bh, float bl, float vh, float vl) {
    const float p = bh * vh;
    const float e = fmaf(bh, vh, -p);
    const float t = fmaf(bh, vl, bl * vh);
    const float s = sh + p;
    const float bb = s - sh;
    const float err = (sh - (s - bb)) + (p - bb);
    sh = s;
    sl += err + (e + t);
}

// (ah, al) + (bh, bl), renormalised by TwoSum of the high parts.
__device__ __forceinline__ void df_add1(float& ah, float& al, float bh, float bl) {
    const float s = ah + bh;
    const float bb = s - ah;
    const float err = (ah - (s - bb)) + (bh - bb);
    ah = s;
    al = (al + bl) + err;
}

__global__ void __launch_bounds__(kGT, 2) gemver_small_kernel(const GsArgs a) {
    extern __shared__ double sm[];        // pass 1: u1, u2, y (m each); pass 2: x (n)
    __shared__ float2 red[kP2Groups * kP2Rows];
    __shared__ int ok_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t m = a.m, n = a.n;
    double* su1 = sm;
    double* su2 = sm + m;
    float2* sy = reinterpret_cast<float2*>(sm + 2 * m);   // y as (hi, lo)
    bool ybad = false;
    // Four elements of each vector per thread at a time, their loads issued
    // together (one round trip to L2 instead of four).
    for (int64_t i0 = tid; i0 < m; i0 += 4 * kGT) {
        double u1r[4], u2r[4], yr[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int64_t i = i0 + (int64_t)u * kGT;
            if (i < m) {
                u1r[u] = __ldg(a.u1 + i);
                u2r[u] = __ldg(a.u2 + i);
                yr[u] = __ldg(a.y + i);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int64_t i = i0 + (int64_t)u * kGT;
            if (i < m) {
                su1[i] = u1r[u];
                su2[i] = u2r[u];
                const uint32_t hw = (uint32_t)__double2hiint(yr[u]), lw = (uint32_t)__double2loint(yr[u]);
                ybad |= df_out_of_range(hw, lw);
                float h, l;
                df::split_words(hw, lw, h, l);
                sy[i] = make_float2(h, l);
            }
        }
    }
    ybad = __syncthreads_or(ybad) != 0;    // y out of range: every x in FP64

    // ---- pass 1: whole columns per warp, dealt over the blocks first
    // (column j to block j mod G), so that every SM gets its share of the
    // FP64 work when there are fewer columns than warps.
    const int64_t nw = (int64_t)gridDim.x * kGW;
    for (int64_t j = (int64_t)warp * gridDim.x + blockIdx.x; j < n; j += nw) {
        const double v1j = __ldg(a.v1 + j), v2j = __ldg(a.v2 + j);
        const double* acol = a.A + j * a.lda;     // plain loads: B may overwrite A
        double* bcol = a.B + j * a.ldb;
        float sh[2] = {0.f, 0.f}, sl[2] = {0.f, 0.f};
        bool bad = ybad;
        auto one = [&](int64_t ii, double av, int k) {
            const double b = fma(su2[ii], v2j, fma(su1[ii], v1j, av));
            bcol[ii] = b;
            const uint32_t hw = (uint32_t)__double2hiint(b), lw = (uint32_t)__double2loint(b);
            bad |= df_out_of_range(hw, lw);
            float bh, bl;
            df::split_words(hw, lw, bh, bl);
            const float2 yv = sy[ii];
            df_mac1(sh[k], sl[k], bh, bl, yv.x, yv.y);
        };
        // Four rows per lane at a time; the next four are loaded before these
        // are processed (other rows than the ones stored, so in-place B is
        // safe), which the compiler cannot do across the stores by itself.
        int64_t i = lane;
        if (i + 96 < m) {
            double av[4];
#pragma unroll
            for (int u = 0; u < 4; u++) av[u] = acol[i + 32 * u];
            while (true) {
                const int64_t in = i + 128;
                const bool more = in + 96 < m;
                double nx[4];
                if (more) {
#pragma unroll
                    for (int u = 0; u < 4; u++) nx[u] = acol[in + 32 * u];
                }
#pragma unroll
                for (int u = 0; u < 4; u++) one(i + 32 * u, av[u], u & 1);
                i = in;
                if (!more) break;
#pragma unroll
                for (int u = 0; u < 4; u++) av[u] = nx[u];
            }
        }
        for (; i < m; i += 32) one(i, acol[i], 0);
        df_add1(sh[0], sl[0], sh[1], sl[1]);
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, sh[0], d), ol = __shfl_xor_sync(0xffffffffu, sl[0], d);
            df_add1(sh[0], sl[0], oh, ol);
        }
        double s = (double)sh[0] + (double)sl[0];
        if (__any_sync(0xffffffffu, bad)) {
            // FP64 over the stored column (this warp's own stores).
            __syncwarp();
            double acc = 0.0;
            for (int64_t ii = lane; ii < m; ii += 32) acc = fma(bcol[ii], __ldg(a.y + ii), acc);
#pragma unroll
            for (int d = 16; d >= 1; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
            s = acc;
        }
        if (lane == 0) a.x[j] = a.beta * s + a.z[j];
    }

    // ---- grid barrier (bounded)
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if ((int)blockIdx.x != a.stall_block) atomicAdd(a.counter, 1u);
        const unsigned long long t0 = gtimer();
        int ok = 1;
        while (ld_acquire_u32(a.counter) < gridDim.x) {
            if (gtimer() - t0 > a.timeout_ns) {
                atomicExch(a.status, (int)BTO_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    if (!ok_s) return;

    // ---- pass 2: 8 rows per block step, 32 column groups per row
    float2* sx = reinterpret_cast<float2*>(sm);    // x as (hi, lo)
    double* sxd = sm + n;                          // and in FP64 (for the fallback)
    bool xbad = false;
    for (int64_t j0 = tid; j0 < n; j0 += 8 * kGT) {
        double xr[8];                              // eight loads in flight per thread
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int64_t j = j0 + (int64_t)u * kGT;
            if (j < n) xr[u] = __ldcg(a.x + j);
        }
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int64_t j = j0 + (int64_t)u * kGT;
            if (j < n) {
                const uint32_t hw = (uint32_t)__double2hiint(xr[u]), lw = (uint32_t)__double2loint(xr[u]);
                xbad |= df_out_of_range(hw, lw);
                float h, l;
                df::split_words(hw, lw, h, l);
                sx[j] = make_float2(h, l);
                sxd[j] = xr[u];
            }
        }
    }
    xbad = __syncthreads_or(xbad) != 0;
    const int r = tid % kP2Rows, g = tid / kP2Rows;
    for (int64_t i0 = (int64_t)blockIdx.x * kP2Rows; i0 < m; i0 += (int64_t)gridDim.x * kP2Rows) {
        const int64_t i = i0 + r;
        float th[2] = {0.f, 0.f}, tl[2] = {0.f, 0.f};
        bool bad = xbad;
        if (i < m && !xbad) {
            const double* brow = a.B + i;
            auto one = [&](int64_t j, int k) {
                const double b = __ldcg(brow + j * a.ldb);
                const uint32_t hw = (uint32_t)__double2hiint(b), lw = (uint32_t)__double2loint(b);
                bad |= df_out_of_range(hw, lw);
                float bh, bl;
                df::split_words(hw, lw, bh, bl);
                const float2 xv = sx[j];
                df_mac1(th[k], tl[k], bh, bl, xv.x, xv.y);
            };
            int64_t j = g;
#pragma unroll 4
            for (; j + kP2Groups < n; j += 2 * kP2Groups) {
                one(j, 0);
                one(j + kP2Groups, 1);
            }
            if (j < n) one(j, 0);
            df_add1(th[0], tl[0], th[1], tl[1]);
        }
        red[g * kP2Rows + r] = make_float2(th[0], tl[0]);
        bad = __syncthreads_or(bad) != 0;
        if (!bad) {
            if (tid < kP2Rows && i0 + tid < m) {
                float2 acc = red[tid];
                for (int gg = 1; gg < kP2Groups; gg++) {
                    const float2 v = red[gg * kP2Rows + tid];
                    df_add1(acc.x, acc.y, v.x, v.y);
                }
                a.w[i0 + tid] = a.alpha * ((double)acc.x + (double)acc.y);
            }
        } else {
            // FP64 for these rows: 32 column groups per row, then their sum.
            double t = 0.0;
            if (i < m)
                for (int64_t j = g; j < n; j += kP2Groups) t = fma(__ldcg(a.B + i + j * a.ldb), sxd[j], t);
            __syncthreads();
            reinterpret_cast<double*>(red)[g * kP2Rows + r] = t;
            __syncthreads();
            if (tid < kP2Rows && i0 + tid < m) {
                double s = reinterpret_cast<double*>(red)[tid];
                for (int gg = 1; gg < kP2Groups; gg++) s += reinterpret_cast<double*>(red)[gg * kP2Rows + tid];
                a.w[i0 + tid] = a.alpha * s;
            }
        }
        __syncthreads();
    }
}

// pass 1: u1, u2 (FP64) and y (hi, lo); pass 2: x as (hi, lo) and in FP64.
size_t gs_smem(int64_t m, int64_t n) { return (size_t)std::max<int64_t>(3 * m, 2 * n) * sizeof(double); }

}  // namespace

bool gemver_small_ok(int64_t m, int64_t n, const DeviceInfo& d) {
    return d.coop && m > 0 && n > 0 && gs_smem(m, n) <= kSmemCap && m * n <= (int64_t(1) << 23);
}

// Returns BTO_ERR_UNSUPPORTED (with nothing launched and no error left
// pending) when the grid cannot be made co-resident; the caller then runs
// the two-pass form.
bto_status gemver_small(int64_t m, int64_t n, double alpha, double beta, const double* A, int64_t lda,
                        const double* u1, const double* v1, const double* u2, const double* v2, const double* y,
                        const double* z, double* B, int64_t ldb, double* x, double* w, void* ws,
                        const DeviceInfo& d, int stall_block, unsigned long long timeout_ns, cudaStream_t st) {
    const size_t smem = gs_smem(m, n);
    if (cudaFuncSetAttribute(gemver_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return BTO_ERR_UNSUPPORTED;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gemver_small_kernel, kGT, smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return BTO_ERR_UNSUPPORTED;
    }
    per_sm = std::min(per_sm, 2);
    GsArgs a;
    a.m = m; a.n = n; a.alpha = alpha; a.beta = beta; a.A = A; a.lda = lda;
    a.u1 = u1; a.v1 = v1; a.u2 = u2; a.v2 = v2; a.y = y; a.z = z;
    a.B = B; a.ldb = ldb; a.x = x; a.w = w;
    a.counter = reinterpret_cast<unsigned*>(static_cast<char*>(ws) + kBarrierOff);
    a.status = static_cast<int*>(ws);
    a.stall_block = stall_block;
    a.timeout_ns = timeout_ns ? timeout_ns : kWaitNs;
    // status word and barrier counter
    if (cudaMemsetAsync(ws, 0, WS_HEADER, st) != cudaSuccess) return BTO_ERR_CUDA;
    void* args[] = {&a};
    const cudaError_t e = cudaLaunchCooperativeKernel((const void*)gemver_small_kernel, dim3(per_sm * d.sms),
                                                      dim3(kGT), args, smem, st);
    if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorNotSupported) {
        cudaGetLastError();
        return BTO_ERR_UNSUPPORTED;
    }
    return e == cudaSuccess ? BTO_OK : BTO_ERR_CUDA;
}

}  // namespace bto
