// Unfused comparison forms: every BLAS call of a sequence is its own kernel
// (or, for dgemv, the panel engine in single-product mode plus its combine),
// and every intermediate result goes through device memory.  The paper's
// unfused baselines are this translation of the BLAS calls into separate
// loops (Section V-B); each kernel here is a full-bandwidth kernel on its
// own, so a fused/unfused comparison measures fusion alone.
#include "check.cuh"

namespace bto {

namespace {

constexpr int kThreads = 256;

__global__ void dcopy_kernel(int64_t n, const double* __restrict__ x, double* __restrict__ y) {
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += stride) y[i] = x[i];
}
__global__ void dcopy2_kernel(int64_t n2, const double2* __restrict__ x, double2* __restrict__ y) {
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n2; i += stride) y[i] = __ldg(x + i);
}
__global__ void dscal_kernel(int64_t n, double a, double* x) {
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += stride) x[i] = a * x[i];
}
__global__ void daxpy_kernel(int64_t n, double a, const double* __restrict__ x, double* y) {
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += stride)
        y[i] = fma(a, __ldg(x + i), y[i]);
}
// A(i,j) += x_i * y_j (dger with alpha = 1), column j per block-iteration.
__global__ void dger_kernel(int64_t m, int64_t n, const double* __restrict__ x,
                            const double* __restrict__ y, double* A, int64_t lda) {
    for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
        const double yj = __ldg(y + j);
        double* col = A + j * lda;
        for (int64_t i = threadIdx.x; i < m; i += kThreads) col[i] = fma(__ldg(x + i), yj, col[i]);
    }
}

}  // namespace

static int egrid(int64_t n, int sms) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 8, ceil_div(n, kThreads)));
}

bto_status dcopy(int64_t n, const double* x, double* y, int sms, cudaStream_t st) {
    if (n <= 0) return BTO_OK;
    if (aligned16(x) && aligned16(y) && n % 2 == 0)
        dcopy2_kernel<<<egrid(n / 2, sms), kThreads, 0, st>>>(n / 2, reinterpret_cast<const double2*>(x),
                                                             reinterpret_cast<double2*>(y));
    else
        dcopy_kernel<<<egrid(n, sms), kThreads, 0, st>>>(n, x, y);
    return launch_status();
}
bto_status dscal(int64_t n, double a, double* x, int sms, cudaStream_t st) {
    if (n <= 0) return BTO_OK;
    dscal_kernel<<<egrid(n, sms), kThreads, 0, st>>>(n, a, x);
    return launch_status();
}
bto_status daxpy(int64_t n, double a, const double* x, double* y, int sms, cudaStream_t st) {
    if (n <= 0) return BTO_OK;
    daxpy_kernel<<<egrid(n, sms), kThreads, 0, st>>>(n, a, x, y);
    return launch_status();
}
bto_status dger(int64_t m, int64_t n, const double* x, const double* y, double* A, int64_t lda,
                int sms, cudaStream_t st) {
    if (m <= 0 || n <= 0) return BTO_OK;
    dger_kernel<<<(int)std::min<int64_t>(n, (int64_t)sms * 8), kThreads, 0, st>>>(m, n, x, y, A, lda);
    return launch_status();
}
// Copies an m x n matrix (lda) into B (ldb), column by column.
bto_status dcopy_mat(int64_t m, int64_t n, const double* A, int64_t lda, double* B, int64_t ldb,
                     int sms, cudaStream_t st) {
    if (m <= 0 || n <= 0) return BTO_OK;
    if (lda == m && ldb == m) return dcopy(m * n, A, B, sms, st);
    for (int64_t j = 0; j < n; j++) {
        bto_status e = dcopy(m, A + j * lda, B + j * ldb, sms, st);
        if (e != BTO_OK) return e;
    }
    return BTO_OK;
}

namespace {

// out = alpha A v (+ beta y if y != NULL): dgemv with trans = 'N'.
bto_status dgemv_n(int64_t m, int64_t n, double alpha, const double* A, int64_t lda,
                   const double* v, double beta, const double* y, double* out, double* qpart,
                   const PanelPlan& pl, cudaStream_t st) {
    if (m <= 0) return BTO_OK;
    PanelArgs a{};
    a.m = m; a.n = n; a.A = A; a.lda = lda; a.p = v; a.qpart = qpart;
    a.ldq = pl.ldq; a.lds = pl.lds; a.NR = pl.NR; a.NC = pl.NC; a.ntiles = pl.ntiles;
    bto_status e = launch_panel(PM_Q, a, pl, st);
    if (e != BTO_OK) return e;
    CombineJob j = {out, m, qpart, pl.ldq, pl.NC, alpha, nullptr, 0, 0, 0.0, y, beta};
    return launch_combine(&j, 1, st);
}
// out = alpha A^T v (+ beta y if y != NULL): dgemv with trans = 'T'.
bto_status dgemv_t(int64_t m, int64_t n, double alpha, const double* A, int64_t lda,
                   const double* v, double beta, const double* y, double* out, double* spart,
                   const PanelPlan& pl, cudaStream_t st) {
    if (n <= 0) return BTO_OK;
    PanelArgs a{};
    a.m = m; a.n = n; a.A = A; a.lda = lda; a.r = v; a.spart = spart;
    a.ldq = pl.ldq; a.lds = pl.lds; a.NR = pl.NR; a.NC = pl.NC; a.ntiles = pl.ntiles;
    bto_status e = launch_panel(PM_S, a, pl, st);
    if (e != BTO_OK) return e;
    CombineJob j = {out, n, spart, pl.lds, pl.NR, alpha, nullptr, 0, 0, 0.0, y, beta};
    return launch_combine(&j, 1, st);
}

struct Ctx {
    DeviceInfo d;
    WsLayout L;
    PanelPlan pl;
    char* w;
    double* at(int k) const { return reinterpret_cast<double*>(w + L.off[k]); }
};

bool make_ctx(int op, int form, int64_t m, int64_t n, void* ws, Ctx* c) {
    if (!device_info(&c->d)) return false;
    if (ws_layout(op, form, m, n, BTO_F64, c->d, &c->L) != BTO_OK) return false;
    c->pl = panel_plan(m, n, c->d.sms, op, BTO_FORM_UNFUSED);
    c->w = static_cast<char*>(ws);
    return true;
}

// The double-float form of an unfused sequence: each dgemv is a
// double-float single-product sweep and its combine, on df_plan's tiles and
// df_ws_layout's regions.  False (the FP64 form runs, on its own regions of
// the same workspace) when a matrix does not suit the tensor-map copies.
bool df_unfused_ready(int form, int op, int64_t m, int64_t n, const double* A, int64_t lda, const double* B,
                      int64_t ldb, Ctx* X, cudaStream_t st, bto_status* e) {
    *e = BTO_OK;
    if (form != BTO_FORM_DF_UNFUSED) return false;
    const PanelPlan dp = df_plan(m, n, X->d.sms);
    DfArgs a = df_args(m, n, A, lda, dp, X->w);
    bool ok = m > 0 && n > 0 && df_layout_ok(DF_Q, a);
    if (ok && B) {
        a.A = B; a.lda = ldb;
        ok = df_layout_ok(DF_Q, a);
    }
    // The status word reads BTO_OK after either path.
    *e = cudaMemsetAsync(X->w, 0, sizeof(int), st) == cudaSuccess ? BTO_OK : BTO_ERR_CUDA;
    if (!ok) {
        // FP64 regions of the same workspace.
        if (*e == BTO_OK && ws_layout(op, BTO_FORM_UNFUSED, m, n, BTO_F64, X->d, &X->L) != BTO_OK)
            *e = BTO_ERR_CUDA;
        return false;
    }
    X->pl = dp;
    return true;
}

#define TRY(x) do { bto_status e_ = (x); if (e_ != BTO_OK) return e_; } while (0)

}  // namespace
}  // namespace bto

using namespace bto;

static bto_status run_unfused_bicgk(int form, int64_t m, int64_t n, const double* A, int64_t lda,
                                        const double* p, const double* r, double* q, double* s,
                                        void* ws, size_t ws_bytes, bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    c.size(1, m); c.size(2, n);
    if (!c.ok()) return c.finish();
    const size_t Ab = mat_extent_bytes(m, n, lda, 8);
    c.ptr(3, A, m > 0 && n > 0); c.ld(4, lda, m);
    c.ptr(5, p, n > 0); c.ptr(6, r, m > 0); c.ptr(7, q, m > 0); c.ptr(8, s, n > 0);
    c.disjoint(7, q, vbytes(m), A, Ab); c.disjoint(7, q, vbytes(m), p, vbytes(n));
    c.disjoint(7, q, vbytes(m), r, vbytes(m)); c.disjoint(7, q, vbytes(m), s, vbytes(n));
    c.disjoint(8, s, vbytes(n), A, Ab); c.disjoint(8, s, vbytes(n), p, vbytes(n));
    c.disjoint(8, s, vbytes(n), r, vbytes(m));
    Ctx x;
    if (c.ok() && !make_ctx(BTO_OP_BICGK, form, m, n, ws, &x)) return BTO_ERR_CUDA;
    if (c.ok()) c.ws(9, ws, ws_bytes, x.L);
    if (!c.ok()) return c.finish();
    cudaStream_t st = (cudaStream_t)stream;
    bto_status e;
    if (df_unfused_ready(form, BTO_OP_BICGK, m, n, A, lda, nullptr, 0, &x, st, &e)) {
        TRY(e);
        TRY(df_gemv_n(m, n, 1.0, A, lda, p, 0.0, nullptr, q, x.at(0), x.pl, ws, 0, st));
        return df_gemv_t(m, n, 1.0, A, lda, r, 0.0, nullptr, s, x.at(1), x.pl, ws, 0, st);
    }
    TRY(e);
    // dgemv('N', m, n, 1.0, A, lda, p, 1, 0.0, q, 1)
    TRY(dgemv_n(m, n, 1.0, A, lda, p, 0.0, nullptr, q, x.at(0), x.pl, st));
    // dgemv('T', m, n, 1.0, A, lda, r, 1, 0.0, s, 1)
    return dgemv_t(m, n, 1.0, A, lda, r, 0.0, nullptr, s, x.at(1), x.pl, st);
}

static bto_status run_unfused_atax(int form, int64_t m, int64_t n, double beta, const double* A,
                                       int64_t lda, const double* x, double* y, void* ws,
                                       size_t ws_bytes, bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    c.size(1, m); c.size(2, n);
    if (!c.ok()) return c.finish();
    const size_t Ab = mat_extent_bytes(m, n, lda, 8);
    c.ptr(4, A, m > 0 && n > 0); c.ld(5, lda, m);
    c.ptr(6, x, n > 0); c.ptr(7, y, n > 0);
    c.disjoint(7, y, vbytes(n), A, Ab); c.disjoint(7, y, vbytes(n), x, vbytes(n));
    Ctx X;
    if (c.ok() && !make_ctx(BTO_OP_ATAX, form, m, n, ws, &X)) return BTO_ERR_CUDA;
    if (c.ok()) c.ws(8, ws, ws_bytes, X.L);
    if (!c.ok()) return c.finish();
    cudaStream_t st = (cudaStream_t)stream;
    bto_status e;
    if (df_unfused_ready(form, BTO_OP_ATAX, m, n, A, lda, nullptr, 0, &X, st, &e)) {
        TRY(e);
        double* t = X.at(0);
        TRY(df_gemv_n(m, n, 1.0, A, lda, x, 0.0, nullptr, t, X.at(1), X.pl, ws, 0, st));   // t0 = A x
        TRY(df_gemv_t(m, n, 1.0, A, lda, t, 0.0, nullptr, y, X.at(2), X.pl, ws, 0, st));   // t1 = A^T t0
        return dscal(n, beta, y, X.d.sms, st);                                              // y = t1 beta
    }
    TRY(e);
    double* t = X.at(0);
    TRY(dgemv_n(m, n, 1.0, A, lda, x, 0.0, nullptr, t, X.at(1), X.pl, st));    // t0 = A x
    TRY(dgemv_t(m, n, 1.0, A, lda, t, 0.0, nullptr, y, X.at(2), X.pl, st));    // t1 = A^T t0
    return dscal(n, beta, y, X.d.sms, st);                                       // y = t1 beta
}

static bto_status run_unfused_gemver(int form, int64_t m, int64_t n, double alpha, double beta,
                                         const double* A, int64_t lda, const double* u1,
                                         const double* v1, const double* u2, const double* v2,
                                         const double* y, const double* z, double* B, int64_t ldb,
                                         double* x, double* w, void* ws, size_t ws_bytes,
                                         bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    c.size(1, m); c.size(2, n);
    if (!c.ok()) return c.finish();
    const size_t Ab = mat_extent_bytes(m, n, lda, 8), Bb = mat_extent_bytes(m, n, ldb, 8);
    c.ptr(5, A, m > 0 && n > 0); c.ld(6, lda, m);
    c.ptr(7, u1, m > 0); c.ptr(8, v1, n > 0); c.ptr(9, u2, m > 0); c.ptr(10, v2, n > 0);
    c.ptr(11, y, m > 0); c.ptr(12, z, n > 0);
    c.ptr(13, B, m > 0 && n > 0); c.ld(14, ldb, m);
    c.ptr(15, x, n > 0); c.ptr(16, w, m > 0);
    const void* ins[6] = {u1, v1, u2, v2, y, z};
    const size_t inb[6] = {vbytes(m), vbytes(n), vbytes(m), vbytes(n), vbytes(m), vbytes(n)};
    c.disjoint(13, B, Bb, A, Ab);
    for (int k = 0; k < 6; k++) c.disjoint(13, B, Bb, ins[k], inb[k]);
    c.disjoint(15, x, vbytes(n), A, Ab); c.disjoint(15, x, vbytes(n), B, Bb);
    for (int k = 0; k < 6; k++) c.disjoint(15, x, vbytes(n), ins[k], inb[k]);
    c.disjoint(16, w, vbytes(m), A, Ab); c.disjoint(16, w, vbytes(m), B, Bb);
    for (int k = 0; k < 6; k++) c.disjoint(16, w, vbytes(m), ins[k], inb[k]);
    c.disjoint(16, w, vbytes(m), x, vbytes(n));
    Ctx X;
    if (c.ok() && !make_ctx(BTO_OP_GEMVER, form, m, n, ws, &X)) return BTO_ERR_CUDA;
    if (c.ok()) c.ws(17, ws, ws_bytes, X.L);
    if (!c.ok()) return c.finish();
    cudaStream_t st = (cudaStream_t)stream;
    const int sms = X.d.sms;
    bto_status e;
    if (df_unfused_ready(form, BTO_OP_GEMVER, m, n, B, ldb, nullptr, 0, &X, st, &e)) {
        TRY(e);
        TRY(dcopy_mat(m, n, A, lda, B, ldb, sms, st));                 // B = A
        TRY(dger(m, n, u1, v1, B, ldb, sms, st));                      // B += u1 v1^T
        TRY(dger(m, n, u2, v2, B, ldb, sms, st));                      // B += u2 v2^T
        TRY(dcopy(n, z, x, sms, st));                                  // x = z
        TRY(df_gemv_t(m, n, beta, B, ldb, y, 1.0, x, x, X.at(1), X.pl, ws, 0, st));      // x = beta B^T y + x
        return df_gemv_n(m, n, alpha, B, ldb, x, 0.0, nullptr, w, X.at(0), X.pl, ws, 0, st);   // w = alpha B x
    }
    TRY(e);
    TRY(dcopy_mat(m, n, A, lda, B, ldb, sms, st));                 // B = A
    TRY(dger(m, n, u1, v1, B, ldb, sms, st));                      // B += u1 v1^T
    TRY(dger(m, n, u2, v2, B, ldb, sms, st));                      // B += u2 v2^T
    TRY(dcopy(n, z, x, sms, st));                                  // x = z
    TRY(dgemv_t(m, n, beta, B, ldb, y, 1.0, x, x, X.at(1), X.pl, st));   // x = beta B^T y + x
    return dgemv_n(m, n, alpha, B, ldb, x, 0.0, nullptr, w, X.at(0), X.pl, st);   // w = alpha B x
}

static bto_status run_unfused_gesummv(int form, int64_t m, int64_t n, double alpha, const double* A,
                                          int64_t lda, double beta, const double* B, int64_t ldb,
                                          const double* x, double* y, void* ws, size_t ws_bytes,
                                          bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    c.size(1, m); c.size(2, n);
    if (!c.ok()) return c.finish();
    const size_t Ab = mat_extent_bytes(m, n, lda, 8), Bb = mat_extent_bytes(m, n, ldb, 8);
    c.ptr(4, A, m > 0 && n > 0); c.ld(5, lda, m);
    c.ptr(7, B, m > 0 && n > 0); c.ld(8, ldb, m);
    c.ptr(9, x, n > 0); c.ptr(10, y, m > 0);
    c.disjoint(10, y, vbytes(m), A, Ab); c.disjoint(10, y, vbytes(m), B, Bb);
    c.disjoint(10, y, vbytes(m), x, vbytes(n));
    Ctx X;
    if (c.ok() && !make_ctx(BTO_OP_GESUMMV, form, m, n, ws, &X)) return BTO_ERR_CUDA;
    if (c.ok()) c.ws(11, ws, ws_bytes, X.L);
    if (!c.ok()) return c.finish();
    cudaStream_t st = (cudaStream_t)stream;
    bto_status e;
    if (df_unfused_ready(form, BTO_OP_GESUMMV, m, n, A, lda, B, ldb, &X, st, &e)) {
        TRY(e);
        TRY(df_gemv_n(m, n, alpha, A, lda, x, 0.0, nullptr, y, X.at(0), X.pl, ws, 0, st));   // y = alpha A x
        return df_gemv_n(m, n, beta, B, ldb, x, 1.0, y, y, X.at(0), X.pl, ws, 0, st);        // y = beta B x + y
    }
    TRY(e);
    TRY(dgemv_n(m, n, alpha, A, lda, x, 0.0, nullptr, y, X.at(0), X.pl, st));   // y = alpha A x
    return dgemv_n(m, n, beta, B, ldb, x, 1.0, y, y, X.at(0), X.pl, st);         // y = beta B x + y
}

static bto_status run_unfused_dgemv(int form, int64_t m, int64_t n, double alpha, const double* A,
                                        int64_t lda, const double* x, double beta,
                                        const double* y, double* z, void* ws, size_t ws_bytes,
                                        bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    c.size(1, m); c.size(2, n);
    if (!c.ok()) return c.finish();
    const size_t Ab = mat_extent_bytes(m, n, lda, 8);
    c.ptr(4, A, m > 0 && n > 0); c.ld(5, lda, m);
    c.ptr(6, x, n > 0); c.ptr(8, y, m > 0); c.ptr(9, z, m > 0);
    c.disjoint(9, z, vbytes(m), A, Ab); c.disjoint(9, z, vbytes(m), x, vbytes(n));
    c.disjoint(9, z, vbytes(m), y, vbytes(m));
    Ctx X;
    if (c.ok() && !make_ctx(BTO_OP_DGEMV, form, m, n, ws, &X)) return BTO_ERR_CUDA;
    if (c.ok()) c.ws(10, ws, ws_bytes, X.L);
    if (!c.ok()) return c.finish();
    cudaStream_t st = (cudaStream_t)stream;
    bto_status e;
    if (df_unfused_ready(form, BTO_OP_DGEMV, m, n, A, lda, nullptr, 0, &X, st, &e)) {
        TRY(e);
        TRY(dcopy(m, y, z, X.d.sms, st));                                                         // z = y
        return df_gemv_n(m, n, alpha, A, lda, x, beta, z, z, X.at(0), X.pl, ws, 0, st);          // z = alpha A x + beta z
    }
    TRY(e);
    TRY(dcopy(m, y, z, X.d.sms, st));                                               // z = y
    return dgemv_n(m, n, alpha, A, lda, x, beta, z, z, X.at(0), X.pl, st);          // z = alpha A x + beta z
}

static bto_status run_unfused_dgemvt(int form, int64_t m, int64_t n, double alpha, double beta,
                                         const double* A, int64_t lda, const double* y,
                                         const double* z, double* x, double* w, void* ws,
                                         size_t ws_bytes, bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    c.size(1, m); c.size(2, n);
    if (!c.ok()) return c.finish();
    const size_t Ab = mat_extent_bytes(m, n, lda, 8);
    c.ptr(5, A, m > 0 && n > 0); c.ld(6, lda, m);
    c.ptr(7, y, m > 0); c.ptr(8, z, n > 0); c.ptr(9, x, n > 0); c.ptr(10, w, m > 0);
    c.disjoint(9, x, vbytes(n), A, Ab); c.disjoint(9, x, vbytes(n), y, vbytes(m));
    c.disjoint(9, x, vbytes(n), z, vbytes(n));
    c.disjoint(10, w, vbytes(m), A, Ab); c.disjoint(10, w, vbytes(m), y, vbytes(m));
    c.disjoint(10, w, vbytes(m), z, vbytes(n)); c.disjoint(10, w, vbytes(m), x, vbytes(n));
    Ctx X;
    if (c.ok() && !make_ctx(BTO_OP_DGEMVT, form, m, n, ws, &X)) return BTO_ERR_CUDA;
    if (c.ok()) c.ws(11, ws, ws_bytes, X.L);
    if (!c.ok()) return c.finish();
    cudaStream_t st = (cudaStream_t)stream;
    const int sms = X.d.sms;
    bto_status e;
    if (df_unfused_ready(form, BTO_OP_DGEMVT, m, n, A, lda, nullptr, 0, &X, st, &e)) {
        TRY(e);
        TRY(dcopy(n, z, x, sms, st));                                                           // x = z
        TRY(df_gemv_t(m, n, beta, A, lda, y, 1.0, x, x, X.at(1), X.pl, ws, 0, st));            // x = beta A^T y + x
        return df_gemv_n(m, n, alpha, A, lda, x, 0.0, nullptr, w, X.at(0), X.pl, ws, 0, st);   // w = alpha A x
    }
    TRY(e);
    TRY(dcopy(n, z, x, sms, st));                                                  // x = z
    TRY(dgemv_t(m, n, beta, A, lda, y, 1.0, x, x, X.at(1), X.pl, st));            // x = beta A^T y + x
    return dgemv_n(m, n, alpha, A, lda, x, 0.0, nullptr, w, X.at(0), X.pl, st);   // w = alpha A x
}

extern "C" bto_status bto_unfused_axpydot(int64_t n, double alpha, const double* w,
                                          const double* v, const double* u, double* z, double* r,
                                          void* ws, size_t ws_bytes, bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    c.size(1, n);
    if (!c.ok()) return c.finish();
    c.ptr(3, w, n > 0); c.ptr(4, v, n > 0); c.ptr(5, u, n > 0); c.ptr(6, z, n > 0); c.ptr(7, r, true);
    c.disjoint(6, z, vbytes(n), w, vbytes(n)); c.disjoint(6, z, vbytes(n), v, vbytes(n));
    c.disjoint(6, z, vbytes(n), u, vbytes(n));
    c.disjoint(7, r, 8, w, vbytes(n)); c.disjoint(7, r, 8, v, vbytes(n));
    c.disjoint(7, r, 8, u, vbytes(n)); c.disjoint(7, r, 8, z, vbytes(n));
    Ctx X;
    if (c.ok() && !make_ctx(BTO_OP_AXPYDOT, BTO_FORM_UNFUSED, 0, n, ws, &X)) return BTO_ERR_CUDA;
    if (c.ok()) c.ws(8, ws, ws_bytes, X.L);
    if (!c.ok()) return c.finish();
    cudaStream_t st = (cudaStream_t)stream;
    const int sms = X.d.sms, grid = vector_grid(sms);
    TRY(dcopy(n, w, z, sms, st));                                   // z = w
    TRY(daxpy(n, -alpha, v, z, sms, st));                           // z = -alpha v + z
    TRY(launch_dot_partials(n, 0.0, z, nullptr, u, nullptr, X.at(0), grid, 1, st));   // r = z^T u
    return launch_dot_final(X.at(0), grid, r, st);
}

extern "C" bto_status bto_unfused_waxpby(int64_t n, double alpha, const double* x, double beta,
                                         const double* y, double* w, bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    c.size(1, n);
    if (!c.ok()) return c.finish();
    c.ptr(3, x, n > 0); c.ptr(5, y, n > 0); c.ptr(6, w, n > 0);
    c.disjoint(6, w, vbytes(n), x, vbytes(n)); c.disjoint(6, w, vbytes(n), y, vbytes(n));
    if (!c.ok()) return c.finish();
    DeviceInfo d;
    if (!device_info(&d)) return BTO_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    TRY(dcopy(n, y, w, d.sms, st));            // w = y
    TRY(dscal(n, beta, w, d.sms, st));         // w = beta w
    return daxpy(n, alpha, x, w, d.sms, st);   // w = alpha x + w
}

extern "C" bto_status bto_unfused_vadd(int64_t n, const double* w, const double* y,
                                       const double* z, double* x, bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    c.size(1, n);
    if (!c.ok()) return c.finish();
    c.ptr(2, w, n > 0); c.ptr(3, y, n > 0); c.ptr(4, z, n > 0); c.ptr(5, x, n > 0);
    c.disjoint(5, x, vbytes(n), w, vbytes(n)); c.disjoint(5, x, vbytes(n), y, vbytes(n));
    c.disjoint(5, x, vbytes(n), z, vbytes(n));
    if (!c.ok()) return c.finish();
    DeviceInfo d;
    if (!device_info(&d)) return BTO_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    TRY(dcopy(n, w, x, d.sms, st));            // x = w
    TRY(daxpy(n, 1.0, y, x, d.sms, st));       // x = y + x
    return daxpy(n, 1.0, z, x, d.sms, st);     // x = z + x
}

extern "C" bto_status bto_unfused_bicgk(int64_t m, int64_t n, const double* A, int64_t lda, const double* p,
                                        const double* r, double* q, double* s, void* ws, size_t ws_bytes,
                                        bto_stream_t stream) {
    return run_unfused_bicgk(BTO_FORM_UNFUSED, m, n, A, lda, p, r, q, s, ws, ws_bytes, stream);
}
extern "C" bto_status bto_unfused_bicgk_df(int64_t m, int64_t n, const double* A, int64_t lda, const double* p,
                                           const double* r, double* q, double* s, void* ws, size_t ws_bytes,
                                           bto_stream_t stream) {
    return run_unfused_bicgk(BTO_FORM_DF_UNFUSED, m, n, A, lda, p, r, q, s, ws, ws_bytes, stream);
}
extern "C" bto_status bto_unfused_atax(int64_t m, int64_t n, double beta, const double* A, int64_t lda,
                                       const double* x, double* y, void* ws, size_t ws_bytes, bto_stream_t stream) {
    return run_unfused_atax(BTO_FORM_UNFUSED, m, n, beta, A, lda, x, y, ws, ws_bytes, stream);
}
extern "C" bto_status bto_unfused_atax_df(int64_t m, int64_t n, double beta, const double* A, int64_t lda,
                                          const double* x, double* y, void* ws, size_t ws_bytes,
                                          bto_stream_t stream) {
    return run_unfused_atax(BTO_FORM_DF_UNFUSED, m, n, beta, A, lda, x, y, ws, ws_bytes, stream);
}
extern "C" bto_status bto_unfused_gemver(int64_t m, int64_t n, double alpha, double beta, const double* A,
                                         int64_t lda, const double* u1, const double* v1, const double* u2,
                                         const double* v2, const double* y, const double* z, double* B,
                                         int64_t ldb, double* x, double* w, void* ws, size_t ws_bytes,
                                         bto_stream_t stream) {
    return run_unfused_gemver(BTO_FORM_UNFUSED, m, n, alpha, beta, A, lda, u1, v1, u2, v2, y, z, B, ldb, x, w,
                              ws, ws_bytes, stream);
}
extern "C" bto_status bto_unfused_gemver_df(int64_t m, int64_t n, double alpha, double beta, const double* A,
                                            int64_t lda, const double* u1, const double* v1, const double* u2,
                                            const double* v2, const double* y, const double* z, double* B,
                                            int64_t ldb, double* x, double* w, void* ws, size_t ws_bytes,
                                            bto_stream_t stream) {
    return run_unfused_gemver(BTO_FORM_DF_UNFUSED, m, n, alpha, beta, A, lda, u1, v1, u2, v2, y, z, B, ldb, x,
                              w, ws, ws_bytes, stream);
}
extern "C" bto_status bto_unfused_gesummv(int64_t m, int64_t n, double alpha, const double* A, int64_t lda,
                                          double beta, const double* B, int64_t ldb, const double* x, double* y,
                                          void* ws, size_t ws_bytes, bto_stream_t stream) {
    return run_unfused_gesummv(BTO_FORM_UNFUSED, m, n, alpha, A, lda, beta, B, ldb, x, y, ws, ws_bytes, stream);
}
extern "C" bto_status bto_unfused_gesummv_df(int64_t m, int64_t n, double alpha, const double* A, int64_t lda,
                                             double beta, const double* B, int64_t ldb, const double* x,
                                             double* y, void* ws, size_t ws_bytes, bto_stream_t stream) {
    return run_unfused_gesummv(BTO_FORM_DF_UNFUSED, m, n, alpha, A, lda, beta, B, ldb, x, y, ws, ws_bytes,
                               stream);
}
extern "C" bto_status bto_unfused_dgemv(int64_t m, int64_t n, double alpha, const double* A, int64_t lda,
                                        const double* x, double beta, const double* y, double* z, void* ws,
                                        size_t ws_bytes, bto_stream_t stream) {
    return run_unfused_dgemv(BTO_FORM_UNFUSED, m, n, alpha, A, lda, x, beta, y, z, ws, ws_bytes, stream);
}
extern "C" bto_status bto_unfused_dgemv_df(int64_t m, int64_t n, double alpha, const double* A, int64_t lda,
                                           const double* x, double beta, const double* y, double* z, void* ws,
                                           size_t ws_bytes, bto_stream_t stream) {
    return run_unfused_dgemv(BTO_FORM_DF_UNFUSED, m, n, alpha, A, lda, x, beta, y, z, ws, ws_bytes, stream);
}
extern "C" bto_status bto_unfused_dgemvt(int64_t m, int64_t n, double alpha, double beta, const double* A,
                                         int64_t lda, const double* y, const double* z, double* x, double* w,
                                         void* ws, size_t ws_bytes, bto_stream_t stream) {
    return run_unfused_dgemvt(BTO_FORM_UNFUSED, m, n, alpha, beta, A, lda, y, z, x, w, ws, ws_bytes, stream);
}
extern "C" bto_status bto_unfused_dgemvt_df(int64_t m, int64_t n, double alpha, double beta, const double* A,
                                            int64_t lda, const double* y, const double* z, double* x, double* w,
                                            void* ws, size_t ws_bytes, bto_stream_t stream) {
    return run_unfused_dgemvt(BTO_FORM_DF_UNFUSED, m, n, alpha, beta, A, lda, y, z, x, w, ws, ws_bytes, stream);
}
