// Storage order and transposition for the FP64 matrix kernels.
//
// The paper's types describe a matrix as a container of containers, a
// column-major one as a row of columns and a row-major one as a column of
// rows (Section II; BATAX's A in Fig. 1 is declared row-major), and BTO
// generates code for either.  Here a row-major m x n matrix A with leading
// dimension lda is the column-major n x m matrix S = A^T with the same lda,
// so every statement is rewritten onto the stored matrix S:
//
//   A x   = S^T x   (the column sums of the panel engine, s partials)
//   A^T y = S y     (the row accumulators of the panel engine, q partials)
//
// and the same fused passes run with the two products' roles exchanged:
// BICGK stays one pass, GEMVER's first pass forms S_B = S_A + v1 u1^T +
// v2 u2^T together with S_B y (mode PM_G1Q), DGEMVT and DGEMV map onto the
// single-product modes.  GESUMMV on row-major storage takes one column-sum
// pass per matrix (each matrix still read once; the paired row-accumulator
// pass has no column-sum twin), and BATAX on row-major storage two passes,
// t = A x then y = beta A^T t (its single-read group-band kernel is written
// for column-major bands).  Column-major calls go to the ordinary entry points.
#include "check.cuh"

namespace bto {
namespace {

bool layout_ok(int layout) { return layout == BTO_COL_MAJOR || layout == BTO_ROW_MAJOR; }

// Workspace of a call on the stored n x m matrix (row-major), or of the
// transposed DGEMV on column-major storage: the plan is the op's fused plan
// on the stored shape.
bto_status layout_ws(int op, int64_t R, int64_t K, const DeviceInfo& d, WsLayout* out) {
    const PanelPlan pl = panel_plan(R, K, d.sms, op, BTO_FORM_FUSED);
    WsLayout L;
    size_t cur = WS_HEADER;
    auto region = [&](size_t bytes) {
        const size_t at = cur;
        cur += round_up((int64_t)bytes, 256);
        return at;
    };
    const size_t qp = (size_t)pl.NC * pl.ldq * sizeof(double);
    const size_t sp = (size_t)pl.NR * pl.lds * sizeof(double);
    L.off[0] = region(qp);
    L.off[1] = region(sp);
    if (op == BTO_OP_GESUMMV) L.off[2] = region(sp);
    if (op == BTO_OP_ATAX) L.off[3] = region((size_t)std::max<int64_t>(K, 1) * sizeof(double));
    L.total = cur;
    *out = L;
    return BTO_OK;
}

double* wsd(void* ws, size_t off) { return reinterpret_cast<double*>(static_cast<char*>(ws) + off); }

// Panel arguments for the stored R x K matrix.
PanelArgs stored(const PanelPlan& pl, int64_t R, int64_t K, const double* S, int64_t lds_mat, void* ws,
                 const WsLayout& L) {
    PanelArgs a{};
    a.m = R; a.n = K; a.A = S; a.lda = lds_mat;
    a.qpart = wsd(ws, L.off[0]); a.spart = wsd(ws, L.off[1]);
    a.ldq = pl.ldq; a.lds = pl.lds; a.NR = pl.NR; a.NC = pl.NC; a.ntiles = pl.ntiles;
    return a;
}

// out = a1 * (row-accumulator result, length R) + b * v.
CombineJob q_job(const PanelArgs& a, double* out, double a1, const double* v, double b) {
    return CombineJob{out, a.m, a.qpart, a.ldq, a.NC, a1, nullptr, 0, 0, 0.0, v, b};
}
// out = a1 * (column-sum result, length K) + b * v.
CombineJob s_job(const PanelArgs& a, double* out, double a1, const double* v, double b) {
    return CombineJob{out, a.n, a.spart, a.lds, a.NR, a1, nullptr, 0, 0, 0.0, v, b};
}

// Shifts the invalid-argument position of a delegated call past the extra
// leading arguments of the layout entry point.
bto_status shifted(bto_status st, int extra) {
    if (st != BTO_OK && last_invalid_arg() > 0) set_invalid_arg(last_invalid_arg() + extra);
    return st;
}

bool prepare(int op, int64_t R, int64_t K, DeviceInfo* d, WsLayout* L) {
    if (!device_info(d)) return false;
    return layout_ws(op, R, K, *d, L) == BTO_OK;
}

bto_status layout_workspace(int op, int layout, int trans, int64_t m, int64_t n, const DeviceInfo& d,
                            WsLayout* out) {
    if (layout == BTO_COL_MAJOR && !(op == BTO_OP_DGEMV && trans == BTO_TRANS))
        return ws_layout(op, BTO_FORM_FUSED, m, n, BTO_F64, d, out);
    if (layout == BTO_COL_MAJOR) return layout_ws(op, m, n, d, out);
    return layout_ws(op, n, m, d, out);
}

}  // namespace
}  // namespace bto

using namespace bto;

extern "C" bto_status bto_layout_workspace_bytes(int op, int layout, int trans, int64_t m, int64_t n,
                                                 size_t* bytes) {
    clear_invalid_arg();
    if (op < BTO_OP_BICGK || op > BTO_OP_DGEMVT) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (!layout_ok(layout)) { set_invalid_arg(2); return BTO_ERR_INVALID_VALUE; }
    if (trans != BTO_NO_TRANS && !(trans == BTO_TRANS && op == BTO_OP_DGEMV)) {
        set_invalid_arg(3);
        return BTO_ERR_INVALID_VALUE;
    }
    if (m < 0) { set_invalid_arg(4); return BTO_ERR_INVALID_VALUE; }
    if (n < 0) { set_invalid_arg(5); return BTO_ERR_INVALID_VALUE; }
    if (!bytes) { set_invalid_arg(6); return BTO_ERR_INVALID_VALUE; }
    DeviceInfo d;
    if (!device_info(&d)) return BTO_ERR_CUDA;
    WsLayout L;
    const bto_status st = layout_workspace(op, layout, trans, m, n, d, &L);
    if (st != BTO_OK) return st;
    *bytes = L.total;
    return BTO_OK;
}

extern "C" bto_status bto_bicgk_layout(int layout, int64_t m, int64_t n, const double* A, int64_t lda,
                                       const double* p, const double* r, double* q, double* s, void* ws,
                                       size_t ws_bytes, bto_stream_t stream) {
    clear_invalid_arg();
    if (!layout_ok(layout)) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (layout == BTO_COL_MAJOR) return shifted(bto_bicgk(m, n, A, lda, p, r, q, s, ws, ws_bytes, stream), 1);
    Check c;
    c.size(2, m); c.size(3, n);
    if (!c.ok()) return c.finish();
    const size_t Ab = mat_extent_bytes(n, m, lda, 8);
    c.ptr(4, A, m > 0 && n > 0); c.ld(5, lda, n);
    c.ptr(6, p, n > 0); c.ptr(7, r, m > 0); c.ptr(8, q, m > 0); c.ptr(9, s, n > 0);
    c.disjoint(8, q, vbytes(m), A, Ab); c.disjoint(8, q, vbytes(m), p, vbytes(n));
    c.disjoint(8, q, vbytes(m), r, vbytes(m)); c.disjoint(8, q, vbytes(m), s, vbytes(n));
    c.disjoint(9, s, vbytes(n), A, Ab); c.disjoint(9, s, vbytes(n), p, vbytes(n));
    c.disjoint(9, s, vbytes(n), r, vbytes(m));
    DeviceInfo d; WsLayout L;
    if (c.ok() && !prepare(BTO_OP_BICGK, n, m, &d, &L)) return BTO_ERR_CUDA;
    if (c.ok()) c.ws(10, ws, ws_bytes, L);
    if (!c.ok()) return c.finish();

    cudaStream_t st = (cudaStream_t)stream;
    const PanelPlan pl = panel_plan(n, m, d.sms, BTO_OP_BICGK, BTO_FORM_FUSED);
    PanelArgs a = stored(pl, n, m, A, lda, ws, L);
    a.p = r;   // A^T r = S r: row accumulators, length n
    a.r = p;   // A p = S^T p: column sums, length m
    bto_status e = launch_panel(PM_QS, a, pl, st);
    if (e != BTO_OK) return e;
    CombineJob j[2] = {s_job(a, q, 1.0, nullptr, 0.0), q_job(a, s, 1.0, nullptr, 0.0)};
    return launch_combine(j, 2, st);
}

extern "C" bto_status bto_dgemv_layout(int layout, int trans, int64_t m, int64_t n, double alpha,
                                       const double* A, int64_t lda, const double* x, double beta,
                                       const double* y, double* z, void* ws, size_t ws_bytes,
                                       bto_stream_t stream) {
    clear_invalid_arg();
    if (!layout_ok(layout)) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (trans != BTO_NO_TRANS && trans != BTO_TRANS) { set_invalid_arg(2); return BTO_ERR_INVALID_VALUE; }
    if (layout == BTO_COL_MAJOR && trans == BTO_NO_TRANS)
        return shifted(bto_dgemv(m, n, alpha, A, lda, x, beta, y, z, ws, ws_bytes, stream), 2);
    Check c;
    c.size(3, m); c.size(4, n);
    if (!c.ok()) return c.finish();
    const bool row = layout == BTO_ROW_MAJOR;
    const int64_t R = row ? n : m, K = row ? m : n;          // stored matrix: R x K, column-major
    const int64_t lx = trans ? m : n, lz = trans ? n : m;    // op(A) x: x has lx, y and z have lz
    const size_t Ab = mat_extent_bytes(R, K, lda, 8);
    c.ptr(6, A, m > 0 && n > 0); c.ld(7, lda, R);
    c.ptr(8, x, lx > 0 && lz > 0); c.ptr(10, y, lz > 0); c.ptr(11, z, lz > 0);
    c.disjoint(11, z, vbytes(lz), A, Ab); c.disjoint(11, z, vbytes(lz), x, vbytes(lx));
    if (z != y) c.disjoint(11, z, vbytes(lz), y, vbytes(lz));
    DeviceInfo d; WsLayout L;
    if (c.ok() && !prepare(BTO_OP_DGEMV, R, K, &d, &L)) return BTO_ERR_CUDA;
    if (c.ok()) c.ws(12, ws, ws_bytes, L);
    if (!c.ok()) return c.finish();

    cudaStream_t st = (cudaStream_t)stream;
    const PanelPlan pl = panel_plan(R, K, d.sms, BTO_OP_DGEMV, BTO_FORM_FUSED);
    PanelArgs a = stored(pl, R, K, A, lda, ws, L);
    // op(A) = S (row-major, transposed): row accumulators; op(A) = S^T: column sums.
    const bool rows = row && trans;
    if (rows) a.p = x; else a.r = x;
    // An empty product plans no tiles, and the combine then gives z = beta y.
    bto_status e = launch_panel(rows ? PM_Q : PM_S, a, pl, st);
    if (e != BTO_OK) return e;
    CombineJob j = rows ? q_job(a, z, alpha, y, beta) : s_job(a, z, alpha, y, beta);
    return launch_combine(&j, 1, st);
}

extern "C" bto_status bto_dgemvt_layout(int layout, int64_t m, int64_t n, double alpha, double beta,
                                        const double* A, int64_t lda, const double* y, const double* z,
                                        double* x, double* w, void* ws, size_t ws_bytes,
                                        bto_stream_t stream) {
    clear_invalid_arg();
    if (!layout_ok(layout)) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (layout == BTO_COL_MAJOR)
        return shifted(bto_dgemvt(m, n, alpha, beta, A, lda, y, z, x, w, ws, ws_bytes, stream), 1);
    Check c;
    c.size(2, m); c.size(3, n);
    if (!c.ok()) return c.finish();
    const size_t Ab = mat_extent_bytes(n, m, lda, 8);
    c.ptr(6, A, m > 0 && n > 0); c.ld(7, lda, n);
    c.ptr(8, y, m > 0); c.ptr(9, z, n > 0); c.ptr(10, x, n > 0); c.ptr(11, w, m > 0);
    c.disjoint(10, x, vbytes(n), A, Ab); c.disjoint(10, x, vbytes(n), y, vbytes(m));
    if (x != z) c.disjoint(10, x, vbytes(n), z, vbytes(n));
    c.disjoint(11, w, vbytes(m), A, Ab); c.disjoint(11, w, vbytes(m), y, vbytes(m));
    c.disjoint(11, w, vbytes(m), z, vbytes(n)); c.disjoint(11, w, vbytes(m), x, vbytes(n));
    DeviceInfo d; WsLayout L;
    if (c.ok() && !prepare(BTO_OP_DGEMVT, n, m, &d, &L)) return BTO_ERR_CUDA;
    if (c.ok()) c.ws(12, ws, ws_bytes, L);
    if (!c.ok()) return c.finish();

    cudaStream_t st = (cudaStream_t)stream;
    const PanelPlan pl = panel_plan(n, m, d.sms, BTO_OP_DGEMVT, BTO_FORM_FUSED);
    PanelArgs a = stored(pl, n, m, A, lda, ws, L);
    // Pass 1: x = beta A^T y + z = beta S y + z (row accumulators, length n).
    a.p = y;
    bto_status e = launch_panel(PM_Q, a, pl, st);
    if (e != BTO_OK) return e;
    CombineJob jx = q_job(a, x, beta, z, 1.0);
    if ((e = launch_combine(&jx, 1, st)) != BTO_OK) return e;
    // Pass 2: w = alpha A x = alpha S^T x (column sums), tiles in reverse so
    // the tail still in L2 is read first.
    a.p = nullptr; a.r = x; a.reverse = 1;
    if ((e = launch_panel(PM_S, a, pl, st)) != BTO_OK) return e;
    CombineJob jw = s_job(a, w, alpha, nullptr, 0.0);
    return launch_combine(&jw, 1, st);
}

extern "C" bto_status bto_gesummv_layout(int layout, int64_t m, int64_t n, double alpha, const double* A,
                                         int64_t lda, double beta, const double* B, int64_t ldb,
                                         const double* x, double* y, void* ws, size_t ws_bytes,
                                         bto_stream_t stream) {
    clear_invalid_arg();
    if (!layout_ok(layout)) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (layout == BTO_COL_MAJOR)
        return shifted(bto_gesummv(m, n, alpha, A, lda, beta, B, ldb, x, y, ws, ws_bytes, stream), 1);
    Check c;
    c.size(2, m); c.size(3, n);
    if (!c.ok()) return c.finish();
    const size_t Ab = mat_extent_bytes(n, m, lda, 8), Bb = mat_extent_bytes(n, m, ldb, 8);
    c.ptr(5, A, m > 0 && n > 0); c.ld(6, lda, n);
    c.ptr(8, B, m > 0 && n > 0); c.ld(9, ldb, n);
    c.ptr(10, x, n > 0); c.ptr(11, y, m > 0);
    c.disjoint(11, y, vbytes(m), A, Ab); c.disjoint(11, y, vbytes(m), B, Bb);
    c.disjoint(11, y, vbytes(m), x, vbytes(n));
    DeviceInfo d; WsLayout L;
    if (c.ok() && !prepare(BTO_OP_GESUMMV, n, m, &d, &L)) return BTO_ERR_CUDA;
    if (c.ok()) c.ws(12, ws, ws_bytes, L);
    if (!c.ok()) return c.finish();

    cudaStream_t st = (cudaStream_t)stream;
    const PanelPlan pl = panel_plan(n, m, d.sms, BTO_OP_GESUMMV, BTO_FORM_FUSED);
    // A x = S_A^T x and B x = S_B^T x: one column-sum pass per matrix.
    PanelArgs a = stored(pl, n, m, A, lda, ws, L);
    a.r = x;
    bto_status e = launch_panel(PM_S, a, pl, st);
    if (e != BTO_OK) return e;
    PanelArgs b = a;
    b.A = B; b.lda = ldb; b.spart = wsd(ws, L.off[2]);
    if ((e = launch_panel(PM_S, b, pl, st)) != BTO_OK) return e;
    CombineJob j = {y, m, a.spart, a.lds, a.NR, alpha, b.spart, b.lds, b.NR, beta, nullptr, 0.0};
    return launch_combine(&j, 1, st);
}

extern "C" bto_status bto_atax_layout(int layout, int64_t m, int64_t n, double beta, const double* A,
                                      int64_t lda, const double* x, double* y, void* ws, size_t ws_bytes,
                                      bto_stream_t stream) {
    clear_invalid_arg();
    if (!layout_ok(layout)) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (layout == BTO_COL_MAJOR) return shifted(bto_atax(m, n, beta, A, lda, x, y, ws, ws_bytes, stream), 1);
    Check c;
    c.size(2, m); c.size(3, n);
    if (!c.ok()) return c.finish();
    const size_t Ab = mat_extent_bytes(n, m, lda, 8);
    c.ptr(5, A, m > 0 && n > 0); c.ld(6, lda, n);
    c.ptr(7, x, n > 0); c.ptr(8, y, n > 0);
    c.disjoint(8, y, vbytes(n), A, Ab); c.disjoint(8, y, vbytes(n), x, vbytes(n));
    DeviceInfo d; WsLayout L;
    if (c.ok() && !prepare(BTO_OP_ATAX, n, m, &d, &L)) return BTO_ERR_CUDA;
    if (c.ok()) c.ws(9, ws, ws_bytes, L);
    if (!c.ok()) return c.finish();

    // An empty matrix plans no tiles; the combines then give t = 0 and y = 0.
    cudaStream_t st = (cudaStream_t)stream;
    const PanelPlan pl = panel_plan(n, m, d.sms, BTO_OP_ATAX, BTO_FORM_FUSED);
    PanelArgs a = stored(pl, n, m, A, lda, ws, L);
    double* t = wsd(ws, L.off[3]);
    // t = A x = S^T x (column sums, length m).
    a.r = x;
    bto_status e = launch_panel(PM_S, a, pl, st);
    if (e != BTO_OK) return e;
    CombineJob jt = s_job(a, t, 1.0, nullptr, 0.0);
    if ((e = launch_combine(&jt, 1, st)) != BTO_OK) return e;
    // y = beta A^T t = beta S t (row accumulators, length n), tiles reversed.
    a.r = nullptr; a.p = t; a.reverse = 1;
    if ((e = launch_panel(PM_Q, a, pl, st)) != BTO_OK) return e;
    CombineJob jy = q_job(a, y, beta, nullptr, 0.0);
    return launch_combine(&jy, 1, st);
}

extern "C" bto_status bto_gemver_layout(int layout, int64_t m, int64_t n, double alpha, double beta,
                                        const double* A, int64_t lda, const double* u1, const double* v1,
                                        const double* u2, const double* v2, const double* y,
                                        const double* z, double* B, int64_t ldb, double* x, double* w,
                                        void* ws, size_t ws_bytes, bto_stream_t stream) {
    clear_invalid_arg();
    if (!layout_ok(layout)) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (layout == BTO_COL_MAJOR)
        return shifted(bto_gemver(m, n, alpha, beta, A, lda, u1, v1, u2, v2, y, z, B, ldb, x, w, ws,
                                  ws_bytes, stream), 1);
    Check c;
    c.size(2, m); c.size(3, n);
    if (!c.ok()) return c.finish();
    const size_t Ab = mat_extent_bytes(n, m, lda, 8), Bb = mat_extent_bytes(n, m, ldb, 8);
    c.ptr(6, A, m > 0 && n > 0); c.ld(7, lda, n);
    c.ptr(8, u1, m > 0); c.ptr(9, v1, n > 0); c.ptr(10, u2, m > 0); c.ptr(11, v2, n > 0);
    c.ptr(12, y, m > 0); c.ptr(13, z, n > 0);
    c.ptr(14, B, m > 0 && n > 0); c.ld(15, ldb, n);
    c.ptr(16, x, n > 0); c.ptr(17, w, m > 0);
    const void* ins[6] = {u1, v1, u2, v2, y, z};
    const size_t inb[6] = {vbytes(m), vbytes(n), vbytes(m), vbytes(n), vbytes(m), vbytes(n)};
    if (!(B == A && ldb == lda)) c.disjoint(14, B, Bb, A, Ab);
    for (int k = 0; k < 6; k++) c.disjoint(14, B, Bb, ins[k], inb[k]);
    c.disjoint(16, x, vbytes(n), A, Ab); c.disjoint(16, x, vbytes(n), B, Bb);
    for (int k = 0; k < 5; k++) c.disjoint(16, x, vbytes(n), ins[k], inb[k]);
    if (x != z) c.disjoint(16, x, vbytes(n), z, vbytes(n));
    c.disjoint(17, w, vbytes(m), A, Ab); c.disjoint(17, w, vbytes(m), B, Bb);
    for (int k = 0; k < 6; k++) c.disjoint(17, w, vbytes(m), ins[k], inb[k]);
    c.disjoint(17, w, vbytes(m), x, vbytes(n));
    DeviceInfo d; WsLayout L;
    if (c.ok() && !prepare(BTO_OP_GEMVER, n, m, &d, &L)) return BTO_ERR_CUDA;
    if (c.ok()) c.ws(18, ws, ws_bytes, L);
    if (!c.ok()) return c.finish();

    // An empty matrix plans no tiles; the combines then give x = z and w = 0.
    cudaStream_t st = (cudaStream_t)stream;
    const PanelPlan pl = panel_plan(n, m, d.sms, BTO_OP_GEMVER, BTO_FORM_FUSED);
    PanelArgs a = stored(pl, n, m, A, lda, ws, L);
    // Pass 1: S_B = S_A + v1 u1^T + v2 u2^T (v row-indexed, u column-indexed
    // in the stored matrix) and x = beta B^T y + z = beta S_B y + z.
    a.Bout = B; a.ldb = ldb;
    a.u1 = v1; a.u2 = v2; a.v1 = u1; a.v2 = u2; a.p = y;
    bto_status e = launch_panel(PM_G1Q, a, pl, st);
    if (e != BTO_OK) return e;
    CombineJob jx = q_job(a, x, beta, z, 1.0);
    if ((e = launch_combine(&jx, 1, st)) != BTO_OK) return e;
    // Pass 2: w = alpha B x = alpha S_B^T x (column sums), tiles reversed.
    PanelArgs b = a;
    b.A = B; b.lda = ldb; b.Bout = nullptr; b.p = nullptr; b.r = x; b.reverse = 1;
    if ((e = launch_panel(PM_S, b, pl, st)) != BTO_OK) return e;
    CombineJob jw = s_job(b, w, alpha, nullptr, 0.0);
    return launch_combine(&jw, 1, st);
}
