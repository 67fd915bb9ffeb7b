// Fused FP64 entry points built on the panel engine (BICGK, GEMVER, GESUMMV,
// DGEMV, DGEMVT) and the workspace layouts of every entry point.
#include "check.cuh"

namespace bto {

namespace {

size_t region(size_t& cur, size_t bytes) {
    size_t at = cur;
    cur += round_up((int64_t)bytes, 256);
    return at;
}

}  // namespace

bto_status ws_layout(int op, int form, int64_t m, int64_t n, int a_type, const DeviceInfo& d,
                     WsLayout* out) {
    if (form == BTO_FORM_DF || form == BTO_FORM_DF_UNFUSED) {
        if (a_type != BTO_F64) return BTO_ERR_UNSUPPORTED;
        return df_ws_layout(op, form, m, n, d, out);
    }
    // Reduced-precision storage exists for the fused BICGK, GEMVER, ATAX and
    // GESUMMV forms (bto_*_ex); their partials take the FP64 form's space.
    if (a_type != BTO_F64 &&
        !(form == BTO_FORM_FUSED && (op == BTO_OP_BICGK || op == BTO_OP_GEMVER || op == BTO_OP_ATAX ||
                                     op == BTO_OP_GESUMMV)))
        return BTO_ERR_UNSUPPORTED;
    WsLayout L;
    size_t cur = WS_HEADER;
    PanelPlan pl = a_type == BTO_F64 ? panel_plan(m, n, d.sms, op, form)
                                     : lp_plan(m, n, d.sms, a_type, lp_blocks_per_sm(op, a_type), false);
    if (a_type != BTO_F64) {
        // Room for the partials of either split (the call picks one by the
        // operands' alignment).
        const PanelPlan pb = lp_plan(m, n, d.sms, a_type, lp_blocks_per_sm(op, a_type), true);
        pl.NC = std::max(pl.NC, pb.NC);
        pl.NR = std::max(pl.NR, pb.NR);
    }
    const size_t qp = (size_t)pl.NC * pl.ldq * sizeof(double);
    const size_t sp = (size_t)pl.NR * pl.lds * sizeof(double);
    switch (op) {
        case BTO_OP_BICGK:
        case BTO_OP_GEMVER:
        case BTO_OP_DGEMVT:
            L.off[0] = region(cur, qp);
            L.off[1] = region(cur, sp);
            break;
        case BTO_OP_DGEMV:
            L.off[0] = region(cur, qp);
            break;
        case BTO_OP_GESUMMV:
            L.off[0] = region(cur, qp);
            if (form == BTO_FORM_FUSED) L.off[1] = region(cur, qp);
            break;
        case BTO_OP_ATAX:
            if (form == BTO_FORM_FUSED && a_type == BTO_F64) {
                const AtaxPlan ap = atax_plan(m, n, d);
                if (ap.fused) {
                    L.off[0] = region(cur, (size_t)std::max(ap.G, 1) * sizeof(unsigned));             // per-block flags
                    L.off[1] = region(cur, (size_t)ap.NG * 2 * ap.D * ap.S * ap.TB * sizeof(double));  // t partial slots
                    L.off[2] = region(cur, (size_t)ap.NG * std::max<int64_t>(ap.ldy, 1) * sizeof(double)); // y partials
                    break;
                }
            }
            L.off[0] = region(cur, (size_t)std::max<int64_t>(m, 1) * sizeof(double));    // t = A x
            L.off[1] = region(cur, qp);
            L.off[2] = region(cur, sp);
            break;
        case BTO_OP_AXPYDOT:
            L.off[0] = region(cur, (size_t)vector_grid(d.sms) * sizeof(double));
            break;
        case BTO_OP_WAXPBY:
        case BTO_OP_VADD:
            cur = 0;
            break;
        default:
            return BTO_ERR_INVALID_VALUE;
    }
    L.total = cur;
    *out = L;
    return BTO_OK;
}

}  // namespace bto

using namespace bto;

namespace {

// Shared preamble: device facts and the workspace layout of op.
bool prepare(int op, int form, int64_t m, int64_t n, DeviceInfo* d, WsLayout* L) {
    if (!device_info(d)) return false;
    return ws_layout(op, form, m, n, BTO_F64, *d, L) == BTO_OK;
}

double* wsd(void* ws, size_t off) { return reinterpret_cast<double*>(static_cast<char*>(ws) + off); }

// The double-float form runs on the plan and workspace regions of df_plan /
// df_ws_layout, after clearing the status word; when the matrices do not suit
// its tensor-map copies, the FP64 form runs instead, on its own regions of
// the same workspace (df_ws_layout makes room for both).
// The status word is cleared on either path (true with *e set on failure).
bool df_ready(int form, int mode, const DfArgs& a, cudaStream_t st, bto_status* e) {
    *e = BTO_OK;
    if (form != BTO_FORM_DF) return false;
    if (cudaMemsetAsync(a.status, 0, sizeof(int), st) != cudaSuccess) {
        *e = BTO_ERR_CUDA;
        return true;
    }
    return a.m > 0 && a.n > 0 && df_layout_ok(mode, a);
}

}  // namespace

// stall_block >= 0 (testing): the double-float sweep's producer in that block
// stops after one ring fill and the ring waits give up after wait_ns; the
// call is then BTO_ERR_UNSUPPORTED unless that sweep runs.
static bto_status run_bicgk(int form, int64_t m, int64_t n, const double* A, int64_t lda,
                            const double* p, const double* r, double* q, double* s,
                            void* ws, size_t ws_bytes, bto_stream_t stream, int stall_block = -1,
                            unsigned long long wait_ns = 0) {
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
    DeviceInfo d; WsLayout L;
    if (c.ok() && !prepare(BTO_OP_BICGK, form, m, n, &d, &L)) return BTO_ERR_CUDA;
    if (c.ok()) c.ws(9, ws, ws_bytes, L);
    if (!c.ok()) return c.finish();

    cudaStream_t st = (cudaStream_t)stream;
    {
        const PanelPlan dp = df_plan(m, n, d.sms);
        DfArgs a = df_args(m, n, A, lda, dp, ws);
        a.p = p; a.r = r; a.qpart = wsd(ws, L.off[0]); a.spart = wsd(ws, L.off[1]);
        if (stall_block >= 0) {
            a.stall_block = stall_block;
            a.wait_ns = wait_ns;
        }
        bto_status e;
        if (df_ready(form, DF_QS, a, st, &e)) {
            if (e != BTO_OK || (e = df_launch(DF_QS, a, dp, st)) != BTO_OK) return e;
            CombineJob j[2] = {};
            j[0] = {q, m, a.qpart, dp.ldq, dp.NC, 1.0, nullptr, 0, 0, 0.0, nullptr, 0.0};
            j[1] = {s, n, a.spart, dp.lds, dp.NR, 1.0, nullptr, 0, 0, 0.0, nullptr, 0.0};
            return launch_combine(j, 2, st);
        }
        if (stall_block >= 0) return BTO_ERR_UNSUPPORTED;
        if (form == BTO_FORM_DF && ws_layout(BTO_OP_BICGK, BTO_FORM_FUSED, m, n, BTO_F64, d, &L) != BTO_OK)
            return BTO_ERR_CUDA;
    }
    const PanelPlan pl = panel_plan(m, n, d.sms, BTO_OP_BICGK, BTO_FORM_FUSED);
    PanelArgs a{};
    a.m = m; a.n = n; a.A = A; a.lda = lda; a.p = p; a.r = r;
    a.qpart = wsd(ws, L.off[0]); a.spart = wsd(ws, L.off[1]);
    a.ldq = pl.ldq; a.lds = pl.lds; a.NR = pl.NR; a.NC = pl.NC; a.ntiles = pl.ntiles;
    bto_status e = launch_panel(PM_QS, a, pl, st);
    if (e != BTO_OK) return e;
    CombineJob j[2] = {};
    j[0] = {q, m, a.qpart, pl.ldq, pl.NC, 1.0, nullptr, 0, 0, 0.0, nullptr, 0.0};
    j[1] = {s, n, a.spart, pl.lds, pl.NR, 1.0, nullptr, 0, 0, 0.0, nullptr, 0.0};
    return launch_combine(j, 2, st);
}

static bto_status run_dgemv(int form, int64_t m, int64_t n, double alpha, const double* A, int64_t lda,
                            const double* x, double beta, const double* y, double* z,
                            void* ws, size_t ws_bytes, bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    c.size(1, m); c.size(2, n);
    if (!c.ok()) return c.finish();
    const size_t Ab = mat_extent_bytes(m, n, lda, 8);
    c.ptr(4, A, m > 0 && n > 0); c.ld(5, lda, m);
    c.ptr(6, x, n > 0); c.ptr(8, y, m > 0); c.ptr(9, z, m > 0);
    c.disjoint(9, z, vbytes(m), A, Ab); c.disjoint(9, z, vbytes(m), x, vbytes(n));
    if (z != y) c.disjoint(9, z, vbytes(m), y, vbytes(m));
    DeviceInfo d; WsLayout L;
    if (c.ok() && !prepare(BTO_OP_DGEMV, form, m, n, &d, &L)) return BTO_ERR_CUDA;
    if (c.ok()) c.ws(10, ws, ws_bytes, L);
    if (!c.ok()) return c.finish();

    cudaStream_t st = (cudaStream_t)stream;
    {
        const PanelPlan dp = df_plan(m, n, d.sms);
        DfArgs a = df_args(m, n, A, lda, dp, ws);
        bto_status e;
        if (df_ready(form, DF_Q, a, st, &e)) {
            if (e != BTO_OK) return e;
            return df_gemv_n(m, n, alpha, A, lda, x, beta, y, z, wsd(ws, L.off[0]), dp, ws, 0, st);
        }
        if (form == BTO_FORM_DF && ws_layout(BTO_OP_DGEMV, BTO_FORM_FUSED, m, n, BTO_F64, d, &L) != BTO_OK)
            return BTO_ERR_CUDA;
    }
    const PanelPlan pl = panel_plan(m, n, d.sms, BTO_OP_DGEMV, BTO_FORM_FUSED);
    PanelArgs a{};
    a.m = m; a.n = n; a.A = A; a.lda = lda; a.p = x;
    a.qpart = wsd(ws, L.off[0]);
    a.ldq = pl.ldq; a.lds = pl.lds; a.NR = pl.NR; a.NC = pl.NC; a.ntiles = pl.ntiles;
    bto_status e = launch_panel(PM_Q, a, pl, st);
    if (e != BTO_OK) return e;
    CombineJob j = {z, m, a.qpart, pl.ldq, pl.NC, alpha, nullptr, 0, 0, 0.0, y, beta};
    return launch_combine(&j, 1, st);
}

static bto_status run_gesummv(int form, int64_t m, int64_t n, double alpha, const double* A,
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
    DeviceInfo d; WsLayout L;
    if (c.ok() && !prepare(BTO_OP_GESUMMV, form, m, n, &d, &L)) return BTO_ERR_CUDA;
    if (c.ok()) c.ws(11, ws, ws_bytes, L);
    if (!c.ok()) return c.finish();

    cudaStream_t st = (cudaStream_t)stream;
    {
        const PanelPlan dp = df_plan(m, n, d.sms);
        DfArgs a = df_args(m, n, A, lda, dp, ws);
        a.B = B; a.ldb = ldb; a.p = x; a.qpart = wsd(ws, L.off[0]); a.qpart2 = wsd(ws, L.off[1]);
        bto_status e;
        if (df_ready(form, DF_Q2, a, st, &e)) {
            if (e != BTO_OK || (e = df_launch(DF_Q2, a, dp, st)) != BTO_OK) return e;
            CombineJob j = {y, m, a.qpart, dp.ldq, dp.NC, alpha, a.qpart2, dp.ldq, dp.NC, beta, nullptr, 0.0};
            return launch_combine(&j, 1, st);
        }
        if (form == BTO_FORM_DF && ws_layout(BTO_OP_GESUMMV, BTO_FORM_FUSED, m, n, BTO_F64, d, &L) != BTO_OK)
            return BTO_ERR_CUDA;
    }
    const PanelPlan pl = panel_plan(m, n, d.sms, BTO_OP_GESUMMV, BTO_FORM_FUSED);
    PanelArgs a{};
    a.m = m; a.n = n; a.A = A; a.lda = lda; a.B = B; a.ldb = ldb; a.p = x;
    a.qpart = wsd(ws, L.off[0]); a.qpart2 = wsd(ws, L.off[1]);
    a.ldq = pl.ldq; a.lds = pl.lds; a.NR = pl.NR; a.NC = pl.NC; a.ntiles = pl.ntiles;
    bto_status e = launch_panel(PM_Q2, a, pl, st);
    if (e != BTO_OK) return e;
    CombineJob j = {y, m, a.qpart, pl.ldq, pl.NC, alpha, a.qpart2, pl.ldq, pl.NC, beta, nullptr, 0.0};
    return launch_combine(&j, 1, st);
}

static bto_status run_dgemvt(int form, int64_t m, int64_t n, double alpha, double beta,
                             const double* A, int64_t lda, const double* y, const double* z,
                             double* x, double* w, void* ws, size_t ws_bytes,
                             bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    c.size(1, m); c.size(2, n);
    if (!c.ok()) return c.finish();
    const size_t Ab = mat_extent_bytes(m, n, lda, 8);
    c.ptr(5, A, m > 0 && n > 0); c.ld(6, lda, m);
    c.ptr(7, y, m > 0); c.ptr(8, z, n > 0); c.ptr(9, x, n > 0); c.ptr(10, w, m > 0);
    c.disjoint(9, x, vbytes(n), A, Ab); c.disjoint(9, x, vbytes(n), y, vbytes(m));
    if (x != z) c.disjoint(9, x, vbytes(n), z, vbytes(n));
    c.disjoint(10, w, vbytes(m), A, Ab); c.disjoint(10, w, vbytes(m), y, vbytes(m));
    c.disjoint(10, w, vbytes(m), z, vbytes(n)); c.disjoint(10, w, vbytes(m), x, vbytes(n));
    DeviceInfo d; WsLayout L;
    if (c.ok() && !prepare(BTO_OP_DGEMVT, form, m, n, &d, &L)) return BTO_ERR_CUDA;
    if (c.ok()) c.ws(11, ws, ws_bytes, L);
    if (!c.ok()) return c.finish();

    cudaStream_t st = (cudaStream_t)stream;
    {
        const PanelPlan dp = df_plan(m, n, d.sms);
        DfArgs a = df_args(m, n, A, lda, dp, ws);
        bto_status e;
        if (df_ready(form, DF_S, a, st, &e)) {
            if (e != BTO_OK) return e;
            // x = beta A^T y + z, then w = alpha A x with panels in reverse (L2 reuse).
            if ((e = df_gemv_t(m, n, beta, A, lda, y, 1.0, z, x, wsd(ws, L.off[1]), dp, ws, 0, st)) != BTO_OK)
                return e;
            return df_gemv_n(m, n, alpha, A, lda, x, 0.0, nullptr, w, wsd(ws, L.off[0]), dp, ws, 1, st);
        }
        if (form == BTO_FORM_DF && ws_layout(BTO_OP_DGEMVT, BTO_FORM_FUSED, m, n, BTO_F64, d, &L) != BTO_OK)
            return BTO_ERR_CUDA;
    }
    const PanelPlan pl = panel_plan(m, n, d.sms, BTO_OP_DGEMVT, BTO_FORM_FUSED);
    PanelArgs a{};
    a.m = m; a.n = n; a.A = A; a.lda = lda; a.r = y;
    a.qpart = wsd(ws, L.off[0]); a.spart = wsd(ws, L.off[1]);
    a.ldq = pl.ldq; a.lds = pl.lds; a.NR = pl.NR; a.NC = pl.NC; a.ntiles = pl.ntiles;
    // Pass 1: x = beta A^T y + z (column sums).  Pass 2 needs the complete x.
    bto_status e = launch_panel(PM_S, a, pl, st);
    if (e != BTO_OK) return e;
    CombineJob jx = {x, n, a.spart, pl.lds, pl.NR, beta, nullptr, 0, 0, 0.0, z, 1.0};
    if ((e = launch_combine(&jx, 1, st)) != BTO_OK) return e;
    // Pass 2: w = alpha A x, panels in reverse so the tail still in L2 is read first.
    a.p = x; a.r = nullptr; a.reverse = 1;
    if ((e = launch_panel(PM_Q, a, pl, st)) != BTO_OK) return e;
    CombineJob jw = {w, m, a.qpart, pl.ldq, pl.NC, alpha, nullptr, 0, 0, 0.0, nullptr, 0.0};
    return launch_combine(&jw, 1, st);
}

static bto_status run_gemver(int form, int64_t m, int64_t n, double alpha, double beta,
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
    const void* ins[7] = {u1, v1, u2, v2, y, z, nullptr};
    const size_t inb[7] = {vbytes(m), vbytes(n), vbytes(m), vbytes(n), vbytes(m), vbytes(n), 0};
    if (!(B == A && ldb == lda)) c.disjoint(13, B, Bb, A, Ab);
    for (int k = 0; k < 6; k++) c.disjoint(13, B, Bb, ins[k], inb[k]);
    c.disjoint(15, x, vbytes(n), A, Ab); c.disjoint(15, x, vbytes(n), B, Bb);
    for (int k = 0; k < 5; k++) c.disjoint(15, x, vbytes(n), ins[k], inb[k]);
    if (x != z) c.disjoint(15, x, vbytes(n), z, vbytes(n));
    c.disjoint(16, w, vbytes(m), A, Ab); c.disjoint(16, w, vbytes(m), B, Bb);
    for (int k = 0; k < 6; k++) c.disjoint(16, w, vbytes(m), ins[k], inb[k]);
    c.disjoint(16, w, vbytes(m), x, vbytes(n));
    DeviceInfo d; WsLayout L;
    if (c.ok() && !prepare(BTO_OP_GEMVER, form, m, n, &d, &L)) return BTO_ERR_CUDA;
    if (c.ok()) c.ws(17, ws, ws_bytes, L);
    if (!c.ok()) return c.finish();

    cudaStream_t st = (cudaStream_t)stream;
    {
        const PanelPlan dp = df_plan(m, n, d.sms);
        DfArgs a = df_args(m, n, A, lda, dp, ws);
        a.Bout = B; a.ldbo = ldb; a.u1 = u1; a.v1 = v1; a.u2 = u2; a.v2 = v2; a.r = y;
        a.spart = wsd(ws, L.off[1]);
        bto_status e;
        if (df_ready(form, DF_G1, a, st, &e)) {
            if (e != BTO_OK || (e = df_launch(DF_G1, a, dp, st)) != BTO_OK) return e;
            CombineJob jx = {x, n, a.spart, dp.lds, dp.NR, beta, nullptr, 0, 0, 0.0, z, 1.0};
            if ((e = launch_combine(&jx, 1, st)) != BTO_OK) return e;
            // w = alpha B x over the new B, last-written panels first (L2 reuse).
            return df_gemv_n(m, n, alpha, B, ldb, x, 0.0, nullptr, w, wsd(ws, L.off[0]), dp, ws, 1, st);
        }
        if (form == BTO_FORM_DF && ws_layout(BTO_OP_GEMVER, BTO_FORM_FUSED, m, n, BTO_F64, d, &L) != BTO_OK)
            return BTO_ERR_CUDA;
    }
    // Matrices whose B stays in L2: both passes in one launch (unless a
    // schedule override asks for the panel engine's tiles).
    if (gemver_small_ok(m, n, d) && !schedule_overridden(BTO_OP_GEMVER, BTO_FORM_FUSED)) {
        const bto_status e = gemver_small(m, n, alpha, beta, A, lda, u1, v1, u2, v2, y, z, B, ldb, x, w, ws, d, -1, 0,
                                          st);
        if (e != BTO_ERR_UNSUPPORTED) return e;
    }
    const PanelPlan pl = panel_plan(m, n, d.sms, BTO_OP_GEMVER, BTO_FORM_FUSED);
    PanelArgs a{};
    a.m = m; a.n = n; a.A = A; a.lda = lda; a.Bout = B; a.ldb = ldb;
    a.u1 = u1; a.v1 = v1; a.u2 = u2; a.v2 = v2; a.r = y;
    a.qpart = wsd(ws, L.off[0]); a.spart = wsd(ws, L.off[1]);
    a.ldq = pl.ldq; a.lds = pl.lds; a.NR = pl.NR; a.NC = pl.NC; a.ntiles = pl.ntiles;
    // Pass 1: B = A + u1 v1^T + u2 v2^T written once, with x = beta B^T y + z
    // fused into the same sweep (column sums of the new B).
    bto_status e = launch_panel(PM_G1, a, pl, st);
    if (e != BTO_OK) return e;
    CombineJob jx = {x, n, a.spart, pl.lds, pl.NR, beta, nullptr, 0, 0, 0.0, z, 1.0};
    if ((e = launch_combine(&jx, 1, st)) != BTO_OK) return e;
    // Pass 2: w = alpha B x over the new B, last-written panels first (L2 reuse).
    PanelArgs b{};
    b.m = m; b.n = n; b.A = B; b.lda = ldb; b.p = x;
    b.qpart = a.qpart; b.ldq = pl.ldq; b.lds = pl.lds; b.NR = pl.NR; b.NC = pl.NC;
    b.ntiles = pl.ntiles; b.reverse = 1;
    if ((e = launch_panel(PM_Q, b, pl, st)) != BTO_OK) return e;
    CombineJob jw = {w, m, b.qpart, pl.ldq, pl.NC, alpha, nullptr, 0, 0, 0.0, nullptr, 0.0};
    return launch_combine(&jw, 1, st);
}

extern "C" bto_status bto_bicgk(int64_t m, int64_t n, const double* A, int64_t lda, const double* p,
                                const double* r, double* q, double* s, void* ws, size_t ws_bytes,
                                bto_stream_t stream) {
    return run_bicgk(BTO_FORM_FUSED, m, n, A, lda, p, r, q, s, ws, ws_bytes, stream);
}
extern "C" bto_status bto_bicgk_df(int64_t m, int64_t n, const double* A, int64_t lda, const double* p,
                                   const double* r, double* q, double* s, void* ws, size_t ws_bytes,
                                   bto_stream_t stream) {
    return run_bicgk(BTO_FORM_DF, m, n, A, lda, p, r, q, s, ws, ws_bytes, stream);
}
// Fault injection for tests (declared in bto.h's testing section): the
// double-float BICGK with block `stall_block`'s producer stopping after one
// ring fill, so its consumers' waits expire after `timeout_ms`.
extern "C" bto_status bto_debug_df_stall(int64_t m, int64_t n, const double* A, int64_t lda, const double* p,
                                         const double* r, double* q, double* s, void* ws, size_t ws_bytes,
                                         int stall_block, int timeout_ms, bto_stream_t stream) {
    clear_invalid_arg();
    if (stall_block < 0) { set_invalid_arg(11); return BTO_ERR_INVALID_VALUE; }
    if (timeout_ms < 1 || timeout_ms > 10000) { set_invalid_arg(12); return BTO_ERR_INVALID_VALUE; }
    return run_bicgk(BTO_FORM_DF, m, n, A, lda, p, r, q, s, ws, ws_bytes, stream, stall_block,
                     (unsigned long long)timeout_ms * 1000000ull);
}
extern "C" bto_status bto_dgemv(int64_t m, int64_t n, double alpha, const double* A, int64_t lda,
                                const double* x, double beta, const double* y, double* z, void* ws,
                                size_t ws_bytes, bto_stream_t stream) {
    return run_dgemv(BTO_FORM_FUSED, m, n, alpha, A, lda, x, beta, y, z, ws, ws_bytes, stream);
}
extern "C" bto_status bto_dgemv_df(int64_t m, int64_t n, double alpha, const double* A, int64_t lda,
                                   const double* x, double beta, const double* y, double* z, void* ws,
                                   size_t ws_bytes, bto_stream_t stream) {
    return run_dgemv(BTO_FORM_DF, m, n, alpha, A, lda, x, beta, y, z, ws, ws_bytes, stream);
}
extern "C" bto_status bto_gesummv(int64_t m, int64_t n, double alpha, const double* A, int64_t lda,
                                  double beta, const double* B, int64_t ldb, const double* x, double* y,
                                  void* ws, size_t ws_bytes, bto_stream_t stream) {
    return run_gesummv(BTO_FORM_FUSED, m, n, alpha, A, lda, beta, B, ldb, x, y, ws, ws_bytes, stream);
}
extern "C" bto_status bto_gesummv_df(int64_t m, int64_t n, double alpha, const double* A, int64_t lda,
                                     double beta, const double* B, int64_t ldb, const double* x, double* y,
                                     void* ws, size_t ws_bytes, bto_stream_t stream) {
    return run_gesummv(BTO_FORM_DF, m, n, alpha, A, lda, beta, B, ldb, x, y, ws, ws_bytes, stream);
}
extern "C" bto_status bto_dgemvt(int64_t m, int64_t n, double alpha, double beta, const double* A,
                                 int64_t lda, const double* y, const double* z, double* x, double* w,
                                 void* ws, size_t ws_bytes, bto_stream_t stream) {
    return run_dgemvt(BTO_FORM_FUSED, m, n, alpha, beta, A, lda, y, z, x, w, ws, ws_bytes, stream);
}
extern "C" bto_status bto_dgemvt_df(int64_t m, int64_t n, double alpha, double beta, const double* A,
                                    int64_t lda, const double* y, const double* z, double* x, double* w,
                                    void* ws, size_t ws_bytes, bto_stream_t stream) {
    return run_dgemvt(BTO_FORM_DF, m, n, alpha, beta, A, lda, y, z, x, w, ws, ws_bytes, stream);
}
extern "C" bto_status bto_gemver(int64_t m, int64_t n, double alpha, double beta, const double* A,
                                 int64_t lda, const double* u1, const double* v1, const double* u2,
                                 const double* v2, const double* y, const double* z, double* B, int64_t ldb,
                                 double* x, double* w, void* ws, size_t ws_bytes, bto_stream_t stream) {
    return run_gemver(BTO_FORM_FUSED, m, n, alpha, beta, A, lda, u1, v1, u2, v2, y, z, B, ldb, x, w, ws,
                      ws_bytes, stream);
}
extern "C" bto_status bto_gemver_df(int64_t m, int64_t n, double alpha, double beta, const double* A,
                                    int64_t lda, const double* u1, const double* v1, const double* u2,
                                    const double* v2, const double* y, const double* z, double* B, int64_t ldb,
                                    double* x, double* w, void* ws, size_t ws_bytes, bto_stream_t stream) {
    return run_gemver(BTO_FORM_DF, m, n, alpha, beta, A, lda, u1, v1, u2, v2, y, z, B, ldb, x, w, ws,
                      ws_bytes, stream);
}

// Fault injection for the bounded grid barrier of the one-launch GEMVER:
// block `stall_block` never arrives, so every block's wait expires after
// `timeout_ms` and the status word reads BTO_ERR_TIMEOUT.
extern "C" bto_status bto_debug_gemver_stall(int64_t m, int64_t n, double alpha, double beta, const double* A,
                                             int64_t lda, const double* u1, const double* v1, const double* u2,
                                             const double* v2, const double* y, const double* z, double* B,
                                             int64_t ldb, double* x, double* w, void* ws, size_t ws_bytes,
                                             int stall_block, int timeout_ms, bto_stream_t stream) {
    clear_invalid_arg();
    Check c;
    c.size(1, m); c.size(2, n);
    c.ptr(5, A, true); c.ld(6, lda, m);
    c.ptr(7, u1, true); c.ptr(8, v1, true); c.ptr(9, u2, true); c.ptr(10, v2, true);
    c.ptr(11, y, true); c.ptr(12, z, true); c.ptr(13, B, true); c.ld(14, ldb, m);
    c.ptr(15, x, true); c.ptr(16, w, true);
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < WS_HEADER) c.fail(17, BTO_ERR_WORKSPACE);
    if (timeout_ms < 1 || timeout_ms > 10000) c.fail(20);
    if (!c.ok()) return c.finish();
    DeviceInfo d;
    if (!device_info(&d)) return BTO_ERR_CUDA;
    if (!gemver_small_ok(m, n, d)) return BTO_ERR_UNSUPPORTED;
    return gemver_small(m, n, alpha, beta, A, lda, u1, v1, u2, v2, y, z, B, ldb, x, w, ws, d, stall_block,
                        (unsigned long long)timeout_ms * 1000000ull, (cudaStream_t)stream);
}
