// Pass programs: the runtime that executes what the sequence generator
// plans.  A program is a list of engine passes (each reads one matrix once
// and forms up to two of its products as per-tile partial sums in numbered
// slots), fixed-order combines of those slots, and WAXPBY steps.  The check
// is structural and runs before any device call; the workspace holds one
// region per slot, sized by the pass's tile plan on the current device.
#include "check.cuh"
#include <vector>

namespace bto {
namespace {

struct Slot {
    int64_t len = -1;      // vector length of the slot's sums (-1: not written yet)
    bool q = false;        // row accumulators (q partials) or column sums (s partials)
    int pass = -1;         // instruction that writes it
};

bool mode_ok(int m) { return m >= BTO_PASS_QS && m <= BTO_PASS_G1Q; }
bool has_q(int m) { return m == BTO_PASS_QS || m == BTO_PASS_Q || m == BTO_PASS_Q2 || m == BTO_PASS_G1Q; }
bool has_s(int m) { return m == BTO_PASS_QS || m == BTO_PASS_S || m == BTO_PASS_G1; }
bool slot_ok(int s) { return s >= 0 && s < BTO_PROGRAM_MAX_SLOTS; }
bool aligned8(const void* x) { return (reinterpret_cast<uintptr_t>(x) & 7) == 0; }

// Structural check; fills slots[] as the program writes them.
int check_program(const bto_instr* prog, int count, Slot* slots) {
    for (int i = 0; i < count; i++) {
        const bto_instr& I = prog[i];
        const void* ptrs[12] = {I.A, I.B, I.Bout, I.p, I.r, I.u1, I.v1, I.u2, I.v2, I.out, I.x, I.y};
        for (const void* x : ptrs)
            if (!aligned8(x)) return i;
        if (I.op == BTO_INSTR_PASS) {
            const int64_t m = I.m, n = I.n;
            if (!mode_ok(I.mode) || m < 0 || n < 0) return i;
            const bool work = m > 0 && n > 0;
            if (work && (!I.A || I.lda < std::max<int64_t>(1, m))) return i;
            const bool gen = I.mode == BTO_PASS_G1 || I.mode == BTO_PASS_G1Q;
            if (work && has_q(I.mode) && !I.p) return i;
            if (work && has_s(I.mode) && !I.r) return i;
            if (work && gen && (!I.Bout || I.ldbo < std::max<int64_t>(1, m) || !I.u1 || !I.v1 || !I.u2 || !I.v2))
                return i;
            if (gen && I.Bout && I.Bout != I.A &&
                overlap(I.Bout, mat_extent_bytes(m, n, I.ldbo, 8), I.A, mat_extent_bytes(m, n, I.lda, 8)))
                return i;
            if (gen && I.Bout == I.A && I.ldbo != I.lda && work) return i;
            if (I.mode == BTO_PASS_Q2 && work && (!I.B || I.ldb < std::max<int64_t>(1, m))) return i;
            // Written vectors never alias the formed matrix.
            if (gen && work) {
                const size_t Bb = mat_extent_bytes(m, n, I.ldbo, 8);
                const void* vs[6] = {I.p, I.r, I.u1, I.v1, I.u2, I.v2};
                const size_t nb[6] = {vbytes(n), vbytes(m), vbytes(m), vbytes(n), vbytes(m), vbytes(n)};
                for (int k = 0; k < 6; k++)
                    if (vs[k] && overlap(I.Bout, Bb, vs[k], nb[k])) return i;
            }
            // Slots: exactly those of the mode, each written once.
            const int want_q = has_q(I.mode), want_q2 = I.mode == BTO_PASS_Q2, want_s = has_s(I.mode);
            if (want_q != (I.slot_q >= 0) || want_q2 != (I.slot_q2 >= 0) || want_s != (I.slot_s >= 0)) return i;
            const int ss[3] = {I.slot_q, I.slot_q2, I.slot_s};
            const bool isq[3] = {true, true, false};
            for (int k = 0; k < 3; k++) {
                if (ss[k] < 0) continue;
                if (!slot_ok(ss[k]) || slots[ss[k]].len >= 0) return i;
                for (int k2 = 0; k2 < k; k2++)
                    if (ss[k2] == ss[k]) return i;
                slots[ss[k]].len = isq[k] ? m : n;
                slots[ss[k]].q = isq[k];
                slots[ss[k]].pass = i;
            }
        } else if (I.op == BTO_INSTR_COMBINE) {
            if (I.n < 0 || (I.n > 0 && !I.out)) return i;
            const int src[2] = {I.src1, I.src2};
            for (int k = 0; k < 2; k++) {
                if (src[k] < 0) continue;
                if (!slot_ok(src[k]) || slots[src[k]].len != I.n) return i;
            }
            if (I.src2 >= 0 && I.src1 < 0) return i;
        } else if (I.op == BTO_INSTR_WAXPBY) {
            if (I.n < 0) return i;
            if (I.n > 0 && (!I.out || !I.x || !I.y)) return i;
            if (overlap(I.out, vbytes(I.n), I.x, vbytes(I.n)) || overlap(I.out, vbytes(I.n), I.y, vbytes(I.n)))
                return i;
        } else {
            return i;
        }
    }
    return -1;
}

struct SlotRegion {
    size_t off = 0;
    int64_t ld = 0;
    int K = 0;
};

// Workspace layout: one region per written slot, after the header.
size_t layout_slots(const bto_instr* prog, int count, const Slot* slots, int sms, SlotRegion* reg,
                    std::vector<PanelPlan>* plans) {
    size_t cur = WS_HEADER;
    if (plans) plans->assign(count, PanelPlan{});
    for (int i = 0; i < count; i++) {
        const bto_instr& I = prog[i];
        if (I.op != BTO_INSTR_PASS) continue;
        // A pass that forms a matrix takes GEMVER's measured plan (row blocks
        // of one chunk); the others the engine's default.
        const bool gen = I.mode == BTO_PASS_G1 || I.mode == BTO_PASS_G1Q;
        const PanelPlan pl = panel_plan(I.m, I.n, sms, gen ? BTO_OP_GEMVER : -1, BTO_FORM_FUSED);
        if (plans) (*plans)[i] = pl;
        const int ss[3] = {I.slot_q, I.slot_q2, I.slot_s};
        for (int k = 0; k < 3; k++) {
            if (ss[k] < 0) continue;
            SlotRegion& R = reg[ss[k]];
            const bool q = slots[ss[k]].q;
            R.ld = q ? pl.ldq : pl.lds;
            R.K = q ? pl.NC : pl.NR;
            R.off = cur;
            cur += round_up((int64_t)((size_t)R.K * R.ld * sizeof(double)), 256);
        }
    }
    return cur;
}

}  // namespace
}  // namespace bto

using namespace bto;

extern "C" bto_status bto_program_check(const bto_instr* prog, int count, int* bad_index) {
    clear_invalid_arg();
    if (!bad_index) { set_invalid_arg(3); return BTO_ERR_INVALID_VALUE; }
    *bad_index = -1;
    if (count < 0 || count > BTO_PROGRAM_MAX_INSTRS) { set_invalid_arg(2); return BTO_ERR_INVALID_VALUE; }
    if (count > 0 && !prog) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    Slot slots[BTO_PROGRAM_MAX_SLOTS];
    const int bad = check_program(prog, count, slots);
    if (bad >= 0) {
        *bad_index = bad;
        set_invalid_arg(1);
        return BTO_ERR_INVALID_VALUE;
    }
    return BTO_OK;
}

extern "C" bto_status bto_program_workspace_bytes(const bto_instr* prog, int count, size_t* bytes) {
    clear_invalid_arg();
    if (count < 0 || count > BTO_PROGRAM_MAX_INSTRS) { set_invalid_arg(2); return BTO_ERR_INVALID_VALUE; }
    if (count > 0 && !prog) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    if (!bytes) { set_invalid_arg(3); return BTO_ERR_INVALID_VALUE; }
    Slot slots[BTO_PROGRAM_MAX_SLOTS];
    if (check_program(prog, count, slots) >= 0) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    DeviceInfo d;
    if (!device_info(&d)) return BTO_ERR_CUDA;
    SlotRegion reg[BTO_PROGRAM_MAX_SLOTS];
    *bytes = layout_slots(prog, count, slots, d.sms, reg, nullptr);
    return BTO_OK;
}

extern "C" bto_status bto_program_run(const bto_instr* prog, int count, void* ws, size_t ws_bytes,
                                      bto_stream_t stream) {
    clear_invalid_arg();
    if (count < 0 || count > BTO_PROGRAM_MAX_INSTRS) { set_invalid_arg(2); return BTO_ERR_INVALID_VALUE; }
    if (count > 0 && !prog) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    Slot slots[BTO_PROGRAM_MAX_SLOTS];
    if (check_program(prog, count, slots) >= 0) { set_invalid_arg(1); return BTO_ERR_INVALID_VALUE; }
    DeviceInfo d;
    if (!device_info(&d)) return BTO_ERR_CUDA;
    SlotRegion reg[BTO_PROGRAM_MAX_SLOTS];
    std::vector<PanelPlan> plans;
    const size_t need = layout_slots(prog, count, slots, d.sms, reg, &plans);
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < need) {
        set_invalid_arg(3);
        return BTO_ERR_WORKSPACE;
    }
    char* base = static_cast<char*>(ws);
    auto slot_ptr = [&](int s) { return reinterpret_cast<double*>(base + reg[s].off); };
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < count; i++) {
        const bto_instr& I = prog[i];
        bto_status e = BTO_OK;
        if (I.op == BTO_INSTR_PASS) {
            const PanelPlan& pl = plans[i];
            PanelArgs a{};
            a.m = I.m; a.n = I.n; a.A = I.A; a.lda = I.lda;
            a.p = I.p; a.r = I.r; a.u1 = I.u1; a.v1 = I.v1; a.u2 = I.u2; a.v2 = I.v2;
            if (I.mode == BTO_PASS_Q2) { a.B = I.B; a.ldb = I.ldb; }
            if (I.mode == BTO_PASS_G1 || I.mode == BTO_PASS_G1Q) { a.Bout = I.Bout; a.ldb = I.ldbo; }
            a.qpart = I.slot_q >= 0 ? slot_ptr(I.slot_q) : nullptr;
            a.qpart2 = I.slot_q2 >= 0 ? slot_ptr(I.slot_q2) : nullptr;
            a.spart = I.slot_s >= 0 ? slot_ptr(I.slot_s) : nullptr;
            a.ldq = pl.ldq; a.lds = pl.lds; a.NR = pl.NR; a.NC = pl.NC; a.ntiles = pl.ntiles;
            a.reverse = I.reverse ? 1 : 0;
            // The engine's modes carry the same numbers as BTO_PASS_*.
            e = launch_panel(I.mode, a, pl, st);
        } else if (I.op == BTO_INSTR_COMBINE) {
            CombineJob j{};
            j.out = I.out; j.len = I.n;
            if (I.src1 >= 0) { j.P1 = slot_ptr(I.src1); j.ld1 = reg[I.src1].ld; j.K1 = reg[I.src1].K; }
            j.a1 = I.a1;
            if (I.src2 >= 0) { j.P2 = slot_ptr(I.src2); j.ld2 = reg[I.src2].ld; j.K2 = reg[I.src2].K; }
            j.a2 = I.a2;
            j.v = I.x; j.b = I.b;
            e = launch_combine(&j, 1, st);
        } else {
            e = launch_waxpby(I.n, I.a1, I.x, I.b, I.y, I.out, d.sms, st);
        }
        if (e != BTO_OK) return e;
    }
    return BTO_OK;
}

static_assert(BTO_PASS_QS == PM_QS && BTO_PASS_Q == PM_Q && BTO_PASS_S == PM_S && BTO_PASS_G1 == PM_G1 &&
                  BTO_PASS_Q2 == PM_Q2 && BTO_PASS_G1Q == PM_G1Q,
              "pass modes and engine modes share their numbers");
