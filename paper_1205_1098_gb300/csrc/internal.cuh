// Internal declarations shared by the translation units of libbto.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include "bto.h"

namespace bto {

// ------------------------------------------------------------ host helpers
void set_invalid_arg(int pos);
void clear_invalid_arg();
int last_invalid_arg();

// Device facts, cached per device.
struct DeviceInfo {
    int sms = 0;
    int max_smem_optin = 0;
    bool coop = false;
};
bool device_info(DeviceInfo* out);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Byte extent touched by an m x n column-major matrix with leading dimension ld.
inline size_t mat_extent_bytes(int64_t m, int64_t n, int64_t ld, size_t esz) {
    if (m <= 0 || n <= 0) return 0;
    return ((size_t)(n - 1) * (size_t)ld + (size_t)m) * esz;
}
inline bool overlap(const void* a, size_t na, const void* b, size_t nb) {
    if (!na || !nb) return false;
    uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + nb && y < x + na;
}

// Workspace header: the first 256 bytes hold the device status word and,
// for kernels with inter-block waits, nothing else (counters follow in
// their own region).
constexpr size_t WS_HEADER = 256;

// Launch status -> bto_status.
inline bto_status launch_status() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BTO_OK : BTO_ERR_CUDA;
}

// Transposing butterfly over 16 column partials: after four rounds lane l
// holds, for column l mod 16, the sum over the 16 lanes that share bit 4 of
// l; one more exchange with lane l ^ 16 completes the warp sum.  16 adds per
// lane for 16 columns (v is destroyed).
__device__ __forceinline__ double transpose_reduce16(double (&v)[16], int lane) {
#pragma unroll
    for (int half = 8; half >= 1; half >>= 1) {
        const bool upper = (lane & half) != 0;
#pragma unroll
        for (int k = 0; k < half; k++) {
            double send = upper ? v[k] : v[k + half];
            double keep = upper ? v[k + half] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, half);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
}

// ------------------------------------------------------------ panel engine
// The matrix is cut into NR row blocks x NC column panels; tile (rb, cb)
// leaves row-vector partials in qpart[cb][.] and column-vector partials in
// spart[rb][.]; a combine kernel adds them in a fixed order.
// PM_G1 forms B = A + u1 v1^T + u2 v2^T with s = B^T r (GEMVER's first pass
// on column-major storage); PM_G1Q forms the same B with q = B p instead (the
// first pass on row-major storage, where the transposed product of the
// statement becomes the non-transposed product of the stored matrix).
enum PanelMode { PM_QS = 0, PM_Q = 1, PM_S = 2, PM_G1 = 3, PM_Q2 = 4, PM_G1Q = 5 };

struct PanelPlan {
    int NR = 0, NC = 0;
    int64_t TCmax = 0;     // widest column panel
    int64_t ntiles = 0;
    int grid = 0;
    int64_t ldq = 0, lds = 0;  // leading dims of the partial arrays
    int bps = 1;               // blocks per SM the tiles are planned for (reduced-precision sweeps)
};
// op and form select a schedule override (bto_schedule_set); op < 0: none.
PanelPlan panel_plan(int64_t m, int64_t n, int sms, int op = -1, int form = BTO_FORM_FUSED);
size_t panel_smem_bytes(int mode, const PanelPlan& pl);

struct PanelArgs {
    int64_t m, n;
    const double* A; int64_t lda;
    const double* B; int64_t ldb;    // second input matrix (PM_Q2)
    double* Bout;                    // output matrix (PM_G1, PM_G1Q), may equal A
    const double* p;                 // column-indexed vector (PM_QS, PM_Q, PM_Q2, PM_G1Q)
    const double* r;                 // row-indexed vector (PM_QS, PM_S, PM_G1: y)
    // PM_G1, PM_G1Q: u1, u2 row-indexed, v1, v2 column-indexed.
    const double* u1; const double* v1; const double* u2; const double* v2;
    double* qpart; double* qpart2; double* spart;
    int64_t ldq, lds;
    int NR, NC; int64_t ntiles; int reverse;
};
bto_status launch_panel(int mode, const PanelArgs& a, const PanelPlan& pl, cudaStream_t st);

// True when bto_schedule_set has replaced the automatic schedule of (op, form).
bool schedule_overridden(int op, int form);

// GEMVER in one cooperative launch for matrices whose B stays in L2
// (gemver_small.cu).  gemver_small returns BTO_ERR_UNSUPPORTED, having
// launched nothing, when the grid cannot be made co-resident.
bool gemver_small_ok(int64_t m, int64_t n, const DeviceInfo& d);
bto_status gemver_small(int64_t m, int64_t n, double alpha, double beta, const double* A, int64_t lda,
                        const double* u1, const double* v1, const double* u2, const double* v2, const double* y,
                        const double* z, double* B, int64_t ldb, double* x, double* w, void* ws,
                        const DeviceInfo& d, int stall_block, unsigned long long timeout_ns, cudaStream_t st);

// out[i] = a1 * sum_k P1[k*ld1 + i] (+ a2 * sum_k P2[k*ld2 + i]) (+ b * v[i])
struct CombineJob {
    double* out; int64_t len;
    const double* P1; int64_t ld1; int K1; double a1;
    const double* P2; int64_t ld2; int K2; double a2;
    const double* v; double b;
};
bto_status launch_combine(const CombineJob* jobs, int njobs, cudaStream_t st);

// ------------------------------------------------------------ reduced-precision form
// Tiles of the FP32/BF16 storage form: column panels are whole multiples of
// `cu` columns (the TMA box width: 16 for FP32, 32 for BF16) and row blocks
// whole multiples of 256 rows (the box height), so no panel's copies spill
// into a neighbour's columns.
__host__ __device__ inline int64_t lp_col_at(int64_t n, int64_t NC, int64_t cb, int64_t cu) {
    const int64_t units = (n + cu - 1) / cu, c = (units * cb / NC) * cu;
    return c < n ? c : n;
}
__host__ __device__ inline int64_t lp_row_at(int64_t m, int64_t NR, int64_t rb) {
    const int64_t units = (m + 255) / 256, r = (units * rb / NR) * 256;
    return r < m ? r : m;
}
inline int64_t lp_col_unit(int a_type) { return a_type == BTO_BF16 ? 32 : 16; }
// Blocks per SM of an op's reduced-precision sweeps (the plan makes tiles for
// that many blocks): two for BICGK and for BF16 ATAX and GESUMMV, whose sweeps
// fit two blocks' registers; one otherwise (GEMVER's first pass needs more).
inline int lp_blocks_per_sm(int op, int a_type) {
    return ((a_type == BTO_BF16 && (op == BTO_OP_BICGK || op == BTO_OP_ATAX || op == BTO_OP_GESUMMV)) ||
            (a_type == BTO_F32 && op == BTO_OP_BICGK)) ? 2 : 1;
}
// balanced: the split of the TMA-fed sweeps (every sweep of the call can
// take that path, see lp_tma_ok); otherwise the load-instruction kernel's.
PanelPlan lp_plan(int64_t m, int64_t n, int sms, int a_type, int bps = 1, bool balanced = false);
// A matrix the TMA-fed sweep can copy (16-byte base and column stride).
bool lp_tma_ok(int a_type, const void* A, int64_t lda, int64_t m, int64_t n);

// TMA path of the batched form (batched_tma.cu): instances whose matrices
// suit the tensor memory accelerator, as tiles through the reduced-precision
// sweep.  bt_plan_add returns false for an instance the path cannot take.
struct BtPlan;
BtPlan* bt_plan_create();
void bt_plan_destroy(BtPlan* p);
void bt_plan_reset(BtPlan* p, int tile_cols);
bool bt_plan_empty(const BtPlan* p);
bool bt_plan_add(BtPlan* p, const bto_batch_desc& d);
int64_t bt_plan_layout_records(BtPlan* p, int64_t cur, int grid);   // grid: the sweep's blocks (#SMs)
// The assignment the layout uses for a (stage, type) list longer than the
// grid: block[k] for items of the given costs (decreasing), longest
// processing time first, ties to the lower block.
void lpt_blocks(const double* cost, int64_t count, int grid, int32_t* block);
int64_t bt_plan_layout_partials(BtPlan* p, int64_t cur);
void bt_plan_write(const BtPlan* p, char* img, char* ws);
bto_status bt_launch(char* ws, const BtPlan* p, cudaStream_t st);
// The one-launch form (bt_fused): the storage type every TMA item has (0 FP32,
// 1 BF16), or -1 when both occur; and its cooperative launch.
int bt_fused_type(const BtPlan* p);
bto_status bt_launch_fused(char* ws, int type, cudaStream_t st, int stall_block = -1,
                           unsigned long long limit_ns = 2000000000ull);

// Batched form, planned once and submitted (the serving runtime's path).
struct BatchPlan;
BatchPlan* batch_plan_create();
void batch_plan_destroy(BatchPlan* b);
// Validates `count` descriptors and builds their work list; *ws_bytes is the
// workspace the plan needs.  False on an invalid descriptor or tile width.
bool batch_plan_build(BatchPlan* b, int count, const bto_batch_desc* descs, int tile_cols, size_t* ws_bytes);
// Copies the plan (status word and counters zeroed) into ws, through the
// pinned `staging` buffer when it is large enough (the caller keeps it until
// the stream has passed the copy) or a pageable copy that is waited for, and
// launches the kernels of the non-empty queues, each grid at most its items.
// Bytes batch_plan_submit copies (it needs that much staging to avoid a wait).
size_t batch_plan_image_bytes(const BatchPlan* b);
bto_status batch_plan_submit(const BatchPlan* b, void* ws, size_t ws_bytes, void* staging, size_t staging_bytes,
                             cudaStream_t st);

// Sweeps of the reduced-precision form: q = A p and s = A^T r together
// (BICGK), q alone, GEMVER's first pass (B, B^T y), s alone (ATAX's second
// pass).
enum LpMode { LP_QS = 0, LP_Q = 1, LP_G1 = 2, LP_S = 3 };

struct LpArgs {
    int64_t m, n;
    const void* A; int64_t lda;
    void* Bout; int64_t ldb;
    const float* p;            // column-indexed vector (LP_QS, LP_Q)
    const float* r;            // row-indexed vector (LP_QS; LP_G1: y)
    const float* u1; const float* v1; const float* u2; const float* v2;
    double* qpart; double* spart;
    int64_t ldq, lds, tcmax, cu;   // cu: panel column unit
    int NR, NC; int64_t ntiles; int reverse;
    int* status;               // device status word (timeouts of bounded waits)
};
// Launches the TMA-fed sweep; returns false (launching nothing) when the
// layout does not meet the tensor-map rules, so the caller uses the
// load-instruction sweep instead.
bool lp_tma_launch(int a_type, int mode, const LpArgs& a, int grid, int bps, cudaStream_t st, bto_status* out);

// ------------------------------------------------------------ double-float form
// Sweeps of the FP64 matrix sequences with double-float arithmetic on the
// FP32 pipes (df_tma.cu): q = A p and s = A^T r together (BICGK), q alone,
// s alone, GEMVER's first pass (B = A + u1 v1^T + u2 v2^T written in FP64,
// s = B^T r), and q over two matrices (GESUMMV).  Tiles as the reduced-
// precision form: column panels of whole 16-column units, row blocks of
// whole 256-row chunks; partials in FP64 for the panel engine's combine.
enum DfMode { DF_QS = 0, DF_Q = 1, DF_S = 2, DF_G1 = 3, DF_Q2 = 4 };

struct DfArgs {
    int64_t m, n;
    const double* A; int64_t lda;
    const double* B; int64_t ldb;      // second matrix (DF_Q2)
    double* Bout; int64_t ldbo;        // formed matrix (DF_G1), may equal A
    const double* p;                   // column-indexed vector (DF_QS, DF_Q, DF_Q2)
    const double* r;                   // row-indexed vector (DF_QS, DF_S; DF_G1: y)
    const double* u1; const double* v1; const double* u2; const double* v2;
    double* qpart; double* qpart2; double* spart;
    int64_t ldq, lds, tcmax;
    int NR, NC; int64_t ntiles; int reverse;
    int* status;                       // device status word (timeouts of bounded waits)
    unsigned long long wait_ns;        // limit of each ring wait (df_args: 2 s)
    int stall_block;                   // testing: this block's producer stops after one ring fill (-1: none)
};
PanelPlan df_plan(int64_t m, int64_t n, int sms);
// True when the matrices suit the tensor-map copies the sweep is built on
// (16-byte aligned bases, even leading dimensions, sizes below 2^31).
bool df_layout_ok(int mode, const DfArgs& a);
// Launches the sweep (the layout must pass df_layout_ok).
bto_status df_launch(int mode, const DfArgs& a, const PanelPlan& pl, cudaStream_t st);
// Arguments of a sweep over A with the plan's tiles; the status word at ws.
DfArgs df_args(int64_t m, int64_t n, const double* A, int64_t lda, const PanelPlan& pl, void* ws);
// out = alpha A v (+ beta y when y != NULL) and out = alpha A^T v (+ beta y):
// a single-product sweep and its combine (m or n = 0: the combine alone).
bto_status df_gemv_n(int64_t m, int64_t n, double alpha, const double* A, int64_t lda, const double* v,
                     double beta, const double* y, double* out, double* qpart, const PanelPlan& pl, void* ws,
                     int reverse, cudaStream_t st);
bto_status df_gemv_t(int64_t m, int64_t n, double alpha, const double* A, int64_t lda, const double* v,
                     double beta, const double* y, double* out, double* spart, const PanelPlan& pl, void* ws,
                     int reverse, cudaStream_t st);

// ------------------------------------------------------------ ATAX group bands
// A cooperative grid of G blocks is cut into NG groups of S; group g takes
// the bands of TB rows g, g + NG, ...; block r of a group owns a fixed slice
// of about n / S columns.  Each group leaves a partial y over all columns.
struct AtaxPlan {
    int G = 0;          // blocks (one per SM, a multiple of S)
    int S = 0;          // blocks per group
    int NG = 0;         // groups
    int TB = 0;         // band height (rows)
    int D = 0;          // bands of lookahead (2 D partial slots per group)
    int64_t nb = 0;     // number of bands
    int64_t cmax = 0;   // widest column slice
    int64_t ldy = 0;    // leading dimension of the group partials of y
    size_t smem = 0;    // dynamic shared memory per block
    bool fused = false; // false: the slices do not fit; the two-pass form runs
};
AtaxPlan atax_plan(int64_t m, int64_t n, const DeviceInfo& d);

// ------------------------------------------------------------ workspace
struct WsLayout {
    size_t total = 0;
    size_t off[6] = {0, 0, 0, 0, 0, 0};
};
bto_status ws_layout(int op, int form, int64_t m, int64_t n, int a_type,
                     const DeviceInfo& d, WsLayout* out);
// Workspace of the double-float forms (form BTO_FORM_DF or BTO_FORM_DF_UNFUSED):
// room for the double-float sweeps' partials and for the FP64 form the call
// runs instead when the layout does not suit the tensor-map copies.
bto_status df_ws_layout(int op, int form, int64_t m, int64_t n, const DeviceInfo& d, WsLayout* out);
// Validates ws against the layout; sets the invalid-arg position on failure.
bto_status check_ws(const void* ws, size_t ws_bytes, const WsLayout& L, int pos_ws);

// ------------------------------------------------------------ BLAS-1/2 building blocks
// Kernels of the unfused forms (unfused_f64.cu), one per BLAS call.
bto_status dcopy(int64_t n, const double* x, double* y, int sms, cudaStream_t st);
bto_status dcopy_mat(int64_t m, int64_t n, const double* A, int64_t lda, double* B, int64_t ldb,
                     int sms, cudaStream_t st);
bto_status dger(int64_t m, int64_t n, const double* x, const double* y, double* A, int64_t lda,
                int sms, cudaStream_t st);

// ------------------------------------------------------------ vector helpers
int vector_grid(int sms);                     // blocks of the reduction kernels
bto_status launch_dot_partials(int64_t n, double alpha, const double* w, const double* v,
                               const double* u, double* z, double* partials, int grid,
                               int mode, cudaStream_t st);   // mode 0: axpydot, 1: plain dot of w,u
bto_status launch_dot_final(const double* partials, int grid, double* r, cudaStream_t st);
bto_status launch_waxpby(int64_t n, double alpha, const double* x, double beta, const double* y,
                         double* w, int sms, cudaStream_t st);
bto_status launch_vadd(int64_t n, const double* w, const double* y, const double* z, double* x,
                       int sms, cudaStream_t st);

}  // namespace bto
