/*
 * bto.h -- C ABI of the fused BLAS-1/2 sequence library for GB300 (sm_103a).
 *
 * The operations are the kernels of Table I (Section V-A, "Test Environment
 * and Kernels") of "Reliable Generation of High-Performance Matrix Algebra"
 * (Belter, Jessup, Nelson, Norris, Siek; the Build to Order BLAS).  Each
 * sequence runs with loop fusion and array contraction (Sections I and III):
 * a matrix is streamed from device memory the fewest times the data
 * dependences allow, and temporary vectors stay on chip.
 *
 * Conventions shared by every entry point:
 *  - Pointers are DEVICE pointers unless a comment says otherwise.  The
 *    caller owns all memory; the library never allocates, frees or
 *    synchronizes (bto_device_status is the one call that waits, on request).
 *  - Matrices are column-major: element (i, j) of A is A[i + j*lda], with
 *    lda >= max(1, m).  Rows m..lda-1 are never read or written.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL is the legacy default
 *    stream) and returns before it finishes.  The returned status covers
 *    argument validation and launch errors; faults inside a kernel surface at
 *    the caller's next synchronization, as for any CUDA launch.
 *  - m = 0 or n = 0 is valid; an empty sum is 0 (so GEMVER with m = 0 gives
 *    x = beta*0 + z).
 *  - Arithmetic is IEEE with no BLAS-style shortcut for zero scalars: alpha*s
 *    is always evaluated, so a NaN or Inf in an operand propagates even when
 *    its scalar is 0.  Kernels may contract a*b + c into one fused
 *    multiply-add and sum in any fixed order; the order depends only on the
 *    sizes and the device's SM count, so repeated calls are bitwise equal.
 *  - Outputs may not overlap inputs, except where an entry point documents an
 *    in-place form.  Violations are rejected with BTO_ERR_INVALID_VALUE.
 *  - Workspace `ws` (device memory, at least bto_workspace_bytes() bytes,
 *    256-byte aligned) holds split partial sums; its contents on entry are
 *    ignored and on exit unspecified.  Calls that share a workspace must be
 *    ordered (same stream or events).
 *  - On an invalid argument nothing is launched, the call returns
 *    BTO_ERR_INVALID_VALUE (or BTO_ERR_WORKSPACE for a short workspace) and
 *    bto_last_invalid_arg() gives the 1-based position of the argument.
 */
#ifndef BTO_H
#define BTO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t (struct CUstream_st *); no CUDA header needed. */
typedef struct CUstream_st *bto_stream_t;

typedef enum {
    BTO_OK = 0,
    BTO_ERR_INVALID_VALUE = 1, /* bad size, pointer, alignment or aliasing      */
    BTO_ERR_UNSUPPORTED = 2,   /* valid request this library does not implement */
    BTO_ERR_WORKSPACE = 3,     /* ws NULL or smaller than bto_workspace_bytes() */
    BTO_ERR_CUDA = 4,          /* a CUDA runtime call or launch failed          */
    BTO_ERR_TIMEOUT = 5,       /* a bounded device-side wait expired            */
    BTO_ERR_BUDGET = 6         /* a request exceeds a configured memory budget  */
} bto_status;

typedef enum { BTO_F64 = 0, BTO_F32 = 1, BTO_BF16 = 2 } bto_dtype;

typedef enum {
    BTO_OP_BICGK = 0,
    BTO_OP_ATAX = 1,
    BTO_OP_GEMVER = 2,
    BTO_OP_GESUMMV = 3,
    BTO_OP_DGEMV = 4,
    BTO_OP_DGEMVT = 5,
    BTO_OP_AXPYDOT = 6,
    BTO_OP_WAXPBY = 7,
    BTO_OP_VADD = 8
} bto_op;

/* Form selector for bto_workspace_bytes: the fused kernels or the unfused
 * one-kernel-per-BLAS-call sequences (bto_unfused_*). */
#define BTO_FORM_FUSED 0
#define BTO_FORM_UNFUSED 1
/* The double-float forms of the FP64 matrix sequences (bto_*_df and
 * bto_unfused_*_df, below): matrix ops BICGK .. DGEMVT, a_type BTO_F64. */
#define BTO_FORM_DF 2
#define BTO_FORM_DF_UNFUSED 3

/* ---------------------------------------------------------------- utilities */

/* Library version, major*10000 + minor*100 + patch. */
int bto_version(void);

/* Static, NUL-terminated description of a status code (never NULL). */
const char *bto_status_string(int status);

/* 1-based position of the argument rejected by the calling thread's most
 * recent failing call (0 if none). Thread-local. */
int bto_last_invalid_arg(void);

/* Bytes of workspace that `op` in `form` needs for an m x n problem (vector
 * kernels: n elements, m ignored) with matrix storage type `a_type`, on the
 * CURRENT device (the split of the matrix follows its SM count).  Writes the
 * size to *bytes.  Returns BTO_ERR_INVALID_VALUE for a negative size or an
 * unknown op/form/type, BTO_ERR_CUDA if the device cannot be queried. */
bto_status bto_workspace_bytes(int op, int form, int64_t m, int64_t n, int a_type,
                               size_t *bytes);

/* Waits for `stream`, then reads the device status word that the kernels
 * with bounded inter-block waits (bto_atax) leave at the start of `ws`:
 * BTO_OK, or BTO_ERR_TIMEOUT if a wait expired (the outputs are then
 * unspecified).  *status receives the value. */
bto_status bto_device_status(const void *ws, bto_stream_t stream, int *status);

/* --------------------------------------------------- fused FP64 sequences */

/* BICGK (Table I): q <- A p ; s <- A^T r.
 * A: m x n (lda); p: n; r: m; q: m (output); s: n (output).
 * One pass over A produces both products (the two dgemv calls of the BICGK
 * BLAS listing in Section V-A, fused). */
bto_status bto_bicgk(int64_t m, int64_t n, const double *A, int64_t lda,
                     const double *p, const double *r, double *q, double *s,
                     void *ws, size_t ws_bytes, bto_stream_t stream);

/* ATAX (Table I, y <- A^T A x) generalised to BATAX (Section II, Fig. 1:
 * y <- beta A^T (A x)); beta = 1 is ATAX.  A: m x n (lda); x: n; y: n (output).
 * The temporary t = A x (length m) is contracted: it never reaches device
 * memory as a vector; A is read from device memory once.  Uses bounded waits
 * between blocks; a timeout is reported through bto_device_status. */
bto_status bto_atax(int64_t m, int64_t n, double beta, const double *A, int64_t lda,
                    const double *x, double *y, void *ws, size_t ws_bytes,
                    bto_stream_t stream);

/* GEMVER (Table I): B <- A + u1 v1^T + u2 v2^T ; x <- beta B^T y + z ;
 * w <- alpha B x  (x uses the new B, w the new x).
 * A: m x n (lda); u1, u2, y: m; v1, v2, z: n; B: m x n (ldb, output);
 * x: n (output); w: m (output).  In place: B == A with ldb == lda, and
 * x == z, are allowed.  B is written once and read back once (w needs the
 * complete x, so a second pass over B is unavoidable). */
bto_status bto_gemver(int64_t m, int64_t n, double alpha, double beta,
                      const double *A, int64_t lda, const double *u1, const double *v1,
                      const double *u2, const double *v2, const double *y, const double *z,
                      double *B, int64_t ldb, double *x, double *w,
                      void *ws, size_t ws_bytes, bto_stream_t stream);

/* GESUMMV (Table I): y <- alpha A x + beta B x.
 * A: m x n (lda); B: m x n (ldb); x: n; y: m (output). */
bto_status bto_gesummv(int64_t m, int64_t n, double alpha, const double *A, int64_t lda,
                       double beta, const double *B, int64_t ldb, const double *x,
                       double *y, void *ws, size_t ws_bytes, bto_stream_t stream);

/* DGEMV (Table I): z <- alpha A x + beta y.
 * A: m x n (lda); x: n; y: m; z: m (output; z == y allowed). */
bto_status bto_dgemv(int64_t m, int64_t n, double alpha, const double *A, int64_t lda,
                     const double *x, double beta, const double *y, double *z,
                     void *ws, size_t ws_bytes, bto_stream_t stream);

/* DGEMVT (Table I): x <- beta A^T y + z ; w <- alpha A x (with the new x).
 * A: m x n (lda); y: m; z: n; x: n (output; x == z allowed); w: m (output). */
bto_status bto_dgemvt(int64_t m, int64_t n, double alpha, double beta,
                      const double *A, int64_t lda, const double *y, const double *z,
                      double *x, double *w, void *ws, size_t ws_bytes, bto_stream_t stream);

/* AXPYDOT (Table I): z <- w - alpha v ; r <- z^T u.  (Table I names the
 * output scalar beta.)  w, v, u: n; z: n (output; z == w allowed);
 * r: one double in device memory (output). */
bto_status bto_axpydot(int64_t n, double alpha, const double *w, const double *v,
                       const double *u, double *z, double *r,
                       void *ws, size_t ws_bytes, bto_stream_t stream);

/* WAXPBY (Table I): w <- alpha x + beta y.  x, y: n; w: n (output). */
bto_status bto_waxpby(int64_t n, double alpha, const double *x, double beta,
                      const double *y, double *w, bto_stream_t stream);

/* VADD (Table I): x <- w + y + z, evaluated as (w + y) + z.
 * w, y, z: n; x: n (output). */
bto_status bto_vadd(int64_t n, const double *w, const double *y, const double *z,
                    double *x, bto_stream_t stream);

/* ------------------------------------------ storage order and transposition
 * The FP64 matrix sequences on row-major as well as column-major storage, and
 * DGEMV with a BLAS-style transposition flag.  The paper's type system treats
 * a matrix as a container of row or column containers and generates code for
 * either order (Section II; BATAX's A in Fig. 1 is declared row-major).
 * layout: BTO_COL_MAJOR (element (i, j) at A[i + j*lda], lda >= max(1, m)) or
 * BTO_ROW_MAJOR (element (i, j) at A[i*lda + j], lda >= max(1, n)); B (GEMVER,
 * GESUMMV) has the same layout with its own ldb.  The statements, vector
 * lengths, aliasing rules and errors are those of the column-major entry point
 * of the same name; argument positions (bto_last_invalid_arg) count the
 * leading layout (and trans) arguments.  A column-major call is the ordinary
 * entry point.  On row-major storage the stored matrix is A^T in column-major
 * order, so the two products of each statement exchange roles in the same
 * fused passes (BICGK: one pass; GEMVER: two, B written once and read back
 * once; DGEMVT: two; DGEMV: one).  GESUMMV on row-major storage runs one pass
 * per matrix (each read once) and BATAX two passes (A read twice: t = A x is
 * formed in the workspace, then y = beta A^T t).
 * The workspace is bto_layout_workspace_bytes(op, layout, trans, m, n); it is
 * the same as bto_workspace_bytes(op, BTO_FORM_FUSED, m, n, BTO_F64) for
 * column-major calls without transposition.  trans must be BTO_NO_TRANS except
 * for op = BTO_OP_DGEMV. */
#define BTO_COL_MAJOR 0
#define BTO_ROW_MAJOR 1
#define BTO_NO_TRANS 0
#define BTO_TRANS 1

bto_status bto_layout_workspace_bytes(int op, int layout, int trans, int64_t m, int64_t n,
                                      size_t *bytes);

/* BICGK: q <- A p ; s <- A^T r (A m x n in `layout`). */
bto_status bto_bicgk_layout(int layout, int64_t m, int64_t n, const double *A, int64_t lda,
                            const double *p, const double *r, double *q, double *s,
                            void *ws, size_t ws_bytes, bto_stream_t stream);

/* BATAX: y <- beta A^T (A x) (A m x n in `layout`; x, y: n). */
bto_status bto_atax_layout(int layout, int64_t m, int64_t n, double beta, const double *A,
                           int64_t lda, const double *x, double *y, void *ws, size_t ws_bytes,
                           bto_stream_t stream);

/* GEMVER: B <- A + u1 v1^T + u2 v2^T ; x <- beta B^T y + z ; w <- alpha B x
 * (A and B m x n in `layout`; B == A with ldb == lda and x == z allowed). */
bto_status bto_gemver_layout(int layout, int64_t m, int64_t n, double alpha, double beta,
                             const double *A, int64_t lda, const double *u1, const double *v1,
                             const double *u2, const double *v2, const double *y, const double *z,
                             double *B, int64_t ldb, double *x, double *w,
                             void *ws, size_t ws_bytes, bto_stream_t stream);

/* GESUMMV: y <- alpha A x + beta B x (A, B m x n in `layout`). */
bto_status bto_gesummv_layout(int layout, int64_t m, int64_t n, double alpha, const double *A,
                              int64_t lda, double beta, const double *B, int64_t ldb,
                              const double *x, double *y, void *ws, size_t ws_bytes,
                              bto_stream_t stream);

/* DGEMV with transposition: z <- alpha op(A) x + beta y, A m x n in `layout`,
 * op(A) = A (trans = BTO_NO_TRANS; x: n, y and z: m) or A^T (BTO_TRANS; x: m,
 * y and z: n).  z == y allowed.  An empty product gives z = beta y. */
bto_status bto_dgemv_layout(int layout, int trans, int64_t m, int64_t n, double alpha,
                            const double *A, int64_t lda, const double *x, double beta,
                            const double *y, double *z, void *ws, size_t ws_bytes,
                            bto_stream_t stream);

/* DGEMVT: x <- beta A^T y + z ; w <- alpha A x (A m x n in `layout`). */
bto_status bto_dgemvt_layout(int layout, int64_t m, int64_t n, double alpha, double beta,
                             const double *A, int64_t lda, const double *y, const double *z,
                             double *x, double *w, void *ws, size_t ws_bytes,
                             bto_stream_t stream);

/* ------------------------------------------------------------ pass programs
 * A program is a list of instructions over the FP64 panel engine, which a
 * generator (paper_1205_1098_gb300.generator) produces from a short
 * description of a BLAS-1/2 sequence, the way the paper's compiler turns its
 * input (Section II, Fig. 1) into fused loop nests: each PASS instruction
 * reads one column-major matrix (two for BTO_PASS_Q2) once and forms up to
 * two products of it, leaving per-tile partial sums in numbered slots; each
 * COMBINE adds the partial sums of one or two slots in a fixed order and
 * scales them (plus a scaled vector); WAXPBY forms a x + b y.
 *
 * PASS over the stored m x n matrix A (lda >= max(1, m)), tiles in reverse
 * order if `reverse`:
 *   BTO_PASS_QS   slot_q <- A p (length m), slot_s <- A^T r (length n)
 *   BTO_PASS_Q    slot_q <- A p
 *   BTO_PASS_S    slot_s <- A^T r
 *   BTO_PASS_G1   Bout <- A + u1 v1^T + u2 v2^T (u length m, v length n;
 *                 ldbo; Bout == A with ldbo == lda allowed),
 *                 slot_s <- Bout^T r
 *   BTO_PASS_Q2   slot_q <- A p, slot_q2 <- B p (B m x n, ldb)
 *   BTO_PASS_G1Q  Bout as for G1, slot_q <- Bout p
 * COMBINE: out[0..n) <- a1 * (sum of slot src1) + a2 * (sum of slot src2)
 *   + b * x, where src2 = -1 and x = NULL drop their terms, src1 = -1 gives
 *   0 for its term; a slot's length must equal n; x may equal out.
 * WAXPBY: out[0..n) <- a1 * x + b * y; out must not overlap x or y.
 * Slots are numbered 0..BTO_PROGRAM_MAX_SLOTS-1; each is written by one PASS
 * and read only by later COMBINEs.  Vectors must not overlap the matrix a
 * PASS writes.  Sums run in a fixed order, so a program gives the same bits
 * on every run. */
#define BTO_INSTR_PASS 0
#define BTO_INSTR_COMBINE 1
#define BTO_INSTR_WAXPBY 2
#define BTO_PASS_QS 0
#define BTO_PASS_Q 1
#define BTO_PASS_S 2
#define BTO_PASS_G1 3
#define BTO_PASS_Q2 4
#define BTO_PASS_G1Q 5
#define BTO_PROGRAM_MAX_SLOTS 64
#define BTO_PROGRAM_MAX_INSTRS 4096

typedef struct bto_instr {
    int32_t op;            /* BTO_INSTR_*                                        */
    int32_t mode;          /* PASS: BTO_PASS_*                                   */
    int32_t reverse;       /* PASS: nonzero = tiles in reverse order             */
    int32_t slot_q;        /* PASS: slot of A p (or Bout p), -1 if none          */
    int32_t slot_q2;       /* PASS: slot of B p (BTO_PASS_Q2), -1 if none        */
    int32_t slot_s;        /* PASS: slot of A^T r (or Bout^T r), -1 if none      */
    int32_t src1, src2;    /* COMBINE: slots read, -1 if none                    */
    int64_t m, n;          /* PASS: matrix rows, columns; COMBINE/WAXPBY: n = length */
    const double *A; int64_t lda;
    const double *B; int64_t ldb;
    double *Bout; int64_t ldbo;
    const double *p, *r;   /* PASS: length n (column-indexed), length m (row-indexed) */
    const double *u1, *v1, *u2, *v2;
    double *out;           /* COMBINE, WAXPBY                                    */
    const double *x, *y;   /* COMBINE: x; WAXPBY: x and y                        */
    double a1, a2, b;
} bto_instr;

/* Structural check of a program (no device access): on an invalid
 * instruction returns BTO_ERR_INVALID_VALUE and writes its index to
 * *bad_index (-1 when the count itself is invalid). */
bto_status bto_program_check(const bto_instr *prog, int count, int *bad_index);

/* Workspace bytes for the slots of a program on the current device. */
bto_status bto_program_workspace_bytes(const bto_instr *prog, int count, size_t *bytes);

/* Checks the program, then enqueues its kernels on `stream` in order (no
 * host synchronisation; a program may be recorded into a CUDA graph). */
bto_status bto_program_run(const bto_instr *prog, int count, void *ws, size_t ws_bytes,
                           bto_stream_t stream);

/* ------------------------------------------------------------ sparse (CSR)
 * BICGK and BATAX on a sparse matrix in compressed sparse row form, one of
 * the matrix formats the paper plans as future work (Section VII).  A is
 * m x n with nnz stored entries: row_ptr has m + 1 int64 entries
 * (nondecreasing, row_ptr[0] = 0, row_ptr[m] = nnz), col and val nnz entries
 * (int32 column indices in [0, n), FP64 values; duplicates are summed, order
 * within a row is free).  The stored entries are divided evenly among the
 * lanes (8 consecutive entries each), whatever the row lengths.  Each row's
 * products are summed in a fixed order (bitwise reproducible); the
 * transposed product is scattered with FP64 atomic adds (reproducible to
 * rounding only).  BATAX forms t = A x in the workspace, then scatters
 * beta t_i A(i, j): the stored entries are read twice.  n <= 2^31 - 1.
 * ws: bto_csr_workspace_bytes bytes (about 24 bytes per 256 stored entries,
 * plus 8 m for BATAX), 256-byte aligned; its first word is the device status
 * (bto_device_status): BTO_ERR_INVALID_VALUE if a row pointer lay outside
 * [0, nnz] or decreased (the call then sums every row with clamped bounds),
 * or a column index outside [0, n) (that entry is skipped, never
 * dereferenced). */

/* Workspace bytes of a CSR call; op is BTO_OP_BICGK or BTO_OP_ATAX. */
bto_status bto_csr_workspace_bytes(int op, int64_t m, int64_t n, int64_t nnz, size_t *bytes);

/* q <- A p (q: m) ; s <- A^T r (s: n); p: n, r: m. */
bto_status bto_csr_bicgk(int64_t m, int64_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col,
                         const double *val, const double *p, const double *r, double *q, double *s,
                         void *ws, size_t ws_bytes, bto_stream_t stream);

/* y <- beta A^T (A x); x: n, y: n. */
bto_status bto_csr_atax(int64_t m, int64_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col,
                        const double *val, double beta, const double *x, double *y, void *ws,
                        size_t ws_bytes, bto_stream_t stream);

/* ------------------------------------------------- banded and triangular
 * BICGK and BATAX on banded and triangular matrices, the other structured
 * formats the paper plans beside sparse ones (Section VII).  A is m x n with
 * A(i, j) = 0 outside j - ku <= i <= j + kl (kl sub-diagonals, ku
 * super-diagonals, both >= 0 and <= 2^40; they may exceed the matrix).  Only
 * entries inside the band are read and only they enter the sums, whatever
 * the storage holds elsewhere: a NaN or Inf in p, r or x meets no product
 * outside the band.  With unit_diag = 1 the diagonal entries are taken as 1
 * and never read.  Storage kinds (all FP64, 8-byte aligned):
 *   BTO_STORE_FULL    column-major, A(i, j) at A[i + j*ld], ld >= max(1, m);
 *   BTO_STORE_BAND    the LAPACK band layout: A(i, j) at A[(ku + i - j) + j*ld],
 *                     ld >= kl + ku + 1 (column j holds its band entries,
 *                     the diagonal in row ku);
 *   BTO_STORE_PACKED  a square triangle (m = n, kl = 0 and ku = n - 1 for the
 *                     upper one, ku = 0 and kl = n - 1 for the lower) packed
 *                     column after column: column j holds rows 0..j (upper)
 *                     or j..n-1 (lower); ld is ignored.
 * Every entry is multiplied in FP64 (two FMAs per stored entry; the sweep is
 * bound by the FP64 pipe).  Each output's partial sums are added in a fixed
 * order, so results are bitwise reproducible.  BATAX forms t = A x in the
 * workspace, then y = beta (A^T t): A is read twice.
 * ws: bto_band_workspace_bytes (or bto_tri_workspace_bytes) bytes, 256-byte
 * aligned, not shared with a call in flight; its first word is the device
 * status (always BTO_OK for these calls).  Argument positions are 1-based as
 * in every entry point (bto_last_invalid_arg). */
#define BTO_STORE_FULL 0
#define BTO_STORE_BAND 1
#define BTO_STORE_PACKED 2
#define BTO_UPPER 0
#define BTO_LOWER 1

/* Workspace bytes of a band call; op is BTO_OP_BICGK or BTO_OP_ATAX. */
bto_status bto_band_workspace_bytes(int op, int64_t m, int64_t n, int64_t kl, int64_t ku, size_t *bytes);

/* q <- A p (q: m), s <- A^T r (s: n); p: n, r: m. */
bto_status bto_band_bicgk(int storage, int64_t m, int64_t n, int64_t kl, int64_t ku, int unit_diag,
                          const double *A, int64_t ld, const double *p, const double *r, double *q, double *s,
                          void *ws, size_t ws_bytes, bto_stream_t stream);

/* y <- beta A^T (A x); x: n, y: n. */
bto_status bto_band_atax(int storage, int64_t m, int64_t n, int64_t kl, int64_t ku, int unit_diag, double beta,
                         const double *A, int64_t ld, const double *x, double *y, void *ws, size_t ws_bytes,
                         bto_stream_t stream);

/* Triangular n x n forms of the same calls: uplo BTO_UPPER or BTO_LOWER,
 * packed 0 (full storage, lda >= max(1, n)) or 1 (packed storage, lda
 * ignored).  Equivalent to the band calls with (kl, ku) = (0, n - 1) or
 * (n - 1, 0). */
bto_status bto_tri_workspace_bytes(int op, int uplo, int64_t n, size_t *bytes);
bto_status bto_tri_bicgk(int uplo, int unit_diag, int packed, int64_t n, const double *A, int64_t lda,
                         const double *p, const double *r, double *q, double *s, void *ws, size_t ws_bytes,
                         bto_stream_t stream);
bto_status bto_tri_atax(int uplo, int unit_diag, int packed, int64_t n, double beta, const double *A,
                        int64_t lda, const double *x, double *y, void *ws, size_t ws_bytes, bto_stream_t stream);

/* --------------------------------------------------------- schedule overrides
 * The FP64 matrix kernels (BICGK, ATAX's two-pass forms, GEMVER, GESUMMV,
 * DGEMV, DGEMVT; op < BTO_OP_AXPYDOT) split A into row blocks x column panels
 * whose partial sums a fixed-order combine adds.  These calls replace the
 * automatic numbers of panels and row blocks for one (op, form), process-wide,
 * so that a measured-cost search (the paper's empirical search, Section IV)
 * can explore the schedules; 0 restores the automatic choice.  Set them before
 * the calls and the bto_workspace_bytes queries they should affect.  Panels are
 * clamped to [ceil(n / 512), n] and row blocks to [1, ceil(m / 64)].  Results
 * stay within the usual tolerance under any schedule (the split changes the
 * summation order).  ATAX's fused group-band kernel has its own plan; its
 * schedule applies to its two-pass form (and to bto_unfused_atax). */
bto_status bto_schedule_set(int op, int form, int panels, int row_blocks);
bto_status bto_schedule_get(int op, int form, int *panels, int *row_blocks);

/* The tile plan the FP64 matrix kernels use for `op` in `form` on an m x n
 * matrix with `sms` multiprocessors (overrides included): writes the number
 * of row blocks and column panels.  Host only; touches no device.  ATAX's
 * fused group-band kernel has its own plan; this is its two-pass plan.  The
 * double-float forms (BTO_FORM_DF, BTO_FORM_DF_UNFUSED) share one plan for
 * every op: panels of at most 1024 columns, at most one tile per
 * multiprocessor where that allows, chosen by the least busiest-block work
 * (256 x 16 units) times one plus the partial-sum bytes over the matrix
 * bytes. */
bto_status bto_panel_plan(int op, int form, int64_t m, int64_t n, int sms, int *row_blocks, int *panels);

/* ------------------------------------------- reduced-precision storage form
 * BICGK, GEMVER, ATAX and GESUMMV (Table I) with the matrices stored in FP32
 * or BF16 to cut the bytes of this bandwidth-bound path (the paper's kernels
 * are FP64; this form has no counterpart there).  a_type is BTO_F32 or BTO_BF16 (raw BF16
 * bits, as uint16).  Vectors and outputs are FP32.  Arithmetic is FP32 with
 * compensated accumulation: products are summed in short FP32 FMA chains
 * (16 columns for A p, 8 rows for A^T r) that are folded into TwoSum
 * (hi, lo) pairs; per-tile results are combined in FP64 in a fixed order and
 * rounded once to FP32.  Against an FP64 evaluation on the same (stored)
 * values the normwise relative error is of order 1e-7.
 * The workspace is bto_workspace_bytes(op, BTO_FORM_FUSED, m, n, a_type).
 * Alignment: A (and B) must be aligned to their element size. */

/* q <- A p ; s <- A^T r, with A m x n (lda) of type a_type. */
bto_status bto_bicgk_ex(int64_t m, int64_t n, int a_type, const void *A, int64_t lda,
                        const float *p, const float *r, float *q, float *s,
                        void *ws, size_t ws_bytes, bto_stream_t stream);

/* B <- A + u1 v1^T + u2 v2^T, formed in FP32 and rounded to a_type (round to
 * nearest even); x <- beta B^T y + z ; w <- alpha B x, both computed from the
 * stored (rounded) B.  B == A with ldb == lda and x == z are allowed. */
bto_status bto_gemver_ex(int64_t m, int64_t n, float alpha, float beta, int a_type,
                         const void *A, int64_t lda, const float *u1, const float *v1,
                         const float *u2, const float *v2, const float *y, const float *z,
                         void *B, int64_t ldb, float *x, float *w,
                         void *ws, size_t ws_bytes, bto_stream_t stream);

/* BATAX (Section II, Fig. 1): y <- beta A^T (A x), A m x n (lda) of type
 * a_type; x: n, y: n (output).  Two sweeps: t = A x is formed and rounded to
 * FP32 in the workspace, then y = beta A^T t, so A is read twice (the FP64
 * form's single-read kernel pays an exchange between blocks that only an
 * arithmetic-bound sweep can hide). */
bto_status bto_atax_ex(int64_t m, int64_t n, float beta, int a_type, const void *A, int64_t lda,
                       const float *x, float *y, void *ws, size_t ws_bytes, bto_stream_t stream);

/* GESUMMV (Table I): y <- alpha A x + beta B x, A and B m x n (lda, ldb) of
 * type a_type; x: n, y: m (output).  One sweep per matrix; a single combine
 * adds both scaled sums in FP64 and rounds once. */
bto_status bto_gesummv_ex(int64_t m, int64_t n, float alpha, float beta, int a_type,
                          const void *A, int64_t lda, const void *B, int64_t ldb,
                          const float *x, float *y, void *ws, size_t ws_bytes,
                          bto_stream_t stream);

/* ------------------------------------------------------------ batched form
 * Many independent, uneven BICGK, GEMVER, ATAX and GESUMMV instances
 * (Table I) in one persistent launch; matrices in FP32 or BF16, vectors FP32
 * (no counterpart in the paper, which times one instance at a time).
 * Arithmetic is that of the reduced-precision form (FP32 FMA chains folded
 * into TwoSum pairs, FP64 for the cross-panel combines); GEMVER's B is
 * rounded to the storage type and x, w use the stored B; ATAX forms
 * t = A x in the workspace (FP32) and reads A a second time for
 * y = beta A^T t.  An instance gives the same bits alone or in a batch
 * planned with the same tile_cols.
 * Use: bto_batch_workspace_bytes -> bto_batch_prepare (host: builds the work
 * list and copies it into ws, waiting for that copy) -> bto_batch_run, as
 * often as wanted while the descriptors' buffers stay valid.  bto_batch_run
 * only enqueues kernels (one cooperative launch, or the few of the
 * multi-launch form) and performs no host synchronisation, so it may be
 * recorded into a CUDA graph.  Calls sharing a ws must be ordered.
 * tile_cols: width of the column panels each work item covers (16..1024, a
 * multiple of 16; 0 picks 128).  Second-stage items (GEMVER's w, ATAX's y)
 * wait for their instance's first stage with a bounded wait (about 2 s); a
 * timeout leaves BTO_ERR_TIMEOUT in the status word (bto_device_status). */
typedef struct bto_batch_desc {
    int32_t op;          /* BTO_OP_BICGK, BTO_OP_GEMVER, BTO_OP_ATAX or BTO_OP_GESUMMV       */
    int32_t a_type;      /* storage type of the matrices: BTO_F32 or BTO_BF16                */
    int64_t m, n;        /* sizes (>= 0)                                                      */
    int64_t lda, ldb;    /* leading dimensions of A and B                                     */
    float alpha, beta;   /* GEMVER, GESUMMV: alpha, beta; ATAX: beta; BICGK: unused           */
    const void *A;       /* m x n, column-major, a_type                                       */
    void *B;             /* GEMVER: output B (ldb, a_type); GESUMMV: second input matrix     */
    const float *in[6];  /* BICGK: p (n), r (m); GEMVER: u1 (m), v1 (n), u2 (m), v2 (n),     */
                         /* y (m), z (n); ATAX: x (n); GESUMMV: x (n)                         */
    float *out[2];       /* BICGK: q (m), s (n); GEMVER: x (n), w (m); ATAX: y (n);          */
                         /* GESUMMV: y (m)                                                    */
} bto_batch_desc;

/* Workspace bytes for a batch of `count` host descriptors. */
bto_status bto_batch_workspace_bytes(int count, const bto_batch_desc *descs, int tile_cols,
                                     size_t *bytes);

/* Validates the host descriptors, builds the work list and copies it into
 * ws (device, 256-byte aligned) on `stream`; returns once the copy is done.
 * A descriptor with a bad size, leading dimension or NULL operand makes the
 * call fail with BTO_ERR_INVALID_VALUE (argument 2). */
bto_status bto_batch_prepare(int count, const bto_batch_desc *descs, int tile_cols, void *ws,
                             size_t ws_bytes, bto_stream_t stream);

/* Runs a prepared batch on `stream`.  When every instance suits the tensor
 * memory accelerator (16-byte aligned matrices and leading dimensions) and
 * all share one storage type, and the device launches cooperatively, the
 * whole batch is one cooperative launch of one block per SM: both stages'
 * sweeps and fixed-order combines, separated by bounded grid barriers (a
 * timeout leaves BTO_ERR_TIMEOUT in the status word; prepare the workspace
 * again before the next run).  Otherwise a reset kernel, the persistent
 * kernels of the load-instruction queues and the tensor-memory sweeps and
 * combines of each stage.  The results are the same either way. */
bto_status bto_batch_run(void *ws, size_t ws_bytes, bto_stream_t stream);

/* Whether bto_batch_run takes the one-launch form for the workspace ws (as
 * last prepared by bto_batch_prepare): *one = 1 or 0.  No device work. */
bto_status bto_batch_one_launch(const void *ws, int *one);

/* Plans and launches a batch in one call: the plan is copied into ws
 * (status word and counters zeroed, so no reset kernel runs) through
 * `staging` when it is pinned host memory of at least the plan's size (the
 * caller keeps it unchanged until the stream has passed the copy), else
 * through a pageable copy that the call waits for; then the one-launch form
 * when it applies (as for bto_batch_run), else only the kernels of the
 * non-empty queues, each grid no larger than its items, so that a small batch
 * leaves the other SMs to other streams.  Same results as
 * bto_batch_prepare + bto_batch_run.  Not for graph capture when staging is
 * NULL (the call waits). */
bto_status bto_batch_submit(int count, const bto_batch_desc *descs, int tile_cols, void *ws,
                            size_t ws_bytes, void *staging, size_t staging_bytes,
                            bto_stream_t stream);

/* ------------------------------------------------------------ serving runtime
 * Continuous batching of BICGK, ATAX, GEMVER and GESUMMV requests (Table I)
 * over resident operands, scheduled by a native polling loop on the calling
 * thread (no counterpart in the paper).  Requests arrive at their times t
 * (seconds after the call starts; non-decreasing); each is an n x n problem
 * on the leading block of a resident nmax x nmax matrix of its storage type
 * (ld nmax) and prefixes of the resident vectors, with FP32 outputs.
 *   - A request with n >= direct_n (direct_n > 0) runs alone through
 *     bto_bicgk_ex / bto_gemver_ex / bto_atax_ex / bto_gesummv_ex.
 *   - Otherwise requests from the head of the arrival queue form a batch
 *     (at most max_batch, stopping before a direct one) launched with the
 *     batched form's plan-and-submit path (tile_cols as there).
 *   - A launch goes to a free slot (one per caller stream); launches on
 *     different slots overlap on the device.
 *   - Outputs, GEMVER's B and workspaces are carved from the caller's device
 *     arena (the HBM budget): admission waits while they do not fit; a request
 *     that cannot fit with nothing in flight ends with BTO_ERR_BUDGET.
 * A request's path and arithmetic depend on the request alone, so its
 * results are the same bits alone and in any mix.  Outputs of finished
 * requests are released unless keep_results (then res->out give their arena
 * offsets, valid until the arena is reused).  Returns BTO_OK, or the first
 * launch or device status that was not BTO_OK (every request still ends). */
typedef struct bto_serve_req {
    double t;            /* arrival, seconds after the start of the call          */
    int32_t op;          /* BTO_OP_BICGK, BTO_OP_ATAX, BTO_OP_GEMVER, BTO_OP_GESUMMV */
    int32_t a_type;      /* BTO_F32 or BTO_BF16: which resident matrices           */
    int64_t n;           /* 1 <= n <= nmax                                         */
} bto_serve_req;

typedef struct bto_serve_res {
    double admit;        /* seconds after the start: launched (-1: never)                  */
    double done;         /* seconds after the start: completion observed (-1: never)       */
    int64_t out[3];      /* arena byte offsets: outputs 0 and 1 (as bto_batch_desc.out),     */
                         /* GEMVER's B (n x n in A's storage type, leading dimension n     */
                         /* rounded up to a multiple of 8); -1 where none                   */
    int32_t status;      /* BTO_OK, the device status of its launch, or BTO_ERR_BUDGET     */
    int32_t direct;      /* 1: served alone by a bto_*_ex entry point                      */
} bto_serve_res;

typedef struct bto_serve_cfg {
    const void *A[2][2];          /* [F32, BF16][A, GESUMMV's B]: nmax x nmax, ld nmax          */
    const float *vec[6];          /* resident vectors (>= nmax): inputs in bto_batch_desc order */
    void *arena;                  /* device memory, 256-byte aligned: the HBM budget             */
    void *staging;                /* pinned host memory, 256-byte aligned (or NULL)              */
    const bto_stream_t *streams;  /* nstreams launch slots                                       */
    size_t arena_bytes, staging_bytes;
    int64_t nmax, direct_n;
    double max_wall;              /* stop admitting after this many seconds (0: no limit)        */
    float alpha, beta;            /* GEMVER, GESUMMV: alpha, beta; ATAX: beta                    */
    int32_t nstreams;             /* 1..64                                                       */
    int32_t max_batch, tile_cols, keep_results;
} bto_serve_cfg;

typedef struct bto_serve_stats {
    int64_t served, batches, direct, rejected;
    double wall_s, peak_bytes;    /* run time; high-water mark of the arena in use */
    /* Diagnostics of the loop itself (seconds on the loop's clock):          */
    double max_gap_s, max_gap_at_s;   /* longest time between two passes of the loop, and when */
    double max_admit_s;               /* longest single admission (plan, copy, launches)      */
    double max_complete_s;            /* longest completion scan                              */
    double max_oversleep_s;           /* longest overshoot of an idle sleep                   */
    int64_t max_fifo;                 /* deepest FIFO of arrived, unadmitted requests         */
    int64_t fifo_at_max_gap;          /* its depth when the longest gap ended                 */
    int64_t sleeps;                   /* idle sleeps taken                                    */
    int64_t blocking_copies;          /* batch plans too large for their staging slice,      */
                                      /* copied with a wait on the stream                    */
    double max_query_s;               /* longest single completion-event query (driver call) */
} bto_serve_stats;

bto_status bto_serve_run(const bto_serve_cfg *cfg, int64_t count, const bto_serve_req *req,
                         bto_serve_res *res, bto_serve_stats *stats);

/* ------------------------------------------------- multi-right-hand-side BICGK
 * The BICGK kernel of Table I with k right-hand sides at once (the paper has
 * one; a block Krylov method or several independent solves sharing A has k):
 *     Q <- A P,   S <- A^T R
 * A m x n, P n x k, R m x k, all BF16 (raw 16-bit words, column-major with
 * leading dimensions lda, ldp, ldr); Q m x k and S n x k FP32 (ldq, lds).
 * Every element of A is read from device memory once and feeds both
 * products, which run on the tensor cores (BF16 products, FP32
 * accumulation); partial sums over 512-column panels and over row ranges are
 * added in compensated FP32 (TwoSum) in a fixed order, so the result is
 * reproducible bit for bit and its normwise error against the exact product
 * of the BF16 inputs is of order 1e-7 for uniform random data.
 *  - k: 16 to 96, a multiple of 16.  m = 0 or n = 0 is accepted (Q or S
 *    becomes 0; the other is empty).
 *  - A, P, R must be 2-byte aligned, Q and S 4-byte aligned.  When A, P and
 *    R are 16-byte aligned with leading dimensions that are multiples of 8,
 *    tiles are copied by the tensor memory accelerator; otherwise a slower
 *    kernel copies 16-byte chunks (element by element where unaligned).  Both
 *    give the same bits.
 *  - Q and S must not overlap each other or any input.
 *  - ws: device memory of bto_bicgk_mrhs_workspace_bytes(m, n, k) bytes,
 *    256-byte aligned, owned by the caller; nothing in it needs to start at
 *    zero.  Its first int is the status word (bto_device_status).
 *  - Waits inside the kernel are bounded (1 s); a timeout leaves
 *    BTO_ERR_TIMEOUT in the status word.
 * Errors: BTO_ERR_INVALID_VALUE with bto_last_invalid_arg() naming the
 * argument (1-based), BTO_ERR_WORKSPACE (argument 14) for a missing, short
 * or misaligned workspace, BTO_ERR_CUDA for a failed launch. */
bto_status bto_bicgk_mrhs_workspace_bytes(int64_t m, int64_t n, int64_t k, size_t *bytes);
bto_status bto_bicgk_mrhs(int64_t m, int64_t n, int64_t k, const uint16_t *A, int64_t lda,
                          const uint16_t *P, int64_t ldp, const uint16_t *R, int64_t ldr,
                          float *Q, int64_t ldq, float *S, int64_t lds,
                          void *ws, size_t ws_bytes, bto_stream_t stream);

/* BICGK without a workspace argument (the paper has no counterpart; this is
 * a convenience of this library).  Some callers cannot call cudaMalloc: a
 * plugin whose host application owns all device memory through its own
 * allocator, code that must keep a device-memory footprint fixed when the
 * library loads, and latency-critical loops, since cudaMalloc and cudaFree
 * may synchronize the device.  This entry point computes exactly what
 * bto_bicgk computes (same kernels, bitwise equal results) but keeps the
 * split partial sums in a file-scope device array of
 * BTO_NOALLOC_SCRATCH_BYTES (4 MiB) inside the library, which every GPU that
 * loads the library holds until the process exits.  It allocates nothing.
 *  - Size limit: the call is accepted when
 *    bto_workspace_bytes(BTO_OP_BICGK, BTO_FORM_FUSED, m, n, BTO_F64) is at
 *    most BTO_NOALLOC_SCRATCH_BYTES (for square FP64 problems on a 152-SM
 *    GB300, every n up to 3427); larger workspaces return BTO_ERR_WORKSPACE
 *    with bto_last_invalid_arg() naming m (1) or n (2), and nothing runs.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.  The address is kept for the life of the
 *    process: do not call this entry point on a device after resetting it
 *    (cudaDeviceReset), since the array may then live elsewhere.
 *  - All calls share the one array, and it keeps the last call's contents;
 *    no part of it needs to start at zero.  Calls whose kernels overlap on
 *    the GPU (different streams, no ordering between them) race on the
 *    array and give undefined results: order them.
 * Arguments, layout and errors are otherwise those of bto_bicgk. */
#define BTO_NOALLOC_SCRATCH_BYTES ((size_t)4 << 20)
bto_status bto_bicgk_noalloc(int64_t m, int64_t n, const double *A, int64_t lda,
                             const double *p, const double *r, double *q, double *s,
                             bto_stream_t stream);

/* ------------------------------------------- unfused comparison sequences
 * Same operations, arguments and results as the fused entry points above,
 * computed as one GPU kernel per BLAS call, the way a program built from
 * separately tuned BLAS routines would (the BICGK listing of Section V-A;
 * the other kernels by the same translation): temporaries and intermediate
 * results round-trip through device memory.
 *   BICGK:   dgemv N (q = A p); dgemv T (s = A^T r)
 *   ATAX:    dgemv N (t = A x, t in ws); dgemv T (y = A^T t); dscal (y = beta y)
 *   GEMVER:  dcopy (B = A); dger (B += u1 v1^T); dger (B += u2 v2^T);
 *            dcopy (x = z); dgemv T (x = beta B^T y + x); dgemv N (w = alpha B x)
 *   GESUMMV: dgemv N (y = alpha A x); dgemv N (y = beta B x + y)
 *   DGEMV:   dgemv N (z = alpha A x + beta y)
 *   DGEMVT:  dcopy (x = z); dgemv T (x = beta A^T y + x); dgemv N (w = alpha A x)
 *   AXPYDOT: dcopy (z = w); daxpy (z = -alpha v + z); ddot (r = z^T u)
 *   WAXPBY:  dcopy (w = y); dscal (w = beta w); daxpy (w = alpha x + w)
 *   VADD:    dcopy (x = w); daxpy (x = y + x); daxpy (x = z + x)
 * In-place forms are not accepted here.  Results agree with the fused forms
 * to rounding (the association of some sums differs). */
bto_status bto_unfused_bicgk(int64_t m, int64_t n, const double *A, int64_t lda,
                             const double *p, const double *r, double *q, double *s,
                             void *ws, size_t ws_bytes, bto_stream_t stream);
bto_status bto_unfused_atax(int64_t m, int64_t n, double beta, const double *A, int64_t lda,
                            const double *x, double *y, void *ws, size_t ws_bytes,
                            bto_stream_t stream);
bto_status bto_unfused_gemver(int64_t m, int64_t n, double alpha, double beta,
                              const double *A, int64_t lda, const double *u1,
                              const double *v1, const double *u2, const double *v2,
                              const double *y, const double *z, double *B, int64_t ldb,
                              double *x, double *w, void *ws, size_t ws_bytes,
                              bto_stream_t stream);
bto_status bto_unfused_gesummv(int64_t m, int64_t n, double alpha, const double *A,
                               int64_t lda, double beta, const double *B, int64_t ldb,
                               const double *x, double *y, void *ws, size_t ws_bytes,
                               bto_stream_t stream);
bto_status bto_unfused_dgemv(int64_t m, int64_t n, double alpha, const double *A, int64_t lda,
                             const double *x, double beta, const double *y, double *z,
                             void *ws, size_t ws_bytes, bto_stream_t stream);
bto_status bto_unfused_dgemvt(int64_t m, int64_t n, double alpha, double beta,
                              const double *A, int64_t lda, const double *y,
                              const double *z, double *x, double *w,
                              void *ws, size_t ws_bytes, bto_stream_t stream);
bto_status bto_unfused_axpydot(int64_t n, double alpha, const double *w, const double *v,
                               const double *u, double *z, double *r,
                               void *ws, size_t ws_bytes, bto_stream_t stream);
bto_status bto_unfused_waxpby(int64_t n, double alpha, const double *x, double beta,
                              const double *y, double *w, bto_stream_t stream);
bto_status bto_unfused_vadd(int64_t n, const double *w, const double *y, const double *z,
                            double *x, bto_stream_t stream);

/* --------------------------------- double-float form of the FP64 sequences
 * The six FP64 matrix sequences of Table I (Section V-A) with the same
 * arguments, outputs, aliasing rules and validation as bto_bicgk ..
 * bto_dgemvt and bto_unfused_* above, computed in double-float arithmetic
 * (each FP64 value carried as a sum of two FP32 numbers) on the FP32 units
 * instead of the FP64 unit, which on this GPU issues two FMAs per clock per
 * SM, too few to keep up with HBM.  Data in and out are FP64; only the
 * arithmetic differs from the FP64 form:
 *   - each matrix and vector element keeps 47 of its 53 significant bits
 *     (the low 6 fraction bits are dropped); each product is exact up to
 *     the dropped low-part product (below 2^-47 of it); sums are
 *     compensated (TwoSum); the final reduction over tiles is FP64.
 *     Normwise relative error against exact FP64 arithmetic: about 1e-14 on
 *     ordinary data (the FP64 form's contract is 1e-12); integer-valued data
 *     below 2^24 in magnitude give exact results, as in the FP64 form.
 *   - GEMVER's B is formed with the FP64 form's two FMAs per element
 *     (the same bits as bto_gemver's B); x and w are double-float sums over
 *     that B.
 *   - FP32's exponent range: values below 2^-127 in magnitude count as zero
 *     and products below about 2^-100 lose low-order bits, an absolute error
 *     below 2^-126 times the other factor per element (the underflow term of
 *     the error bound).  Values of 2^128 or more, Inf, NaN, and products or
 *     sums beyond FP32's range make a 256-row chunk's results non-finite;
 *     such a chunk is recomputed in FP64, so those inputs propagate as in
 *     the FP64 form.
 *   - Layout: the matrices are copied by the tensor memory accelerator, which
 *     needs 16-byte aligned matrix pointers and even leading dimensions (and
 *     m, n < 2^31).  Otherwise the call runs the FP64 form with the same
 *     arguments (the workspace is large enough for either).
 * Workspace: bto_workspace_bytes(op, BTO_FORM_DF, m, n, BTO_F64) for the
 * fused calls, BTO_FORM_DF_UNFUSED for the unfused ones.  The status word at
 * the start of ws is cleared by the call and reads BTO_ERR_TIMEOUT
 * (bto_device_status) if a bounded wait of the sweep expired.
 * ATAX in this form reads A twice (t = A x, then y = beta A^T t), as its
 * unfused form; the other fused forms read each matrix as often as the FP64
 * fused form.  The unfused forms follow the decompositions listed above,
 * with every dgemv a double-float sweep (dcopy, dger, dscal stay FP64). */
bto_status bto_bicgk_df(int64_t m, int64_t n, const double *A, int64_t lda,
                        const double *p, const double *r, double *q, double *s,
                        void *ws, size_t ws_bytes, bto_stream_t stream);
bto_status bto_atax_df(int64_t m, int64_t n, double beta, const double *A, int64_t lda,
                       const double *x, double *y, void *ws, size_t ws_bytes,
                       bto_stream_t stream);
bto_status bto_gemver_df(int64_t m, int64_t n, double alpha, double beta,
                         const double *A, int64_t lda, const double *u1,
                         const double *v1, const double *u2, const double *v2,
                         const double *y, const double *z, double *B, int64_t ldb,
                         double *x, double *w, void *ws, size_t ws_bytes,
                         bto_stream_t stream);
bto_status bto_gesummv_df(int64_t m, int64_t n, double alpha, const double *A, int64_t lda,
                          double beta, const double *B, int64_t ldb, const double *x,
                          double *y, void *ws, size_t ws_bytes, bto_stream_t stream);
bto_status bto_dgemv_df(int64_t m, int64_t n, double alpha, const double *A, int64_t lda,
                        const double *x, double beta, const double *y, double *z,
                        void *ws, size_t ws_bytes, bto_stream_t stream);
bto_status bto_dgemvt_df(int64_t m, int64_t n, double alpha, double beta,
                         const double *A, int64_t lda, const double *y,
                         const double *z, double *x, double *w,
                         void *ws, size_t ws_bytes, bto_stream_t stream);
bto_status bto_unfused_bicgk_df(int64_t m, int64_t n, const double *A, int64_t lda,
                                const double *p, const double *r, double *q, double *s,
                                void *ws, size_t ws_bytes, bto_stream_t stream);
bto_status bto_unfused_atax_df(int64_t m, int64_t n, double beta, const double *A, int64_t lda,
                               const double *x, double *y, void *ws, size_t ws_bytes,
                               bto_stream_t stream);
bto_status bto_unfused_gemver_df(int64_t m, int64_t n, double alpha, double beta,
                                 const double *A, int64_t lda, const double *u1,
                                 const double *v1, const double *u2, const double *v2,
                                 const double *y, const double *z, double *B, int64_t ldb,
                                 double *x, double *w, void *ws, size_t ws_bytes,
                                 bto_stream_t stream);
bto_status bto_unfused_gesummv_df(int64_t m, int64_t n, double alpha, const double *A,
                                  int64_t lda, double beta, const double *B, int64_t ldb,
                                  const double *x, double *y, void *ws, size_t ws_bytes,
                                  bto_stream_t stream);
bto_status bto_unfused_dgemv_df(int64_t m, int64_t n, double alpha, const double *A, int64_t lda,
                                const double *x, double beta, const double *y, double *z,
                                void *ws, size_t ws_bytes, bto_stream_t stream);
bto_status bto_unfused_dgemvt_df(int64_t m, int64_t n, double alpha, double beta,
                                 const double *A, int64_t lda, const double *y,
                                 const double *z, double *x, double *w,
                                 void *ws, size_t ws_bytes, bto_stream_t stream);

/* ------------------------------------------------ synthetic input fills
 * Not part of any Table I operation: device-side generation of the seeded
 * test and benchmark inputs, so that matrices of several GiB need no host
 * copy.  Element (i, j) of an m x n array receives value(seed, aid, i + j*m)
 * (multiplied by colscale[j] when colscale is non-NULL), where value() is
 * the SplitMix64 counter stream of Steele, Lea and Flood (OOPSLA 2014):
 *   key = fmix(seed * 2^32 + aid); u = fmix(key + (k + 1) * 0x9E3779B97F4A7C15)
 *   kind 0: 2 * ((u >> 11) * 2^-53) - 1   (uniform in [-1, 1))
 *   kind 1: ((u >> 11) mod 17) - 8         (integers in [-8, 8])
 * `out` is column-major with leading dimension ld >= max(1, m); padding rows
 * are left untouched.  The f32/bf16 forms round the FP64 value to nearest
 * even (one rounding).  colscale, when given, is a device vector of n doubles. */
bto_status bto_fill_f64(uint64_t seed, uint64_t aid, int kind, int64_t m, int64_t n,
                        const double *colscale, double *out, int64_t ld, bto_stream_t stream);
bto_status bto_fill_f32(uint64_t seed, uint64_t aid, int kind, int64_t m, int64_t n,
                        const double *colscale, float *out, int64_t ld, bto_stream_t stream);
bto_status bto_fill_bf16(uint64_t seed, uint64_t aid, int kind, int64_t m, int64_t n,
                         const double *colscale, uint16_t *out, int64_t ld,
                         bto_stream_t stream);

/* ------------------------------------------------------------ testing
 * Fault injection for the bounded inter-block waits of bto_atax (no
 * counterpart in the paper).  Runs bto_atax, except that the ready flag of
 * row band `stall_band` (bands are the kernel's internal row groups; 0 is
 * the first) is never published, so every wait for it expires after
 * `timeout_ms` (1..10000) milliseconds instead of about two seconds.  The
 * kernel then returns early, y is unspecified, and bto_device_status reads
 * BTO_ERR_TIMEOUT.  No fault is raised on the device.  With stall_band < 0
 * the call is bto_atax with a shorter wait limit. */
bto_status bto_debug_atax_stall(int64_t m, int64_t n, double beta, const double *A, int64_t lda,
                                const double *x, double *y, void *ws, size_t ws_bytes,
                                int64_t stall_band, int timeout_ms, bto_stream_t stream);

/* Fault injection for the grid barriers of the batched form's one-launch
 * form (see bto_batch_run; the workspace must have been prepared for it,
 * else BTO_ERR_UNSUPPORTED).  Runs it with block `stall_block` never
 * arriving at the barriers, so every wait expires after `timeout_ms`
 * (1..10000) milliseconds: the outputs are unspecified and
 * bto_device_status reads BTO_ERR_TIMEOUT; prepare the workspace again before
 * the next run.  No fault is raised on the device. */
bto_status bto_debug_batch_stall(void *ws, size_t ws_bytes, int stall_block, int timeout_ms,
                                 bto_stream_t stream);

/* The batched sweep's assignment of one list of work items to the `grid`
 * (1..65536) blocks of its launch, computed on the host as bto_batch_prepare
 * does for a list longer than the grid: items in decreasing cost (count >=
 * 0 costs, each >= 0 and none above the one before it, else
 * BTO_ERR_INVALID_VALUE, argument 2), each to the block with the least cost
 * so far, ties to the lower block (longest processing time first).  Writes
 * block[k] in [0, grid) for every item.  No device work. */
bto_status bto_debug_lpt(int64_t count, const double *cost, int grid, int32_t *block);

/* Fault injection for the ring waits of the double-float sweeps.  Runs
 * bto_bicgk_df, except that in block `stall_block` (>= 0; a block of the
 * sweep's grid) the producer stops after filling the ring once, so that
 * block's consumer waits expire after `timeout_ms` (1..10000) milliseconds
 * instead of about two seconds: q and s are unspecified and
 * bto_device_status reads BTO_ERR_TIMEOUT when that block had more than one
 * ring fill (five stages of 256 x 16) of work.  The next call clears the
 * status word.  No fault is raised on the device.  BTO_ERR_UNSUPPORTED when
 * the sizes or layout send the call to the FP64 form. */
bto_status bto_debug_df_stall(int64_t m, int64_t n, const double *A, int64_t lda, const double *p,
                              const double *r, double *q, double *s, void *ws, size_t ws_bytes,
                              int stall_block, int timeout_ms, bto_stream_t stream);

/* Fault injection for the grid barrier of the one-launch GEMVER (bto_gemver
 * takes it for matrices with m n <= 2^23 and max(3 m, 2 n) <= 12800 when the
 * device allows a cooperative launch).  Runs that form with block
 * `stall_block` never arriving at the barrier, so every wait expires after
 * `timeout_ms` (1..10000) milliseconds: the kernel returns without the second
 * pass, w is unspecified (B and x are complete) and bto_device_status reads
 * BTO_ERR_TIMEOUT.  No fault is raised on the device.  stall_block < 0 runs
 * the form normally.  BTO_ERR_UNSUPPORTED when the sizes do not qualify.
 * ws: at least 256 bytes, 256-byte aligned. */
bto_status bto_debug_gemver_stall(int64_t m, int64_t n, double alpha, double beta, const double *A, int64_t lda,
                                  const double *u1, const double *v1, const double *u2, const double *v2,
                                  const double *y, const double *z, double *B, int64_t ldb, double *x, double *w,
                                  void *ws, size_t ws_bytes, int stall_block, int timeout_ms,
                                  bto_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* BTO_H */
