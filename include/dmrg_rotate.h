/*
 * dmrg_rotate.h -- C ABI of the GB300 (sm_103a) DMRG operator-rotation library.
 *
 * The library performs the density-matrix rotation and decimation step of
 * the DMRG (Rincon, Garcia, Hallberg, "Improved parallelization techniques
 * for the density matrix renormalization group", Sec. 2, algorithm step 5,
 * and the paragraph after it):
 *
 *     O'_k = U^T (O_k (x) I_d) U,        k = 0 .. K-1,
 *
 * where O_k is an m x m block operator, I_d the identity of the added site
 * (the "blocking" Z_[B a] <- Z_[B (+) a]), and U = R^+ the (m*d) x m'
 * matrix of kept density-matrix eigenvectors (step 4; real data, so
 * R^+ = R^T).  Sec. 3.2 identifies the two matrix products Z R^+ and
 * R (Z R^+) over the K stored Z_i and Z_i Z_j operators as the most
 * expensive part of a DMRG run that measures correlation functions.
 *
 * Conventions shared by every entry point
 *   - Index convention of [B a]: row r = i*d + s (block state i, site state
 *     s), i.e. the blocked operator is kron(O, I_d).  All matrices row-major.
 *   - Every data pointer is a DEVICE pointer owned by the caller.  The
 *     library never keeps a reference to caller memory after a call returns.
 *   - Calls are asynchronous on `stream` (NULL = legacy default stream).
 *     Argument and shape errors are returned synchronously, before anything
 *     is launched.  A kernel that gives up waiting (bounded spin on an
 *     mbarrier) records DMRG_ERR_TIMEOUT in a device status word owned by
 *     the handle; dmrg_sync_status() reads and clears it.
 *   - The hot-path calls allocate nothing: scratch memory is the caller's
 *     workspace `ws` of at least the size returned by the matching
 *     *_workspace query.  Workspace pointers must be 256-byte aligned.
 *   - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef DMRG_ROTATE_H
#define DMRG_ROTATE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DMRG_API __attribute__((visibility("default")))
#else
#define DMRG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
/* Same type as cudaStream_t. */
typedef struct CUstream_st* dmrg_stream_t;

typedef enum {
    DMRG_OK = 0,
    DMRG_ERR_INVALID_ARG = 1,      /* null pointer, bad enum, misaligned pointer        */
    DMRG_ERR_SHAPE = 2,            /* inconsistent or unsupported sizes                  */
    DMRG_ERR_NOT_ORTHONORMAL = 3,  /* ||U^T U - I||_F above the checked tolerance       */
    DMRG_ERR_WORKSPACE = 4,        /* workspace missing or smaller than the query says   */
    DMRG_ERR_CUDA = 5,             /* a CUDA runtime/driver call failed                  */
    DMRG_ERR_TIMEOUT = 6,          /* a device-side bounded wait expired                 */
    DMRG_ERR_UNSUPPORTED = 7       /* combination not implemented (e.g. GPU too old)     */
} dmrg_status;

/* Arithmetic of the two products.
 *   FP64   : plain FP64 FMA on the GPU (reference path).
 *   FP32   : plain FP32 FMA.
 *   TF32   : tcgen05 tensor cores, kind::tf32, FP32 accumulate.
 *   BF16X3 : tcgen05 tensor cores, kind::f16 with every operand split into a
 *            BF16 pair x = hi + lo and hi*hi + hi*lo + lo*hi accumulated in FP32. */
typedef enum {
    DMRG_PREC_FP64 = 0,
    DMRG_PREC_FP32 = 1,
    DMRG_PREC_TF32 = 2,
    DMRG_PREC_BF16X3 = 3
} dmrg_precision;

typedef struct dmrg_handle_s* dmrg_handle;

/* Creates a handle bound to the current CUDA device.  It owns a small device
 * status word, the autotuner's cache and any captured CUDA graphs. */
DMRG_API dmrg_status dmrg_create(dmrg_handle* handle);
DMRG_API dmrg_status dmrg_destroy(dmrg_handle handle);
DMRG_API const char* dmrg_status_string(dmrg_status status);
/* Human-readable detail of the last error returned on this handle ("" if none). */
DMRG_API const char* dmrg_last_error(dmrg_handle handle);
/* Synchronises `stream`, then reads and clears the device status word:
 * DMRG_ERR_TIMEOUT if a kernel gave up on a bounded wait since the last check. */
DMRG_API dmrg_status dmrg_sync_status(dmrg_handle handle, dmrg_stream_t stream);

/* Options (value is a double for uniformity).
 *   DMRG_OPT_GRAPH           : 1 = capture each distinct call (pointers + sizes)
 *                              in a CUDA graph on first use and replay it after.
 *   DMRG_OPT_KERNEL_TIMING   : 1 = record CUDA events around every kernel the
 *                              library launches (read with dmrg_kernel_timing).
 *   DMRG_OPT_WAIT_TIMEOUT_MS : device-side bounded-wait limit (default 2000 ms).
 *   DMRG_OPT_CHECK_ORTHO     : tolerance > 0 makes dmrg_rotate_ops verify
 *                              ||U^T U - I||_F <= tol first (synchronises the
 *                              stream); 0 = off (default).
 *   DMRG_OPT_DETERMINISTIC   : 1 = bit-reproducible results.  By default the
 *                              tiles left over after the last full wave of the
 *                              second product are split along the reduction and
 *                              accumulated with FP32 atomics, so the last few
 *                              operators' rounding order may differ between runs
 *                              (within the precision's tolerance).
 *   DMRG_OPT_ACCUM_CHAIN     : longest reduction (in elements) that one tensor-core
 *                              FP32 accumulator sums in the BF16x3 dense products
 *                              (default 1024, accepted 1 .. 1024).  A longer
 *                              reduction (and longer than 512) is cut into chains of
 *                              this length whose results are added in FP32 with
 *                              round to nearest; the tensor core's own accumulation
 *                              error grows with the chain length, and chains longer
 *                              than 1024 (or one chain per tile) break the 1e-5
 *                              BF16x3 bound at m*d = 4800, so such values return
 *                              DMRG_ERR_INVALID_ARG.  Products whose reduction needs
 *                              chains always run on the CTA-pair kernel, whatever
 *                              tiling is cached.
 *   DMRG_OPT_BLOCKED_SMALL   : 1 (default) = blocked plans whose sectors all hold at
 *                              most 32 states (site dimension <= 8) run one fused
 *                              kernel, one warp per (operator, output block), in FP32
 *                              for the reduced precisions (more accurate than they
 *                              ask) and FP64 for DMRG_PREC_FP64; 0 = the grouped GEMMs.
 *   DMRG_OPT_TRUNCATION_JACOBI : 1 = dmrg_truncation diagonalises rho by cyclic Jacobi
 *                              sweeps; 0 (default) = Householder tridiagonalisation,
 *                              bisection and inverse iteration (rows <= 6144; larger
 *                              matrices take the Jacobi sweeps).
 *   DMRG_OPT_FUSED_ROTATION  : 1 = dmrg_rotate_ops runs DMRG_PREC_BF16X3 with
 *                              mp <= 256 as one kernel per call that keeps the
 *                              intermediate (O_k (x) I_d) U on chip (tensor memory and
 *                              shared memory) instead of writing it to global memory.
 *                              Same precision and workspace as the two-product path.
 *                              0 (default) = the two products (mp > 256 always).
 *                              Other values return DMRG_ERR_INVALID_ARG.
 *   DMRG_OPT_PACK_OPERATORS  : how the TF32 and BF16x3 dense products take FP32
 *                              operators whose rows are whole 16-byte units
 *                              (m % 4 == 0, 16-byte aligned base).  Either a separate
 *                              pass packs them (BF16 hi/lo split or TF32 rounding), or
 *                              the first product reads them as they are and converts
 *                              each tile in shared memory into the same values (results
 *                              are bit-identical).  The conversion is repeated for
 *                              every N tile of the first product, so it pays only for
 *                              few tiles.  0 (default) = convert for BF16x3 when d*mp
 *                              fits in two N tiles, else pack; 1 = always pack;
 *                              2 = convert whenever the layout allows.  FP64 operators
 *                              and other rows are always packed.
 *   DMRG_OPT_STORE_EPILOGUE  : how the tensor-core products on CTA pairs write their
 *                              results: the first product's T = O_k U_r (BF16 hi/lo
 *                              or TF32; d = 2 or 4, m a multiple of 16), the second
 *                              product's O'_k (FP32, m' a multiple of 16, at most two
 *                              accumulation chains per tile) and the adjoint's W'_k,
 *                              W_k and dO_k.  0 (default) = each epilogue warp stages a
 *                              32 x 32 chunk in shared memory and one lane sends it out
 *                              with TMA bulk tensor stores (a second accumulation chain,
 *                              or a part of a split tile, with TMA reductions) where
 *                              the layout and the shared memory allow (else as 1);
 *                              1 = every thread stores its own values.  The values
 *                              written are the same (FP32 sums flush subnormal results
 *                              to zero either way).  Other values return
 *                              DMRG_ERR_INVALID_ARG.
 *   DMRG_OPT_TEST_WITHHOLD_ARRIVAL : test hook for failure detection.  1 makes
 *                              the next dense tensor-core launch withhold one
 *                              shared-memory stage release in its first CTA, so
 *                              a bounded wait expires: the kernel winds down
 *                              (waiting, with a fixed limit, for copies and MMAs
 *                              already issued) and dmrg_sync_status() returns
 *                              DMRG_ERR_TIMEOUT.  No fault, trap or hang. */
typedef enum {
    DMRG_OPT_GRAPH = 1,
    DMRG_OPT_KERNEL_TIMING = 2,
    DMRG_OPT_WAIT_TIMEOUT_MS = 3,
    DMRG_OPT_CHECK_ORTHO = 4,
    DMRG_OPT_TEST_WITHHOLD_ARRIVAL = 5,
    DMRG_OPT_DETERMINISTIC = 6,
    DMRG_OPT_ACCUM_CHAIN = 7,
    DMRG_OPT_BLOCKED_SMALL = 8,
    DMRG_OPT_TRUNCATION_JACOBI = 9,
    DMRG_OPT_FUSED_ROTATION = 10,
    DMRG_OPT_PACK_OPERATORS = 11,
    DMRG_OPT_STORE_EPILOGUE = 12
} dmrg_option;
DMRG_API dmrg_status dmrg_set_option(dmrg_handle handle, dmrg_option option, double value);

/* Writes a JSON array [{"kernel": name, "launches": n, "total_ms": t}, ...]
 * of the events recorded since the last reset into buf (synchronises the
 * recorded events).  reset != 0 clears the record afterwards. */
DMRG_API dmrg_status dmrg_kernel_timing(dmrg_handle handle, char* buf, size_t buf_len, int reset);

/* ------------------------------------------------------------------------
 * Dense rotation (Sec. 2 step 5; Sec. 3.2 two-product order).
 *
 *   U    : (m*d) x mp, FP64, orthonormal columns, row-major.
 *   O    : K x m x m, FP64 if in_is_fp64 else FP32.  The FP64 precision needs
 *          FP64 input.
 *   Oout : K x mp x mp; FP64 for DMRG_PREC_FP64, FP32 for every other
 *          precision.  Must not overlap O, U or ws.
 *   Requires m >= 1, d >= 1, 1 <= mp <= m*d, K >= 0 (K = 0 is a no-op),
 *   and (tensor-core precisions) m*d <= 2^31 - 1 and K*max(m, mp) <= 2^31 - 1.
 *
 * Implementation: the blocking is never materialised.  With U viewed as the
 * m x (d*mp) matrix U_r[j][s*mp + b] = U[j*d + s][b], the first product is
 * T_k = O_k U_r (= (O_k (x) I_d) U), the second O'_k = U^T T_k.  Tensor-core
 * precisions stack all K operators into one GEMM per product.
 * ------------------------------------------------------------------------ */
DMRG_API dmrg_status dmrg_rotate_ops_workspace(dmrg_handle handle, int64_t K, int64_t m, int d, int64_t mp,
                                      dmrg_precision precision, size_t* bytes);
DMRG_API dmrg_status dmrg_rotate_ops(dmrg_handle handle, const double* U, int64_t m, int d, int64_t mp,
                            const void* O, int in_is_fp64, int64_t K, void* Oout,
                            dmrg_precision precision, void* ws, size_t ws_bytes,
                            dmrg_stream_t stream);

/* The same rotation with U, O and Oout in HOST memory (page-locked for the copies
 * to overlap the computation; pageable memory works but serialises).  The batch is
 * processed in chunks of `chunk` consecutive operators (0 = about K/5): while chunk
 * c is rotated, chunk c+1 is copied in and chunk c-1 copied out on two streams
 * owned by the handle, and rotations alternate between `stream` and a third
 * handle stream, so host-to-device copies, kernels and device-to-host copies
 * overlap.  Operators are independent given U, which is what
 * makes the split exact (the paper's UMD distribution rests on the same fact,
 * Sec. 3.2).  ws: device workspace of dmrg_rotate_ops_host_workspace() bytes.
 * Asynchronous on `stream`: Oout is complete once `stream` is. */
DMRG_API dmrg_status dmrg_rotate_ops_host_workspace(dmrg_handle handle, int64_t K, int64_t m, int d,
                                                    int64_t mp, dmrg_precision precision,
                                                    int in_is_fp64, int64_t chunk, size_t* bytes);
DMRG_API dmrg_status dmrg_rotate_ops_host(dmrg_handle handle, const double* U, int64_t m, int d,
                                          int64_t mp, const void* O, int in_is_fp64, int64_t K,
                                          void* Oout, dmrg_precision precision, int64_t chunk,
                                          void* ws, size_t ws_bytes, dmrg_stream_t stream);

/* Runs every candidate tiling of the tensor-core kernels on these buffers,
 * times them with CUDA events and caches the fastest for this shape in the
 * handle (and in the JSON file named by $DMRG_AUTOTUNE_CACHE, if set).
 * Overwrites Oout and ws.  Synchronous.  FP64/FP32 precisions: no-op. */
DMRG_API dmrg_status dmrg_autotune_rotate_ops(dmrg_handle handle, const double* U, int64_t m, int d,
                                     int64_t mp, const void* O, int in_is_fp64, int64_t K,
                                     void* Oout, dmrg_precision precision, void* ws,
                                     size_t ws_bytes, dmrg_stream_t stream);

/* ------------------------------------------------------------------------
 * Adjoint of the dense rotation for a loss L with dL/dO'_k = G_k:
 *   dO_k = Tr_d(U G_k U^T)        i.e. dO_k[i][j] = sum_s (U G_k U^T)[i*d+s][j*d+s]
 *   dU   = sum_k (O_k (x) I_d) U G_k^T + (O_k (x) I_d)^T U G_k
 * (chain rule of the rotation of Sec. 2 step 5; the paper has no gradient).
 * Nothing from the forward pass is stored; only U and O are read again.
 *   G (dOout) : K x mp x mp and O : K x m x m, both FP64 if in_is_fp64 else FP32
 *               (FP64 precision needs FP64).
 *   dO        : K x m x m, FP64 for DMRG_PREC_FP64 else FP32.  May be NULL.
 *   dU        : (m*d) x mp FP64, overwritten.  May be NULL.
 * ------------------------------------------------------------------------ */
DMRG_API dmrg_status dmrg_rotate_ops_backward_workspace(dmrg_handle handle, int64_t K, int64_t m, int d,
                                               int64_t mp, dmrg_precision precision, size_t* bytes);
DMRG_API dmrg_status dmrg_rotate_ops_backward(dmrg_handle handle, const double* U, int64_t m, int d,
                                     int64_t mp, const void* O, const void* dOout, int in_is_fp64,
                                     int64_t K, void* dO, double* dU, dmrg_precision precision,
                                     void* ws, size_t ws_bytes, dmrg_stream_t stream);

/* ------------------------------------------------------------------------
 * FP64 checks and measurements (kept in FP64 whatever the rotation used).
 * ------------------------------------------------------------------------ */
/* out_fro (device, 1 double) = ||U^T U - I_mp||_F for U (rows x mp).  The
 * kept |w_alpha> must be orthonormal for the rotation to be a projection
 * (Sec. 2: the block basis is only approximately complete). */
DMRG_API dmrg_status dmrg_orthonormality_error(dmrg_handle handle, const double* U, int64_t rows,
                                      int64_t mp, double* out_fro, void* ws, size_t ws_bytes,
                                      dmrg_stream_t stream);
DMRG_API dmrg_status dmrg_orthonormality_error_workspace(dmrg_handle handle, int64_t rows, int64_t mp,
                                                size_t* bytes);

/* Two-point functions of Sec. 3.2, C[i][j] = <psi| O'_i O'_j |psi>, computed in
 * FP64 as (O'_i^T psi) . (O'_j psi) (real data).  Op: K x mp x mp (FP64 if
 * in_is_fp64 else FP32); psi: mp FP64; C: K x K FP64 (device). */
DMRG_API dmrg_status dmrg_correlations_workspace(dmrg_handle handle, int64_t K, int64_t mp, size_t* bytes);
DMRG_API dmrg_status dmrg_correlations(dmrg_handle handle, const void* Op, int in_is_fp64,
                              const double* psi, int64_t K, int64_t mp, double* C, void* ws,
                              size_t ws_bytes, dmrg_stream_t stream);

/* ------------------------------------------------------------------------
 * Block-sparse U(1) x U(1) rotation (operators labelled by quantum numbers,
 * Sec. 3.1 Eq. (hache); the paper did not distribute these sub-blocks
 * "because of their dissimilar dimensions" -- here they all go into one
 * grouped launch per product).
 *
 * Canonical storage (all row-major, FP64 U, operators FP64/FP32):
 *   block sectors q (given order): label (n_up, n_dn), size m_q;
 *   site states s = 0..d-1 with label shifts delta_s;
 *   kept sectors Q (given order): label, size m'_Q (0 < m'_Q <= D_Q).
 *   [B a] sector of kept Q: for s = 0..d-1 in order, the states of block
 *     sector (Q - delta_s) if present; D_Q = number of such states.
 *   U blocks : kept sector after kept sector, U_Q of D_Q x m'_Q.
 *   O blocks : operator after operator; operator k (label shift delta_k)
 *     stores, for every block sector q in order with q + delta_k present,
 *     the m_{q+delta_k} x m_q block O_k[q + delta_k, q].
 *   Output   : operator after operator; operator k stores, for every kept
 *     sector Q in order with Q + delta_k kept, the m'_{Q+delta_k} x m'_Q block
 *     O'_k[Q + delta_k, Q] = sum_s U_{Q+delta_k}[seg s]^T
 *                            O_k[Q + delta_k - delta_s, Q - delta_s] U_Q[seg s].
 * Labels must be distinct within each list.  The plan precomputes the
 * grouped problem lists (device tables; allocated at plan creation, not on
 * the hot path) and is tied to the handle's device.
 * ------------------------------------------------------------------------ */
typedef struct {
    int32_t n_up;
    int32_t n_dn;
    int64_t dim;
} dmrg_qn_sector;

typedef struct {
    int32_t d_up;
    int32_t d_dn;
} dmrg_qn_shift;

typedef struct dmrg_blocked_plan_s* dmrg_blocked_plan;

DMRG_API dmrg_status dmrg_blocked_plan_create(dmrg_handle handle, const dmrg_qn_sector* block_sectors,
                                     int32_t n_block_sectors, const dmrg_qn_shift* site_shifts,
                                     int32_t d, const dmrg_qn_sector* kept_sectors, int32_t n_kept,
                                     const dmrg_qn_shift* op_shifts, int64_t K,
                                     dmrg_blocked_plan* plan);
DMRG_API dmrg_status dmrg_blocked_plan_destroy(dmrg_blocked_plan plan);
/* Element counts of the three storages and the workspace bytes for `precision`
 * (DMRG_PREC_FP64, DMRG_PREC_FP32 or DMRG_PREC_BF16X3). */
DMRG_API dmrg_status dmrg_blocked_plan_sizes(dmrg_blocked_plan plan, dmrg_precision precision,
                                    int64_t* u_elems, int64_t* in_elems, int64_t* out_elems,
                                    size_t* ws_bytes);
/* Realised problem statistics: number of grouped GEMM problems of each
 * product, and the logical flops of one call. */
DMRG_API dmrg_status dmrg_blocked_plan_stats(dmrg_blocked_plan plan, int64_t* n_problems_first,
                                    int64_t* n_problems_second, double* flops);
/* Oout_blocks: FP64 for DMRG_PREC_FP64, else FP32. */
DMRG_API dmrg_status dmrg_rotate_ops_blocked(dmrg_handle handle, dmrg_blocked_plan plan,
                                    const double* U_blocks, const void* O_blocks, int in_is_fp64,
                                    void* Oout_blocks, dmrg_precision precision, void* ws,
                                    size_t ws_bytes, dmrg_stream_t stream);

/* ------------------------------------------------------------------------
 * Measurement stage (Sec. 3.2: one- and two-point functions <psi0|Z_i|psi0>,
 * <psi0|Z_i Z_j|psi0>; Sec. 2: the structure factors N(q), S^z(q)).
 *
 * The superblock ground state psi0 = sum_{a,e} Psi[a][e] |a>|e> is a rows x cols
 * FP64 matrix on the device: system basis a (rows), environment basis e (cols).
 * All results are FP64.
 * ------------------------------------------------------------------------ */

/* <Z_k> = <psi0| Z_k (x) I |psi0> (side 0: Z_k rows x rows, system) or
 * <psi0| I (x) Z_k |psi0> (side 1: cols x cols, environment), for K operators Z
 * (device, K x n x n, FP64 or FP32, row-major) -- single-site operators and the
 * stored products Z_i Z_j of one block alike.  Computed as Tr(rho Z_k) with the
 * reduced density matrix rho = Psi Psi^T (side 0) or Psi^T Psi (side 1), formed in
 * the workspace.  out: device, K doubles.  Errors: DMRG_ERR_INVALID_ARG for NULL
 * pointers or side not in {0, 1}; DMRG_ERR_SHAPE for K < 0 or empty Psi. */
DMRG_API dmrg_status dmrg_expectation_workspace(dmrg_handle handle, int64_t K, int64_t rows,
                                       int64_t cols, int side, size_t* bytes);
DMRG_API dmrg_status dmrg_expectation(dmrg_handle handle, const void* Z, int in_is_fp64, int64_t K,
                             const double* Psi, int64_t rows, int64_t cols, int side,
                             double* out, void* ws, size_t ws_bytes, dmrg_stream_t stream);

/* Two-point functions across the two blocks:
 *   C[i][j] = <psi0| Z_i (x) W_j |psi0> = <Psi^T Z_i Psi, W_j>_F,
 * Z: device, Ks x rows x rows (system operators), W: device, Ke x cols x cols
 * (environment operators), each FP64 or FP32; C: device, Ks x Ke FP64 row-major.
 * Operators that are odd under fermion parity need the string of the block in
 * front of them folded into W by the caller (number and spin operators need none). */
DMRG_API dmrg_status dmrg_cross_correlations_workspace(dmrg_handle handle, int64_t Ks, int64_t Ke,
                                              int64_t rows, int64_t cols, int z_is_fp64,
                                              int w_is_fp64, size_t* bytes);
DMRG_API dmrg_status dmrg_cross_correlations(dmrg_handle handle, const void* Z, int z_is_fp64,
                                    int64_t Ks, const void* W, int w_is_fp64, int64_t Ke,
                                    const double* Psi, int64_t rows, int64_t cols, double* C,
                                    void* ws, size_t ws_bytes, dmrg_stream_t stream);

/* Structure factor (Sec. 2):
 *   F(q_p) = (1/L) sum_{k,j} e^{i q_p (k - j)} (G[k][j] - c v[k] - c v[j] + c^2),
 *   q_p = 2 pi p / L, p = 0 .. L-1,
 * from G[k][j] = <X_k X_j> (device, L x L FP64) and v[k] = <X_k> (device, L FP64, or
 * NULL for v = 0): N(q) with X = n and c = n, the mean charge; S^z(q) with X = S^z
 * and c = 0.  Fre, Fim: device, L doubles each (real and imaginary parts; the
 * imaginary part vanishes for symmetric G). */
DMRG_API dmrg_status dmrg_structure_factor(dmrg_handle handle, const double* G, const double* v,
                                  double c, int64_t L, double* Fre, double* Fim,
                                  dmrg_stream_t stream);

/* ------------------------------------------------------------------------
 * Truncation matrix (Sec. 2, steps 3-4; Eq. rho and Eq. error).
 *
 * From the superblock ground state Psi (device, rows x cols FP64: system states i,
 * environment states j), forms the system's reduced density matrix
 * rho[i][i'] = sum_j Psi[i][j] Psi[i'][j], diagonalises it by cyclic Jacobi
 * rotations in FP64, and returns
 *   U       device, rows x mp FP64 row-major: the mp eigenvectors with the largest
 *           eigenvalues as columns, in decreasing eigenvalue order, each with its
 *           largest-magnitude component positive (U = R^+ of the rotation);
 *   lambda  device, rows FP64: all eigenvalues in decreasing order;
 *   eps     device, 1 FP64: the discarded weight sum_{a >= mp} lambda[a]
 *           (= 1 - sum of the kept eigenvalues for a normalized state);
 *   sweeps  host (may be NULL): 0 for the tridiagonal solver (the default, see
 *           DMRG_OPT_TRUNCATION_JACOBI); for the Jacobi sweeps, the sweeps done;
 *           -max_sweeps if the off-diagonal part
 *           did not fall below tol * ||rho||_F (the outputs then hold the last
 *           iterate).  A pair is rotated only if |rho_ab| exceeds both
 *           DBL_EPSILON * sqrt(|rho_aa rho_bb|) and (from the second sweep on)
 *           DBL_EPSILON * ||rho||_F / sqrt(rows); a sweep that rotates no pair also
 *           ends the iteration.
 * Each sweep is one cooperative launch whose rounds meet at a grid-wide barrier with
 * a bounded wait.  The call waits for the stream once per sweep (the convergence
 * test), so it is not graph-capturable.  Errors: DMRG_ERR_SHAPE unless
 * 1 <= mp <= rows; DMRG_ERR_INVALID_ARG for NULL outputs, tol <= 0 or
 * max_sweeps < 1; DMRG_ERR_TIMEOUT if a barrier wait expired (the outputs are then
 * undefined); DMRG_ERR_CUDA if the device cannot run cooperative launches. */
DMRG_API dmrg_status dmrg_truncation_workspace(dmrg_handle handle, int64_t rows, int64_t cols,
                                      size_t* bytes);
DMRG_API dmrg_status dmrg_truncation(dmrg_handle handle, const double* Psi, int64_t rows,
                            int64_t cols, int64_t mp, double* U, double* lambda, double* eps,
                            double tol, int max_sweeps, int* sweeps, void* ws, size_t ws_bytes,
                            dmrg_stream_t stream);

/* ------------------------------------------------------------------------
 * Blocked site and cross operators (Sec. 2, the blocking of operators into the
 * [B a] basis that follows step 5; task ii of the rotation step in Sec. 3.2).
 *
 * Operators acting on the added site, and products of a block operator with a
 * site operator, are written in [B a] as Z_k = (A_k P^f) (x) S, where S is a
 * d x d site matrix and P = diag(parity) the block's fermion parity (-1)^{N_B}:
 * with the Jordan-Wigner order block modes before the site's, a fermion operator
 * of the added site carries that string on the block.  This call rotates them:
 *
 *     O'_k = U^T ((A_k P^{f_c}) (x) S_c) U
 *
 * The K operators come in n_class consecutive classes: class c has counts[c]
 * operators, site matrix S + c*d*d and parity flag flags[c] (0 or 1).
 *
 *   U       device, (m*d) x mp FP64, row-major, orthonormal columns.
 *   A       device, K x m x m, FP64 (in_is_fp64 = 1) or FP32, row-major.
 *   S       HOST, n_class x d x d FP64 (copied into kernel arguments; d <= 8).
 *   counts  HOST, n_class entries >= 0 summing to K.
 *   flags   HOST, n_class entries in {0, 1}.
 *   parity  device, m entries of +1 / -1 (signed char); may be NULL when every
 *           flag is 0.
 *   Oout    device, K x mp x mp: FP64 for DMRG_PREC_FP64, else FP32.
 * Errors: DMRG_ERR_INVALID_ARG for NULL pointers, counts not summing to K, a flag
 * outside {0, 1} or a set flag without parity; DMRG_ERR_SHAPE as for
 * dmrg_rotate_ops or d > 8; DMRG_ERR_WORKSPACE when ws_bytes is too small.  With
 * every S = I and every flag 0 the result equals dmrg_rotate_ops.  Not captured
 * into CUDA graphs (S, counts and flags are host data of the call).
 * ------------------------------------------------------------------------ */
DMRG_API dmrg_status dmrg_rotate_site_ops_workspace(dmrg_handle handle, int64_t K, int64_t m, int d,
                                           int64_t mp, dmrg_precision precision, size_t* bytes);
DMRG_API dmrg_status dmrg_rotate_site_ops(dmrg_handle handle, const double* U, int64_t m, int d,
                                 int64_t mp, const void* A, int in_is_fp64, int64_t K,
                                 int n_class, const double* S, const int64_t* counts,
                                 const int32_t* flags, const signed char* parity, void* Oout,
                                 dmrg_precision precision, void* ws, size_t ws_bytes,
                                 dmrg_stream_t stream);

/* ------------------------------------------------------------------------
 * Diagnostic: the reciprocal used by the Sturm counts of dmrg_truncation's
 * eigenvalue multisection (Sec. 2, the diagonalisation of rho in Eq. rho).
 *
 * out[i] = 1 / q[i] computed as the truncation kernels compute it: the
 * hardware's approximate reciprocal refined by two Newton-Raphson steps.
 *   q, out  device, n FP64 values each (caller-owned).
 * For normal |q| <= 1/DBL_MIN the result is within a few ulps of correctly
 * rounded division; larger |q| flush to zero.  Asynchronous on stream.
 * Errors: DMRG_ERR_INVALID_ARG for n < 0 or NULL pointers with n > 0,
 * DMRG_ERR_CUDA if the launch fails.
 * ------------------------------------------------------------------------ */
DMRG_API dmrg_status dmrg_debug_reciprocal(const double* q, double* out, int64_t n,
                                           dmrg_stream_t stream);

/* ------------------------------------------------------------------------
 * Dense rotation without any allocation (the paper has no counterpart; this
 * entry point exists for callers of the library, not for the method).
 *
 * For callers that cannot call cudaMalloc -- a plug-in inside a host program
 * whose device memory is fully reserved by that program's own pool, code
 * under a fixed per-client memory limit, or a latency-critical loop where an
 * allocation would synchronise the device.  Same arguments and result as
 * dmrg_rotate_ops(), but no handle and no workspace: the scratch lives in a
 * static device array of 32 MiB that every GPU loading the library holds
 * until the process exits.  Problems whose dmrg_rotate_ops_workspace() size
 * exceeds 32 MiB are rejected with DMRG_ERR_WORKSPACE before any launch.
 * The first call on each device (with that device current) looks up the
 * array's device address; make that first call before any stream capture.
 * All calls share the array, so calls that overlap on the GPU race on it:
 * serialise them (one stream, one host thread at a time).  A device-side
 * bounded-wait timeout cannot be reported by this entry point (there is no
 * handle to read it from); the kernels still return.
 * ------------------------------------------------------------------------ */
DMRG_API dmrg_status dmrg_rotate_ops_noalloc(const double* U, int64_t m, int d, int64_t mp,
                                             const void* O, int in_is_fp64, int64_t K, void* Oout,
                                             dmrg_precision precision, dmrg_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* DMRG_ROTATE_H */
