// internal.h -- host-side structures shared by the translation units of the library.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "dmrg_rotate.h"

namespace dmrg {

// ---------------------------------------------------------------- SIMT GEMM
// C[b](i, j) (+)= sum_k A[b](i, k) * B[b](k, j) with arbitrary element strides.
// Used by the FP64 and FP32 paths (plain FMA, no tensor cores).
struct SimtGemm {
    const void* A;
    const void* B;
    void* C;
    int64_t M, N, K;
    int64_t sAb, sAi, sAk;
    int64_t sBb, sBk, sBj;
    int64_t sCb, sCi, sCj;
    int32_t accumulate;   // 1: C += A B, 0: C = A B
    int32_t tile_start;   // first tile (grouped launches)
    int32_t tiles_m, tiles_n;
    int32_t batch;
    int32_t reduce_batch; // 1: C = sum_b A[b] B[b] (one output, batch folded into the reduction)
    // Grouped launches: A, B and C hold element offsets from bases[a_sel / b_sel / c_sel]
    // of the launch (sel < 0: absolute pointers); a_boff / c_boff, when set, give the
    // element offset of each batch entry instead of b * sAb / b * sCb.
    int32_t a_sel, b_sel, c_sel;
    int32_t small;        // grouped launches: M, N <= 32, one warp per batch entry, 8 per block
    int32_t lower;        // symmetric C: only tiles on and below the diagonal (the caller mirrors)
    const int64_t* a_boff;
    const int64_t* c_boff;
};

enum class Real { F64, F32 };

// Launches one batched GEMM (or a grouped list already in device memory).
cudaError_t simt_gemm_launch(Real t, const SimtGemm& g, cudaStream_t s);
cudaError_t simt_gemm_grouped_launch(Real t, const SimtGemm* d_problems, int nprob,
                                     int total_tiles, const void* const bases[4], cudaStream_t s);
// Grouped problems with M, N <= kSimtSmall and no batch reduction take the small path
// (set SimtGemm::small and count ceil(batch / kSimtSmallPerBlock) tiles).
constexpr int kSimtSmall = 32;
constexpr int kSimtSmallPerBlock = 8;
int simt_tile_m();
int simt_tile_n();

// Fused ||U^T U - I||_F: G = U^T U tile-wise, squares of (G - I) reduced into
// *acc (device double, zeroed inside), then sqrt into *out.
cudaError_t ortho_error_launch(const double* U, int64_t rows, int64_t mp, double* acc, double* out,
                               cudaStream_t s);
// x_k = O'_k^T psi and y_k = O'_k psi (FP64 results) for every k.
cudaError_t corr_matvec_launch(const void* Op, bool f64, const double* psi, int64_t K, int64_t mp,
                               double* x, double* y, cudaStream_t s);
// dO-style partial trace helper etc. live in the api translation unit.
cudaError_t convert_f32_to_f64_launch(const float* src, double* dst, int64_t n, cudaStream_t s);
// Reduced density matrix of the superblock state Psi (rows x cols, FP64):
// rho = Psi Psi^T (side 0, rows x rows) or Psi^T Psi (side 1, cols x cols).
cudaError_t rho_launch(const double* Psi, int64_t rows, int64_t cols, int side, double* rho,
                       cudaStream_t s);
cudaError_t fill_zero_launch(void* p, size_t bytes, cudaStream_t s);

// ---------------------------------------------------------------- tensor-core GEMM
// One grouped GEMM problem for the tcgen05 kernel:
//   D (M x N) = sum_{z < nbatch} A_z (M x Kred) B_z (N x Kred)^T,
// both operands K-major and stored as BF16 hi/lo pairs (BF16X3) or FP32 (TF32),
// seen through 3-D tensor maps (reduction, rows, z).  The epilogue writes D through
// the scatter map sc[0], which sends element (row R, col n) to
//   out + out_off + (op_off ? op_off[R / rows_per_op] : (R / rows_per_op) * s_op)
//       + (R % rows_per_op) * s_row + (n / col_div) * s_col_hi + (n % col_div) * s_col_lo.
struct TcScatter {
    int64_t out_off, s_op, s_row, s_col_hi, s_col_lo;
    const int64_t* op_off;
    int32_t rows_per_op, col_div;
    int64_t s_split;   // CTA-pair kernel: output offset per reduction split (0: the splits
                       // of a tile add into one output, atomically when the problem says so)
};

struct TcProblem {  // 64-byte aligned through its CUtensorMap members
    CUtensorMap tmA[2];  // hi, lo (lo unused for TF32)
    CUtensorMap tmB[2];
    int32_t M, N, Kred;  // Kred: reduction length of one z slice
    int32_t nbatch;      // reduction also runs over z = 0 .. nbatch-1
    int32_t tile_n;      // N tile width (multiple of 16, <= 256)
    int32_t m_tiles, n_tiles, k_splits, kb_per_split;
    int32_t tile_start;  // first global tile of this problem
    int32_t m_tile0;     // first M tile (the problem covers M tiles m_tile0 .. m_tile0 + m_tiles - 1)
    int32_t atomic;      // FP32 epilogues: accumulate with atomics (split-K parts of a tile)
    int32_t kb_chunk;    // CTA-pair kernel: k-blocks per tensor-core accumulation chain; the
                         // chains of a tile are summed in FP32 registers (0: one chain)
    int32_t a_mn, b_mn;  // CTA-pair kernel, BF16 operands: A / B stored MN-major (its M / N
                         // index contiguous in memory), read in 64-column boxes
    int32_t store_z0;    // with TcLaunch::t_store: operator index of this problem's first
                         // operator in the store maps
    TcScatter sc[1];
};

enum TcMode : int { TC_BF16X3 = 0, TC_TF32 = 1, TC_BF16 = 2 };
enum TcEpi : int { EPI_SPLIT_BF16 = 0, EPI_TF32 = 1, EPI_F32 = 2, EPI_F32_ATOMIC = 3 };

struct TcConfig {
    int tile_n_max = 256;   // upper bound on the N tile (the split picks <= this)
    int stages = 3;
    int grid = 0;           // 0 = number of SMs
    int row_bytes = 128;    // 128: 128-byte swizzle; 64: 64-byte swizzle, half-depth k-blocks
    int pair = 0;           // 1: CTA-pair kernel (256-row tiles on two SMs, cta_group::2)
    bool operator==(const TcConfig& o) const {
        return tile_n_max == o.tile_n_max && stages == o.stages && grid == o.grid &&
               row_bytes == o.row_bytes && pair == o.pair;
    }
};

constexpr int kMaxInlineProblems = 6;
// MN-major operands are loaded in boxes of this many rows (64 BF16: one 128-byte row per
// reduction index).
constexpr int kMnBox = 64;   // keeps TcLaunch (the kernel parameters) under 4 KB
// Running-sum scratch of the CTA-pair kernel's chained accumulation: kChainScratchCtas
// CTAs x 128 rows x 256 FP32 columns.
constexpr int kChainScratchCtas = 160;
constexpr size_t kChainScratchBytes = size_t(kChainScratchCtas) * 128 * 256 * 4;
// Reductions up to this length always run as one chain (no scratch is reserved for them).
constexpr int64_t kChainMinRed = 512;
// Longest accumulation chain the BF16x3 products accept (DMRG_OPT_ACCUM_CHAIN).
constexpr int kMaxAccumChain = 1024;

struct TcLaunch {
    TcProblem inline_prob[kMaxInlineProblems];  // used when table == nullptr
    const TcProblem* table;       // grouped problems in device memory
    const int32_t* tile_problem;  // with a table: problem index of every tile (nullptr: search)
    int32_t nprob;
    int32_t total_tiles;
    void* out[1][2];              // [scatter][hi, lo]: FP32/TF32 output in [0][0]
    unsigned* status;
    uint64_t timeout_ns;
    int32_t drop_arrival;   // test hook: CTA 0 withholds its first stage release
    int32_t row_bytes;      // 128 or 64: must match the problems' tensor maps
    float* chunk_scratch;   // CTA-pair kernel with kb_chunk: gridDim.x x 128 x 256 FP32 running
                            // sums (nullptr: every tile is one accumulation chain)
    int32_t convert_a;      // CTA-pair kernel: every problem's A map is an FP32 source that
                            // the converter warps turn into the MMA operand (f32_source)
    int32_t reverse_m;      // 1: each problem's M tiles run from the last to the first (the
                            // rows a preceding kernel wrote last are the likeliest in L2)
    // CTA-pair kernel, EPI_SPLIT_BF16 / EPI_TF32: a second, site-major copy of the result
    // (null: none).  Element (row R, column c) also goes to
    //   out2 + (R / o2_rows_per_op) * o2_s_op + (R % o2_rows_per_op) * o2_s_row
    //        + (c / o2_m) * o2_s_site + c % o2_m
    // i.e. for rows (k, a) and columns c = s * m + j: copy_k[s * m' + a][j], j contiguous.
    void* out2[2];
    int64_t o2_s_op, o2_s_row, o2_s_site;
    int32_t o2_rows_per_op, o2_m;
    // CTA-pair kernel, EPI_SPLIT_BF16 (EPI_TF32: site-interleaved layout only; EPI_F32:
    // columns layout only): the result leaves by TMA bulk stores instead of stores from
    // registers (t_store = 0: off).  Each epilogue warp stages one 32-column
    // chunk (hi and lo) of its 32 rows in shared memory; launches whose shared memory
    // cannot hold the staging store from registers.  Rows R = k_local * rows_per_op + i
    // (rows_per_op a multiple of 16); t_store_map[hi, lo] are 3-D maps whose third
    // coordinate is the operator k = store_z0 + k_local.  The scatter must be one of:
    //   kStoreSiteInterleaved (t_store_d = d, 2 or 4): column n = b * d + s goes to
    //     T[k][b][i * d + s], as in the first product; map (i * d + s, b, k), box
    //     16 d x 32 / d x 1 (EPI_SPLIT_BF16: BF16 hi and lo maps; EPI_TF32: one FP32 map);
    //   kStoreRowContiguous: column n = s * col_div + j goes to
    //     W[k][j][s * s_col_hi + i] (s_row = 1, col_div a multiple of 16); maps
    //     (s * s_col_hi + i, j, k), boxes 32 x 16 x 1 ([0], [1]: a warp's 32 rows in one
    //     operator) and 16 x 16 x 1 ([2], [3]);
    //   kStoreSiteMajor: the site-major copy alone (out[0] null, out2 set; o2_m and
    //     o2_rows_per_op multiples of 16): column n = s * o2_m + j goes to
    //     out2_k[s * o2_rows_per_op + i][j]; maps (j, s * o2_rows_per_op + i, k), boxes
    //     32 x 16 x 1 with the 64-byte swizzle ([0], [1]: a chunk's 32 columns in one
    //     site) and 16 x 16 x 1 with the 32-byte swizzle ([2], [3]);
    //   kStoreColumnsF32 (EPI_F32 / EPI_F32_ATOMIC, chains summed in the output): column
    //     n of row (k, i) goes to out_k[n][i] (s_row = 1, col_div = 1, s_op = N s_col_hi);
    //     map (i, n, k), FP32 box 16 x 16 x 1; a tile's later chains and the parts of a
    //     split tile add with TMA reductions.
    // t_store_map[hi, lo, hi narrow, lo narrow] (one FP32 map: [0]).
    CUtensorMap t_store_map[4];
    int32_t t_store;
    int32_t t_store_d;
};
constexpr int32_t kStoreSiteInterleaved = 1;
constexpr int32_t kStoreRowContiguous = 2;
constexpr int32_t kStoreSiteMajor = 3;
constexpr int32_t kStoreColumnsF32 = 4;
// Shared memory of the CTA-pair kernel's store staging: per epilogue warp, the hi and lo
// halves of a 32-row x 32-column BF16 chunk (or the FP32 chunk).
constexpr size_t kStoreStagingBytes = size_t(8) * 2 * 32 * 32 * 2;

// One operand seen by the kernel: `nbatch` slices of rows x cols (cols = the
// reduction, contiguous), row stride ld elements, slice stride in elements.
struct TcOperand {
    const void* hi;
    const void* lo;
    int64_t rows, cols, ld;
    int64_t nbatch = 1;
    int64_t batch_stride = 0;
    // A operand of the CTA-pair kernel only: `hi` is an unconverted FP32 matrix (row
    // stride ld floats, a multiple of 4, 16-byte aligned) that the kernel's converter
    // warps split into BF16 hi/lo (BF16X3) or round to TF32 in shared memory.
    int32_t f32_source = 0;
    // CTA-pair kernel, BF16 operands (BF16X3, 128-byte rows): the operand is stored
    // MN-major, element (row r, reduction index c) of slice z at z * batch_stride +
    // c * ld + r (its rows contiguous), ld a multiple of 8.
    int32_t mn_major = 0;
};

cudaError_t tc_gemm_launch(TcMode mode, TcEpi epi, const TcLaunch& L, int stages, int grid,
                           cudaStream_t s);
int tc_max_stages(TcMode mode, int tile_n_max, int row_bytes = 128);
// One-CTA kernel with two CTAs per SM (N tiles <= 128, 64-byte rows): the deepest
// pipeline that fits, or 0 if none does.
int tc_stages_two_per_sm(TcMode mode, int tile_n_max);
// CTA-pair form: problems made with make_problem(..., pair_form = 1); `grid` counts
// CTAs (rounded down to whole pairs, capped by the pairs that fit at once).
cudaError_t tc_gemm_launch_pair(TcMode mode, TcEpi epi, const TcLaunch& L, int stages, int grid,
                                cudaStream_t s);
int tc_pair_max_stages(TcMode mode, int tile_n_max, int row_bytes = 128);
// Dispatch on cfg.pair.
inline int tc_stages_for(TcMode mode, const TcConfig& c) {
    return c.pair ? tc_pair_max_stages(mode, c.tile_n_max, c.row_bytes)
                  : tc_max_stages(mode, c.tile_n_max, c.row_bytes);
}

// Encodes a K-major operand map (3-D: cols, rows, batch), box = box_rows x 128 bytes.
bool encode_operand_map(CUtensorMap* map, const void* base, bool fp32, int64_t rows, int64_t cols,
                        int64_t ld, int box_rows, int64_t nbatch = 1, int64_t batch_stride = 0,
                        int row_bytes = 128);
// Encodes a store map (BF16, or FP32 with fp32) for the CTA-pair kernel's TMA-store
// epilogue: nz slices of ny rows x nx elements (row stride ld elements, slice stride
// ny * ld), box bx x by x 1; swizzle: 0, or the shared-memory swizzle span in bytes (the
// box row: 32 or 64).
bool encode_store_map(CUtensorMap* map, void* base, int64_t nx, int64_t ny, int64_t nz, int64_t ld,
                      int bx, int by, int swizzle = 0, bool fp32 = false);
// Chooses an N tile (multiple of 16, <= tile_n_max) that splits N evenly.
int choose_tile_n(int64_t N, int tile_n_max);
// Fills operand maps and tiling fields of a problem: D (M x N) += A B^T over Kred x nbatch.
// pair_form: 0 for the one-CTA kernel, 1 for the CTA-pair kernel (other values fail).
bool make_problem(TcProblem& p, TcMode mode, const TcOperand& A, const TcOperand& B,
                  int tile_n_max, int k_splits, int row_bytes = 128, int pair_form = 0);
// Scatter for a plain row-major (rows x cols, leading dimension ld) destination.
TcScatter scatter_rowmajor(int64_t ld);

// ---------------------------------------------------------------- packer
// Gathers and converts a strided source matrix into K-major tensor-core
// operands: dst row r, column c  <-  src[base + op_part(r) + (r % rdiv') ...].
// For row r: g = r / rows_per_op (operand group), rr = r % rows_per_op;
//   src index = src_off + (op_off ? op_off[g] : g * s_op) + (rr / rdiv) * s_r_hi
//               + (rr % rdiv) * s_r_lo + c * s_c.
constexpr int32_t kPackZero = 3;   // PackJob::mode: clear rows x cols FP32 values at dst0

struct PackJob {
    const void* src;
    int32_t src_f64;
    int32_t mode;          // 0: BF16 hi/lo pair, 1: FP32 rounded to TF32, 2: FP32, 3: zero fill
    int64_t rows, cols;
    int64_t src_off;
    int64_t rows_per_op;
    int64_t s_op;
    const int64_t* op_off;
    int64_t rdiv, s_r_hi, s_r_lo, s_c;
    void* dst0;            // hi (BF16) or TF32 (FP32)
    void* dst1;            // lo (BF16)
    int64_t ld;            // dst row stride in elements
    int64_t block_start;   // first CUDA block of this job (grouped launch)
    // Grouped launches from a device table: src holds an element offset from
    // srcs[src_sel] of the launch and dst0 / dst1 hold byte offsets from its
    // workspace base (rel = 1); rel = 0 means absolute pointers.
    int32_t rel, src_sel;
    int32_t vec8;          // set by the launcher: contiguous rows, 8 elements per thread
    int32_t tiled;         // set by the launcher: transposing gather through 32 x 32 tiles
    // Set by pack_prepare: n / d == (n * m) >> s for 0 <= n < 2^31 (Granlund-Montgomery
    // round-up multipliers) for d = cols, rows_per_op, rdiv, when the job fits 31 bits.
    int32_t fastdiv;
    int32_t s_cols, s_rpo, s_rdiv;
    uint64_t m_cols, m_rpo, m_rdiv;
    // Set by pack_prepare_grouped (grouped launches): the job's rows are contiguous runs
    // of its source (s_c = 1, rdiv = 1) and are copied one warp per row.
    int32_t rowwise;
    int32_t late;          // single-launch packer: placed after every other job (its output
                           // is the likeliest to be in L2 when the launch ends)
    // Single-launch packer, tiled (transposing) jobs with rdiv = 1: st0 / st1 (null: none)
    // also receive the untransposed copy, element (row g * cols + c, column r) for the
    // job's element (row g * rows_per_op + r, column c), row stride st_ld (even).
    void* st0;
    void* st1;
    int64_t st_ld;
    // Set by the single-launch packer (pack_launch): multiply-shift divisors, in 32-bit
    // index arithmetic, of the tiled path's geometry (tiles per operator group, per
    // residue and per row of tiles) and of the 8-wide path's units per row (fast8).
    uint64_t m_pg, m_hc, m_ct, m_u8;
    int32_t s_pg, s_hc, s_ct, s_u8;
    int32_t t_pg, t_hc, t_ct, fast8;
    int64_t t_hrows;
};
void pack_prepare(PackJob& j);
// The single-launch packer takes j through shared-memory tiles (FP32 source, transposing).
bool pack_job_tiled(const PackJob& j);
// pack_prepare, and for grouped launches the row-by-row copy of contiguous rows.
void pack_prepare_grouped(PackJob& j);
cudaError_t pack_launch(const PackJob* jobs_host, int njobs, PackJob* jobs_dev_or_null,
                        cudaStream_t s);
int64_t pack_blocks_for(const PackJob& j);
cudaError_t pack_grouped_launch(const PackJob* jobs_dev, int njobs, int64_t total_blocks,
                                const void* const srcs[2], void* ws_base, int src1_f64,
                                cudaStream_t s);

// ---------------------------------------------------------------- fused rotation (fused.cu)
// Both products in one kernel, the intermediate kept in TMEM and shared memory (BF16x3).
constexpr int kFusedMaxMp = 256;
struct FusedArgs {
    const void* Op[2];   // O hi/lo (BF16): K*m rows of m, row stride ld
    const void* Pu[2];   // U hi/lo (BF16): Pu[s][x][j] = U[j d + s][x], d*mp rows of m, stride ld
    float* out;          // K x mp x mp
    int64_t K, m, mp, ld;
    int d, grid, accum_chain;
    unsigned* status;
    uint64_t timeout_ns;
};
cudaError_t fused_rotate_launch(const FusedArgs& a, cudaStream_t s);

// ---------------------------------------------------------------- backward helpers
cudaError_t f32_to_f64_strided_launch(const float* src, double* dst, int64_t n, cudaStream_t s);

}  // namespace dmrg

// ---------------------------------------------------------------- handle
struct dmrg_handle_s {
    int device = 0;
    int num_sms = 0;
    int cc_major = 0, cc_minor = 0;
    unsigned* d_status = nullptr;   // device status word (+ scratch doubles after it)
    double* d_scratch = nullptr;    // 8 doubles of scratch for reductions
    std::string last_error;
    bool graph_mode = false;
    bool timing = false;
    double wait_timeout_ms = 2000.0;
    double check_ortho_tol = 0.0;
    int drop_arrival_next = 0;      // test hook, consumed by the next tensor-core launch
    bool deterministic = false;     // no atomically accumulated split tiles
    bool trunc_jacobi = false;      // truncation: cyclic Jacobi instead of the tridiagonal solver
    bool blocked_small = true;      // plans with sectors <= 32 states: fused small-sector kernel
    int pack_operators = 0;         // dense tensor-core products, FP32 operators: 0 = convert
                                    // them in the first product's shared memory where that
                                    // was measured faster (BF16x3, at most two N tiles),
                                    // 1 = always pack them in a separate pass, 2 = convert
                                    // whenever their layout allows
    int fused_rotation = 0;         // dense BF16x3, mp <= 256: both products in one kernel
                                    // (0 = off)
    int accum_chain = 1024;         // BF16x3 dense products: reduction elements per accumulator
                                    // chain (0 = one chain per tile)
    int store_epilogue = 0;         // BF16x3 first product: 0 = TMA bulk stores where the
                                    // layout allows, 1 = stores from registers

    struct Timed {
        std::string name;
        cudaEvent_t a, b;
    };
    std::vector<Timed> pending;
    std::vector<cudaEvent_t> event_pool;
    std::map<std::string, std::pair<long, double>> timing_acc;

    std::map<std::string, dmrg::TcConfig> tune_cache;
    bool tune_cache_loaded = false;

    std::map<std::string, cudaGraphExec_t> graphs;
    cudaStream_t capture_stream = nullptr;
    bool capturing = false;

    // host-buffer pipeline: copy-in and copy-out streams and their events
    cudaStream_t copy_in = nullptr, copy_out = nullptr, compute2 = nullptr;
    cudaEvent_t ev_start = nullptr, ev_u = nullptr;
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr},
                ev_out[2] = {nullptr, nullptr};
};

struct dmrg_blocked_plan_s;
