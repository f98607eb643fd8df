// api_common.h -- helpers shared by the host translation units of the C ABI.
#pragma once
#include <functional>
#include <string>
#include <vector>

#include "internal.h"

namespace dmrg {

// Sections of a caller workspace, each 256-byte aligned.
struct WsLayout {
    std::vector<size_t> offsets;
    size_t total = 0;
    void add(const char* name, size_t bytes);
};

struct DenseDims {
    int64_t K, m, mp, md, ld1, ld2;
    int d;
    WsLayout ws;
};

dmrg_status fail(dmrg_handle h, dmrg_status st, const std::string& msg);
dmrg_status cuda_fail(dmrg_handle h, cudaError_t e, const char* where);
cudaError_t timed_launch(dmrg_handle h, const char* name, cudaStream_t s,
                         const std::function<cudaError_t()>& f);
size_t align_up(size_t x, size_t a);
bool tc_supported(dmrg_handle h);
uint64_t timeout_ns(dmrg_handle h);
int take_drop_arrival(dmrg_handle h);
dmrg_status run_maybe_graph(dmrg_handle h, const std::string& key, cudaStream_t stream,
                            const std::function<dmrg_status(cudaStream_t)>& body);
DenseDims dense_dims(int64_t K, int64_t m, int d, int64_t mp, dmrg_precision p);
dmrg_status check_dense_args(dmrg_handle h, int64_t K, int64_t m, int d, int64_t mp,
                             dmrg_precision p);
dmrg_status check_ws(dmrg_handle h, const void* ws, size_t have, size_t need);
TcConfig tuned_config(dmrg_handle h, const std::string& key, TcMode mode);
void load_tune_file(dmrg_handle h);
void save_tune_file(dmrg_handle h);
std::string shape_key(const char* tag, int64_t K, int64_t m, int d, int64_t mp, dmrg_precision p);
// Operator classes of the first product (blocked site operators): class c holds the
// operators k0[c] .. k0[c] + kc[c] - 1 of the call (consecutive, covering all K) and
// uses its own U1_c = U1 + c * (m d mp) in place of U.  The packed U1_c go to b1
// (hi, lo; class c at c * d * mp * ld1 elements), a caller scratch for n classes.
struct FirstClasses {
    int n = 0;   // 1 .. kMaxInlineProblems
    int64_t k0[kMaxInlineProblems] = {};
    int64_t kc[kMaxInlineProblems] = {};
    const double* U1 = nullptr;
    void* b1[2] = {nullptr, nullptr};
    bool b1_ready = false;   // b1 already holds the packed U1_c (U1 is then not read)
};

// The dense rotation O'_k = U^T (O_k (x) I_d) U.  With U1 != nullptr the first
// product uses U1 in place of U, i.e. O'_k = U^T (O_k (x) I_d) U1 (the blocked site
// operators pass U1 = (P (x) S) U); the FP32 plain-FMA path then needs U1_32, an
// (m*d) x mp FP32 scratch for U1's conversion.  With cls != nullptr (tensor-core
// paths) the first product runs one problem per class in one launch.
dmrg_status dense_tc_forward(dmrg_handle h, const double* U, int64_t m, int d, int64_t mp,
                             const void* O, int in_is_fp64, int64_t K, void* Oout,
                             dmrg_precision p, void* ws, const TcConfig& c1, const TcConfig& c2,
                             cudaStream_t s, bool pack_u = true, const double* U1 = nullptr,
                             const FirstClasses* cls = nullptr);

dmrg_status dense_fused_forward(dmrg_handle h, const double* U, int64_t m, int d, int64_t mp,
                                const void* O, int in_is_fp64, int64_t K, void* Oout, void* ws,
                                cudaStream_t s);
dmrg_status dense_simt_forward(dmrg_handle h, const double* U, int64_t m, int d, int64_t mp,
                               const void* O, int in_is_fp64, int64_t K, void* Oout,
                               dmrg_precision p, void* ws, cudaStream_t s, bool pack_u = true,
                               const double* U1 = nullptr, float* U1_32 = nullptr);

// The truncation's eigen-decomposition by tridiagonalisation (tridiag.cu): workspace
// layout for n rows and mp kept vectors (rho goes into its first section), and the
// solver: U (n x mp), lambda (n, decreasing).
WsLayout tridiag_layout(int64_t n, int64_t mp);
dmrg_status tridiag_eigen(dmrg_handle h, int64_t n, int64_t mp, char* ws, double* U, double* lambda,
                          double* eps, cudaStream_t s);

// two_per_sm: the variant with 128-column accumulators and 64-byte rows, two CTAs per
// SM (grid may then be twice the SM count; needs row_bytes 64 and bn_smem <= 128).
cudaError_t tc_gemm_launch_grouped(TcMode mode, TcEpi epi, const TcLaunch& L, int stages, int grid,
                                   int bn_smem, cudaStream_t s, bool two_per_sm = false);

}  // namespace dmrg
