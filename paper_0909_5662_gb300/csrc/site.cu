// site.cu -- rotation of blocked site and cross operators (dmrg_rotate_site_ops).
//
// Operators of the added site and block x site products are written in the [B a]
// basis as Z_k = (A_k P^f) (x) S (Sec. 2, the blocking that follows step 5), with P
// the block's fermion parity carried by odd site operators (block modes ordered
// first).  Since (A P) (x) S = (A (x) I)(P (x) S), the rotation is
//
//     O'_k = U^T (A_k (x) I_d) U_c,     U_c = (P^{f_c} (x) S_c) U,
//
// i.e. the plain block rotation of A_k with U_c in the first product.  Each class
// of operators sharing (S_c, f_c) gets U_c from one small FP64 kernel and then runs
// the dense rotation (pack, first product, second product) on its operators.
#include <cuda_runtime.h>

#include <algorithm>

#include "api_common.h"

using namespace dmrg;

namespace {

constexpr int kMaxSiteDim = 8;

struct SiteMatrix {
    double s[kMaxSiteDim * kMaxSiteDim];
};

// Uc[(j, s)][b] = p_j * sum_t S[s][t] U[(j, t)][b], one thread per (j, b).
__global__ void site_u_kernel(const double* __restrict__ U, double* __restrict__ Uc, int64_t m,
                              int d, int64_t mp, const __grid_constant__ SiteMatrix S,
                              const signed char* __restrict__ parity) {
    const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= m * mp) return;
    const int64_t j = idx / mp, b = idx - j * mp;
    double u[kMaxSiteDim];
#pragma unroll
    for (int t = 0; t < kMaxSiteDim; ++t) u[t] = t < d ? U[(j * d + t) * mp + b] : 0.0;
    const double pj = parity ? double(parity[j]) : 1.0;
#pragma unroll
    for (int s = 0; s < kMaxSiteDim; ++s) {
        if (s >= d) break;
        double v = 0.0;
#pragma unroll
        for (int t = 0; t < kMaxSiteDim; ++t)
            if (t < d) v = fma(S.s[s * d + t], u[t], v);
        Uc[(j * d + s) * mp + b] = pj * v;
    }
}

struct SiteDims {
    WsLayout ws;   // Uc (FP64), Uc in FP32 (plain-FMA FP32 path), dense rotation workspace
};

SiteDims site_dims(int64_t K, int64_t m, int d, int64_t mp, dmrg_precision p) {
    SiteDims D;
    D.ws.add("Uc", size_t(m) * d * mp * 8);
    D.ws.add("Uc32", p == DMRG_PREC_FP32 ? size_t(m) * d * mp * 4 : 0);
    D.ws.add("dense", dense_dims(std::max<int64_t>(K, 1), m, d, mp, p).ws.total);
    return D;
}

}  // namespace

extern "C" {

dmrg_status dmrg_rotate_site_ops_workspace(dmrg_handle h, int64_t K, int64_t m, int d, int64_t mp,
                                           dmrg_precision p, size_t* bytes) {
    if (!bytes) return fail(h, DMRG_ERR_INVALID_ARG, "bytes is NULL");
    dmrg_status st = check_dense_args(h, K, m, d, mp, p);
    if (st != DMRG_OK) return st;
    if (d > kMaxSiteDim) return fail(h, DMRG_ERR_SHAPE, "site dimension d must be <= 8");
    *bytes = site_dims(K, m, d, mp, p).ws.total;
    return DMRG_OK;
}

dmrg_status dmrg_rotate_site_ops(dmrg_handle h, const double* U, int64_t m, int d, int64_t mp,
                                 const void* A, int in_is_fp64, int64_t K, int n_class,
                                 const double* S, const int64_t* counts, const int32_t* flags,
                                 const signed char* parity, void* Oout, dmrg_precision p, void* ws,
                                 size_t ws_bytes, dmrg_stream_t stream) {
    dmrg_status st = check_dense_args(h, K, m, d, mp, p);
    if (st != DMRG_OK) return st;
    if (d > kMaxSiteDim) return fail(h, DMRG_ERR_SHAPE, "site dimension d must be <= 8");
    if (K == 0) return DMRG_OK;
    if (!U || !A || !Oout || !S || !counts || !flags || n_class < 1)
        return fail(h, DMRG_ERR_INVALID_ARG, "null pointer or no operator class");
    if (p == DMRG_PREC_FP64 && !in_is_fp64)
        return fail(h, DMRG_ERR_INVALID_ARG, "the FP64 precision needs FP64 operators");
    int64_t total = 0;
    for (int c = 0; c < n_class; ++c) {
        if (counts[c] < 0 || (flags[c] != 0 && flags[c] != 1))
            return fail(h, DMRG_ERR_INVALID_ARG, "class counts must be >= 0 and flags 0 or 1");
        if (flags[c] && !parity) return fail(h, DMRG_ERR_INVALID_ARG, "a parity flag needs the parity");
        total += counts[c];
    }
    if (total != K) return fail(h, DMRG_ERR_INVALID_ARG, "class counts must sum to K");
    const bool tc = (p == DMRG_PREC_TF32 || p == DMRG_PREC_BF16X3);
    if (tc && !tc_supported(h)) return fail(h, DMRG_ERR_UNSUPPORTED, "tensor cores need sm_103");
    const SiteDims D = site_dims(K, m, d, mp, p);
    st = check_ws(h, ws, ws_bytes, D.ws.total);
    if (st != DMRG_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char* base = static_cast<char*>(ws);
    double* Uc = reinterpret_cast<double*>(base + D.ws.offsets[0]);
    float* Uc32 = p == DMRG_PREC_FP32 ? reinterpret_cast<float*>(base + D.ws.offsets[1]) : nullptr;
    void* wsd = base + D.ws.offsets[2];
    const size_t es_in = in_is_fp64 ? 8 : 4, es_out = p == DMRG_PREC_FP64 ? 8 : 4;
    const TcMode mode = (p == DMRG_PREC_BF16X3) ? TC_BF16X3 : TC_TF32;
    int64_t k0 = 0;
    for (int c = 0; c < n_class; ++c) {
        const int64_t kc = counts[c];
        if (kc == 0) continue;
        SiteMatrix Sm{};
        for (int x = 0; x < d * d; ++x) Sm.s[x] = S[int64_t(c) * d * d + x];
        const int64_t n = m * mp;
        cudaError_t e = timed_launch(h, "site_u_transform", s, [&] {
            site_u_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(U, Uc, m, d, mp, Sm,
                                                                    flags[c] ? parity : nullptr);
            return cudaGetLastError();
        });
        if (e != cudaSuccess) return cuda_fail(h, e, "site transform");
        const void* Ac = static_cast<const char*>(A) + size_t(k0) * m * m * es_in;
        void* Oc = static_cast<char*>(Oout) + size_t(k0) * mp * mp * es_out;
        if (tc) {
            const TcConfig c1 = tuned_config(h, shape_key("g1", kc, m, d, mp, p), mode);
            const TcConfig c2 = tuned_config(h, shape_key("g2", kc, m, d, mp, p), mode);
            st = dense_tc_forward(h, U, m, d, mp, Ac, in_is_fp64, kc, Oc, p, wsd, c1, c2, s, true, Uc);
        } else {
            st = dense_simt_forward(h, U, m, d, mp, Ac, in_is_fp64, kc, Oc, p, wsd, s, true, Uc, Uc32);
        }
        if (st != DMRG_OK) return st;
        k0 += kc;
    }
    return DMRG_OK;
}

}  // extern "C"
