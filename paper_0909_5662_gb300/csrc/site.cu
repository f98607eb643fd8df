// site.cu -- rotation of blocked site and cross operators (dmrg_rotate_site_ops).
//
// Operators of the added site and block x site products are written in the [B a]
// basis as Z_k = (A_k P^f) (x) S (Sec. 2, the blocking that follows step 5), with P
// the block's fermion parity carried by odd site operators (block modes ordered
// first).  Since (A P) (x) S = (A (x) I)(P (x) S), the rotation is
//
//     O'_k = U^T (A_k (x) I_d) U_c,     U_c = (P^{f_c} (x) S_c) U,
//
// i.e. the plain block rotation of A_k with U_c in the first product.  On the
// tensor-core paths the classes go in groups of up to six: one kernel forms the
// group's U_c straight into the first product's packed operand, and one dense rotation
// packs the operators and runs the first product as one problem per class (each with
// its own U_c) and the second product over the group.
#include <cuda_runtime.h>

#include <algorithm>

#include "api_common.h"
#include "tc_common.cuh"

using namespace dmrg;

namespace {

constexpr int kMaxSiteDim = 8;

constexpr int kGroup = kMaxInlineProblems;   // classes per first-product launch

struct SiteMatrices {
    double s[kGroup][kMaxSiteDim * kMaxSiteDim];
    unsigned long long nz[kGroup];   // bit s * d + t set where S_c[s][t] != 0
    int odd[kGroup];                 // 1: the class carries the block parity
};

// Uc_c[(j, s)][b] = p_j^{f_c} * sum_t S_c[s][t] U[(j, t)][b] for class c = blockIdx.z of
// the group (Uc_c at c * m * d * mp), one thread per (j, b): b from blockIdx.x, rows j
// from blockIdx.y onwards in steps of gridDim.y.
__global__ void site_u_kernel(const double* __restrict__ U, double* __restrict__ Uc, int64_t m,
                              int d, int64_t mp, const __grid_constant__ SiteMatrices S,
                              const signed char* __restrict__ parity) {
    const int c = blockIdx.z;
    const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= mp) return;
    double* out = Uc + int64_t(c) * m * d * mp;
    for (int64_t j = blockIdx.y; j < m; j += gridDim.y) {
        double u[kMaxSiteDim];
#pragma unroll
        for (int t = 0; t < kMaxSiteDim; ++t) u[t] = t < d ? U[(j * d + t) * mp + b] : 0.0;
        // the parity is a sign: applied to the bits, off the (slow) FP64 pipe
        const long long flip = (S.odd[c] && parity && parity[j] < 0) ? (1ll << 63) : 0ll;
#pragma unroll
        for (int s = 0; s < kMaxSiteDim; ++s) {
            if (s >= d) break;
            double v = 0.0;
#pragma unroll
            for (int t = 0; t < kMaxSiteDim; ++t) {
                // site operators are sparse (one entry per row for c, c+): the zero test is
                // an integer mask, uniform over the grid
                if (t < d && ((S.nz[c] >> (s * d + t)) & 1ull)) v = fma(S.s[c][s * d + t], u[t], v);
            }
            out[(j * d + s) * mp + b] = __longlong_as_double(__double_as_longlong(v) ^ flip);
        }
    }
}

// Tensor-core paths: U_c formed and written straight into the first product's packed
// operand.  Packed row b * d + s, column j of class c holds
//   U_c[(j, s)][b] = p_j^{f_c} * sum_t S_c[s][t] U[(j, t)][b]
// as a BF16 hi/lo pair (split) or TF32-rounded FP32 (tf32), row stride ld.  A block
// takes 16 columns j and 32 rows b of one class (blockIdx.z): it reads U along b,
// forms the d values per (j, b) in FP64 and writes them along j through shared memory.
constexpr int kSpJ = 16, kSpB = 32;

__global__ void __launch_bounds__(256) site_pack_kernel(const double* __restrict__ U, int64_t m, int d,
                                                        int64_t mp, const __grid_constant__ SiteMatrices S,
                                                        const signed char* __restrict__ parity, int split,
                                                        void* __restrict__ dst0, void* __restrict__ dst1,
                                                        int64_t ld) {
    __shared__ double tile[kMaxSiteDim][kSpJ][kSpB + 1];
    const int c = blockIdx.z;
    const int64_t j0 = int64_t(blockIdx.x) * kSpJ, b0 = int64_t(blockIdx.y) * kSpB;
    const int tb = threadIdx.x % kSpB, tj = threadIdx.x / kSpB;   // 8 column rows per pass
    for (int jj = tj; jj < kSpJ; jj += 256 / kSpB) {
        const int64_t j = j0 + jj, b = b0 + tb;
        if (j >= m || b >= mp) continue;
        double u[kMaxSiteDim];
#pragma unroll
        for (int t = 0; t < kMaxSiteDim; ++t) u[t] = t < d ? U[(j * d + t) * mp + b] : 0.0;
        const long long flip = (S.odd[c] && parity && parity[j] < 0) ? (1ll << 63) : 0ll;
#pragma unroll
        for (int s = 0; s < kMaxSiteDim; ++s) {
            if (s >= d) break;
            double v = 0.0;
#pragma unroll
            for (int t = 0; t < kMaxSiteDim; ++t)
                if (t < d && ((S.nz[c] >> (s * d + t)) & 1ull)) v = fma(S.s[c][s * d + t], u[t], v);
            tile[s][jj][tb] = __longlong_as_double(__double_as_longlong(v) ^ flip);
        }
    }
    __syncthreads();
    // write: packed row (b, s), columns j0 .. j0 + 15
    const size_t cls_off = size_t(c) * d * mp * ld;
    for (int x = threadIdx.x; x < kSpB * d * kSpJ; x += 256) {
        const int jj = x % kSpJ, rs = x / kSpJ;
        const int tbb = rs / d, s = rs % d;
        const int64_t j = j0 + jj, b = b0 + tbb;
        if (j >= m || b >= mp) continue;
        const size_t at = cls_off + size_t(b * d + s) * ld + j;
        const double v = tile[s][jj][tbb];
        if (split) {
            __nv_bfloat16 h, l;
            tcdev::split_bf16(v, h, l);
            static_cast<__nv_bfloat16*>(dst0)[at] = h;
            static_cast<__nv_bfloat16*>(dst1)[at] = l;
        } else {
            static_cast<float*>(dst0)[at] = tcdev::tf32_round(float(v));
        }
    }
}

struct SiteDims {
    // Uc (FP64, plain-FMA paths), Uc in FP32 (plain-FMA FP32 path), the group's packed
    // U_c (tensor-core paths), dense rotation workspace
    WsLayout ws;
};

SiteDims site_dims(int64_t K, int64_t m, int d, int64_t mp, dmrg_precision p) {
    SiteDims D;
    const bool tc = (p == DMRG_PREC_TF32 || p == DMRG_PREC_BF16X3);
    const DenseDims dd = dense_dims(std::max<int64_t>(K, 1), m, d, mp, p);
    const size_t es = (p == DMRG_PREC_TF32) ? 4 : 2;
    D.ws.add("Uc", tc ? 0 : size_t(m) * d * mp * 8);
    D.ws.add("Uc32", p == DMRG_PREC_FP32 ? size_t(m) * d * mp * 4 : 0);
    for (int i = 0; i < 2; ++i)
        D.ws.add("B1", (tc && (i == 0 || p == DMRG_PREC_BF16X3)) ? size_t(kGroup) * d * mp * dd.ld1 * es : 0);
    D.ws.add("dense", dd.ws.total);
    return D;
}

cudaError_t site_u_launch(dmrg_handle h, const double* U, double* Uc, int64_t m, int d, int64_t mp,
                          const SiteMatrices& S, int nclass, const signed char* parity,
                          cudaStream_t s) {
    const dim3 grid(unsigned((mp + 127) / 128), unsigned(std::min<int64_t>(m, 65535)), unsigned(nclass));
    return timed_launch(h, "site_u_transform", s, [&] {
        site_u_kernel<<<grid, 128, 0, s>>>(U, Uc, m, d, mp, S, parity);
        return cudaGetLastError();
    });
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
    void* b1[2] = {base + D.ws.offsets[2], p == DMRG_PREC_BF16X3 ? base + D.ws.offsets[3] : nullptr};
    void* wsd = base + D.ws.offsets[4];
    const size_t es_in = in_is_fp64 ? 8 : 4, es_out = p == DMRG_PREC_FP64 ? 8 : 4;
    const TcMode mode = (p == DMRG_PREC_BF16X3) ? TC_BF16X3 : TC_TF32;
    auto site_matrix = [&](SiteMatrices& Sm, int slot, int c) {
        Sm.nz[slot] = 0;
        for (int x = 0; x < d * d; ++x) {
            Sm.s[slot][x] = S[int64_t(c) * d * d + x];
            if (Sm.s[slot][x] != 0.0) Sm.nz[slot] |= 1ull << x;
        }
        Sm.odd[slot] = flags[c];
    };
    int64_t k0 = 0;
    if (!tc) {
        // plain-FMA paths: one class at a time
        for (int c = 0; c < n_class; ++c) {
            const int64_t kc = counts[c];
            if (kc == 0) continue;
            SiteMatrices Sm{};
            site_matrix(Sm, 0, c);
            cudaError_t e = site_u_launch(h, U, Uc, m, d, mp, Sm, 1, parity, s);
            if (e != cudaSuccess) return cuda_fail(h, e, "site transform");
            const void* Ac = static_cast<const char*>(A) + size_t(k0) * m * m * es_in;
            void* Oc = static_cast<char*>(Oout) + size_t(k0) * mp * mp * es_out;
            st = dense_simt_forward(h, U, m, d, mp, Ac, in_is_fp64, kc, Oc, p, wsd, s, true, Uc, Uc32);
            if (st != DMRG_OK) return st;
            k0 += kc;
        }
        return DMRG_OK;
    }
    // tensor-core paths: the classes with operators in groups of at most kGroup, the
    // groups as even as possible
    int live = 0;
    for (int x = 0; x < n_class; ++x) live += counts[x] > 0 ? 1 : 0;
    const int ngroups = (live + kGroup - 1) / kGroup;
    const int per_group = ngroups ? (live + ngroups - 1) / ngroups : 1;
    int c = 0;
    while (c < n_class) {
        SiteMatrices Sm{};
        FirstClasses cls;   // U1_c are formed straight into b1 by site_pack_kernel
        cls.b1[0] = b1[0];
        cls.b1[1] = b1[1];
        const int64_t g0 = k0;
        for (; c < n_class && cls.n < per_group; ++c) {
            if (counts[c] == 0) continue;
            site_matrix(Sm, cls.n, c);
            cls.k0[cls.n] = k0 - g0;
            cls.kc[cls.n] = counts[c];
            k0 += counts[c];
            ++cls.n;
        }
        if (cls.n == 0) break;
        const int64_t ld1 = dense_dims(1, m, d, mp, p).ld1;
        cudaError_t e = timed_launch(h, "site_pack", s, [&] {
            const dim3 grid(unsigned((m + kSpJ - 1) / kSpJ), unsigned((mp + kSpB - 1) / kSpB), unsigned(cls.n));
            site_pack_kernel<<<grid, 256, 0, s>>>(U, m, d, mp, Sm, parity, p == DMRG_PREC_BF16X3 ? 1 : 0, b1[0],
                                                  b1[1], ld1);
            return cudaGetLastError();
        });
        if (e != cudaSuccess) return cuda_fail(h, e, "site transform");
        cls.b1_ready = true;
        const int64_t kg = k0 - g0;
        const void* Ag = static_cast<const char*>(A) + size_t(g0) * m * m * es_in;
        void* Og = static_cast<char*>(Oout) + size_t(g0) * mp * mp * es_out;
        const TcConfig c1 = tuned_config(h, shape_key("g1", kg, m, d, mp, p), mode);
        const TcConfig c2 = tuned_config(h, shape_key("g2", kg, m, d, mp, p), mode);
        st = dense_tc_forward(h, U, m, d, mp, Ag, in_is_fp64, kg, Og, p, wsd, c1, c2, s, true, nullptr, &cls);
        if (st != DMRG_OK) return st;
    }
    return DMRG_OK;
}

}  // extern "C"
