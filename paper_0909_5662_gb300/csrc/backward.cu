// backward.cu -- adjoint of the dense rotation (dmrg_rotate_ops_backward).
//
// For a loss L with dL/dO'_k = G_k and O'_k = U^T (O_k (x) I_d) U (Sec. 2, step 5),
// the chain rule gives
//   dO_k = Tr_d(U G_k U^T) = sum_s U_s G_k U_s^T          (U_s: rows j*d + s of U)
//   dU   = sum_k (O_k (x) I) U G_k^T + (O_k (x) I)^T U G_k.
// Nothing from the forward pass is kept: only U, O and G are read.
//
// Tensor-core schedule (TF32; BF16x3 as noted below), CTA-pair kernel, with
// W_k = U G_k and W'_k = U G_k^T (md x m' each; W_{k,s} = rows j*d + s):
//   1. W'_k: M = K*m' rows (k, a), N = d*m columns ordered (s, j) (U packed with rows
//      s*m + j), reduction m'.  The epilogue writes it twice: row-major (rows (k, j),
//      columns (s, a): the dO operand) and site-major, WT'_k[s*m' + a][j] (j contiguous:
//      the dU operand), where a 32-column chunk is a run of 32 consecutive j;
//   2. W_k the same way from G^T, written site-major only (WT_k);
//   3. dO_k[i][j] = sum_(s,a) W'_k[j*d+s][a] U[i*d+s][a] : M = K*m rows (k, j), N = m;
//   4. dU_r^T[(s,n)][i] = sum_(k,j) WT'_k[(s,n)][j] O_k[i][j] + WT_k[(s,n)][j] O_k[j][i]:
//      one problem whose reduction runs over 2K slices ([WT' | WT] against [O | O^T]),
//      split into P parts that write their own partial sums;
//   5. dU[i*d+s][n] = sum_p partial_p[(s,n)][i], summed in a fixed order.
// BF16x3 reads 16-bit operands in either order (MN-major operands of the pair kernel):
// W' is written row-major only and dU's first K slices read it MN-major; the last K
// slices read O MN-major as O^T, so O^T is not packed.  The two halves are separate
// problems with their own parts.
// BF16x3 reductions longer than one accumulation chain (dO: d*m'; dU: 2*K*m) are cut
// into chains as in the forward products, and nothing is accumulated atomically, so dO
// and dU are reproducible bit for bit.
// Plain FMA schedule (FP64, FP32): the same formulas as strided batched GEMMs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "api_common.h"
#include "ptx.cuh"

using namespace dmrg;

namespace {

// dU's reduction over 2K*m terms is split into at most this many parts, each written to
// its own partial sum.
constexpr int kBwdMaxParts = 16;

struct BwdDims {
    int64_t K, m, mp, md, dmp;
    int d;
    int64_t ld_u, ld_n, ld_j;  // packed leading dimensions (elements)
    WsLayout ws;
    // section indices
    int i_U, i_Ur, i_G, i_GT, i_O, i_Wp, i_WT, i_dU, i_conv;
};

BwdDims bwd_dims(int64_t K, int64_t m, int d, int64_t mp, dmrg_precision p) {
    BwdDims B{};
    B.K = K; B.m = m; B.d = d; B.mp = mp; B.md = m * d; B.dmp = int64_t(d) * mp;
    WsLayout& W = B.ws;
    if (p == DMRG_PREC_FP64 || p == DMRG_PREC_FP32) {
        const size_t es = (p == DMRG_PREC_FP64) ? 8 : 4;
        B.i_Wp = int(W.offsets.size()); W.add("W", size_t(K) * B.md * mp * es);
        B.i_WT = int(W.offsets.size()); W.add("Wp", size_t(K) * B.md * mp * es);
        B.i_dU = int(W.offsets.size()); W.add("dU", size_t(B.md) * mp * es);
        B.i_conv = int(W.offsets.size());
        if (p == DMRG_PREC_FP32) {  // FP32 copies of U, O and G
            W.add("U32", size_t(B.md) * mp * 4);
            W.add("O32", size_t(K) * m * m * 4);
            W.add("G32", size_t(K) * mp * mp * 4);
        }
        return B;
    }
    const bool split = (p == DMRG_PREC_BF16X3);
    const int64_t al = split ? 8 : 4;
    const size_t es = split ? 2 : 4;
    const int ns = split ? 2 : 1;
    auto ld = [&](int64_t x) { return (x + al - 1) / al * al; };
    B.ld_u = ld(mp);
    B.ld_n = ld(B.dmp);
    B.ld_j = ld(m);
    auto add = [&](int& idx, size_t elems) {
        idx = int(W.offsets.size());
        for (int i = 0; i < ns; ++i) W.add("x", elems * es);
    };
    add(B.i_U, size_t(B.md) * B.ld_u);
    add(B.i_Ur, size_t(m) * B.ld_n);
    add(B.i_G, size_t(K) * mp * B.ld_u);
    add(B.i_GT, size_t(K) * mp * B.ld_u);
    // BF16x3 reads O^T from O and W' row-major (MN-major operands): only O and WT are kept
    const int64_t slices = split ? K : 2 * K;
    add(B.i_O, size_t(slices) * m * B.ld_j);       // [O | O^T], slices of m x ld_j
    add(B.i_Wp, size_t(K) * m * B.ld_n);           // W' row-major: rows (k, j), cols (s, a)
    add(B.i_WT, size_t(slices) * B.dmp * B.ld_j);  // [WT' | WT], slices of d*m' x ld_j
    B.i_dU = int(W.offsets.size());
    W.add("dUpart", size_t(kBwdMaxParts) * B.md * mp * 4);
    B.i_conv = int(W.offsets.size());
    W.add("chain", split ? kChainScratchBytes : 0);
    return B;
}

dmrg_status bwd_simt(dmrg_handle h, const double* U, const void* O, const void* G, int in_is_fp64,
                     void* dO, double* dU, const BwdDims& B, dmrg_precision p, void* ws,
                     cudaStream_t s) {
    const bool f64 = (p == DMRG_PREC_FP64);
    const Real rt = f64 ? Real::F64 : Real::F32;
    char* base = static_cast<char*>(ws);
    void* W = base + B.ws.offsets[B.i_Wp];
    void* Wp = base + B.ws.offsets[B.i_WT];
    void* dUr = base + B.ws.offsets[B.i_dU];
    const void* Uu = U;
    const void* Ou = O;
    const void* Gu = G;
    const int64_t K = B.K, m = B.m, mp = B.mp, md = B.md, dmp = B.dmp;
    cudaError_t e = cudaSuccess;
    if (!f64) {
        float* U32 = reinterpret_cast<float*>(base + B.ws.offsets[B.i_conv]);
        float* O32 = reinterpret_cast<float*>(base + B.ws.offsets[B.i_conv + 1]);
        float* G32 = reinterpret_cast<float*>(base + B.ws.offsets[B.i_conv + 2]);
        PackJob jobs[3] = {};
        int nj = 0;
        auto conv = [&](const void* src, float* dst, int64_t rows, int64_t cols) {
            PackJob& j = jobs[nj++];
            j.src = src; j.src_f64 = 1; j.mode = 2; j.rows = rows; j.cols = cols;
            j.rows_per_op = rows; j.rdiv = 1; j.s_r_hi = cols; j.s_c = 1; j.dst0 = dst; j.ld = cols;
        };
        conv(U, U32, md, mp);
        Uu = U32;
        if (in_is_fp64) {
            conv(O, O32, K * m, m);
            conv(G, G32, K * mp, mp);
            Ou = O32;
            Gu = G32;
        }
        e = timed_launch(h, "bwd_convert_fp32", s, [&] { return pack_launch(jobs, nj, nullptr, s); });
        if (e != cudaSuccess) return cuda_fail(h, e, "convert");
    }
    // W_k = U G_k and W'_k = U G_k^T (md x mp each)
    SimtGemm g{};
    g.A = Uu; g.M = md; g.N = mp; g.K = mp;
    g.sAb = 0; g.sAi = mp; g.sAk = 1;
    g.B = Gu; g.sBb = mp * mp; g.sBk = mp; g.sBj = 1;
    g.C = W; g.sCb = md * mp; g.sCi = mp; g.sCj = 1;
    g.batch = int32_t(K);
    e = timed_launch(h, "bwd_simt_W", s, [&] { return simt_gemm_launch(rt, g, s); });
    if (e != cudaSuccess) return cuda_fail(h, e, "W");
    g.sBk = 1; g.sBj = mp; g.C = Wp;
    e = timed_launch(h, "bwd_simt_Wp", s, [&] { return simt_gemm_launch(rt, g, s); });
    if (e != cudaSuccess) return cuda_fail(h, e, "W'");
    if (dO) {
        // dO_k[i][j] = sum_n (W_k)_r[i][n] U_r[j][n]
        SimtGemm q{};
        q.A = W; q.M = m; q.N = m; q.K = dmp;
        q.sAb = md * mp; q.sAi = dmp; q.sAk = 1;
        q.B = Uu; q.sBb = 0; q.sBk = 1; q.sBj = dmp;
        q.C = dO; q.sCb = m * m; q.sCi = m; q.sCj = 1;
        q.batch = int32_t(K);
        e = timed_launch(h, "bwd_simt_dO", s, [&] { return simt_gemm_launch(rt, q, s); });
        if (e != cudaSuccess) return cuda_fail(h, e, "dO");
    }
    if (dU) {
        void* target = f64 ? static_cast<void*>(dU) : dUr;
        // dU_r = sum_k O_k (W'_k)_r   then   += sum_k O_k^T (W_k)_r
        SimtGemm q{};
        q.A = Ou; q.M = m; q.N = dmp; q.K = m;
        q.sAb = m * m; q.sAi = m; q.sAk = 1;
        q.B = Wp; q.sBb = md * mp; q.sBk = dmp; q.sBj = 1;
        q.C = target; q.sCb = 0; q.sCi = dmp; q.sCj = 1;
        q.batch = int32_t(K);
        q.reduce_batch = 1;
        e = timed_launch(h, "bwd_simt_dU", s, [&] { return simt_gemm_launch(rt, q, s); });
        if (e != cudaSuccess) return cuda_fail(h, e, "dU");
        q.sAi = 1; q.sAk = m; q.B = W; q.accumulate = 1;
        e = timed_launch(h, "bwd_simt_dU", s, [&] { return simt_gemm_launch(rt, q, s); });
        if (e != cudaSuccess) return cuda_fail(h, e, "dU");
        if (!f64) {
            e = timed_launch(h, "bwd_dU_to_fp64", s, [&] {
                return convert_f32_to_f64_launch(static_cast<const float*>(dUr), dU, md * mp, s);
            });
            if (e != cudaSuccess) return cuda_fail(h, e, "dU convert");
        }
    }
    return DMRG_OK;
}

// dU[(i d + s) m' + n] = sum_p part[p][(s m' + n) m + i], p in order: the partial sums
// of dU_r^T are transposed back through a shared-memory tile.  The sum is compensated
// (Neumaier's variant of Kahan summation) in FP32: an FP64 addition per part would make
// the kernel FP64-bound on this part, and the compensated sum's error stays at the final
// rounding to FP32 for the few parts there are.
__global__ void __launch_bounds__(256) bwd_du_reduce_kernel(const float* __restrict__ part,
                                                            int nparts, int64_t dmp, int64_t m,
                                                            int64_t mp, int d,
                                                            double* __restrict__ dU) {
    __shared__ double t[32][33];
    const int64_t R0 = int64_t(blockIdx.y) * 32, I0 = int64_t(blockIdx.x) * 32;
    for (int rr = threadIdx.y; rr < 32; rr += 8) {
        const int64_t R = R0 + rr, I = I0 + threadIdx.x;
        float sum = 0.f, comp = 0.f;
        if (R < dmp && I < m) {
            float x[kBwdMaxParts];   // every part's load in flight before the sum
#pragma unroll
            for (int q = 0; q < kBwdMaxParts; ++q)
                x[q] = q < nparts ? part[(int64_t(q) * dmp + R) * m + I] : 0.f;
#pragma unroll
            for (int q = 0; q < kBwdMaxParts; ++q) {
                if (q >= nparts) break;
                const float u = sum + x[q];
                comp += fabsf(sum) >= fabsf(x[q]) ? (sum - u) + x[q] : (x[q] - u) + sum;
                sum = u;
            }
        }
        t[rr][threadIdx.x] = double(sum) + double(comp);
    }
    __syncthreads();
    for (int ii = threadIdx.y; ii < 32; ii += 8) {
        const int64_t I = I0 + ii, R = R0 + threadIdx.x;
        if (R < dmp && I < m) {
            const int64_t sidx = R / mp, n = R - sidx * mp;
            dU[(I * d + sidx) * mp + n] = t[threadIdx.x][ii];
        }
    }
}

// The same sum with four consecutive i per thread (m % 4 == 0, 16-byte aligned parts):
// each thread has every part's 16-byte load in flight at once (one round of loads where
// the one-element form has four).  Per element the parts are added in the same order, so
// the two forms agree bit for bit.  Launched as a programmatic dependent of the product
// that writes the parts.
__global__ void __launch_bounds__(256) bwd_du_reduce4_kernel(const float* __restrict__ part,
                                                             int nparts, int64_t dmp, int64_t m,
                                                             int64_t mp, int d,
                                                             double* __restrict__ dU) {
    __shared__ double t[32][33];
    griddep_wait();
    const int64_t R0 = int64_t(blockIdx.y) * 32, I0 = int64_t(blockIdx.x) * 32;
    const int rl = threadIdx.x >> 3, i4 = (threadIdx.x & 7) * 4;
    const int64_t R = R0 + rl, I = I0 + i4;
    float sum[4] = {0.f, 0.f, 0.f, 0.f}, comp[4] = {0.f, 0.f, 0.f, 0.f};
    if (R < dmp && I < m) {
        float4 x[kBwdMaxParts];
#pragma unroll
        for (int q = 0; q < kBwdMaxParts; ++q)
            x[q] = q < nparts ? *reinterpret_cast<const float4*>(part + (int64_t(q) * dmp + R) * m + I)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < kBwdMaxParts; ++q) {
            if (q >= nparts) break;
            const float xs[4] = {x[q].x, x[q].y, x[q].z, x[q].w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float u = sum[e] + xs[e];
                comp[e] += fabsf(sum[e]) >= fabsf(xs[e]) ? (sum[e] - u) + xs[e] : (xs[e] - u) + sum[e];
                sum[e] = u;
            }
        }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) t[rl][i4 + e] = double(sum[e]) + double(comp[e]);
    __syncthreads();
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int ii = ty; ii < 32; ii += 8) {
        const int64_t Iw = I0 + ii, Rw = R0 + tx;
        if (Rw < dmp && Iw < m) {
            const int64_t sidx = Rw / mp, n = Rw - sidx * mp;
            dU[(Iw * d + sidx) * mp + n] = t[tx][ii];
        }
    }
}

dmrg_status bwd_tc(dmrg_handle h, const double* U, const void* O, const void* G, int in_is_fp64,
                   void* dO, double* dU, const BwdDims& B, dmrg_precision p, void* ws,
                   cudaStream_t s) {
    const bool split = (p == DMRG_PREC_BF16X3);
    const TcMode mode = split ? TC_BF16X3 : TC_TF32;
    const int pmode = split ? 0 : 1;
    const TcEpi epi_op = split ? EPI_SPLIT_BF16 : EPI_TF32;
    const int64_t K = B.K, m = B.m, mp = B.mp, md = B.md, dmp = B.dmp;
    const int d = B.d;
    const size_t es = split ? 2 : 4;
    char* base = static_cast<char*>(ws);
    auto sec = [&](int idx, int half) -> char* {
        return base + B.ws.offsets[idx + (split ? half : 0)];
    };
    auto lo = [&](int idx) -> char* { return split ? sec(idx, 1) : sec(idx, 0); };
    // BF16x3: dU reads W' and W row-major and O^T from O, as MN-major operands of the
    // CTA-pair kernel (its tensor core takes 16-bit operands in either order), so neither
    // the transposed pack of O nor site-major copies of W' and W are made.
    const bool mn = split;
    cudaError_t e;
    // ---- packs: U, U_r (dO), G, and for dU G^T, O and O^T, in one launch
    {
        PackJob jobs[6] = {};
        int nj = 0;
        PackJob& ju = jobs[nj++];   // U site-major: row s*m + j, cols a = U[j*d + s][a]
        ju.src = U; ju.src_f64 = 1; ju.mode = pmode; ju.rows = md; ju.cols = mp; ju.rows_per_op = m;
        ju.s_op = mp; ju.rdiv = 1; ju.s_r_hi = int64_t(d) * mp; ju.s_c = 1;
        ju.dst0 = sec(B.i_U, 0); ju.dst1 = lo(B.i_U); ju.ld = B.ld_u;
        if (dO) {
            PackJob& jr = jobs[nj++];   // U_r: rows j, cols (s, a)
            jr.src = U; jr.src_f64 = 1; jr.mode = pmode; jr.rows = m; jr.cols = dmp; jr.rows_per_op = m;
            jr.rdiv = 1; jr.s_r_hi = dmp; jr.s_c = 1; jr.dst0 = sec(B.i_Ur, 0); jr.dst1 = lo(B.i_Ur);
            jr.ld = B.ld_n;
        }
        if (dU) {
            PackJob& jt = jobs[nj++];   // G^T: rows (k, b), cols a = G_k[a][b]
            jt.src = G; jt.src_f64 = in_is_fp64; jt.mode = pmode; jt.rows = K * mp; jt.cols = mp;
            jt.rows_per_op = mp; jt.s_op = mp * mp; jt.rdiv = 1; jt.s_r_hi = 1; jt.s_c = mp;
            jt.dst0 = sec(B.i_GT, 0); jt.dst1 = lo(B.i_GT); jt.ld = B.ld_u;
            const size_t oT = size_t(K) * m * B.ld_j * es;   // O^T slices follow the O slices
            PackJob& jo = jobs[nj++];   // O: rows (k, i), cols j
            jo.src = O; jo.src_f64 = in_is_fp64; jo.mode = pmode; jo.rows = K * m; jo.cols = m;
            jo.rows_per_op = K * m; jo.rdiv = 1; jo.s_r_hi = m; jo.s_c = 1;
            jo.dst0 = sec(B.i_O, 0); jo.dst1 = lo(B.i_O); jo.ld = B.ld_j;
            if (!mn) {   // (BF16x3 reads O MN-major instead)
                PackJob& jq = jobs[nj++];   // O^T: rows (k, i), cols j = O_k[j][i]
                jq.src = O; jq.src_f64 = in_is_fp64; jq.mode = pmode; jq.rows = K * m; jq.cols = m;
                jq.rows_per_op = m; jq.s_op = m * m; jq.rdiv = 1; jq.s_r_hi = 1; jq.s_c = m;
                jq.dst0 = sec(B.i_O, 0) + oT; jq.dst1 = lo(B.i_O) + (split ? oT : 0); jq.ld = B.ld_j;
            }
        }
        // G last: its last rows are still in L2 when the W' product, which runs its M tiles
        // from the last to the first, starts reading them.  Where G^T goes through
        // shared-memory tiles, the same tiles also give G (G is read once).
        PackJob* jgt = nullptr;
        for (int i = 0; i < nj; ++i)
            if (jobs[i].dst0 == sec(B.i_GT, 0)) jgt = &jobs[i];
        if (jgt != nullptr && pack_job_tiled(*jgt) && (B.ld_u % 2) == 0) {
            jgt->st0 = sec(B.i_G, 0);
            jgt->st1 = split ? lo(B.i_G) : nullptr;
            jgt->st_ld = B.ld_u;
            jgt->late = 1;
        } else {
            PackJob& jg = jobs[nj++];   // G: rows (k, a), cols b = G_k[a][b]
            jg.src = G; jg.src_f64 = in_is_fp64; jg.mode = pmode; jg.rows = K * mp; jg.cols = mp;
            jg.rows_per_op = K * mp; jg.rdiv = 1; jg.s_r_hi = mp; jg.s_c = 1;
            jg.dst0 = sec(B.i_G, 0); jg.dst1 = lo(B.i_G); jg.ld = B.ld_u;
            jg.late = 1;
        }
        e = timed_launch(h, "bwd_pack", s, [&] { return pack_launch(jobs, nj, nullptr, s); });
        if (e != cudaSuccess) return cuda_fail(h, e, "pack");
    }
    // Every product runs on CTA pairs: only that kernel writes the site-major copy, the
    // per-split partial sums and the chained accumulation.
    TcConfig cfg = tuned_config(h, shape_key("bwd", K, m, d, mp, p), mode);
    if (!cfg.pair || cfg.row_bytes != 128) {
        cfg.pair = 1;
        cfg.row_bytes = 128;
        cfg.stages = tc_stages_for(mode, cfg);
    }
    const int grid = std::min(cfg.grid > 0 ? cfg.grid : h->num_sms, kChainScratchCtas) / 2 * 2;
    float* chain_scr = split ? reinterpret_cast<float*>(base + B.ws.offsets[B.i_conv]) : nullptr;
    const int chain_kb = split ? std::max(1, h->accum_chain / 64) : 0;   // 64 BF16 per k-block
    auto launch = [&](const char* name, TcLaunch& L, TcEpi epi, int64_t red) -> dmrg_status {
        L.table = nullptr;
        int tiles = 0;
        for (int i = 0; i < L.nprob; ++i) {
            TcProblem& P = L.inline_prob[i];
            P.tile_start = tiles;
            P.kb_chunk = (chain_scr && red > std::max<int64_t>(kChainMinRed, h->accum_chain)) ? chain_kb : 0;
            tiles += P.m_tiles * P.n_tiles * P.k_splits;
        }
        L.total_tiles = tiles;
        L.status = h->d_status;
        L.timeout_ns = timeout_ns(h);
        L.row_bytes = cfg.row_bytes;
        // FP32 output with at most two chains per tile sums them in the output (the first
        // chain stores, the second adds), as the forward's second product does
        const int64_t kbt = (red + cfg.row_bytes / int64_t(es) - 1) / (cfg.row_bytes / int64_t(es));
        const int64_t chains = chain_kb > 0 ? (kbt + chain_kb - 1) / chain_kb : 1;
        L.chunk_scratch = (L.inline_prob[0].kb_chunk && !(epi == EPI_F32 && chains <= 2)) ? chain_scr
                                                                                         : nullptr;
        cudaError_t ee = timed_launch(h, name, s, [&] {
            return tc_gemm_launch_pair(mode, epi, L, cfg.stages, grid, s);
        });
        return cuda_fail(h, ee, name);
    };
    dmrg_status st;
    char* wt_hi = sec(B.i_WT, 0);
    char* wt_lo = lo(B.i_WT);
    // WT slices follow the WT' slices (BF16x3 keeps WT alone)
    const size_t wt_second = mn ? 0 : size_t(K) * dmp * B.ld_j * es;
    // site-major copy of a W product: rows (k, a), columns c = s m + j -> slice k, row
    // s m' + a, column j
    auto site_major = [&](TcLaunch& L, char* hi, char* lo_) {
        L.out2[0] = hi;
        L.out2[1] = split ? lo_ : nullptr;
        L.o2_rows_per_op = int32_t(mp);
        L.o2_s_op = dmp * B.ld_j;
        L.o2_s_row = B.ld_j;
        L.o2_s_site = mp * B.ld_j;
        L.o2_m = int32_t(m);
    };
    {
        // 1. W'_k[j d + s][a] = sum_b G_k[a][b] U[j d + s][b], rows (k, a), columns (s, j):
        //    row-major into Wp (rows (k, j), cols (s, a)), and site-major into the first K
        //    slices of WT.
        TcLaunch L{};
        TcProblem& P = L.inline_prob[0];
        TcOperand A{sec(B.i_G, 0), lo(B.i_G), K * mp, mp, B.ld_u};
        TcOperand Bo{sec(B.i_U, 0), lo(B.i_U), md, mp, B.ld_u};
        if (!make_problem(P, mode, A, Bo, cfg.tile_n_max, 1, cfg.row_bytes, 1))
            return fail(h, DMRG_ERR_CUDA, "tensor map");
        TcScatter& S = P.sc[0];
        S.rows_per_op = int32_t(mp); S.s_op = m * B.ld_n; S.s_row = 1;
        S.col_div = int32_t(m); S.s_col_hi = mp; S.s_col_lo = B.ld_n;
        L.nprob = 1;
        // last M tile first (G's last rows are the packer's latest writes); the W' rows of
        // the first operators, written last, are then in L2 for the dO product
        L.reverse_m = 1;
        const bool rowmajor = dO || (dU && mn);
        L.out[0][0] = rowmajor ? sec(B.i_Wp, 0) : nullptr;
        L.out[0][1] = rowmajor ? lo(B.i_Wp) : nullptr;
        if (dU && !mn) site_major(L, wt_hi, wt_lo);
        // BF16x3, row-major only: W' leaves by TMA bulk stores (W'_k rows j, columns
        // s m' + a; a lane's values run down a column), staged per warp in shared memory
        if (split && rowmajor && L.out2[0] == nullptr && h->store_epilogue == 0 && m % 16 == 0 &&
            mp % 16 == 0 &&
            encode_store_map(&L.t_store_map[0], L.out[0][0], dmp, m, K, B.ld_n, 32, 16) &&
            encode_store_map(&L.t_store_map[1], L.out[0][1], dmp, m, K, B.ld_n, 32, 16) &&
            encode_store_map(&L.t_store_map[2], L.out[0][0], dmp, m, K, B.ld_n, 16, 16) &&
            encode_store_map(&L.t_store_map[3], L.out[0][1], dmp, m, K, B.ld_n, 16, 16))
            L.t_store = kStoreRowContiguous;
        if ((st = launch("bwd_tc_Wp", L, epi_op, mp)) != DMRG_OK) return st;
    }
    if (dO) {
        // 3. dO_k[i][j] = sum_(s,a) W'_k[j*d+s][a] U[i*d+s][a], rows (k, j), cols i.
        TcLaunch L2{};
        TcProblem& P2 = L2.inline_prob[0];
        TcOperand A2{sec(B.i_Wp, 0), lo(B.i_Wp), K * m, dmp, B.ld_n};
        TcOperand B2{sec(B.i_Ur, 0), lo(B.i_Ur), m, dmp, B.ld_n};
        if (!make_problem(P2, mode, A2, B2, cfg.tile_n_max, 1, cfg.row_bytes, 1))
            return fail(h, DMRG_ERR_CUDA, "tensor map");
        TcScatter& S2 = P2.sc[0];
        S2.rows_per_op = int32_t(m); S2.s_op = m * m; S2.s_row = 1;
        S2.col_div = 1; S2.s_col_hi = m; S2.s_col_lo = 0;
        L2.nprob = 1;
        L2.out[0][0] = dO;
        // dO leaves by TMA bulk stores (and its second chain by TMA reductions) where the
        // launch sums its chains in the output
        if (split && h->store_epilogue == 0 && m % 16 == 0 &&
            encode_store_map(&L2.t_store_map[0], dO, m, m, K, m, 16, 16, 0, true))
            L2.t_store = kStoreColumnsF32;
        if ((st = launch("bwd_tc_dO", L2, EPI_F32, dmp)) != DMRG_OK) return st;
    }
    if (dU) {
        // 2. W_k[r][b] = sum_a G_k[a][b] U[r][a], rows (k, b), site-major into the last K
        //    slices of WT only.
        {
            TcLaunch L{};
            TcProblem& P = L.inline_prob[0];
            TcOperand A{sec(B.i_GT, 0), lo(B.i_GT), K * mp, mp, B.ld_u};
            TcOperand Bo{sec(B.i_U, 0), lo(B.i_U), md, mp, B.ld_u};
            if (!make_problem(P, mode, A, Bo, cfg.tile_n_max, 1, cfg.row_bytes, 1))
                return fail(h, DMRG_ERR_CUDA, "tensor map");
            L.nprob = 1;
            L.out[0][0] = nullptr;   // no row-major copy
            site_major(L, wt_hi + wt_second, split ? wt_lo + wt_second : nullptr);
            // BF16x3: the site-major W leaves by TMA bulk stores (a lane's values of a
            // column half are 32 contiguous bytes of a row of W_k), staged per warp
            if (split && h->store_epilogue == 0 && m % 16 == 0 && mp % 16 == 0 &&
                encode_store_map(&L.t_store_map[0], L.out2[0], m, dmp, K, B.ld_j, 32, 16, 64) &&
                encode_store_map(&L.t_store_map[1], L.out2[1], m, dmp, K, B.ld_j, 32, 16, 64) &&
                encode_store_map(&L.t_store_map[2], L.out2[0], m, dmp, K, B.ld_j, 16, 16, 32) &&
                encode_store_map(&L.t_store_map[3], L.out2[1], m, dmp, K, B.ld_j, 16, 16, 32))
                L.t_store = kStoreSiteMajor;
            if ((st = launch("bwd_tc_W", L, epi_op, mp)) != DMRG_OK) return st;
        }
        // 4. dU_r^T[(s,n)][i] over 2K slices, split into parts with their own partial sums.
        float* part = reinterpret_cast<float*>(base + B.ws.offsets[B.i_dU]);
        if (mn) {
            // Two problems of K slices each, written to parts [0, pa) and [pa, pa + pb):
            //   sum_(k,j) W'_k[j*d+s][n] O_k[i][j]  (A: W' row-major read MN-major,
            //                                        B: O K-major),
            //   sum_(k,j) WT_k[s*m'+n][j] O_k[j][i] (A: W site-major, K-major,
            //                                        B: O read MN-major).
            TcLaunch L{};
            TcOperand Ap{sec(B.i_Wp, 0), lo(B.i_Wp), dmp, m, B.ld_n, K, m * B.ld_n};
            Ap.mn_major = 1;
            TcOperand Aw{wt_hi + wt_second, wt_lo + wt_second, dmp, m, B.ld_j, K, dmp * B.ld_j};
            TcOperand Bk{sec(B.i_O, 0), lo(B.i_O), m, m, B.ld_j, K, m * B.ld_j};
            TcOperand Bt = Bk;
            Bt.mn_major = 1;
            TcProblem& Pa = L.inline_prob[0];
            TcProblem& Pb = L.inline_prob[1];
            if (!make_problem(Pa, mode, Ap, Bk, cfg.tile_n_max, 1, cfg.row_bytes, 1))
                return fail(h, DMRG_ERR_CUDA, "tensor map");
            // parts per problem: the fewest waves of tiles per unit of reduction length
            // (waves over the CTA pairs x reduction per part), fewer parts on ties
            const int tiles = Pa.m_tiles * Pa.n_tiles;
            const int pairs = std::max(1, grid / 2);
            int each = 1;
            double best = 1e300;
            for (int e = 1; e <= kBwdMaxParts / 2; ++e) {
                const double cost = double((2 * e * tiles + pairs - 1) / pairs) / e + 1e-3 * e;
                if (cost < best) {
                    best = cost;
                    each = e;
                }
            }
            if (!make_problem(Pa, mode, Ap, Bk, cfg.tile_n_max, each, cfg.row_bytes, 1) ||
                !make_problem(Pb, mode, Aw, Bt, cfg.tile_n_max, each, cfg.row_bytes, 1))
                return fail(h, DMRG_ERR_CUDA, "tensor map");
            Pa.sc[0] = scatter_rowmajor(m);
            Pa.sc[0].s_split = dmp * m;
            Pb.sc[0] = Pa.sc[0];
            Pb.sc[0].out_off = int64_t(Pa.k_splits) * dmp * m;
            L.nprob = 2;
            L.out[0][0] = part;
            if ((st = launch("bwd_tc_dU", L, EPI_F32, K * m)) != DMRG_OK) return st;
            const int nparts = Pa.k_splits + Pb.k_splits;
            e = timed_launch(h, "bwd_dU_reduce", s, [&] {
                dim3 grd(unsigned((m + 31) / 32), unsigned((dmp + 31) / 32));
                if (m % 4 != 0 || (reinterpret_cast<uintptr_t>(part) & 15) != 0) {
                    bwd_du_reduce_kernel<<<grd, dim3(32, 8), 0, s>>>(part, nparts, dmp, m, mp, d, dU);
                    return cudaGetLastError();
                }
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = grd;
                cfg.blockDim = dim3(256, 1, 1);
                cfg.stream = s;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
                attr[0].val.programmaticStreamSerializationAllowed = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                return cudaLaunchKernelEx(&cfg, bwd_du_reduce4_kernel, (const float*)part, nparts, dmp,
                                          m, mp, d, dU);
            });
            if (e != cudaSuccess) return cuda_fail(h, e, "dU reduce");
            return DMRG_OK;
        }
        TcLaunch L{};
        TcProblem& P = L.inline_prob[0];
        TcOperand A{wt_hi, split ? wt_lo : nullptr, dmp, m, B.ld_j, 2 * K, dmp * B.ld_j};
        TcOperand Bo{sec(B.i_O, 0), split ? lo(B.i_O) : nullptr, m, m, B.ld_j, 2 * K, m * B.ld_j};
        if (!make_problem(P, mode, A, Bo, cfg.tile_n_max, 1, cfg.row_bytes, 1))
            return fail(h, DMRG_ERR_CUDA, "tensor map");
        // parts: enough to give every CTA pair a tile, at most kBwdMaxParts
        const int tiles = P.m_tiles * P.n_tiles;
        const int parts = std::max(1, std::min(kBwdMaxParts, (grid / 2) / std::max(1, tiles)));
        if (!make_problem(P, mode, A, Bo, cfg.tile_n_max, parts, cfg.row_bytes, 1))
            return fail(h, DMRG_ERR_CUDA, "tensor map");
        P.sc[0] = scatter_rowmajor(m);
        P.sc[0].s_split = dmp * m;
        L.nprob = 1;
        L.out[0][0] = part;
        if ((st = launch("bwd_tc_dU", L, EPI_F32, int64_t(2) * K * m)) != DMRG_OK) return st;
        // 5. dU = the sum of the parts, transposed back, in FP64.
        const int nparts = P.k_splits;
        e = timed_launch(h, "bwd_dU_reduce", s, [&] {
            dim3 grd(unsigned((m + 31) / 32), unsigned((dmp + 31) / 32));
            bwd_du_reduce_kernel<<<grd, dim3(32, 8), 0, s>>>(part, nparts, dmp, m, mp, d, dU);
            return cudaGetLastError();
        });
        if (e != cudaSuccess) return cuda_fail(h, e, "dU reduce");
    }
    return DMRG_OK;
}

}  // namespace

extern "C" {

dmrg_status dmrg_rotate_ops_backward_workspace(dmrg_handle h, int64_t K, int64_t m, int d,
                                               int64_t mp, dmrg_precision p, size_t* bytes) {
    if (!bytes) return fail(h, DMRG_ERR_INVALID_ARG, "bytes is NULL");
    dmrg_status st = check_dense_args(h, K, m, d, mp, p);
    if (st != DMRG_OK) return st;
    *bytes = bwd_dims(K, m, d, mp, p).ws.total;
    return DMRG_OK;
}

dmrg_status dmrg_rotate_ops_backward(dmrg_handle h, const double* U, int64_t m, int d, int64_t mp,
                                     const void* O, const void* G, int in_is_fp64, int64_t K,
                                     void* dO, double* dU, dmrg_precision p, void* ws,
                                     size_t ws_bytes, dmrg_stream_t stream) {
    dmrg_status st = check_dense_args(h, K, m, d, mp, p);
    if (st != DMRG_OK) return st;
    if (!U || !O || !G) return fail(h, DMRG_ERR_INVALID_ARG, "null data pointer");
    if (p == DMRG_PREC_FP64 && !in_is_fp64)
        return fail(h, DMRG_ERR_INVALID_ARG, "the FP64 precision needs FP64 operators");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (K == 0) {
        if (dU) {
            cudaError_t e = cudaMemsetAsync(dU, 0, size_t(m) * d * mp * sizeof(double), s);
            return cuda_fail(h, e, "memset");
        }
        return DMRG_OK;
    }
    const BwdDims B = bwd_dims(K, m, d, mp, p);
    st = check_ws(h, ws, ws_bytes, B.ws.total);
    if (st != DMRG_OK) return st;
    const bool tc = (p == DMRG_PREC_TF32 || p == DMRG_PREC_BF16X3);
    if (tc && !tc_supported(h))
        return fail(h, DMRG_ERR_UNSUPPORTED, "tensor-core precisions need an sm_103 GPU");
    char key[256];
    snprintf(key, sizeof key, "bwd:%p:%p:%p:%p:%p:%p:%p:%lld:%lld:%d:%lld:%d:%d", (const void*)U, O,
             G, dO, (void*)dU, ws, (void*)s, (long long)K, (long long)m, d, (long long)mp, int(p),
             in_is_fp64);
    return run_maybe_graph(h, key, s, [&](cudaStream_t cs) -> dmrg_status {
        if (tc) return bwd_tc(h, U, O, G, in_is_fp64, dO, dU, B, p, ws, cs);
        return bwd_simt(h, U, O, G, in_is_fp64, dO, dU, B, p, ws, cs);
    });
}

}  // extern "C"
