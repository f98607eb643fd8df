// api.cu -- C ABI of the library (declared in include/dmrg_rotate.h): handle,
// argument checks, workspace layout and the dense forward rotation
//   O'_k = U^T (O_k (x) I_d) U        (Sec. 2 step 5; two products of Sec. 3.2).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "api_common.h"
#include "internal.h"

using namespace dmrg;

namespace dmrg {

dmrg_status fail(dmrg_handle h, dmrg_status st, const std::string& msg) {
    if (h) h->last_error = msg;
    return st;
}

dmrg_status cuda_fail(dmrg_handle h, cudaError_t e, const char* where) {
    if (e == cudaSuccess) return DMRG_OK;
    return fail(h, DMRG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

cudaEvent_t pooled_event(dmrg_handle h) {
    if (!h->event_pool.empty()) {
        cudaEvent_t e = h->event_pool.back();
        h->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

cudaError_t timed_launch(dmrg_handle h, const char* name, cudaStream_t s,
                         const std::function<cudaError_t()>& f) {
    if (!h->timing || h->capturing) return f();
    cudaEvent_t a = pooled_event(h), b = pooled_event(h);
    cudaEventRecord(a, s);
    cudaError_t e = f();
    cudaEventRecord(b, s);
    h->pending.push_back({name, a, b});
    return e;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

void WsLayout::add(const char* name, size_t bytes) {
    (void)name;
    offsets.push_back(total);
    total = align_up(total + align_up(bytes, 256), 256);
}

bool tc_supported(dmrg_handle h) { return h->cc_major == 10 && h->cc_minor == 3; }

uint64_t timeout_ns(dmrg_handle h) {
    double ms = h->wait_timeout_ms;
    if (!(ms > 0)) ms = 2000.0;
    return uint64_t(ms * 1e6);
}

int take_drop_arrival(dmrg_handle h) {
    const int v = h->drop_arrival_next;
    h->drop_arrival_next = 0;
    return v;
}

// Runs `body` directly, or (graph mode) captures it once per key into a CUDA
// graph on the handle's private stream and replays the graph on `stream`.
dmrg_status run_maybe_graph(dmrg_handle h, const std::string& key, cudaStream_t stream,
                            const std::function<dmrg_status(cudaStream_t)>& body) {
    if (!h->graph_mode) return body(stream);
    auto it = h->graphs.find(key);
    if (it == h->graphs.end()) {
        if (!h->capture_stream) {
            cudaError_t e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamCreate");
        }
        cudaError_t e = cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamBeginCapture");
        h->capturing = true;
        dmrg_status st = body(h->capture_stream);
        h->capturing = false;
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(h->capture_stream, &g);
        if (st != DMRG_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
        it = h->graphs.emplace(key, ex).first;
    }
    return cuda_fail(h, cudaGraphLaunch(it->second, stream), "cudaGraphLaunch");
}

// ------------------------------------------------------------------ dense layout
DenseDims dense_dims(int64_t K, int64_t m, int d, int64_t mp, dmrg_precision p) {
    DenseDims D;
    D.K = K; D.m = m; D.d = d; D.mp = mp; D.md = m * d;
    const int64_t align = (p == DMRG_PREC_TF32) ? 4 : 8;
    D.ld1 = (m + align - 1) / align * align;
    D.ld2 = (D.md + align - 1) / align * align;
    const size_t es = (p == DMRG_PREC_TF32) ? 4 : 2;
    WsLayout& W = D.ws;
    // Sections that depend only on U come first, so that calls on slices of one
    // operator batch (the host-buffer pipeline) can share them.
    if (p == DMRG_PREC_FP64) {
        W.add("T", size_t(K) * D.md * mp * 8);
    } else if (p == DMRG_PREC_FP32) {
        W.add("U32", size_t(D.md) * mp * 4);
        W.add("O32", size_t(K) * m * m * 4);
        W.add("T", size_t(K) * D.md * mp * 4);
    } else {
        const int nsplit = (p == DMRG_PREC_BF16X3) ? 2 : 1;
        for (int s = 0; s < nsplit; ++s) W.add("B1", size_t(d) * mp * D.ld1 * es);
        for (int s = 0; s < nsplit; ++s) W.add("B2", size_t(mp) * D.ld2 * es);
        for (int s = 0; s < nsplit; ++s) W.add("Op", size_t(K) * m * D.ld1 * es);
        for (int s = 0; s < nsplit; ++s) W.add("T", size_t(K) * mp * D.ld2 * es);
        // running sums of chained accumulation (BF16x3 reductions longer than 512)
        W.add("chain", (p == DMRG_PREC_BF16X3 && D.md > kChainMinRed) ? kChainScratchBytes : 0);
    }
    return D;
}

dmrg_status check_dense_args(dmrg_handle h, int64_t K, int64_t m, int d, int64_t mp,
                             dmrg_precision p) {
    if (!h) return DMRG_ERR_INVALID_ARG;
    if (p < DMRG_PREC_FP64 || p > DMRG_PREC_BF16X3)
        return fail(h, DMRG_ERR_INVALID_ARG, "unknown precision");
    if (m < 1 || d < 1 || mp < 1 || K < 0)
        return fail(h, DMRG_ERR_SHAPE, "need m >= 1, d >= 1, mp >= 1, K >= 0");
    if (mp > m * d) return fail(h, DMRG_ERR_SHAPE, "mp must not exceed m*d");
    if (p == DMRG_PREC_TF32 || p == DMRG_PREC_BF16X3) {
        const int64_t lim = 0x7fffffffLL;
        if (m * d > lim || K * std::max(m, mp) > lim || int64_t(d) * mp > lim)
            return fail(h, DMRG_ERR_SHAPE, "sizes exceed the 32-bit tile index range");
    }
    return DMRG_OK;
}

TcConfig tuned_config(dmrg_handle h, const std::string& key, TcMode mode) {
    load_tune_file(h);
    auto it = h->tune_cache.find(key);
    if (it != h->tune_cache.end()) {
        TcConfig c = it->second;  // a cached depth that no longer fits is reduced
        c.stages = std::min(c.stages, tc_stages_for(mode, c));
        return c;
    }
    // Untuned default: 128-byte rows, N tiles up to 256, the deepest pipeline that
    // fits; the dense products and the adjoint's products run on CTA pairs (half of B
    // staged per SM).
    TcConfig c;
    c.tile_n_max = 256;
    c.row_bytes = 128;
    c.pair = (key.compare(0, 3, "g1:") == 0 || key.compare(0, 3, "g2:") == 0 ||
              key.compare(0, 4, "bwd:") == 0) ? 1 : 0;
    c.stages = tc_stages_for(mode, c);
    c.grid = 0;
    return c;
}

std::string shape_key(const char* tag, int64_t K, int64_t m, int d, int64_t mp, dmrg_precision p) {
    char buf[160];
    snprintf(buf, sizeof buf, "%s:K%lld:m%lld:d%d:mp%lld:p%d", tag, (long long)K, (long long)m, d,
             (long long)mp, int(p));
    return buf;
}

// Dense tensor-core forward with explicit tilings (the autotuner calls this directly).
dmrg_status dense_tc_forward(dmrg_handle h, const double* U, int64_t m, int d, int64_t mp,
                             const void* O, int in_is_fp64, int64_t K, void* Oout,
                             dmrg_precision p, void* ws, const TcConfig& c1_in,
                             const TcConfig& c2_in, cudaStream_t s, bool pack_u, const double* U1,
                             const FirstClasses* cls) {
    const DenseDims D = dense_dims(K, m, d, mp, p);
    // Only the CTA-pair kernel cuts long BF16x3 reductions into accumulation chains, so
    // a product whose reduction is longer than one chain runs on CTA pairs whatever
    // tiling was tuned or cached (the 1e-5 accuracy of BF16x3 depends on the chains).
    TcConfig c1 = c1_in, c2 = c2_in;
    if (p == DMRG_PREC_BF16X3) {
        const int64_t one_chain = std::max<int64_t>(kChainMinRed, h->accum_chain);
        TcConfig* cs[2] = {&c1, &c2};
        const int64_t red[2] = {m, D.md};
        for (int i = 0; i < 2; ++i) {
            if (red[i] > one_chain && !cs[i]->pair) {
                cs[i]->pair = 1;
                cs[i]->stages = tc_stages_for(TC_BF16X3, *cs[i]);
            }
        }
    }
    if (cls && (cls->n < 1 || cls->n > kMaxInlineProblems || (!cls->U1 && !cls->b1_ready) || !pack_u))
        return fail(h, DMRG_ERR_INVALID_ARG, "bad operator classes");
    const bool split = (p == DMRG_PREC_BF16X3);
    const TcMode mode = split ? TC_BF16X3 : TC_TF32;
    const int pmode = split ? 0 : 1;
    char* base = static_cast<char*>(ws);
    int si = 0;
    void* Op[2] = {nullptr, nullptr};
    void* B1[2] = {nullptr, nullptr};
    void* B2[2] = {nullptr, nullptr};
    void* Tt[2] = {nullptr, nullptr};
    const int ns = split ? 2 : 1;
    for (int i = 0; i < ns; ++i) B1[i] = base + D.ws.offsets[si++];
    for (int i = 0; i < ns; ++i) B2[i] = base + D.ws.offsets[si++];
    for (int i = 0; i < ns; ++i) Op[i] = base + D.ws.offsets[si++];
    for (int i = 0; i < ns; ++i) Tt[i] = base + D.ws.offsets[si++];
    // Chained accumulation (CTA-pair kernel, BF16x3): reductions longer than the handle's
    // chain length are cut into chains summed in FP32 through a per-CTA scratch.
    float* chain_scr =
        (split && D.md > kChainMinRed) ? reinterpret_cast<float*>(base + D.ws.offsets[si]) : nullptr;
    auto chain_kb = [&](const TcConfig& c, int64_t red, int grid) -> int {
        if (!chain_scr || !c.pair || h->accum_chain <= 0 || red <= h->accum_chain ||
            grid > kChainScratchCtas)
            return 0;
        const int64_t epr = c.row_bytes / 2;   // BF16 elements per k-block
        return int(std::max<int64_t>(1, h->accum_chain / epr));
    };

    // ---- second product's problem first: its split tail decides which outputs the
    //      packing launch clears.  O'_k^T rows = T_all rows (k*mp + b), columns a.
    TcLaunch L2{};
    TcProblem& P2 = L2.inline_prob[0];
    {
        TcOperand A{Tt[0], Tt[1], K * mp, D.md, D.ld2};
        TcOperand B{B2[0], B2[1], mp, D.md, D.ld2};
        if (!make_problem(P2, mode, A, B, c2.tile_n_max, 1, c2.row_bytes, c2.pair))
            return fail(h, DMRG_ERR_CUDA, "cuTensorMapEncodeTiled failed (second product)");
    }
    TcScatter& S2 = P2.sc[0];
    S2.rows_per_op = int32_t(mp);
    S2.s_op = mp * mp;
    S2.s_row = 1;
    S2.col_div = 1;
    S2.s_col_hi = mp;
    S2.s_col_lo = 0;
    L2.table = nullptr;
    L2.nprob = 1;
    L2.total_tiles = P2.m_tiles * P2.n_tiles * P2.k_splits;
    L2.out[0][0] = Oout;
    const int grid2 = c2.grid > 0 ? c2.grid : h->num_sms;
    P2.kb_chunk = chain_kb(c2, D.md, grid2);
    // Up to two chains per tile are summed in the FP32 output itself (the first chain
    // stores, the second adds with reductions): 0.161 -> 0.156 ms against the scratch at
    // m = m' = 400, d = 4, K = 150.  More chains go through the scratch: at m = m' = 1200
    // (five chains) the reductions made the step 3 % slower.
    {
        const int64_t epr = c2.row_bytes / (split ? 2 : 4);
        const int64_t kb = (D.md + epr - 1) / epr;
        const int64_t chains = P2.kb_chunk > 0 ? (kb + P2.kb_chunk - 1) / P2.kb_chunk : 1;
        L2.chunk_scratch = chains > 2 ? chain_scr : nullptr;
    }
    // summed in the output: O' leaves by TMA bulk stores, the second chain (and the parts
    // of split tiles) by TMA reductions, staged per warp in shared memory
    if (c2.pair && h->store_epilogue == 0 && L2.chunk_scratch == nullptr && mp % 16 == 0 &&
        encode_store_map(&L2.t_store_map[0], Oout, mp, mp, K, mp, 16, 16, 0, true))
        L2.t_store = kStoreColumnsF32;
    int64_t k_clear = K;   // outputs k >= k_clear are accumulated atomically: cleared first
    // Tail wave: the tiles left after the last full wave over the persistent CTAs (or
    // CTA pairs) are whole M tiles whose reduction is split so the last round is short;
    // a problem smaller than one wave is split as a whole.  The parts accumulate with
    // atomics into outputs cleared first (so the summation order of those outputs may
    // differ between runs; DMRG_OPT_DETERMINISTIC turns the split off).
    {
        const int slots = c2.pair ? grid2 / 2 : grid2;
        const int bm = c2.pair ? 256 : 128;
        const int tiles = P2.m_tiles * P2.n_tiles;
        const int full_mt = (tiles / slots) * slots / P2.n_tiles;
        const int tail_mt = P2.m_tiles - full_mt;
        const int64_t epr = c2.row_bytes / (split ? 2 : 4);   // reduction elements per k-block
        const int kb = int((D.md + epr - 1) / epr);
        const int parts = tail_mt > 0 ? std::min(kb, slots / (tail_mt * P2.n_tiles)) : 0;
        if (!h->deterministic && tail_mt > 0 && parts >= 2) {
            TcProblem& T2 = L2.inline_prob[1];
            T2 = P2;
            P2.m_tiles = full_mt;
            T2.m_tile0 = full_mt;
            T2.m_tiles = tail_mt;
            T2.kb_per_split = (kb + parts - 1) / parts;
            T2.k_splits = (kb + T2.kb_per_split - 1) / T2.kb_per_split;
            T2.atomic = 1;
            T2.tile_start = P2.m_tiles * P2.n_tiles;
            L2.nprob = 2;
            L2.total_tiles = T2.tile_start + T2.m_tiles * T2.n_tiles * T2.k_splits;
            k_clear = int64_t(full_mt) * bm / mp;
        }
    }

    // ---- FP32 operators with 16-byte rows feed the first product as they are: the
    //      CTA-pair kernel converts each tile in shared memory, so O is not packed.
    //      Each A tile is converted once per N tile, so this pays only when the first
    //      product has few N tiles (measured: BF16x3 wins at d*m' <= 512, loses at 1600;
    //      TF32, with half as many MMA cycles per converted byte, loses everywhere).
    const int n1_tile = std::max(32, choose_tile_n(int64_t(d) * mp, c1.tile_n_max));
    const int64_t n1_tiles = (int64_t(d) * mp + n1_tile - 1) / n1_tile;
    const bool can_convert = !in_is_fp64 && (m % 4) == 0 &&
                             (reinterpret_cast<uintptr_t>(O) & 15) == 0 && c1.pair &&
                             c1.row_bytes == 128;
    const bool convert_a = can_convert && (h->pack_operators == 2 ||
                                           (h->pack_operators == 0 && split && n1_tiles <= 2));

    // ---- operand packing: O (stacked K*m x m) unless converted in the first product,
    //      U_r' (rows b*d + s, cols j), U^T, and the clearing of the split tail's outputs,
    //      in one launch (the two small U gathers run alongside the O stream).
    PackJob jobs[4] = {};
    int nj = 0;
    if (!convert_a) {
        PackJob& jo = jobs[nj++];
        jo.src = O; jo.src_f64 = in_is_fp64; jo.mode = pmode;
        jo.rows = K * m; jo.cols = m; jo.rows_per_op = K * m; jo.s_op = 0; jo.op_off = nullptr;
        jo.rdiv = 1; jo.s_r_hi = m; jo.s_r_lo = 0; jo.s_c = 1;
        jo.dst0 = Op[0]; jo.dst1 = Op[1]; jo.ld = D.ld1;
    }
    if (pack_u) {
        if (!(cls && cls->b1_ready)) {
            PackJob& j1 = jobs[nj++];
            j1.src = U1 ? U1 : U; j1.src_f64 = 1; j1.mode = pmode;
            j1.rows = int64_t(d) * mp; j1.cols = m; j1.rows_per_op = j1.rows;
            j1.rdiv = d; j1.s_r_hi = 1; j1.s_r_lo = mp; j1.s_c = int64_t(d) * mp;
            j1.dst0 = B1[0]; j1.dst1 = B1[1]; j1.ld = D.ld1;
            if (cls) {   // the classes' U1_c, stacked
                j1.src = cls->U1;
                j1.rows = int64_t(cls->n) * d * mp;
                j1.s_op = m * d * mp;
                j1.dst0 = cls->b1[0]; j1.dst1 = cls->b1[1];
            }
        }
        PackJob& j2 = jobs[nj++];
        j2.src = U; j2.src_f64 = 1; j2.mode = pmode;
        j2.rows = mp; j2.cols = D.md; j2.rows_per_op = mp;
        j2.rdiv = 1; j2.s_r_hi = 1; j2.s_r_lo = 0; j2.s_c = mp;
        j2.dst0 = B2[0]; j2.dst1 = B2[1]; j2.ld = D.ld2;
    }
    if (k_clear < K) {
        PackJob& jz = jobs[nj++];
        jz.mode = kPackZero;
        jz.rows = 1; jz.cols = (K - k_clear) * mp * mp; jz.rows_per_op = 1; jz.rdiv = 1;
        jz.dst0 = static_cast<float*>(Oout) + k_clear * mp * mp; jz.ld = jz.cols;
    }
    cudaError_t e = cudaSuccess;
    if (nj > 0) {
        e = timed_launch(h, convert_a ? "pack_u" : "pack_operands", s,
                         [&] { return pack_launch(jobs, nj, nullptr, s); });
        if (e != cudaSuccess) return cuda_fail(h, e, "pack");
    }

    // ---- first product: T = O U_r, written straight into the second product's
    //      K-major operand layout: T_all[k*mp + b][i*d + s].
    TcLaunch L1{};
    const int nprob1 = cls ? cls->n : 1;
    const size_t es = split ? 2 : 4;
    const int grid1 = c1.grid > 0 ? c1.grid : h->num_sms;
    L1.total_tiles = 0;
    for (int c = 0; c < nprob1; ++c) {
        TcProblem& P1 = L1.inline_prob[c];
        const int64_t k0 = cls ? cls->k0[c] : 0, kc = cls ? cls->kc[c] : K;
        const size_t a_off = size_t(k0) * m * D.ld1 * es;
        const size_t b_off = cls ? size_t(c) * d * mp * D.ld1 * es : 0;
        void* const* bsrc = cls ? cls->b1 : B1;
        TcOperand A{static_cast<char*>(Op[0]) + a_off, Op[1] ? static_cast<char*>(Op[1]) + a_off : nullptr,
                    kc * m, m, D.ld1};
        if (convert_a) {
            A.hi = static_cast<const float*>(O) + k0 * m * m;
            A.lo = nullptr;
            A.ld = m;
            A.f32_source = 1;
        }
        TcOperand B{static_cast<char*>(bsrc[0]) + b_off,
                    bsrc[1] ? static_cast<char*>(bsrc[1]) + b_off : nullptr, int64_t(d) * mp, m, D.ld1};
        if (!make_problem(P1, mode, A, B, c1.tile_n_max, 1, c1.row_bytes, c1.pair))
            return fail(h, DMRG_ERR_CUDA, "cuTensorMapEncodeTiled failed (first product)");
        TcScatter& S1 = P1.sc[0];
        S1.out_off = k0 * mp * D.ld2;
        S1.rows_per_op = int32_t(m);
        S1.s_op = mp * D.ld2;
        S1.s_row = d;
        S1.col_div = d;
        S1.s_col_hi = D.ld2;
        S1.s_col_lo = 1;
        P1.tile_start = L1.total_tiles;
        P1.kb_chunk = chain_kb(c1, m, grid1);
        L1.total_tiles += P1.m_tiles * P1.n_tiles * P1.k_splits;
    }
    L1.table = nullptr;
    L1.nprob = nprob1;
    L1.out[0][0] = Tt[0];
    L1.out[0][1] = Tt[1];
    L1.status = h->d_status;
    L1.timeout_ns = timeout_ns(h);
    L1.drop_arrival = take_drop_arrival(h);
    L1.row_bytes = c1.row_bytes;
    L1.chunk_scratch = L1.inline_prob[0].kb_chunk ? chain_scr : nullptr;
    L1.convert_a = convert_a ? 1 : 0;
    // On CTA pairs T leaves through TMA bulk stores (staged per warp in shared memory)
    // rather than stores from registers, where the layout allows it (BF16 hi and lo, or
    // the TF32-rounded FP32 T)
    if (c1.pair && h->store_epilogue == 0 && (d == 2 || d == 4) && m % 16 == 0) {
        bool ok = true;
        for (int c = 0; c < (split ? 2 : 1) && ok; ++c)
            ok = encode_store_map(&L1.t_store_map[c], Tt[c], D.md, mp, K, D.ld2, 16 * d, 32 / d, 0,
                                  !split);
        if (ok) {
            L1.t_store = kStoreSiteInterleaved;
            L1.t_store_d = d;
            for (int c = 0; c < nprob1; ++c) L1.inline_prob[c].store_z0 = int32_t(cls ? cls->k0[c] : 0);
        }
    }
    // The packing pass wrote the operators in row order and the rows it wrote last are
    // the ones still in L2: the first product starts from the last M tile.  It then leaves
    // the first operators' T rows in L2 for the second product, which starts there.
    L1.reverse_m = convert_a ? 0 : 1;
    e = timed_launch(h, "tc_gemm_first_product", s, [&] {
        const TcEpi epi = split ? EPI_SPLIT_BF16 : EPI_TF32;
        return c1.pair ? tc_gemm_launch_pair(mode, epi, L1, c1.stages, grid1, s)
                       : tc_gemm_launch(mode, epi, L1, c1.stages, grid1, s);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "first product");

    L2.status = h->d_status;
    L2.timeout_ns = timeout_ns(h);
    L2.row_bytes = c2.row_bytes;
    e = timed_launch(h, "tc_gemm_second_product", s, [&] {
        return c2.pair ? tc_gemm_launch_pair(mode, EPI_F32, L2, c2.stages, grid2, s)
                       : tc_gemm_launch(mode, EPI_F32, L2, c2.stages, grid2, s);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "second product");
    return DMRG_OK;
}

// Both products in one kernel (BF16x3, mp <= kFusedMaxMp).  It uses the dense
// workspace's sections for the packed U_r (whose size fits the packed Pu) and O.
dmrg_status dense_fused_forward(dmrg_handle h, const double* U, int64_t m, int d, int64_t mp,
                                const void* O, int in_is_fp64, int64_t K, void* Oout, void* ws,
                                cudaStream_t s) {
    const DenseDims D = dense_dims(K, m, d, mp, DMRG_PREC_BF16X3);
    char* base = static_cast<char*>(ws);
    void* Pu[2] = {base + D.ws.offsets[0], base + D.ws.offsets[1]};   // "B1" sections
    void* Op[2] = {base + D.ws.offsets[4], base + D.ws.offsets[5]};   // "Op" sections
    PackJob jobs[2] = {};
    PackJob& jo = jobs[0];
    jo.src = O; jo.src_f64 = in_is_fp64; jo.mode = 0;
    jo.rows = K * m; jo.cols = m; jo.rows_per_op = K * m; jo.s_op = 0; jo.op_off = nullptr;
    jo.rdiv = 1; jo.s_r_hi = m; jo.s_r_lo = 0; jo.s_c = 1;
    jo.dst0 = Op[0]; jo.dst1 = Op[1]; jo.ld = D.ld1;
    // Pu row s*mp + x, column j  <-  U[(j d + s) mp + x]
    PackJob& ju = jobs[1];
    ju.src = U; ju.src_f64 = 1; ju.mode = 0;
    ju.rows = int64_t(d) * mp; ju.cols = m; ju.rows_per_op = mp; ju.s_op = mp; ju.op_off = nullptr;
    ju.rdiv = 1; ju.s_r_hi = 1; ju.s_r_lo = 0; ju.s_c = int64_t(d) * mp;
    ju.dst0 = Pu[0]; ju.dst1 = Pu[1]; ju.ld = D.ld1;
    cudaError_t e = timed_launch(h, "pack_operands", s,
                                 [&] { return pack_launch(jobs, 2, nullptr, s); });
    if (e != cudaSuccess) return cuda_fail(h, e, "pack");
    FusedArgs a{};
    a.Op[0] = Op[0]; a.Op[1] = Op[1];
    a.Pu[0] = Pu[0]; a.Pu[1] = Pu[1];
    a.out = static_cast<float*>(Oout);
    a.K = K; a.m = m; a.mp = mp; a.ld = D.ld1; a.d = d;
    a.grid = h->num_sms;
    a.accum_chain = h->accum_chain;
    a.status = h->d_status;
    a.timeout_ns = timeout_ns(h);
    e = timed_launch(h, "tc_fused_rotation", s, [&] { return fused_rotate_launch(a, s); });
    if (e != cudaSuccess) return cuda_fail(h, e, "fused rotation");
    return DMRG_OK;
}

dmrg_status dense_simt_forward(dmrg_handle h, const double* U, int64_t m, int d, int64_t mp,
                               const void* O, int in_is_fp64, int64_t K, void* Oout,
                               dmrg_precision p, void* ws, cudaStream_t s, bool pack_u,
                               const double* U1, float* U1_32) {
    const DenseDims D = dense_dims(K, m, d, mp, p);
    char* base = static_cast<char*>(ws);
    const bool f64 = (p == DMRG_PREC_FP64);
    const void* Ouse = O;
    const void* Uuse = U;
    const void* U1use = U1 ? U1 : U;
    void* T = nullptr;
    cudaError_t e = cudaSuccess;
    if (f64) {
        T = base + D.ws.offsets[0];
    } else {
        float* U32 = reinterpret_cast<float*>(base + D.ws.offsets[0]);
        float* O32 = reinterpret_cast<float*>(base + D.ws.offsets[1]);
        T = base + D.ws.offsets[2];
        if (U1 && !U1_32) return fail(h, DMRG_ERR_INVALID_ARG, "FP32 path needs a scratch for U1");
        PackJob jobs[3] = {};
        int nj = 0;
        if (in_is_fp64) {
            PackJob& j = jobs[nj++];
            j.src = O; j.src_f64 = 1; j.mode = 2; j.rows = K * m; j.cols = m; j.rows_per_op = K * m;
            j.rdiv = 1; j.s_r_hi = m; j.s_c = 1; j.dst0 = O32; j.ld = m;
            Ouse = O32;
        }
        if (pack_u) {
            PackJob& j = jobs[nj++];
            j.src = U; j.src_f64 = 1; j.mode = 2; j.rows = D.md; j.cols = mp; j.rows_per_op = D.md;
            j.rdiv = 1; j.s_r_hi = mp; j.s_c = 1; j.dst0 = U32; j.ld = mp;
        }
        Uuse = U32;
        U1use = U32;
        if (U1) {
            PackJob& j = jobs[nj++];
            j.src = U1; j.src_f64 = 1; j.mode = 2; j.rows = D.md; j.cols = mp; j.rows_per_op = D.md;
            j.rdiv = 1; j.s_r_hi = mp; j.s_c = 1; j.dst0 = U1_32; j.ld = mp;
            U1use = U1_32;
        }
        if (nj > 0) {
            e = timed_launch(h, "convert_fp32", s, [&] { return pack_launch(jobs, nj, nullptr, s); });
            if (e != cudaSuccess) return cuda_fail(h, e, "convert");
        }
    }
    const Real rt = f64 ? Real::F64 : Real::F32;
    // First product: T_k (m x d*mp) = O_k (m x m) * U_r (m x d*mp).
    SimtGemm g1{};
    g1.A = Ouse; g1.B = U1use; g1.C = T;
    g1.M = m; g1.N = int64_t(d) * mp; g1.K = m;
    g1.sAb = m * m; g1.sAi = m; g1.sAk = 1;
    g1.sBb = 0; g1.sBk = int64_t(d) * mp; g1.sBj = 1;
    g1.sCb = D.md * mp; g1.sCi = int64_t(d) * mp; g1.sCj = 1;
    g1.batch = int32_t(K);
    e = timed_launch(h, "simt_gemm_first_product", s, [&] { return simt_gemm_launch(rt, g1, s); });
    if (e != cudaSuccess) return cuda_fail(h, e, "first product");
    // Second product: O'_k (mp x mp) = U^T (mp x md) * T_k (md x mp).
    SimtGemm g2{};
    g2.A = Uuse; g2.B = T; g2.C = Oout;
    g2.M = mp; g2.N = mp; g2.K = D.md;
    g2.sAb = 0; g2.sAi = 1; g2.sAk = mp;
    g2.sBb = D.md * mp; g2.sBk = mp; g2.sBj = 1;
    g2.sCb = mp * mp; g2.sCi = mp; g2.sCj = 1;
    g2.batch = int32_t(K);
    e = timed_launch(h, "simt_gemm_second_product", s, [&] { return simt_gemm_launch(rt, g2, s); });
    if (e != cudaSuccess) return cuda_fail(h, e, "second product");
    return DMRG_OK;
}

dmrg_status check_ws(dmrg_handle h, const void* ws, size_t have, size_t need) {
    if (need == 0) return DMRG_OK;
    if (!ws || have < need) {
        char b[128];
        snprintf(b, sizeof b, "workspace too small: need %zu bytes, got %zu", need, have);
        return fail(h, DMRG_ERR_WORKSPACE, b);
    }
    if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0)
        return fail(h, DMRG_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    return DMRG_OK;
}

}  // namespace dmrg

// =================================================================== C ABI
extern "C" {

const char* dmrg_status_string(dmrg_status s) {
    switch (s) {
        case DMRG_OK: return "DMRG_OK";
        case DMRG_ERR_INVALID_ARG: return "DMRG_ERR_INVALID_ARG";
        case DMRG_ERR_SHAPE: return "DMRG_ERR_SHAPE";
        case DMRG_ERR_NOT_ORTHONORMAL: return "DMRG_ERR_NOT_ORTHONORMAL";
        case DMRG_ERR_WORKSPACE: return "DMRG_ERR_WORKSPACE";
        case DMRG_ERR_CUDA: return "DMRG_ERR_CUDA";
        case DMRG_ERR_TIMEOUT: return "DMRG_ERR_TIMEOUT";
        case DMRG_ERR_UNSUPPORTED: return "DMRG_ERR_UNSUPPORTED";
    }
    return "DMRG_ERR_UNKNOWN";
}

const char* dmrg_last_error(dmrg_handle h) { return h ? h->last_error.c_str() : ""; }

dmrg_status dmrg_create(dmrg_handle* out) {
    if (!out) return DMRG_ERR_INVALID_ARG;
    *out = nullptr;
    dmrg_handle h = new dmrg_handle_s();
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->cc_major, cudaDevAttrComputeCapabilityMajor, h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->cc_minor, cudaDevAttrComputeCapabilityMinor, h->device);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&h->d_status), 256);
    if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, 256);
    if (e != cudaSuccess) {
        if (h->d_status) cudaFree(h->d_status);
        delete h;
        return DMRG_ERR_CUDA;
    }
    h->d_scratch = reinterpret_cast<double*>(reinterpret_cast<char*>(h->d_status) + 64);
    *out = h;
    return DMRG_OK;
}

dmrg_status dmrg_destroy(dmrg_handle h) {
    if (!h) return DMRG_ERR_INVALID_ARG;
    for (auto& t : h->pending) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (auto ev : h->event_pool) cudaEventDestroy(ev);
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.second);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    if (h->copy_in) cudaStreamDestroy(h->copy_in);
    if (h->copy_out) cudaStreamDestroy(h->copy_out);
    if (h->compute2) cudaStreamDestroy(h->compute2);
    for (cudaEvent_t ev : {h->ev_start, h->ev_u, h->ev_in[0], h->ev_in[1], h->ev_comp[0],
                           h->ev_comp[1], h->ev_out[0], h->ev_out[1]})
        if (ev) cudaEventDestroy(ev);
    if (h->d_status) cudaFree(h->d_status);
    delete h;
    return DMRG_OK;
}

dmrg_status dmrg_set_option(dmrg_handle h, dmrg_option o, double v) {
    if (!h) return DMRG_ERR_INVALID_ARG;
    switch (o) {
        case DMRG_OPT_GRAPH: h->graph_mode = v != 0; return DMRG_OK;
        case DMRG_OPT_KERNEL_TIMING: h->timing = v != 0; return DMRG_OK;
        case DMRG_OPT_WAIT_TIMEOUT_MS:
            if (!(v > 0)) return fail(h, DMRG_ERR_INVALID_ARG, "timeout must be > 0");
            h->wait_timeout_ms = v;
            return DMRG_OK;
        case DMRG_OPT_CHECK_ORTHO:
            if (v < 0) return fail(h, DMRG_ERR_INVALID_ARG, "tolerance must be >= 0");
            h->check_ortho_tol = v;
            return DMRG_OK;
        case DMRG_OPT_DETERMINISTIC:
            h->deterministic = v != 0;
            return DMRG_OK;
        case DMRG_OPT_ACCUM_CHAIN:
            // Longer chains (or one chain per tile) let the tensor core's FP32 accumulation
            // error of the BF16x3 products exceed 1e-5 at m*d = 4800 (2.05e-5 measured with
            // one chain), so they are refused.
            if (!(v >= 1 && v <= kMaxAccumChain))
                return fail(h, DMRG_ERR_INVALID_ARG, "accum_chain must be in [1, 1024]");
            h->accum_chain = int(v);
            return DMRG_OK;
        case DMRG_OPT_TRUNCATION_JACOBI:
            h->trunc_jacobi = v != 0;
            return DMRG_OK;
        case DMRG_OPT_BLOCKED_SMALL:
            h->blocked_small = v != 0;
            return DMRG_OK;
        case DMRG_OPT_PACK_OPERATORS:
            if (!(v == 0 || v == 1 || v == 2))
                return fail(h, DMRG_ERR_INVALID_ARG, "pack_operators must be 0, 1 or 2");
            h->pack_operators = int(v);
            return DMRG_OK;
        case DMRG_OPT_STORE_EPILOGUE:
            if (!(v == 0 || v == 1))
                return fail(h, DMRG_ERR_INVALID_ARG, "store_epilogue must be 0 or 1");
            h->store_epilogue = int(v);
            return DMRG_OK;
        case DMRG_OPT_FUSED_ROTATION:
            if (!(v == 0 || v == 1))
                return fail(h, DMRG_ERR_INVALID_ARG, "fused_rotation must be 0 or 1");
            h->fused_rotation = int(v);
            return DMRG_OK;
        case DMRG_OPT_TEST_WITHHOLD_ARRIVAL:
            h->drop_arrival_next = v != 0;
            return DMRG_OK;
    }
    return fail(h, DMRG_ERR_INVALID_ARG, "unknown option");
}

dmrg_status dmrg_sync_status(dmrg_handle h, dmrg_stream_t stream) {
    if (!h) return DMRG_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    unsigned st = 0;
    e = cudaMemcpy(&st, h->d_status, sizeof st, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "status read");
    if (st != 0) {
        cudaMemset(h->d_status, 0, sizeof st);
        return fail(h, DMRG_ERR_TIMEOUT, "a device-side bounded wait expired");
    }
    return DMRG_OK;
}

dmrg_status dmrg_kernel_timing(dmrg_handle h, char* buf, size_t len, int reset) {
    if (!h || !buf || len == 0) return DMRG_ERR_INVALID_ARG;
    for (auto& t : h->pending) {
        cudaEventSynchronize(t.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t.a, t.b);
        auto& acc = h->timing_acc[t.name];
        acc.first += 1;
        acc.second += ms;
        h->event_pool.push_back(t.a);
        h->event_pool.push_back(t.b);
    }
    h->pending.clear();
    std::string js = "[";
    bool first = true;
    for (auto& kv : h->timing_acc) {
        char b[256];
        snprintf(b, sizeof b, "%s{\"kernel\": \"%s\", \"launches\": %ld, \"total_ms\": %.6f}",
                 first ? "" : ", ", kv.first.c_str(), kv.second.first, kv.second.second);
        js += b;
        first = false;
    }
    js += "]";
    if (reset) h->timing_acc.clear();
    if (js.size() + 1 > len) return fail(h, DMRG_ERR_INVALID_ARG, "timing buffer too small");
    memcpy(buf, js.c_str(), js.size() + 1);
    return DMRG_OK;
}

dmrg_status dmrg_rotate_ops_workspace(dmrg_handle h, int64_t K, int64_t m, int d, int64_t mp,
                                      dmrg_precision p, size_t* bytes) {
    if (!bytes) return fail(h, DMRG_ERR_INVALID_ARG, "bytes is NULL");
    dmrg_status st = check_dense_args(h, K, m, d, mp, p);
    if (st != DMRG_OK) return st;
    *bytes = dense_dims(K, m, d, mp, p).ws.total;
    return DMRG_OK;
}

dmrg_status dmrg_rotate_ops(dmrg_handle h, const double* U, int64_t m, int d, int64_t mp,
                            const void* O, int in_is_fp64, int64_t K, void* Oout,
                            dmrg_precision p, void* ws, size_t ws_bytes, dmrg_stream_t stream) {
    dmrg_status st = check_dense_args(h, K, m, d, mp, p);
    if (st != DMRG_OK) return st;
    if (K == 0) return DMRG_OK;
    if (!U || !O || !Oout) return fail(h, DMRG_ERR_INVALID_ARG, "null data pointer");
    if (p == DMRG_PREC_FP64 && !in_is_fp64)
        return fail(h, DMRG_ERR_INVALID_ARG, "the FP64 precision needs FP64 operators");
    const DenseDims D = dense_dims(K, m, d, mp, p);
    st = check_ws(h, ws, ws_bytes, D.ws.total);
    if (st != DMRG_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool tc = (p == DMRG_PREC_TF32 || p == DMRG_PREC_BF16X3);
    if (tc && !tc_supported(h))
        return fail(h, DMRG_ERR_UNSUPPORTED, "tensor-core precisions need an sm_103 GPU");
    if (h->check_ortho_tol > 0) {
        cudaError_t e = ortho_error_launch(U, D.md, mp, h->d_scratch, h->d_scratch + 1, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "orthonormality check");
        double err = 0;
        e = cudaMemcpyAsync(&err, h->d_scratch + 1, sizeof err, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(h, e, "orthonormality check");
        if (!(err <= h->check_ortho_tol)) {
            char b[128];
            snprintf(b, sizeof b, "||U^T U - I||_F = %.3e exceeds %.3e", err, h->check_ortho_tol);
            return fail(h, DMRG_ERR_NOT_ORTHONORMAL, b);
        }
    }
    // the options that change the launches are part of the key
    char key[256];
    snprintf(key, sizeof key, "dense:%p:%p:%p:%p:%p:%lld:%lld:%d:%lld:%d:%d:%d%d%d%d:%d", (const void*)U,
             O, Oout, ws, (void*)s, (long long)K, (long long)m, d, (long long)mp, int(p), in_is_fp64,
             int(h->deterministic), h->pack_operators, h->fused_rotation, h->store_epilogue,
             h->accum_chain);
    return run_maybe_graph(h, key, s, [&](cudaStream_t cs) -> dmrg_status {
        if (!tc) return dense_simt_forward(h, U, m, d, mp, O, in_is_fp64, K, Oout, p, ws, cs, true);
        if (h->fused_rotation && p == DMRG_PREC_BF16X3 && mp <= kFusedMaxMp)
            return dense_fused_forward(h, U, m, d, mp, O, in_is_fp64, K, Oout, ws, cs);
        const TcMode mode = (p == DMRG_PREC_BF16X3) ? TC_BF16X3 : TC_TF32;
        const TcConfig c1 = tuned_config(h, shape_key("g1", K, m, d, mp, p), mode);
        const TcConfig c2 = tuned_config(h, shape_key("g2", K, m, d, mp, p), mode);
        return dense_tc_forward(h, U, m, d, mp, O, in_is_fp64, K, Oout, p, ws, c1, c2, cs, true);
    });
}

dmrg_status dmrg_orthonormality_error_workspace(dmrg_handle h, int64_t rows, int64_t mp,
                                                size_t* bytes) {
    if (!h || !bytes) return DMRG_ERR_INVALID_ARG;
    if (rows < 1 || mp < 1) return fail(h, DMRG_ERR_SHAPE, "need rows >= 1 and mp >= 1");
    *bytes = 256;
    return DMRG_OK;
}

dmrg_status dmrg_orthonormality_error(dmrg_handle h, const double* U, int64_t rows, int64_t mp,
                                      double* out, void* ws, size_t ws_bytes,
                                      dmrg_stream_t stream) {
    if (!h) return DMRG_ERR_INVALID_ARG;
    if (rows < 1 || mp < 1) return fail(h, DMRG_ERR_SHAPE, "need rows >= 1 and mp >= 1");
    if (!U || !out) return fail(h, DMRG_ERR_INVALID_ARG, "null pointer");
    dmrg_status st = check_ws(h, ws, ws_bytes, 256);
    if (st != DMRG_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    double* acc = static_cast<double*>(ws);
    cudaError_t e = timed_launch(h, "ortho_error", s,
                                 [&] { return ortho_error_launch(U, rows, mp, acc, out, s); });
    return cuda_fail(h, e, "orthonormality error");
}

dmrg_status dmrg_correlations_workspace(dmrg_handle h, int64_t K, int64_t mp, size_t* bytes) {
    if (!h || !bytes) return DMRG_ERR_INVALID_ARG;
    if (K < 0 || mp < 1) return fail(h, DMRG_ERR_SHAPE, "need K >= 0 and mp >= 1");
    WsLayout W;
    W.add("x", size_t(K) * mp * 8);
    W.add("y", size_t(K) * mp * 8);
    *bytes = W.total;
    return DMRG_OK;
}

dmrg_status dmrg_correlations(dmrg_handle h, const void* Op, int in_is_fp64, const double* psi,
                              int64_t K, int64_t mp, double* C, void* ws, size_t ws_bytes,
                              dmrg_stream_t stream) {
    if (!h) return DMRG_ERR_INVALID_ARG;
    if (K < 0 || mp < 1) return fail(h, DMRG_ERR_SHAPE, "need K >= 0 and mp >= 1");
    if (K == 0) return DMRG_OK;
    if (!Op || !psi || !C) return fail(h, DMRG_ERR_INVALID_ARG, "null pointer");
    WsLayout W;
    W.add("x", size_t(K) * mp * 8);
    W.add("y", size_t(K) * mp * 8);
    dmrg_status st = check_ws(h, ws, ws_bytes, W.total);
    if (st != DMRG_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    double* x = reinterpret_cast<double*>(static_cast<char*>(ws) + W.offsets[0]);
    double* y = reinterpret_cast<double*>(static_cast<char*>(ws) + W.offsets[1]);
    cudaError_t e = timed_launch(h, "corr_matvec", s, [&] {
        return corr_matvec_launch(Op, in_is_fp64 != 0, psi, K, mp, x, y, s);
    });
    if (e != cudaSuccess) return cuda_fail(h, e, "correlation mat-vecs");
    // C = X Y^T: C[i][j] = sum_g x[i][g] y[j][g]
    SimtGemm g{};
    g.A = x; g.B = y; g.C = C;
    g.M = K; g.N = K; g.K = mp;
    g.sAi = mp; g.sAk = 1;
    g.sBk = 1; g.sBj = mp;
    g.sCi = K; g.sCj = 1;
    g.batch = 1;
    e = timed_launch(h, "corr_gemm", s, [&] { return simt_gemm_launch(Real::F64, g, s); });
    return cuda_fail(h, e, "correlation contraction");
}

}  // extern "C"
