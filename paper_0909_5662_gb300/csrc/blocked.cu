// blocked.cu -- block-sparse U(1) x U(1) rotation (dmrg_rotate_ops_blocked).
//
// Operators labelled by quantum numbers (Sec. 3.1, Eq. (hache)): operator k maps
// block sector q to q + delta_k, U is block diagonal over the kept sectors Q of the
// new block, and the [B a] sector of Q stacks the block sectors Q - delta_s of the
// added site's states s.  The rotation restricted to sectors is
//   O'_k[Q2, Q] = sum_s U_Q2[seg s]^T O_k[Q2 - delta_s, Q - delta_s] U_Q[seg s],
// with Q2 = Q + delta_k.  The paper left these sub-blocks undistributed because of
// their dissimilar dimensions (Sec. 3.1); here every block of every operator goes
// into one grouped launch per product.
//
// Planner: operators are grouped into classes of equal shift delta.  Inside a class
// the blocks O_k[q2, q] of all operators are stacked along M, so one problem per
// (class, output block, site state) computes the first product
//   T[(k, x), b] = sum_y O_k[q2, q][x][y] U_Q[seg s][y][b]
// for every operator of the class, and one problem per (class, output block) the
// second, O'_k[Q2, Q] = U_Q2^T T_k.  FP64 / FP32 run the problems as grouped
// plain-FMA GEMMs; BF16x3 / TF32 pack the stacked operands into K-major tensor-core
// layouts and run two grouped tcgen05 launches.
//
// Plans whose sectors all hold at most 32 states have nothing for a tensor-core tile:
// there one warp per (operator, output block) computes sum_s U_Q2[seg s]^T O_k U_Q[seg s]
// through shared memory in one launch, in FP64 for the FP64 precision and in FP32 (more
// accurate than BF16x3 and TF32 ask for) otherwise.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <vector>

#include "api_common.h"

using namespace dmrg;

namespace {

struct ShiftClass {
    int32_t du, dd;
    std::vector<int64_t> ops;        // operator indices, in order
    std::vector<int64_t> in_base;    // per class op: offset of its input storage
    std::vector<int64_t> out_base;   // per class op: offset of its output storage
    std::vector<int64_t> in_local;   // per block sector q: offset of block (q + delta, q) in an op, or -1
    std::vector<int64_t> out_local;  // per kept sector Q: offset of block (Q + delta, Q) in an op, or -1
    int64_t in_size = 0, out_size = 0;
    int64_t* d_in_base = nullptr;    // device copies (owned by the plan's device arena)
    int64_t* d_out_base = nullptr;
};

struct First {   // first-product problem
    int c, Q2, Q, s, q, q2, p2;
};
struct Second {  // second-product problem
    int c, Q2, Q;
};

struct TcTables {
    TcProblem* d_first = nullptr;
    TcProblem* d_second = nullptr;
    int32_t* d_map_first = nullptr;    // problem of every tile (one load per tile to decode)
    int32_t* d_map_second = nullptr;
    int tiles_first = 0, tiles_second = 0;
    int bn_first = 16, bn_second = 16;
    // first product with every N tile <= 128: 64-byte rows and two CTAs per SM (its
    // reductions are a block sector, at most a few k-blocks, so its tiles are short and
    // two CTAs overlap each other's per-tile latency; the second product, reducing over
    // a whole [B a] sector, keeps 128-byte rows and one CTA per SM, which measured faster)
    bool two_per_sm = false;
    int row_bytes = 128;   // of the first product
};

// ---- fused small-sector path
constexpr int kSmallMax = 32;    // largest sector (states) of the fused kernel
constexpr int kSmallSegs = 8;    // largest site dimension of the fused path
constexpr int kSmallWarps = 8;   // warps (work items) per block

struct SmallProb {   // one output block (class, Q2 = Q + delta, Q)
    const int64_t* in_base;    // the class's per-operator input offsets (device)
    const int64_t* out_base;   // the class's per-operator output offsets (device)
    int64_t out_local;         // O'_k[Q2, Q] within an operator's output
    int64_t uQ, uQ2;           // element offsets of U_Q and U_Q2
    int64_t in_local[kSmallSegs];   // per site state: block (q2, q) in an operator's input, -1: none
    int32_t bq[kSmallSegs], bq2[kSmallSegs];      // rows of the block sectors q and q2
    int32_t segQ[kSmallSegs], segQ2[kSmallSegs];  // first rows of segment s in U_Q and U_Q2
    int32_t kQ, kQ2, nseg;
};

// Work item x = (problem, operator of its class) goes to warp x % kSmallWarps of block
// x / kSmallWarps.  A lane owns output entries o = lane + 32 i of the kQ2 x kQ block:
//   T_s[x][j] = sum_y O_k[q2, q][x][y] U_Q[seg s + y][j]        (shared memory)
//   A[e][j]  += sum_x U_Q2[seg s + x][e] T_s[x][j]                (shared memory, own entries)
// Dynamic shared memory: per warp, T_s and A of cap = (largest sector)^2 entries each.
template <typename T>
__global__ void __launch_bounds__(kSmallWarps * 32)
blocked_small_kernel(const SmallProb* __restrict__ probs, const int2* __restrict__ items,
                     int64_t nitems, const T* __restrict__ U, const T* __restrict__ O,
                     T* __restrict__ Oout, int cap) {
    extern __shared__ __align__(16) unsigned char small_smem[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = int64_t(blockIdx.x) * kSmallWarps + w;
    if (item >= nitems) return;   // whole warps only; no block-wide barrier below
    const int2 it = items[item];
    const SmallProb& P = probs[it.x];
    const int kQ = P.kQ, kQ2 = P.kQ2, nout = kQ2 * kQ;
    const int64_t ib = P.in_base[it.y];
    T* Tw = reinterpret_cast<T*>(small_smem) + int64_t(w) * 2 * cap;
    T* Aw = Tw + cap;
    for (int o = lane; o < nout; o += 32) Aw[o] = T(0);
    for (int s = 0; s < P.nseg; ++s) {
        const int64_t il = P.in_local[s];
        if (il < 0) continue;
        const int bq = P.bq[s], bq2 = P.bq2[s];
        const T* Ob = O + ib + il;
        const T* Us = U + P.uQ + int64_t(P.segQ[s]) * kQ;
        __syncwarp();
        for (int o = lane; o < bq2 * kQ; o += 32) {
            const int x = o / kQ, j = o - x * kQ;
            T t = T(0);
            for (int y = 0; y < bq; ++y) t = fma(Ob[x * bq + y], Us[y * kQ + j], t);
            Tw[o] = t;
        }
        __syncwarp();
        const T* U2 = U + P.uQ2 + int64_t(P.segQ2[s]) * kQ2;
        for (int o = lane; o < nout; o += 32) {
            const int e = o / kQ, j = o - e * kQ;
            T a = Aw[o];
            for (int x = 0; x < bq2; ++x) a = fma(U2[x * kQ2 + e], Tw[x * kQ + j], a);
            Aw[o] = a;
        }
    }
    T* out = Oout + P.out_base[it.y] + P.out_local;
    for (int o = lane; o < nout; o += 32) out[o] = Aw[o];
}

int64_t ld_for(int64_t x, int64_t align) { return (x + align - 1) / align * align; }
size_t a128(size_t x) { return (x + 127) / 128 * 128; }

}  // namespace

struct dmrg_blocked_plan_s {
    dmrg_handle h = nullptr;
    int S = 0, d = 0, P = 0;
    int64_t K = 0;
    std::vector<int32_t> bu, bd, ku, kd, su, sd, ou, od;
    std::vector<int64_t> bm, km;
    std::vector<int64_t> D, segoff, uoff;
    std::vector<int> segq;
    std::vector<ShiftClass> classes;
    std::vector<First> first;
    std::vector<Second> second;
    int64_t u_elems = 0, in_elems = 0, out_elems = 0;
    double flops = 0.0;
    bool needs_zero = false;
    // device arena: op offset arrays + SIMT problem tables + pack-job table
    char* d_arena = nullptr;
    SimtGemm* d_simt_first = nullptr;
    SimtGemm* d_simt_second = nullptr;
    int simt_tiles_first = 0, simt_tiles_second = 0;
    std::vector<SimtGemm> simt_first_h, simt_second_h;
    PackJob* d_pack = nullptr;
    int n_pack = 0;
    int64_t pack_blocks = 0;
    std::vector<PackJob> pack_h;
    // workspace layout
    int64_t simt_T_elems = 0;           // per-element count of the plain-FMA intermediate
    std::vector<int64_t> simt_T_off;    // per second problem
    size_t tc_bytes_split = 0, tc_bytes_tf32 = 0;
    // tensor-core layout (element offsets, identical for hi and lo halves)
    struct TcLayout {
        std::vector<int64_t> a_off, a_ld;      // per (class, q) index -> packed A
        std::vector<int64_t> b1_off;           // per (Q, s)
        std::vector<int64_t> b2_off, b2_ld;    // per kept Q
        std::vector<int64_t> t2_off, t2_ld;    // per second problem
        int64_t t2_start = 0;                  // intermediates occupy [t2_start, half_elems)
        int64_t half_elems = 0;                // elements of one half (hi or lo)
    };
    TcLayout tl[2];                          // [0] BF16 (ld multiple of 8), [1] TF32 (of 4)
    // fused small-sector path (every sector <= kSmallMax states, d <= kSmallSegs)
    bool route_small = true;           // the handle's DMRG_OPT_BLOCKED_SMALL at plan creation
    std::vector<Second> small_second;  // output blocks of the fused kernel (all sectors <= 32)
    int64_t n_first_all = 0, n_second_all = 0;   // problems of both routes (statistics)
    bool small_ok = false;             // small_second is non-empty and its tables are uploaded
    int small_cap = 0;                 // (largest sector of the fused problems)^2
    SmallProb* d_small = nullptr;
    int2* d_small_items = nullptr;
    int64_t n_small_items = 0;
    std::map<std::pair<const void*, int>, TcTables> tc_cache;
    std::vector<void*> device_allocs;
};

namespace {

int find_label(const std::vector<int32_t>& u, const std::vector<int32_t>& d, int32_t a, int32_t b) {
    for (size_t i = 0; i < u.size(); ++i)
        if (u[i] == a && d[i] == b) return int(i);
    return -1;
}

// Tensor-core layout of packed operands and intermediates for element alignment `al`.
void build_tc_layout(dmrg_blocked_plan_s& pl, dmrg_blocked_plan_s::TcLayout& L, int64_t al) {
    const int S = pl.S, d = pl.d, P = pl.P;
    int64_t off = 0;
    auto take = [&](int64_t elems) {
        const int64_t o = off;
        off += int64_t(a128(size_t(elems) * 4) / 4);  // 128-byte granularity for 32-bit, finer for 16-bit
        return o;
    };
    const int C = int(pl.classes.size());
    // only the operands of the grouped problems (the fused kernel reads its own)
    std::vector<char> need_a(size_t(C) * S, 0), need_b1(size_t(P) * d, 0), need_b2(P, 0);
    for (const First& f : pl.first) {
        need_a[size_t(f.c) * S + f.q] = 1;
        need_b1[size_t(f.Q) * d + f.s] = 1;
    }
    for (const Second& p : pl.second) need_b2[p.Q2] = 1;
    L.a_off.assign(size_t(C) * S, -1);
    L.a_ld.assign(size_t(C) * S, 0);
    for (int c = 0; c < C; ++c) {
        const ShiftClass& cl = pl.classes[c];
        for (int q = 0; q < S; ++q) {
            if (cl.in_local[q] < 0 || !need_a[size_t(c) * S + q]) continue;
            const int q2 = find_label(pl.bu, pl.bd, pl.bu[q] + cl.du, pl.bd[q] + cl.dd);
            const int64_t ld = ld_for(pl.bm[q], al);
            L.a_ld[size_t(c) * S + q] = ld;
            L.a_off[size_t(c) * S + q] = take(int64_t(cl.ops.size()) * pl.bm[q2] * ld);
        }
    }
    L.b1_off.assign(size_t(P) * d, -1);
    for (int Q = 0; Q < P; ++Q)
        for (int s = 0; s < d; ++s) {
            const int q = pl.segq[size_t(Q) * d + s];
            if (q < 0 || !need_b1[size_t(Q) * d + s]) continue;
            L.b1_off[size_t(Q) * d + s] = take(pl.km[Q] * ld_for(pl.bm[q], al));
        }
    L.b2_off.assign(P, -1);
    L.b2_ld.assign(P, 0);
    for (int Q = 0; Q < P; ++Q) {
        if (!need_b2[Q]) continue;
        L.b2_ld[Q] = ld_for(pl.D[Q], al);
        L.b2_off[Q] = take(pl.km[Q] * L.b2_ld[Q]);
    }
    L.t2_off.assign(pl.second.size(), 0);
    L.t2_ld.assign(pl.second.size(), 0);
    L.t2_start = off;
    for (size_t i = 0; i < pl.second.size(); ++i) {
        const Second& p = pl.second[i];
        L.t2_ld[i] = ld_for(pl.D[p.Q2], al);
        L.t2_off[i] = take(int64_t(pl.classes[p.c].ops.size()) * pl.km[p.Q] * L.t2_ld[i]);
    }
    L.half_elems = off;
}

dmrg_status build_plan(dmrg_blocked_plan_s& pl) {
    const int S = pl.S, d = pl.d, P = pl.P;
    // [B a] sectors of the kept sectors
    pl.D.assign(P, 0);
    pl.segq.assign(size_t(P) * d, -1);
    pl.segoff.assign(size_t(P) * d, 0);
    pl.uoff.assign(P + 1, 0);
    for (int Q = 0; Q < P; ++Q) {
        int64_t rows = 0;
        for (int s = 0; s < d; ++s) {
            const int q = find_label(pl.bu, pl.bd, pl.ku[Q] - pl.su[s], pl.kd[Q] - pl.sd[s]);
            pl.segq[size_t(Q) * d + s] = q;
            pl.segoff[size_t(Q) * d + s] = rows;
            if (q >= 0) rows += pl.bm[q];
        }
        if (pl.km[Q] > rows) return DMRG_ERR_SHAPE;  // more kept states than [B a] states
        pl.D[Q] = rows;
        pl.uoff[Q + 1] = pl.uoff[Q] + rows * pl.km[Q];
    }
    pl.u_elems = pl.uoff[P];
    // shift classes and storage offsets
    std::vector<int> op_class(pl.K);
    for (int64_t k = 0; k < pl.K; ++k) {
        int c = -1;
        for (size_t i = 0; i < pl.classes.size(); ++i)
            if (pl.classes[i].du == pl.ou[k] && pl.classes[i].dd == pl.od[k]) c = int(i);
        if (c < 0) {
            ShiftClass cl;
            cl.du = pl.ou[k];
            cl.dd = pl.od[k];
            cl.in_local.assign(S, -1);
            cl.out_local.assign(P, -1);
            for (int q = 0; q < S; ++q) {
                const int q2 = find_label(pl.bu, pl.bd, pl.bu[q] + cl.du, pl.bd[q] + cl.dd);
                if (q2 < 0) continue;
                cl.in_local[q] = cl.in_size;
                cl.in_size += pl.bm[q2] * pl.bm[q];
            }
            for (int Q = 0; Q < P; ++Q) {
                const int Q2 = find_label(pl.ku, pl.kd, pl.ku[Q] + cl.du, pl.kd[Q] + cl.dd);
                if (Q2 < 0) continue;
                cl.out_local[Q] = cl.out_size;
                cl.out_size += pl.km[Q2] * pl.km[Q];
            }
            pl.classes.push_back(cl);
            c = int(pl.classes.size()) - 1;
        }
        op_class[k] = c;
    }
    int64_t in_off = 0, out_off = 0;
    for (int64_t k = 0; k < pl.K; ++k) {
        ShiftClass& cl = pl.classes[op_class[k]];
        cl.ops.push_back(k);
        cl.in_base.push_back(in_off);
        cl.out_base.push_back(out_off);
        in_off += cl.in_size;
        out_off += cl.out_size;
    }
    pl.in_elems = in_off;
    pl.out_elems = out_off;
    // problems: all to the fused kernel when every sector holds at most kSmallMax states
    // (mixing both routes measured slower: the grouped launch's time is set by its
    // largest blocks, and the fused kernel's work grows as the cube of the sector size)
    bool all_small = pl.route_small && d <= kSmallSegs;
    for (int64_t m : pl.bm) all_small = all_small && m <= kSmallMax;
    for (int64_t m : pl.km) all_small = all_small && m <= kSmallMax;
    for (int c = 0; c < int(pl.classes.size()); ++c) {
        const ShiftClass& cl = pl.classes[c];
        const double nc = double(cl.ops.size());
        for (int Q = 0; Q < P; ++Q) {
            if (cl.out_local[Q] < 0) continue;
            const int Q2 = find_label(pl.ku, pl.kd, pl.ku[Q] + cl.du, pl.kd[Q] + cl.dd);
            pl.flops += 2.0 * nc * pl.km[Q2] * pl.D[Q2] * pl.km[Q];
            ++pl.n_second_all;
            // output blocks whose sectors all hold at most kSmallMax states: fused kernel
            if (all_small) {
                pl.small_second.push_back({c, Q2, Q});
                for (int s = 0; s < d; ++s) {
                    const int q = pl.segq[size_t(Q) * d + s];
                    const int q2 = pl.segq[size_t(Q2) * d + s];
                    if (q < 0 || q2 < 0) continue;
                    ++pl.n_first_all;
                    pl.flops += 2.0 * nc * pl.bm[q2] * pl.bm[q] * pl.km[Q];
                }
                continue;
            }
            const int p2 = int(pl.second.size());
            pl.second.push_back({c, Q2, Q});
            for (int s = 0; s < d; ++s) {
                const int q = pl.segq[size_t(Q) * d + s];
                const int q2 = pl.segq[size_t(Q2) * d + s];
                if (q2 < 0) continue;
                if (q < 0) {
                    pl.needs_zero = true;  // rows of T_Q2 with no source block stay zero
                    continue;
                }
                pl.first.push_back({c, Q2, Q, s, q, q2, p2});
                ++pl.n_first_all;
                pl.flops += 2.0 * nc * pl.bm[q2] * pl.bm[q] * pl.km[Q];
            }
        }
    }
    build_tc_layout(pl, pl.tl[0], 8);
    build_tc_layout(pl, pl.tl[1], 4);
    pl.tc_bytes_split = size_t(pl.tl[0].half_elems) * 2 * 2;
    pl.tc_bytes_tf32 = size_t(pl.tl[1].half_elems) * 4;
    // plain-FMA intermediate: per second problem, n_c x D_Q2 x km[Q]
    pl.simt_T_off.assign(pl.second.size(), 0);
    int64_t t = 0;
    for (size_t i = 0; i < pl.second.size(); ++i) {
        const Second& p = pl.second[i];
        pl.simt_T_off[i] = t;
        t += int64_t(pl.classes[p.c].ops.size()) * pl.D[p.Q2] * pl.km[p.Q];
    }
    pl.simt_T_elems = t;
    return DMRG_OK;
}

// Tiling of one grouped plain-FMA problem: blocks of small outputs go one warp per
// operator (8 operators per CTA), the others 64 x 64 tiles per operator.
void set_simt_tiles(SimtGemm& g) {
    g.small = (g.M <= kSimtSmall && g.N <= kSimtSmall && !g.reduce_batch) ? 1 : 0;
    g.tiles_m = int((g.M + simt_tile_m() - 1) / simt_tile_m());
    g.tiles_n = int((g.N + simt_tile_n() - 1) / simt_tile_n());
}

int simt_tile_count(const SimtGemm& g) {
    if (g.small) return (g.batch + kSimtSmallPerBlock - 1) / kSimtSmallPerBlock;
    return g.tiles_m * g.tiles_n * g.batch;
}

// Device arena: class offset arrays, grouped plain-FMA problem tables and the pack-job
// table (all element offsets, independent of the caller's pointers).
// Tables of the fused small-sector path: one problem per routed output block and one
// work item per (problem, operator of its class).  Needs the class arrays on the device.
dmrg_status upload_small(dmrg_blocked_plan_s& pl) {
    const int d = pl.d;
    pl.small_ok = false;
    if (pl.small_second.empty()) return DMRG_OK;
    int64_t kmax = 1;
    std::vector<SmallProb> probs(pl.small_second.size());
    std::vector<int2> items;
    for (size_t i = 0; i < pl.small_second.size(); ++i) {
        const Second& p = pl.small_second[i];
        const ShiftClass& cl = pl.classes[p.c];
        SmallProb& sp = probs[i];
        sp = SmallProb{};
        sp.in_base = cl.d_in_base;
        sp.out_base = cl.d_out_base;
        sp.out_local = cl.out_local[p.Q];
        sp.uQ = pl.uoff[p.Q];
        sp.uQ2 = pl.uoff[p.Q2];
        sp.kQ = int32_t(pl.km[p.Q]);
        sp.kQ2 = int32_t(pl.km[p.Q2]);
        sp.nseg = d;
        kmax = std::max({kmax, pl.km[p.Q], pl.km[p.Q2]});
        for (int s = 0; s < d; ++s) {
            const int q = pl.segq[size_t(p.Q) * d + s];
            const int q2 = pl.segq[size_t(p.Q2) * d + s];
            sp.in_local[s] = (q >= 0 && q2 >= 0) ? cl.in_local[q] : -1;
            sp.bq[s] = q >= 0 ? int32_t(pl.bm[q]) : 0;
            sp.bq2[s] = q2 >= 0 ? int32_t(pl.bm[q2]) : 0;
            sp.segQ[s] = int32_t(pl.segoff[size_t(p.Q) * d + s]);
            sp.segQ2[s] = int32_t(pl.segoff[size_t(p.Q2) * d + s]);
            kmax = std::max<int64_t>({kmax, sp.bq[s], sp.bq2[s]});
        }
        for (size_t k = 0; k < cl.ops.size(); ++k) items.push_back(make_int2(int(i), int(k)));
    }
    pl.small_cap = int(kmax * kmax);
    pl.n_small_items = int64_t(items.size());
    if (pl.n_small_items == 0) return DMRG_OK;
    if ((pl.n_small_items + kSmallWarps - 1) / kSmallWarps > 0x7fffffffLL) return DMRG_ERR_SHAPE;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&pl.d_small), probs.size() * sizeof(SmallProb));
    if (e != cudaSuccess) return DMRG_ERR_CUDA;
    pl.device_allocs.push_back(pl.d_small);
    e = cudaMalloc(reinterpret_cast<void**>(&pl.d_small_items), items.size() * sizeof(int2));
    if (e != cudaSuccess) return DMRG_ERR_CUDA;
    pl.device_allocs.push_back(pl.d_small_items);
    e = cudaMemcpy(pl.d_small, probs.data(), probs.size() * sizeof(SmallProb), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(pl.d_small_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return DMRG_ERR_CUDA;
    pl.small_ok = true;
    return DMRG_OK;
}

dmrg_status upload_static(dmrg_blocked_plan_s& pl) {
    const int S = pl.S, d = pl.d;
    // plain-FMA problems
    int tiles = 0;
    for (const First& f : pl.first) {
        const ShiftClass& cl = pl.classes[f.c];
        SimtGemm g{};
        g.M = pl.bm[f.q2]; g.N = pl.km[f.Q]; g.K = pl.bm[f.q];
        g.A = reinterpret_cast<const void*>(intptr_t(cl.in_local[f.q]));
        g.a_sel = 1; g.sAi = pl.bm[f.q]; g.sAk = 1;
        g.B = reinterpret_cast<const void*>(intptr_t(pl.uoff[f.Q] + pl.segoff[size_t(f.Q) * d + f.s] * pl.km[f.Q]));
        g.b_sel = 0; g.sBb = 0; g.sBk = pl.km[f.Q]; g.sBj = 1;
        g.C = reinterpret_cast<void*>(intptr_t(pl.simt_T_off[f.p2] + pl.segoff[size_t(f.Q2) * d + f.s] * pl.km[f.Q]));
        g.c_sel = 2; g.sCb = pl.D[f.Q2] * pl.km[f.Q]; g.sCi = pl.km[f.Q]; g.sCj = 1;
        g.batch = int32_t(cl.ops.size());
        set_simt_tiles(g);
        g.tile_start = tiles;
        tiles += simt_tile_count(g);
        pl.simt_first_h.push_back(g);
    }
    pl.simt_tiles_first = tiles;
    tiles = 0;
    for (size_t i = 0; i < pl.second.size(); ++i) {
        const Second& p = pl.second[i];
        const ShiftClass& cl = pl.classes[p.c];
        SimtGemm g{};
        g.M = pl.km[p.Q2]; g.N = pl.km[p.Q]; g.K = pl.D[p.Q2];
        g.A = reinterpret_cast<const void*>(intptr_t(pl.uoff[p.Q2]));
        g.a_sel = 0; g.sAb = 0; g.sAi = 1; g.sAk = pl.km[p.Q2];
        g.B = reinterpret_cast<const void*>(intptr_t(pl.simt_T_off[i]));
        g.b_sel = 2; g.sBb = pl.D[p.Q2] * pl.km[p.Q]; g.sBk = pl.km[p.Q]; g.sBj = 1;
        g.C = reinterpret_cast<void*>(intptr_t(cl.out_local[p.Q]));
        g.c_sel = 3; g.sCi = pl.km[p.Q]; g.sCj = 1;
        g.batch = int32_t(cl.ops.size());
        set_simt_tiles(g);
        g.tile_start = tiles;
        tiles += simt_tile_count(g);
        pl.simt_second_h.push_back(g);
    }
    pl.simt_tiles_second = tiles;
    if (int64_t(pl.simt_tiles_first) > 0x7fffffff || int64_t(tiles) > 0x7fffffff) return DMRG_ERR_SHAPE;
    // pack jobs (BF16 layout offsets; the TF32 layout is selected at launch time by a
    // second table) -- built per layout below
    // arena size
    size_t bytes = 0;
    for (auto& cl : pl.classes) bytes += a128(cl.ops.size() * 8) * 2;
    bytes += a128(pl.simt_first_h.size() * sizeof(SimtGemm)) + a128(pl.simt_second_h.size() * sizeof(SimtGemm));
    // pack jobs for both layouts
    auto make_jobs = [&](const dmrg_blocked_plan_s::TcLayout& L, int li, std::vector<PackJob>& jobs) {
        const int C = int(pl.classes.size());
        for (int c = 0; c < C; ++c) {
            const ShiftClass& cl = pl.classes[c];
            for (int q = 0; q < S; ++q) {
                const int64_t ao = L.a_off[size_t(c) * S + q];
                if (ao < 0) continue;
                const int q2 = find_label(pl.bu, pl.bd, pl.bu[q] + cl.du, pl.bd[q] + cl.dd);
                PackJob j{};
                j.rel = 1; j.src_sel = 1; j.mode = li == 0 ? 0 : 1;
                j.src = reinterpret_cast<const void*>(intptr_t(0));
                j.src_off = cl.in_local[q];
                j.rows = int64_t(cl.ops.size()) * pl.bm[q2];
                j.cols = pl.bm[q];
                j.rows_per_op = pl.bm[q2];
                j.op_off = nullptr;  // patched to the device class array below
                j.s_op = c;          // temporary: class index
                j.rdiv = 1; j.s_r_hi = pl.bm[q]; j.s_r_lo = 0; j.s_c = 1;
                j.ld = L.a_ld[size_t(c) * S + q];
                j.dst0 = reinterpret_cast<void*>(intptr_t(ao));  // element offsets; scaled later
                j.dst1 = reinterpret_cast<void*>(intptr_t(ao));
                jobs.push_back(j);
            }
        }
        for (int Q = 0; Q < pl.P; ++Q)
            for (int s = 0; s < d; ++s) {
                const int64_t bo = L.b1_off[size_t(Q) * d + s];
                if (bo < 0) continue;
                const int q = pl.segq[size_t(Q) * d + s];
                PackJob j{};
                j.rel = 1; j.src_sel = 0; j.src_f64 = 1; j.mode = li == 0 ? 0 : 1;
                j.src_off = pl.uoff[Q] + pl.segoff[size_t(Q) * d + s] * pl.km[Q];
                j.rows = pl.km[Q]; j.cols = pl.bm[q]; j.rows_per_op = j.rows; j.s_op = -1;
                j.rdiv = 1; j.s_r_hi = 1; j.s_r_lo = 0; j.s_c = pl.km[Q];
                j.ld = ld_for(pl.bm[q], li == 0 ? 8 : 4);
                j.dst0 = reinterpret_cast<void*>(intptr_t(bo));
                j.dst1 = reinterpret_cast<void*>(intptr_t(bo));
                jobs.push_back(j);
            }
        for (int Q = 0; Q < pl.P; ++Q) {
            if (L.b2_off[Q] < 0) continue;
            PackJob j{};
            j.rel = 1; j.src_sel = 0; j.src_f64 = 1; j.mode = li == 0 ? 0 : 1;
            j.src_off = pl.uoff[Q];
            j.rows = pl.km[Q]; j.cols = pl.D[Q]; j.rows_per_op = j.rows; j.s_op = -1;
            j.rdiv = 1; j.s_r_hi = 1; j.s_r_lo = 0; j.s_c = pl.km[Q];
            j.ld = L.b2_ld[Q];
            j.dst0 = reinterpret_cast<void*>(intptr_t(L.b2_off[Q]));
            j.dst1 = reinterpret_cast<void*>(intptr_t(L.b2_off[Q]));
            jobs.push_back(j);
        }
    };
    std::vector<PackJob> jobs0, jobs1;
    make_jobs(pl.tl[0], 0, jobs0);
    make_jobs(pl.tl[1], 1, jobs1);
    bytes += a128(jobs0.size() * sizeof(PackJob)) * 2;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&pl.d_arena), std::max<size_t>(bytes, 256));
    if (e != cudaSuccess) return DMRG_ERR_CUDA;
    pl.device_allocs.push_back(pl.d_arena);
    std::vector<char> host(std::max<size_t>(bytes, 256), 0);
    size_t pos = 0;
    for (auto& cl : pl.classes) {
        cl.d_in_base = reinterpret_cast<int64_t*>(pl.d_arena + pos);
        memcpy(host.data() + pos, cl.in_base.data(), cl.in_base.size() * 8);
        pos += a128(cl.ops.size() * 8);
        cl.d_out_base = reinterpret_cast<int64_t*>(pl.d_arena + pos);
        memcpy(host.data() + pos, cl.out_base.data(), cl.out_base.size() * 8);
        pos += a128(cl.ops.size() * 8);
    }
    // class offset arrays into the plain-FMA problems
    for (size_t i = 0; i < pl.first.size(); ++i)
        pl.simt_first_h[i].a_boff = pl.classes[pl.first[i].c].d_in_base;
    for (size_t i = 0; i < pl.second.size(); ++i)
        pl.simt_second_h[i].c_boff = pl.classes[pl.second[i].c].d_out_base;
    pl.d_simt_first = reinterpret_cast<SimtGemm*>(pl.d_arena + pos);
    memcpy(host.data() + pos, pl.simt_first_h.data(), pl.simt_first_h.size() * sizeof(SimtGemm));
    pos += a128(pl.simt_first_h.size() * sizeof(SimtGemm));
    pl.d_simt_second = reinterpret_cast<SimtGemm*>(pl.d_arena + pos);
    memcpy(host.data() + pos, pl.simt_second_h.data(), pl.simt_second_h.size() * sizeof(SimtGemm));
    pos += a128(pl.simt_second_h.size() * sizeof(SimtGemm));
    // pack tables: fix the class arrays and block starts, byte offsets of the destinations
    for (int li = 0; li < 2; ++li) {
        std::vector<PackJob>& jobs = li == 0 ? jobs0 : jobs1;
        const size_t es = li == 0 ? 2 : 4;
        const int64_t half_bytes = pl.tl[li].half_elems * int64_t(es);
        int64_t blocks = 0;
        for (PackJob& j : jobs) {
            if (j.s_op >= 0) {
                j.op_off = pl.classes[size_t(j.s_op)].d_in_base;
            } else {
                j.op_off = nullptr;
            }
            j.s_op = 0;
            const int64_t eo = reinterpret_cast<intptr_t>(j.dst0);
            j.dst0 = reinterpret_cast<void*>(intptr_t(eo * int64_t(es)));
            j.dst1 = li == 0 ? reinterpret_cast<void*>(intptr_t(half_bytes + eo * int64_t(es))) : nullptr;
            j.block_start = blocks;
            pack_prepare_grouped(j);
            blocks += pack_blocks_for(j);
        }
        if (li == 0) pl.pack_blocks = blocks;
        PackJob* dst = reinterpret_cast<PackJob*>(pl.d_arena + pos);
        memcpy(host.data() + pos, jobs.data(), jobs.size() * sizeof(PackJob));
        pos += a128(jobs0.size() * sizeof(PackJob));
        if (li == 0) pl.d_pack = dst;
        pl.n_pack = int(jobs.size());
    }
    e = cudaMemcpy(pl.d_arena, host.data(), host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return DMRG_ERR_CUDA;
    return upload_small(pl);
}

PackJob* pack_table(dmrg_blocked_plan_s& pl, bool tf32) {
    // the TF32 table follows the BF16 one in the arena
    if (!tf32) return pl.d_pack;
    return reinterpret_cast<PackJob*>(reinterpret_cast<char*>(pl.d_pack) + a128(pl.n_pack * sizeof(PackJob)));
}

// Tensor-core problem tables for one workspace pointer (tensor maps hold addresses).
dmrg_status tc_tables(dmrg_blocked_plan_s& pl, void* ws, bool tf32, TcTables*& out) {
    auto key = std::make_pair(static_cast<const void*>(ws), int(tf32));
    auto it = pl.tc_cache.find(key);
    if (it != pl.tc_cache.end()) {
        out = &it->second;
        return DMRG_OK;
    }
    const dmrg_blocked_plan_s::TcLayout& L = pl.tl[tf32 ? 1 : 0];
    const TcMode mode = tf32 ? TC_TF32 : TC_BF16X3;
    const size_t es = tf32 ? 4 : 2;
    char* hi = static_cast<char*>(ws);
    char* lo = tf32 ? hi : hi + L.half_elems * int64_t(es);
    auto ptr = [&](char* base, int64_t eoff) { return static_cast<void*>(base + eoff * int64_t(es)); };
    const int S = pl.S, d = pl.d;
    std::vector<TcProblem> first(pl.first.size()), second(pl.second.size());
    TcTables T;
    int bn_max = 16;
    for (const First& f : pl.first) bn_max = std::max(bn_max, choose_tile_n(pl.km[f.Q], 256));
    T.two_per_sm = bn_max <= 128 && tc_stages_two_per_sm(mode, bn_max) >= 2;
    T.row_bytes = T.two_per_sm ? 64 : 128;
    int tiles = 0;
    for (size_t i = 0; i < pl.first.size(); ++i) {
        const First& f = pl.first[i];
        const ShiftClass& cl = pl.classes[f.c];
        const int64_t nc = int64_t(cl.ops.size());
        const int64_t ao = L.a_off[size_t(f.c) * S + f.q];
        const int64_t bo = L.b1_off[size_t(f.Q) * d + f.s];
        const int64_t ald = L.a_ld[size_t(f.c) * S + f.q];
        TcOperand A{ptr(hi, ao), ptr(lo, ao), nc * pl.bm[f.q2], pl.bm[f.q], ald};
        TcOperand B{ptr(hi, bo), ptr(lo, bo), pl.km[f.Q], pl.bm[f.q],
                    ld_for(pl.bm[f.q], tf32 ? 4 : 8)};
        TcProblem& P = first[i];
        if (!make_problem(P, mode, A, B, 256, 1, T.row_bytes)) return DMRG_ERR_CUDA;
        TcScatter& sc = P.sc[0];
        sc.out_off = L.t2_off[f.p2] + pl.segoff[size_t(f.Q2) * d + f.s];
        sc.rows_per_op = int32_t(pl.bm[f.q2]);
        sc.s_op = pl.km[f.Q] * L.t2_ld[f.p2];
        sc.s_row = 1;
        sc.col_div = 1;
        sc.s_col_hi = L.t2_ld[f.p2];
        sc.s_col_lo = 0;
        P.tile_start = tiles;
        tiles += P.m_tiles * P.n_tiles * P.k_splits;
        T.bn_first = std::max(T.bn_first, P.tile_n);
    }
    T.tiles_first = tiles;
    tiles = 0;
    for (size_t i = 0; i < pl.second.size(); ++i) {
        const Second& p = pl.second[i];
        const ShiftClass& cl = pl.classes[p.c];
        const int64_t nc = int64_t(cl.ops.size());
        TcOperand A{ptr(hi, L.t2_off[i]), ptr(lo, L.t2_off[i]), nc * pl.km[p.Q], pl.D[p.Q2], L.t2_ld[i]};
        TcOperand B{ptr(hi, L.b2_off[p.Q2]), ptr(lo, L.b2_off[p.Q2]), pl.km[p.Q2], pl.D[p.Q2],
                    L.b2_ld[p.Q2]};
        TcProblem& P = second[i];
        if (!make_problem(P, mode, A, B, 256, 1)) return DMRG_ERR_CUDA;
        TcScatter& sc = P.sc[0];
        sc.out_off = cl.out_local[p.Q];
        sc.op_off = cl.d_out_base;
        sc.rows_per_op = int32_t(pl.km[p.Q]);
        sc.s_op = 0;
        sc.s_row = 1;
        sc.col_div = 1;
        sc.s_col_hi = pl.km[p.Q];
        sc.s_col_lo = 0;
        P.tile_start = tiles;
        tiles += P.m_tiles * P.n_tiles * P.k_splits;
        T.bn_second = std::max(T.bn_second, P.tile_n);
    }
    T.tiles_second = tiles;
    std::vector<int32_t> map1(size_t(T.tiles_first)), map2(size_t(T.tiles_second));
    for (size_t i = 0; i < first.size(); ++i) {
        const TcProblem& P = first[i];
        std::fill(map1.begin() + P.tile_start, map1.begin() + P.tile_start + P.m_tiles * P.n_tiles * P.k_splits,
                  int32_t(i));
    }
    for (size_t i = 0; i < second.size(); ++i) {
        const TcProblem& P = second[i];
        std::fill(map2.begin() + P.tile_start, map2.begin() + P.tile_start + P.m_tiles * P.n_tiles * P.k_splits,
                  int32_t(i));
    }
    const size_t b1 = a128(first.size() * sizeof(TcProblem)), b2 = a128(second.size() * sizeof(TcProblem));
    const size_t m1 = a128(map1.size() * 4), m2 = a128(map2.size() * 4);
    char* dev = nullptr;
    if (cudaMalloc(reinterpret_cast<void**>(&dev), std::max<size_t>(b1 + b2 + m1 + m2, 256)) != cudaSuccess)
        return DMRG_ERR_CUDA;
    pl.device_allocs.push_back(dev);
    if ((!first.empty() && cudaMemcpy(dev, first.data(), first.size() * sizeof(TcProblem),
                                      cudaMemcpyHostToDevice) != cudaSuccess) ||
        (!second.empty() && cudaMemcpy(dev + b1, second.data(), second.size() * sizeof(TcProblem),
                                       cudaMemcpyHostToDevice) != cudaSuccess) ||
        (!map1.empty() && cudaMemcpy(dev + b1 + b2, map1.data(), map1.size() * 4, cudaMemcpyHostToDevice) !=
                              cudaSuccess) ||
        (!map2.empty() && cudaMemcpy(dev + b1 + b2 + m1, map2.data(), map2.size() * 4,
                                     cudaMemcpyHostToDevice) != cudaSuccess))
        return DMRG_ERR_CUDA;
    T.d_first = reinterpret_cast<TcProblem*>(dev);
    T.d_second = reinterpret_cast<TcProblem*>(dev + b1);
    T.d_map_first = reinterpret_cast<int32_t*>(dev + b1 + b2);
    T.d_map_second = reinterpret_cast<int32_t*>(dev + b1 + b2 + m1);
    out = &pl.tc_cache.emplace(key, T).first->second;
    return DMRG_OK;
}

size_t simt_ws_bytes(const dmrg_blocked_plan_s& pl, dmrg_precision p) {
    const size_t es = p == DMRG_PREC_FP64 ? 8 : 4;
    WsLayout W;
    W.add("T", size_t(pl.simt_T_elems) * es);
    if (p == DMRG_PREC_FP32) {
        W.add("U32", size_t(pl.u_elems) * 4);
        W.add("O32", size_t(pl.in_elems) * 4);
    }
    return W.total;
}

// The fused small-sector path in FP32: U and (FP64 inputs) O converted first.
WsLayout small_layout(const dmrg_blocked_plan_s& pl) {
    WsLayout W;
    W.add("U32", size_t(pl.u_elems) * 4);
    W.add("O32", size_t(pl.in_elems) * 4);
    return W;
}

size_t ws_bytes(const dmrg_blocked_plan_s& pl, dmrg_precision p) {
    const size_t small = (pl.small_ok && p != DMRG_PREC_FP64) ? small_layout(pl).total : 0;
    if (p == DMRG_PREC_FP64 || p == DMRG_PREC_FP32) return std::max(small, simt_ws_bytes(pl, p));
    return std::max<size_t>({256, small, p == DMRG_PREC_BF16X3 ? pl.tc_bytes_split : pl.tc_bytes_tf32});
}

// The fused small-sector kernel over the plan's routed output blocks.
dmrg_status run_small(dmrg_handle h, const dmrg_blocked_plan_s* pl, const double* U, const void* O,
                      int in_is_fp64, void* Oout, dmrg_precision p, void* ws, cudaStream_t cs) {
    const unsigned blocks = unsigned((pl->n_small_items + kSmallWarps - 1) / kSmallWarps);
    const size_t smem = size_t(kSmallWarps) * 2 * pl->small_cap * (p == DMRG_PREC_FP64 ? 8 : 4);
    cudaError_t e;
    if (p == DMRG_PREC_FP64) {
        e = cudaFuncSetAttribute(blocked_small_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(smem));
        if (e == cudaSuccess)
            e = timed_launch(h, "blk_small", cs, [&] {
                blocked_small_kernel<double><<<blocks, kSmallWarps * 32, smem, cs>>>(
                    pl->d_small, pl->d_small_items, pl->n_small_items, U, static_cast<const double*>(O),
                    static_cast<double*>(Oout), pl->small_cap);
                return cudaGetLastError();
            });
        return cuda_fail(h, e, "small-sector rotation");
    }
    const WsLayout W = small_layout(*pl);
    char* base = static_cast<char*>(ws);
    float* U32 = reinterpret_cast<float*>(base + W.offsets[0]);
    const float* O32 = in_is_fp64 ? reinterpret_cast<const float*>(base + W.offsets[1])
                                  : static_cast<const float*>(O);
    PackJob jobs[2] = {};
    int nj = 0;
    auto conv = [&](const void* src, float* dst, int64_t n) {
        PackJob& j = jobs[nj++];
        j.src = src; j.src_f64 = 1; j.mode = 2; j.rows = 1; j.cols = n; j.rows_per_op = 1;
        j.rdiv = 1; j.s_r_hi = n; j.s_c = 1; j.dst0 = dst; j.ld = n;
    };
    conv(U, U32, pl->u_elems);
    if (in_is_fp64) conv(O, reinterpret_cast<float*>(base + W.offsets[1]), pl->in_elems);
    e = timed_launch(h, "blk_convert_fp32", cs, [&] { return pack_launch(jobs, nj, nullptr, cs); });
    if (e != cudaSuccess) return cuda_fail(h, e, "convert");
    e = cudaFuncSetAttribute(blocked_small_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(smem));
    if (e == cudaSuccess)
        e = timed_launch(h, "blk_small", cs, [&] {
            blocked_small_kernel<float><<<blocks, kSmallWarps * 32, smem, cs>>>(
                pl->d_small, pl->d_small_items, pl->n_small_items, U32, O32, static_cast<float*>(Oout),
                pl->small_cap);
            return cudaGetLastError();
        });
    return cuda_fail(h, e, "small-sector rotation");
}

}  // namespace

extern "C" {

dmrg_status dmrg_blocked_plan_create(dmrg_handle h, const dmrg_qn_sector* bs, int32_t nb,
                                     const dmrg_qn_shift* ss, int32_t d, const dmrg_qn_sector* ks,
                                     int32_t nk, const dmrg_qn_shift* os, int64_t K,
                                     dmrg_blocked_plan* out) {
    if (!h || !out) return DMRG_ERR_INVALID_ARG;
    *out = nullptr;
    if (nb < 1 || d < 1 || nk < 1 || K < 0) return fail(h, DMRG_ERR_SHAPE, "empty sector lists");
    if (!bs || !ss || !ks || (K > 0 && !os)) return fail(h, DMRG_ERR_INVALID_ARG, "null array");
    auto* pl = new dmrg_blocked_plan_s();
    pl->h = h;
    pl->route_small = h->blocked_small;
    pl->S = nb; pl->d = d; pl->P = nk; pl->K = K;
    for (int i = 0; i < nb; ++i) {
        if (bs[i].dim < 1) { delete pl; return fail(h, DMRG_ERR_SHAPE, "block sector of size < 1"); }
        if (find_label(pl->bu, pl->bd, bs[i].n_up, bs[i].n_dn) >= 0) {
            delete pl;
            return fail(h, DMRG_ERR_INVALID_ARG, "repeated block sector label");
        }
        pl->bu.push_back(bs[i].n_up); pl->bd.push_back(bs[i].n_dn); pl->bm.push_back(bs[i].dim);
    }
    for (int i = 0; i < nk; ++i) {
        if (ks[i].dim < 1) { delete pl; return fail(h, DMRG_ERR_SHAPE, "kept sector of size < 1"); }
        if (find_label(pl->ku, pl->kd, ks[i].n_up, ks[i].n_dn) >= 0) {
            delete pl;
            return fail(h, DMRG_ERR_INVALID_ARG, "repeated kept sector label");
        }
        pl->ku.push_back(ks[i].n_up); pl->kd.push_back(ks[i].n_dn); pl->km.push_back(ks[i].dim);
    }
    for (int s = 0; s < d; ++s) { pl->su.push_back(ss[s].d_up); pl->sd.push_back(ss[s].d_dn); }
    for (int64_t k = 0; k < K; ++k) { pl->ou.push_back(os[k].d_up); pl->od.push_back(os[k].d_dn); }
    dmrg_status st = build_plan(*pl);
    if (st != DMRG_OK) {
        delete pl;
        return fail(h, st, "a kept sector is larger than its [B a] sector");
    }
    st = upload_static(*pl);
    if (st != DMRG_OK) {
        for (void* p : pl->device_allocs) cudaFree(p);
        delete pl;
        return fail(h, st, "plan tables");
    }
    *out = pl;
    return DMRG_OK;
}

dmrg_status dmrg_blocked_plan_destroy(dmrg_blocked_plan pl) {
    if (!pl) return DMRG_ERR_INVALID_ARG;
    for (void* p : pl->device_allocs) cudaFree(p);
    delete pl;
    return DMRG_OK;
}

dmrg_status dmrg_blocked_plan_sizes(dmrg_blocked_plan pl, dmrg_precision p, int64_t* u, int64_t* in,
                                    int64_t* o, size_t* ws) {
    if (!pl) return DMRG_ERR_INVALID_ARG;
    if (p < DMRG_PREC_FP64 || p > DMRG_PREC_BF16X3) return DMRG_ERR_INVALID_ARG;
    if (u) *u = pl->u_elems;
    if (in) *in = pl->in_elems;
    if (o) *o = pl->out_elems;
    if (ws) *ws = ws_bytes(*pl, p);
    return DMRG_OK;
}

dmrg_status dmrg_blocked_plan_stats(dmrg_blocked_plan pl, int64_t* n1, int64_t* n2, double* flops) {
    if (!pl) return DMRG_ERR_INVALID_ARG;
    if (n1) *n1 = pl->n_first_all;
    if (n2) *n2 = pl->n_second_all;
    if (flops) *flops = pl->flops;
    return DMRG_OK;
}

dmrg_status dmrg_rotate_ops_blocked(dmrg_handle h, dmrg_blocked_plan pl, const double* U,
                                    const void* O, int in_is_fp64, void* Oout, dmrg_precision p,
                                    void* ws, size_t ws_len, dmrg_stream_t stream) {
    if (!h || !pl) return DMRG_ERR_INVALID_ARG;
    if (pl->h != h) return fail(h, DMRG_ERR_INVALID_ARG, "plan belongs to another handle");
    if (p < DMRG_PREC_FP64 || p > DMRG_PREC_BF16X3) return fail(h, DMRG_ERR_INVALID_ARG, "precision");
    if (pl->K == 0 || pl->out_elems == 0) return DMRG_OK;
    if (!U || !O || !Oout) return fail(h, DMRG_ERR_INVALID_ARG, "null data pointer");
    if (p == DMRG_PREC_FP64 && !in_is_fp64)
        return fail(h, DMRG_ERR_INVALID_ARG, "the FP64 precision needs FP64 operators");
    dmrg_status st = check_ws(h, ws, ws_len, ws_bytes(*pl, p));
    if (st != DMRG_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool tc = (p == DMRG_PREC_TF32 || p == DMRG_PREC_BF16X3);
    if (tc && !tc_supported(h)) return fail(h, DMRG_ERR_UNSUPPORTED, "tensor cores need sm_103");
    TcTables* T = nullptr;
    if (tc && !pl->second.empty() && (st = tc_tables(*pl, ws, p == DMRG_PREC_TF32, T)) != DMRG_OK)
        return fail(h, st, "tensor-core tables");
    char key[200];
    snprintf(key, sizeof key, "blk:%p:%p:%p:%p:%p:%p:%d:%d", (void*)pl, (const void*)U, O, Oout, ws,
             (void*)s, int(p), in_is_fp64);
    return run_maybe_graph(h, key, s, [&](cudaStream_t cs) -> dmrg_status {
        cudaError_t e;
        if (pl->small_ok) {
            const dmrg_status rs = run_small(h, pl, U, O, in_is_fp64, Oout, p, ws, cs);
            if (rs != DMRG_OK) return rs;
        }
        if (pl->second.empty()) return DMRG_OK;
        if (!tc) {
            const bool f64 = (p == DMRG_PREC_FP64);
            const Real rt = f64 ? Real::F64 : Real::F32;
            WsLayout W;
            const size_t es = f64 ? 8 : 4;
            W.add("T", size_t(pl->simt_T_elems) * es);
            char* base = static_cast<char*>(ws);
            void* Tbuf = base + W.offsets[0];
            const void* Uu = U;
            const void* Ou = O;
            if (!f64) {
                W.add("U32", size_t(pl->u_elems) * 4);
                W.add("O32", size_t(pl->in_elems) * 4);
                float* U32 = reinterpret_cast<float*>(base + W.offsets[1]);
                float* O32 = reinterpret_cast<float*>(base + W.offsets[2]);
                PackJob jobs[2] = {};
                int nj = 0;
                auto conv = [&](const void* src, float* dst, int64_t n) {
                    PackJob& j = jobs[nj++];
                    j.src = src; j.src_f64 = 1; j.mode = 2; j.rows = 1; j.cols = n; j.rows_per_op = 1;
                    j.rdiv = 1; j.s_r_hi = n; j.s_c = 1; j.dst0 = dst; j.ld = n;
                };
                conv(U, U32, pl->u_elems);
                Uu = U32;
                if (in_is_fp64) {
                    conv(O, O32, pl->in_elems);
                    Ou = O32;
                }
                e = timed_launch(h, "blk_convert_fp32", cs, [&] { return pack_launch(jobs, nj, nullptr, cs); });
                if (e != cudaSuccess) return cuda_fail(h, e, "convert");
            }
            if (pl->needs_zero) {
                e = cudaMemsetAsync(Tbuf, 0, size_t(pl->simt_T_elems) * es, cs);
                if (e != cudaSuccess) return cuda_fail(h, e, "memset");
            }
            const void* bases[4] = {Uu, Ou, Tbuf, Oout};
            e = timed_launch(h, "blk_simt_first_product", cs, [&] {
                return simt_gemm_grouped_launch(rt, pl->d_simt_first, int(pl->first.size()),
                                                pl->simt_tiles_first, bases, cs);
            });
            if (e != cudaSuccess) return cuda_fail(h, e, "first product");
            e = timed_launch(h, "blk_simt_second_product", cs, [&] {
                return simt_gemm_grouped_launch(rt, pl->d_simt_second, int(pl->second.size()),
                                                pl->simt_tiles_second, bases, cs);
            });
            return cuda_fail(h, e, "second product");
        }
        const bool tf32 = (p == DMRG_PREC_TF32);
        const TcMode mode = tf32 ? TC_TF32 : TC_BF16X3;
        const size_t es = tf32 ? 4 : 2;
        const dmrg_blocked_plan_s::TcLayout& L = pl->tl[tf32 ? 1 : 0];
        char* hi = static_cast<char*>(ws);
        char* lo = tf32 ? hi : hi + L.half_elems * int64_t(es);
        const void* srcs[2] = {U, O};
        // Table jobs read U as FP64 and O in the caller's precision.
        e = timed_launch(h, "blk_pack", cs, [&] {
            return pack_grouped_launch(pack_table(*pl, tf32), pl->n_pack, pl->pack_blocks, srcs, ws,
                                       in_is_fp64, cs);
        });
        if (e != cudaSuccess) return cuda_fail(h, e, "pack");
        if (pl->needs_zero) {  // intermediate rows that no source block writes must read as 0
            const size_t t2 = size_t(L.t2_start) * es, t2n = size_t(L.half_elems - L.t2_start) * es;
            e = cudaMemsetAsync(hi + t2, 0, t2n, cs);
            if (e == cudaSuccess && !tf32) e = cudaMemsetAsync(lo + t2, 0, t2n, cs);
            if (e != cudaSuccess) return cuda_fail(h, e, "memset");
        }
        TcLaunch L1{};
        L1.table = T->d_first;
        L1.tile_problem = T->d_map_first;
        L1.nprob = int(pl->first.size());
        L1.total_tiles = T->tiles_first;
        L1.out[0][0] = hi;
        L1.out[0][1] = lo;
        L1.status = h->d_status;
        L1.timeout_ns = timeout_ns(h);
        L1.row_bytes = T->row_bytes;
        const bool two = T->two_per_sm;
        const int st1 = two ? tc_stages_two_per_sm(mode, T->bn_first)
                            : std::min(tc_max_stages(mode, T->bn_first), 4);
        e = timed_launch(h, "blk_tc_first_product", cs, [&] {
            return tc_gemm_launch_grouped(mode, tf32 ? EPI_TF32 : EPI_SPLIT_BF16, L1, st1,
                                          (two ? 2 : 1) * h->num_sms, T->bn_first, cs, two);
        });
        if (e != cudaSuccess) return cuda_fail(h, e, "first product");
        TcLaunch L2{};
        L2.table = T->d_second;
        L2.tile_problem = T->d_map_second;
        L2.nprob = int(pl->second.size());
        L2.total_tiles = T->tiles_second;
        L2.out[0][0] = Oout;
        L2.status = h->d_status;
        L2.timeout_ns = timeout_ns(h);
        L2.row_bytes = 128;
        const int st2 = std::min(tc_max_stages(mode, T->bn_second), 4);
        e = timed_launch(h, "blk_tc_second_product", cs, [&] {
            return tc_gemm_launch_grouped(mode, EPI_F32, L2, st2, h->num_sms, T->bn_second, cs);
        });
        return cuda_fail(h, e, "second product");
    });
}

}  // extern "C"
