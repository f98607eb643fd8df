// tc.cu -- tcgen05 tensor-core GEMM pipeline and operand packer (sm_103a).
//
// Both products of the rotation (Sec. 3.2: Z R^+ then R (Z R^+)) run through one
// persistent, warp-specialised kernel:
//   warp 0   : TMA producer  -- 128-byte-swizzled K-major tiles of A and B into a
//              ring of shared-memory stages (cp.async.bulk.tensor, mbarrier tx count);
//   warp 1   : MMA issuer    -- one thread issues tcgen05.mma (M = 128, N <= 256)
//              into one of two TMEM accumulators, tcgen05.commit frees the stage;
//   warps 2-9: epilogue      -- tcgen05.ld of the finished accumulator, conversion
//              (FP32 / TF32 / BF16 hi-lo split) and a strided scatter to global memory,
//              overlapping the next tile's main loop (two warps per TMEM lane quadrant,
//              alternate 32-column chunks).
// Precision forms: BF16x3 (A = Ah + Al, B = Bh + Bl, D += Al Bh + Ah Bl + Ah Bh with
// FP32 accumulation), TF32 (kind::tf32) and plain BF16 (one product, for comparison).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "internal.h"
#include "ptx.cuh"
#include "tc_common.cuh"

namespace dmrg {
namespace {

using namespace tcdev;

constexpr int kThreads = 320;        // 10 warps: producer, MMA issuer, 8 epilogue warps
constexpr int kEpiWarps = 8;         // two per TMEM lane quadrant, alternate 32-column chunks
constexpr int kBM = 128;             // rows per tile (TMEM lanes)
// ACC (template): FP32 columns per TMEM accumulator; two accumulators.  256 is the
// default; 128 (N tiles of at most 128) halves the TMEM and, with 64-byte rows, the
// shared memory, so that two CTAs share an SM and overlap each other's per-tile latency.
// Winding down after an expired wait: copies and MMAs already issued are waited for
// with this fixed limit, whatever limit the caller chose for the main waits.
constexpr uint64_t kDrainTimeoutNs = 2000000000ull;

// RB: bytes of reduction per shared-memory row and k-block (128 -> 128-byte swizzle,
// 64 -> 64-byte swizzle with half-depth k-blocks and twice the pipeline stages).
template <int MODE, int EPI, int RB, int ACC>
__global__ void __launch_bounds__(kThreads, ACC == 128 ? 2 : 1)
    tc_gemm_kernel(const __grid_constant__ TcLaunch L, int stages, int bn_smem) {
    constexpr uint32_t kTmemCols = 2 * ACC;
    constexpr uint32_t kAccStride = ACC;
    constexpr int kRowBytes = RB;
    constexpr bool kSplit = (MODE == TC_BF16X3);
    constexpr int kElem = (MODE == TC_TF32) ? 4 : 2;
    constexpr int kElemsPerRow = kRowBytes / kElem;      // reduction elements per k-block
    constexpr int kUmmaK = 32 / kElem;                   // reduction elements per MMA
    constexpr int kStepsPerBlock = kElemsPerRow / kUmmaK;  // 4
    constexpr uint32_t kFmt = (MODE == TC_TF32) ? 2u : 1u;

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t a_bytes = kBM * kRowBytes;
    const uint32_t b_bytes = uint32_t(bn_smem) * kRowBytes;
    const uint32_t stage_bytes = (a_bytes + b_bytes) * (kSplit ? 2 : 1);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + size_t(stages) * stage_bytes);
    uint64_t* empty = full + stages;
    uint64_t* tfull = empty + stages;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
    int* zero_flag = abort_flag + 1;  // never raised: drain waits ignore the abort flag

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], kEpiWarps);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        *zero_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc<kTmemCols>(tmem_slot);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    volatile int* vabort = abort_flag;
    const uint64_t tmo = L.timeout_ns;
    // The set-up above may overlap the previous kernel's tail; nothing in global
    // memory is touched before that kernel has completed.
    griddep_wait();
    griddep_launch_dependents();

    auto stage_a = [&](int s, int half) -> uint8_t* {
        return smem + size_t(s) * stage_bytes + size_t(half) * (a_bytes + b_bytes);
    };
    auto stage_b = [&](int s, int half) -> uint8_t* { return stage_a(s, half) + a_bytes; };

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            if (L.table == nullptr) {
                for (int i = 0; i < L.nprob; ++i) {
                    tma_prefetch_desc(&L.inline_prob[i].tmA[0]);
                    tma_prefetch_desc(&L.inline_prob[i].tmB[0]);
                    if (kSplit) {
                        tma_prefetch_desc(&L.inline_prob[i].tmA[1]);
                        tma_prefetch_desc(&L.inline_prob[i].tmB[1]);
                    }
                }
            }
            int stage = 0;
            uint32_t phase = 0;
            uint32_t armed = 0;  // bit s: stage s holds an issued, unconfirmed load
            uint32_t armed_parity = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < L.total_tiles && ok; t += gridDim.x) {
                const Decoded dt = decode_tile(L, t, kElemsPerRow);
                const TcProblem* P = dt.P;
                const uint32_t bytes =
                    (a_bytes + uint32_t(P->tile_n) * kRowBytes) * (kSplit ? 2u : 1u);
                const int ya = dt.mt * kBM;
                const int yb = dt.nt * P->tile_n;
                for (int kb = dt.kb_begin; kb < dt.kb_end; ++kb) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, tmo, L.status, vabort)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[stage], bytes);
                    const int z = kb / dt.kb_per_batch;
                    const int x = (kb - z * dt.kb_per_batch) * kElemsPerRow;
                    tma_load_3d(stage_a(stage, 0), &P->tmA[0], &full[stage], x, ya, z);
                    tma_load_3d(stage_b(stage, 0), &P->tmB[0], &full[stage], x, yb, z);
                    if (kSplit) {
                        tma_load_3d(stage_a(stage, 1), &P->tmA[1], &full[stage], x, ya, z);
                        tma_load_3d(stage_b(stage, 1), &P->tmB[1], &full[stage], x, yb, z);
                    }
                    armed |= 1u << stage;
                    armed_parity = (armed_parity & ~(1u << stage)) | (phase << stage);
                    if (++stage == stages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            // Never leave the CTA with bulk copies still landing in shared memory.
            for (int s = 0; s < stages; ++s)
                if (armed & (1u << s))
                    mbar_wait(&full[s], (armed_parity >> s) & 1u, kDrainTimeoutNs, L.status,
                              zero_flag);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < L.total_tiles && ok; t += gridDim.x, ++it) {
                const Decoded dt = decode_tile(L, t, kElemsPerRow);
                const TcProblem* P = dt.P;
                const int acc = it & 1;
                const uint32_t acc_parity = uint32_t(it >> 1) & 1u;
                // (everything that does not depend on a barrier is formed before its wait)
                int n_eff = min(P->tile_n, P->N - dt.nt * P->tile_n);
                n_eff = (n_eff + 15) & ~15;
                const uint32_t idesc = make_idesc(kFmt, uint32_t(n_eff));
                const uint32_t tmem_d = tmem_base + uint32_t(acc) * kAccStride;
                if (!mbar_wait(&tempty[acc], acc_parity ^ 1u, tmo, L.status, vabort)) break;
                tc_fence_after();
                for (int kb = dt.kb_begin; kb < dt.kb_end; ++kb) {
                    const int rem = P->Kred - (kb % dt.kb_per_batch) * kElemsPerRow;
                    const int steps = min(kStepsPerBlock, (rem + kUmmaK - 1) / kUmmaK);
                    const uint64_t ah = smem_desc_kmajor<RB>(smem_u32(stage_a(stage, 0)));
                    const uint64_t bh = smem_desc_kmajor<RB>(smem_u32(stage_b(stage, 0)));
                    const uint64_t al = kSplit ? smem_desc_kmajor<RB>(smem_u32(stage_a(stage, 1))) : 0;
                    const uint64_t bl = kSplit ? smem_desc_kmajor<RB>(smem_u32(stage_b(stage, 1))) : 0;
                    if (!mbar_wait(&full[stage], phase, tmo, L.status, vabort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    for (int k = 0; k < steps; ++k) {
                        const uint64_t off = uint64_t(k) * 2;  // 32 bytes in 16-byte units
                        const uint32_t accum = (kb > dt.kb_begin || k > 0) ? 1u : 0u;
                        if (MODE == TC_BF16X3) {
                            mma_bf16(tmem_d, al + off, bh + off, idesc, accum);
                            mma_bf16(tmem_d, ah + off, bl + off, idesc, 1u);
                            mma_bf16(tmem_d, ah + off, bh + off, idesc, 1u);
                        } else if (MODE == TC_TF32) {
                            mma_tf32(tmem_d, ah + off, bh + off, idesc, accum);
                        } else {
                            mma_bf16(tmem_d, ah + off, bh + off, idesc, accum);
                        }
                    }
                    // Test hook: withhold one release so that the producer's bounded wait on
                    // this stage expires (a barrier that nothing arrives on).
                    const bool withhold = L.drop_arrival && blockIdx.x == 0 && it == 0 &&
                                          kb == dt.kb_begin;
                    if (!withhold) mma_commit(&empty[stage]);
                    if (++stage == stages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit(&tfull[acc]);
            }
            // Every issued MMA has finished before TMEM is released.
            mma_commit(drain);
            mbar_wait(drain, 0, kDrainTimeoutNs, L.status, zero_flag);
        }
    } else {
        // ------------------------------------------------------------ epilogue (warps 2..9)
        const int quad = warp & 3;            // TMEM lanes [32*quad, 32*quad + 32)
        const int half = (warp - 2) >> 2;     // 0: even 32-column chunks, 1: odd ones
        int it = 0;
        for (int t = blockIdx.x; t < L.total_tiles; t += gridDim.x, ++it) {
            const Decoded dt = decode_tile(L, t, kElemsPerRow);
            const TcProblem* P = dt.P;
            const int acc = it & 1;
            const uint32_t acc_parity = uint32_t(it >> 1) & 1u;
            // One lane waits and the warp follows its verdict, so the warp-collective
            // tcgen05.ld below is always executed by all 32 lanes or by none.
            int ok = 1;
            if (lane == 0) ok = mbar_wait(&tfull[acc], acc_parity, tmo, L.status, vabort) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tc_fence_after();
            const int row = dt.mt * kBM + quad * 32 + lane;
            // a tile whose reduction range is empty has an uninitialised accumulator
            const bool row_ok = row < P->M && dt.kb_begin < dt.kb_end;
            const int n0 = dt.nt * P->tile_n;
            const int ncols = min(P->tile_n, P->N - n0);
            const TcScatter& S = P->sc[0];
            int64_t row_base = 0;
            if (row_ok) {
                const int g = row / S.rows_per_op;
                const int rr = row - g * S.rows_per_op;
                row_base = S.out_off + (S.op_off ? S.op_off[g] : int64_t(g) * S.s_op) +
                           int64_t(rr) * S.s_row;
            }
            const int cdiv = S.col_div;
            const int64_t sch = S.s_col_hi, scl = S.s_col_lo;
            const bool tile_atomic = P->atomic != 0;
            for (int c = half * 32; c < ncols; c += 64) {
                uint32_t r[32];
                tmem_ld_32x32b_x32(tmem_base + uint32_t(acc) * kAccStride +
                                       (uint32_t(quad * 32) << 16) + uint32_t(c),
                                   r);
                tmem_ld_wait();
                if (!row_ok) continue;
                const int cmax = min(32, ncols - c);
                store_chunk<EPI>(L, r, row_base, n0, c, cmax, cdiv, sch, scl, tile_atomic);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc<kTmemCols>(tmem_base);
    }
}

// ---------------------------------------------------------------- packer
constexpr int kMaxPackJobs = 8;

struct PackLaunch {
    PackJob inline_jobs[kMaxPackJobs];
    const PackJob* table;
    int njobs;
    const void* srcs[2];
    char* ws_base;
    int src1_f64;  // precision of srcs[1] for relative jobs
};

constexpr int kPackThreads = 256;
constexpr int kPackElems = 4;  // elements per thread


template <typename S>
__device__ __forceinline__ void pack_store(const PackJob& j, int64_t dst, S x) {
    if (j.mode == 0) {
        __nv_bfloat16 h, l;
        split_bf16(x, h, l);
        static_cast<__nv_bfloat16*>(j.dst0)[dst] = h;
        static_cast<__nv_bfloat16*>(j.dst1)[dst] = l;
    } else if (j.mode == 1) {
        static_cast<float*>(j.dst0)[dst] = tf32_round(float(x));
    } else {
        static_cast<float*>(j.dst0)[dst] = float(x);
    }
}

// General gather of one block's kPackThreads * kPackElems elements, thread-strided so
// that neighbouring threads take neighbouring elements (coalesced stores, and loads where
// source rows are contiguous).  The row / group / sub-row split uses the host's
// multiply-shift divisors when the job fits 31 bits (a division is a long instruction
// sequence, and this path is instruction-bound).
__device__ __forceinline__ void pack_general(const PackJob& j, int64_t blk) {
    const int64_t total = j.rows * j.cols;
    const int64_t base = blk * (int64_t(kPackThreads) * kPackElems) + threadIdx.x;
#pragma unroll
    for (int q = 0; q < kPackElems; ++q) {
        const int64_t e = base + int64_t(q) * kPackThreads;
        if (e >= total) break;
        int64_t r, c, g, hi, lo;
        if (j.fastdiv) {
            const uint32_t eu = uint32_t(e), cu = uint32_t(j.cols);
            const uint32_t ru = uint32_t((uint64_t(eu) * j.m_cols) >> j.s_cols);
            const uint32_t rpo = uint32_t(j.rows_per_op), rd = uint32_t(j.rdiv);
            const uint32_t gu = uint32_t((uint64_t(ru) * j.m_rpo) >> j.s_rpo);
            const uint32_t rr = ru - gu * rpo;
            const uint32_t h = uint32_t((uint64_t(rr) * j.m_rdiv) >> j.s_rdiv);
            r = ru;
            c = eu - ru * cu;
            g = gu;
            hi = h;
            lo = rr - h * rd;
        } else {
            r = e / j.cols;
            c = e - r * j.cols;
            g = r / j.rows_per_op;
            const int64_t rr = r - g * j.rows_per_op;
            hi = rr / j.rdiv;
            lo = rr - hi * j.rdiv;
        }
        const int64_t src = j.src_off + (j.op_off ? j.op_off[g] : g * j.s_op) + hi * j.s_r_hi +
                            lo * j.s_r_lo + c * j.s_c;
        if (j.src_f64)
            pack_store(j, r * j.ld + c, static_cast<const double*>(j.src)[src]);
        else
            pack_store(j, r * j.ld + c, static_cast<const float*>(j.src)[src]);
    }
}

// Rows whose elements are a contiguous run of the source (s_c = 1, rdiv = 1): one warp
// per row, kPackRowWarps rows per block, lanes along the row, so loads and stores are
// coalesced and the row split costs one division per row instead of per element.
constexpr int kPackRows = 32;   // rows per block (four per warp)

__device__ __forceinline__ void pack_rows(const PackJob& j, int64_t blk) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t cols = j.cols;
    for (int rr = warp; rr < kPackRows; rr += kPackThreads / 32) {
        const int64_t r = blk * kPackRows + rr;
        if (r >= j.rows) break;
        int64_t g, x;
        if (j.fastdiv) {
            const uint32_t ru = uint32_t(r);
            const uint32_t gu = uint32_t((uint64_t(ru) * j.m_rpo) >> j.s_rpo);
            g = gu;
            x = ru - gu * uint32_t(j.rows_per_op);
        } else {
            g = r / j.rows_per_op;
            x = r - g * j.rows_per_op;
        }
        const int64_t src = j.src_off + (j.op_off ? j.op_off[g] : g * j.s_op) + x * j.s_r_hi;
        const int64_t dst = r * j.ld;
        for (int64_t c0 = 0; c0 < cols; c0 += 128) {
            if (j.src_f64) {
                double v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t c = c0 + lane + 32 * u;
                    v[u] = c < cols ? static_cast<const double*>(j.src)[src + c] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t c = c0 + lane + 32 * u;
                    if (c < cols) pack_store(j, dst + c, v[u]);
                }
            } else {
                float v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t c = c0 + lane + 32 * u;
                    v[u] = c < cols ? static_cast<const float*>(j.src)[src + c] : 0.f;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t c = c0 + lane + 32 * u;
                    if (c < cols) pack_store(j, dst + c, v[u]);
                }
            }
        }
    }
}

// The block's job is found once (thread 0), copied word by word into shared memory by
// the block, resolved (relative addresses) by thread 0, and read from there.
__global__ void __launch_bounds__(kPackThreads) pack_kernel(const __grid_constant__ PackLaunch L) {
    __shared__ __align__(16) PackJob sj;
    __shared__ int sk;
    const int b = blockIdx.x;
    if (threadIdx.x == 0) {
        int lo = 0;
        if (L.table == nullptr) {
            for (int i = 1; i < L.njobs; ++i)
                if (L.inline_jobs[i].block_start <= b) lo = i;
        } else {
            int hi = L.njobs - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (L.table[mid].block_start <= b) lo = mid; else hi = mid - 1;
            }
        }
        sk = lo;
    }
    __syncthreads();
    const PackJob* J = L.table ? &L.table[sk] : &L.inline_jobs[sk];
    static_assert(sizeof(PackJob) % 4 == 0, "PackJob is copied in 32-bit words");
    for (int w = threadIdx.x; w < int(sizeof(PackJob) / 4); w += blockDim.x)
        reinterpret_cast<uint32_t*>(&sj)[w] = reinterpret_cast<const uint32_t*>(J)[w];
    __syncthreads();
    if (threadIdx.x == 0 && sj.rel) {
        if (sj.src_sel == 1) sj.src_f64 = L.src1_f64;
        const size_t es = sj.src_f64 ? 8 : 4;
        sj.src = static_cast<const char*>(L.srcs[sj.src_sel]) + reinterpret_cast<intptr_t>(sj.src) * es;
        sj.dst0 = L.ws_base + reinterpret_cast<intptr_t>(sj.dst0);
        sj.dst1 = sj.dst1 ? L.ws_base + reinterpret_cast<intptr_t>(sj.dst1) : nullptr;
    }
    __syncthreads();
    if (sj.rowwise) pack_rows(sj, int64_t(b - sj.block_start));
    else pack_general(sj, int64_t(b - sj.block_start));
}

// Contiguous fast path: one 8-element unit v of a job whose source rows are
// contiguous (16/32-byte loads, 16-byte stores of the BF16 hi and lo halves or
// 2 x 16-byte stores of TF32 / FP32), in two halves so that a thread can issue the
// loads of several units before converting.
// Row and column of 8-element unit v of a contiguous job.
__device__ __forceinline__ void vec8_rc(const PackJob& j, int64_t v, int64_t& r, int64_t& c) {
    const int64_t per_row = j.cols >> 3;
    if (j.fast8) {
        const uint32_t vu = uint32_t(v);
        const uint32_t ru = uint32_t((uint64_t(vu) * j.m_u8) >> j.s_u8);
        r = ru;
        c = int64_t(vu - ru * uint32_t(per_row)) << 3;
    } else {
        r = v / per_row;
        c = (v - r * per_row) << 3;
    }
}

template <typename S>
__device__ __forceinline__ void pack_vec8_load(const PackJob& j, int64_t v, S (&x)[8]) {
    int64_t r, c;
    vec8_rc(j, v, r, c);
    const S* sp = static_cast<const S*>(j.src) + j.src_off + r * j.s_r_hi + c;
    if (sizeof(S) == 4) {
        const float4 a = reinterpret_cast<const float4*>(sp)[0];
        const float4 b = reinterpret_cast<const float4*>(sp)[1];
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
        x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double2 a = reinterpret_cast<const double2*>(sp)[q];
            x[2 * q] = S(a.x);
            x[2 * q + 1] = S(a.y);
        }
    }
}

template <typename S>
__device__ __forceinline__ void pack_vec8_store(const PackJob& j, int64_t v, const S (&x)[8]) {
    int64_t r, c;
    vec8_rc(j, v, r, c);
    const int64_t dst = r * j.ld + c;
    if (j.mode == 0) {
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t hh[2], ll[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                __nv_bfloat16 h, l;
                split_bf16(x[2 * q + e], h, l);
                hh[e] = __bfloat16_as_ushort(h);
                ll[e] = __bfloat16_as_ushort(l);
            }
            hw[q] = hh[0] | (hh[1] << 16);
            lw[q] = ll[0] | (ll[1] << 16);
        }
        *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(j.dst0) + dst) =
            make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(j.dst1) + dst) =
            make_uint4(lw[0], lw[1], lw[2], lw[3]);
    } else {
        float y[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) y[e] = (j.mode == 1) ? tf32_round(float(x[e])) : float(x[e]);
        float4* d4 = reinterpret_cast<float4*>(static_cast<float*>(j.dst0) + dst);
        d4[0] = make_float4(y[0], y[1], y[2], y[3]);
        d4[1] = make_float4(y[4], y[5], y[6], y[7]);
    }
}

// kVec8Units units per thread, block-strided, all loads issued before the stores.
constexpr int kVec8Units = 2;

template <typename S>
__device__ __forceinline__ void pack_vec8_block(const PackJob& j, int64_t blk) {
    const int64_t total = j.rows * (j.cols >> 3);
    const int64_t v0 = blk * (int64_t(kPackThreads) * kVec8Units) + threadIdx.x;
    S x[kVec8Units][8];
#pragma unroll
    for (int u = 0; u < kVec8Units; ++u) {
        const int64_t v = v0 + int64_t(u) * kPackThreads;
        if (v < total) pack_vec8_load<S>(j, v, x[u]);
    }
#pragma unroll
    for (int u = 0; u < kVec8Units; ++u) {
        const int64_t v = v0 + int64_t(u) * kPackThreads;
        if (v < total) pack_vec8_store<S>(j, v, x[u]);
    }
}

// Transposing gathers of FP32 sources (contiguous along the row index, strided along
// the column index, e.g. O_k -> O_k^T) go through shared memory in 64 x 64 tiles, so
// that both the reads and the writes are coalesced: each thread has 16 loads in flight
// and writes column pairs (packed BF16 pairs, or FP32 pairs).  Tile t of a job covers,
// in operator group g and for one residue rem = rr mod rdiv, the rows
// rr = (h0 + 0..63) * rdiv + rem of the group and the columns c0 + 0..63.
constexpr int kTile = 64;

__device__ __forceinline__ void pack_store2_to(int mode, void* d0, void* d1, int64_t dst, float x0,
                                               float x1) {
    if (mode == 0) {
        __nv_bfloat16 h0, l0, h1, l1;
        split_bf16(x0, h0, l0);
        split_bf16(x1, h1, l1);
        *reinterpret_cast<uint32_t*>(static_cast<__nv_bfloat16*>(d0) + dst) =
            uint32_t(__bfloat16_as_ushort(h0)) | (uint32_t(__bfloat16_as_ushort(h1)) << 16);
        *reinterpret_cast<uint32_t*>(static_cast<__nv_bfloat16*>(d1) + dst) =
            uint32_t(__bfloat16_as_ushort(l0)) | (uint32_t(__bfloat16_as_ushort(l1)) << 16);
    } else {
        const bool t = (mode == 1);
        *reinterpret_cast<float2*>(static_cast<float*>(d0) + dst) =
            make_float2(t ? tf32_round(x0) : x0, t ? tf32_round(x1) : x1);
    }
}

__device__ __forceinline__ void pack_store_to(int mode, void* d0, void* d1, int64_t dst, float x) {
    if (mode == 0) {
        __nv_bfloat16 h, l;
        split_bf16(x, h, l);
        static_cast<__nv_bfloat16*>(d0)[dst] = h;
        static_cast<__nv_bfloat16*>(d1)[dst] = l;
    } else {
        static_cast<float*>(d0)[dst] = (mode == 1) ? tf32_round(x) : x;
    }
}

__device__ __forceinline__ void pack_store2(const PackJob& j, int64_t dst, float x0, float x1) {
    if (j.mode == 0) {
        __nv_bfloat16 h0, l0, h1, l1;
        split_bf16(x0, h0, l0);
        split_bf16(x1, h1, l1);
        *reinterpret_cast<uint32_t*>(static_cast<__nv_bfloat16*>(j.dst0) + dst) =
            uint32_t(__bfloat16_as_ushort(h0)) | (uint32_t(__bfloat16_as_ushort(h1)) << 16);
        *reinterpret_cast<uint32_t*>(static_cast<__nv_bfloat16*>(j.dst1) + dst) =
            uint32_t(__bfloat16_as_ushort(l0)) | (uint32_t(__bfloat16_as_ushort(l1)) << 16);
    } else {
        const bool t = (j.mode == 1);
        *reinterpret_cast<float2*>(static_cast<float*>(j.dst0) + dst) =
            make_float2(t ? tf32_round(x0) : x0, t ? tf32_round(x1) : x1);
    }
}

// The tile's coordinates come from host-computed multiply-shift divisors (32-bit index
// arithmetic): 64-bit divisions here made the launch instruction-bound.
__device__ __forceinline__ void pack_tile(const PackJob& j, int64_t t, float (*tile)[kTile + 1]) {
    const int64_t rpo = j.rows_per_op < j.rows ? j.rows_per_op : j.rows;
    const int64_t hrows = j.t_hrows;
    const uint32_t tu = uint32_t(t);
    const uint32_t gu = uint32_t((uint64_t(tu) * j.m_pg) >> j.s_pg);
    const uint32_t u0 = tu - gu * uint32_t(j.t_pg);
    const uint32_t remu = uint32_t((uint64_t(u0) * j.m_hc) >> j.s_hc);
    const uint32_t u = u0 - remu * uint32_t(j.t_hc);
    const uint32_t hq = uint32_t((uint64_t(u) * j.m_ct) >> j.s_ct);
    const int64_t g = gu, rem = remu;
    const int64_t h0 = int64_t(hq) * kTile, c0 = int64_t(u - hq * uint32_t(j.t_ct)) * kTile;
    const float* src = static_cast<const float*>(j.src) + j.src_off + g * j.s_op + rem * j.s_r_lo;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 warps
    float v[16];
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int64_t c = c0 + ty + 8 * q, hr = h0 + tx + 32 * hh;
            v[2 * q + hh] = (c < j.cols && hr < hrows) ? src[hr + c * j.s_c] : 0.f;
        }
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) tile[ty + 8 * q][tx + 32 * hh] = v[2 * q + hh];
    __syncthreads();
    const int64_t c = c0 + 2 * tx;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int64_t hr = h0 + ty + 8 * q;
        if (hr >= hrows || c >= j.cols) continue;
        const int64_t dst = (g * rpo + hr * j.rdiv + rem) * j.ld + c;
        const float x0 = tile[2 * tx][ty + 8 * q];
        if (c + 1 < j.cols) pack_store2(j, dst, x0, tile[2 * tx + 1][ty + 8 * q]);
        else pack_store(j, dst, x0);
    }
    if (j.st0 != nullptr) {
        // the untransposed copy from the same tile: row g * cols + c, columns hs, hs + 1
        const int64_t hs = h0 + 2 * tx;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int cl = ty + 8 * q;
            const int64_t cc = c0 + cl;
            if (cc >= j.cols || hs >= hrows) continue;
            const int64_t dst = (g * j.cols + cc) * j.st_ld + hs;
            const float x0 = tile[cl][2 * tx];
            if (hs + 1 < hrows) pack_store2_to(j.mode, j.st0, j.st1, dst, x0, tile[cl][2 * tx + 1]);
            else pack_store_to(j.mode, j.st0, j.st1, dst, x0);
        }
    }
}

// Several jobs in one launch: block ranges per job; contiguous jobs take the 8-wide
// path, transposing gathers the tiled path, the others the general gather.  Small
// gathers placed first run alongside the bandwidth-bound contiguous job instead of
// after it.
__global__ void __launch_bounds__(kPackThreads) pack_mixed_kernel(const __grid_constant__ PackLaunch L) {
    __shared__ float tile[kTile][kTile + 1];
    griddep_wait();   // launched as a programmatic dependent of the previous kernel
    const int b = blockIdx.x;
    int k = 0;
    for (int i = 1; i < L.njobs; ++i)
        if (L.inline_jobs[i].block_start <= b) k = i;
    const PackJob& j = L.inline_jobs[k];
    if (j.mode == kPackZero) {
        // rows x cols FP32 zeros at row stride ld; 8 values per thread, coalesced
        float* d = static_cast<float*>(j.dst0);
        const int64_t total = j.rows * j.cols;
        const int64_t e0 = int64_t(b - j.block_start) * kPackThreads * 8 + threadIdx.x;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t e = e0 + int64_t(q) * kPackThreads;
            if (e < total) {
                const int64_t r = e / j.cols;
                d[r * j.ld + (e - r * j.cols)] = 0.f;
            }
        }
        return;
    }
    if (j.tiled) {
        pack_tile(j, int64_t(b - j.block_start), tile);
        return;
    }
    if (j.vec8) {
        if (j.src_f64) pack_vec8_block<double>(j, int64_t(b - j.block_start));
        else pack_vec8_block<float>(j, int64_t(b - j.block_start));
        return;
    }
    pack_general(j, int64_t(b - j.block_start));
}

// FP32 sources in groups of rows_per_op rows at source stride s_op (no offset table),
// whole groups only; even destination strides (pair stores).
bool pack_tiled_ok(const PackJob& j) {
    if (j.mode == kPackZero) return false;
    const int64_t rpo = j.rows_per_op < j.rows ? j.rows_per_op : j.rows;
    const bool aligned = (j.ld % 2) == 0 && (reinterpret_cast<uintptr_t>(j.dst0) % 8) == 0 &&
                         (j.dst1 == nullptr || (reinterpret_cast<uintptr_t>(j.dst1) % 4) == 0);
    return !j.src_f64 && j.op_off == nullptr && rpo > 0 && (j.rows % rpo) == 0 && j.s_r_hi == 1 &&
           j.s_c != 1 && j.rdiv >= 1 && (rpo % j.rdiv) == 0 && j.cols >= 8 && aligned;
}

int64_t pack_tiles_host(const PackJob& j) {
    const int64_t rpo = j.rows_per_op < j.rows ? j.rows_per_op : j.rows;
    const int64_t hrows = rpo / j.rdiv;
    return (j.rows / rpo) * int64_t(j.rdiv) * ((hrows + kTile - 1) / kTile) *
           ((j.cols + kTile - 1) / kTile);
}

bool pack_vec8_ok(const PackJob& j) {
    if (j.mode == kPackZero) return false;
    const size_t es = j.src_f64 ? 8 : 4;
    const bool single_group = (j.rows_per_op >= j.rows) && j.op_off == nullptr;
    return single_group && j.rdiv == 1 && j.s_c == 1 && (j.cols % 8) == 0 && (j.s_r_hi % 8) == 0 &&
           (j.ld % 8) == 0 && (j.src_off % 8) == 0 &&
           (reinterpret_cast<uintptr_t>(j.src) % (8 * es)) == 0 &&
           (reinterpret_cast<uintptr_t>(j.dst0) % 32) == 0 &&
           (j.dst1 == nullptr || (reinterpret_cast<uintptr_t>(j.dst1) % 16) == 0);
}

template <int MODE, int EPI>
cudaError_t launch_one(const TcLaunch& L, int stages, int grid, int bn_smem, size_t smem,
                       cudaStream_t s, bool two_per_sm = false) {
    auto k = two_per_sm ? tc_gemm_kernel<MODE, EPI, 64, 128>
             : L.row_bytes == 64 ? tc_gemm_kernel<MODE, EPI, 64, 256>
                                 : tc_gemm_kernel<MODE, EPI, 128, 256>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(grid), 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, L, stages, bn_smem);
}

size_t tc_smem_bytes(TcMode mode, int stages, int bn, int rb) {
    const size_t a = size_t(kBM) * rb, b = size_t(bn) * rb;
    const size_t stage = (a + b) * (mode == TC_BF16X3 ? 2 : 1);
    return 1024 + stage * stages + 8 * (2 * size_t(stages) + 5) + 32;
}

}  // namespace

bool pack_job_tiled(const PackJob& j) { return !pack_vec8_ok(j) && pack_tiled_ok(j); }

int tc_max_stages(TcMode mode, int tile_n_max, int row_bytes) {
    int s = 1;
    while (s < 8 && tc_smem_bytes(mode, s + 1, tile_n_max, row_bytes) <= 232448) ++s;
    return s;
}

// Shared memory of one CTA when two share an SM (228 KB per SM, 1 KB reserved per CTA).
constexpr size_t kTwoPerSmSmem = 112 * 1024;

int tc_stages_two_per_sm(TcMode mode, int tile_n_max) {
    if (tile_n_max > 128 || tc_smem_bytes(mode, 2, tile_n_max, 64) > kTwoPerSmSmem) return 0;
    int s = 2;
    while (s < 8 && tc_smem_bytes(mode, s + 1, tile_n_max, 64) <= kTwoPerSmSmem) ++s;
    return s;
}

cudaError_t tc_gemm_launch(TcMode mode, TcEpi epi, const TcLaunch& L, int stages, int grid,
                           cudaStream_t s) {
    if (L.total_tiles <= 0) return cudaSuccess;
    int bn = 16;
    if (L.table == nullptr && L.nprob >= 1 && L.nprob <= kMaxInlineProblems) {
        for (int i = 0; i < L.nprob; ++i) bn = std::max(bn, L.inline_prob[i].tile_n);
    } else {
        return cudaErrorInvalidValue;  // device-table launches go through tc_gemm_launch_grouped
    }
    const size_t smem = tc_smem_bytes(mode, stages, bn, L.row_bytes);
    if (smem > 232448) return cudaErrorInvalidConfiguration;
    grid = std::max(1, std::min(grid, L.total_tiles));
#define DMRG_TC_CASE(M, E) \
    if (mode == M && epi == E) return launch_one<M, E>(L, stages, grid, bn, smem, s);
    DMRG_TC_CASE(TC_BF16X3, EPI_SPLIT_BF16)
    DMRG_TC_CASE(TC_BF16X3, EPI_F32)
    DMRG_TC_CASE(TC_BF16X3, EPI_F32_ATOMIC)
    DMRG_TC_CASE(TC_TF32, EPI_TF32)
    DMRG_TC_CASE(TC_TF32, EPI_F32)
    DMRG_TC_CASE(TC_TF32, EPI_F32_ATOMIC)
    DMRG_TC_CASE(TC_BF16, EPI_F32)
#undef DMRG_TC_CASE
    return cudaErrorNotSupported;
}

cudaError_t tc_gemm_launch_grouped(TcMode mode, TcEpi epi, const TcLaunch& L, int stages, int grid,
                                   int bn_smem, cudaStream_t s, bool two_per_sm) {
    if (L.total_tiles <= 0) return cudaSuccess;
    const size_t smem = tc_smem_bytes(mode, stages, bn_smem, L.row_bytes);
    if (smem > 232448) return cudaErrorInvalidConfiguration;
    if (two_per_sm && (L.row_bytes != 64 || bn_smem > 128 || smem > kTwoPerSmSmem))
        return cudaErrorInvalidConfiguration;
    grid = std::max(1, std::min(grid, L.total_tiles));
#define DMRG_TC_CASE(M, E) \
    if (mode == M && epi == E) return launch_one<M, E>(L, stages, grid, bn_smem, smem, s, two_per_sm);
    DMRG_TC_CASE(TC_BF16X3, EPI_SPLIT_BF16)
    DMRG_TC_CASE(TC_BF16X3, EPI_F32)
    DMRG_TC_CASE(TC_BF16X3, EPI_F32_ATOMIC)
    DMRG_TC_CASE(TC_TF32, EPI_TF32)
    DMRG_TC_CASE(TC_TF32, EPI_F32)
    DMRG_TC_CASE(TC_TF32, EPI_F32_ATOMIC)
#undef DMRG_TC_CASE
    return cudaErrorNotSupported;
}

namespace {
// Round-up multiplier for n / d with 0 <= n < 2^31, 1 <= d < 2^31 (Granlund and
// Montgomery, "Division by invariant integers using multiplication", Thm. 4.2):
// l = ceil(log2 d), s = 31 + l, m = ceil(2^s / d); then n / d == (n * m) >> s and
// n * m < 2^64.
void div_magic(int64_t d, uint64_t& m, int32_t& s) {
    int l = 0;
    while ((int64_t(1) << l) < d) ++l;
    s = 31 + l;
    m = ((uint64_t(1) << s) + uint64_t(d) - 1) / uint64_t(d);
}
}  // namespace

void pack_prepare(PackJob& j) {
    const int64_t lim = int64_t(1) << 31;
    j.fastdiv = j.cols >= 1 && j.rows_per_op >= 1 && j.rdiv >= 1 && j.rows * j.cols < lim &&
                j.cols < lim && j.rows_per_op < lim && j.rdiv < lim;
    if (!j.fastdiv) return;
    div_magic(j.cols, j.m_cols, j.s_cols);
    div_magic(j.rows_per_op, j.m_rpo, j.s_rpo);
    div_magic(j.rdiv, j.m_rdiv, j.s_rdiv);
}

void pack_prepare_grouped(PackJob& j) {
    pack_prepare(j);
    j.rowwise = (j.s_c == 1 && j.rdiv == 1 && j.mode != kPackZero && j.cols >= 16) ? 1 : 0;
}

int64_t pack_blocks_for(const PackJob& j) {
    if (j.rowwise) return (j.rows + kPackRows - 1) / kPackRows;
    const int64_t per = int64_t(kPackThreads) * kPackElems;
    return (j.rows * j.cols + per - 1) / per;
}

cudaError_t pack_launch(const PackJob* jobs, int njobs, PackJob* /*unused*/, cudaStream_t s) {
    if (njobs <= 0) return cudaSuccess;
    if (njobs > kMaxPackJobs) return cudaErrorInvalidValue;
    PackLaunch L{};
    int64_t blocks = 0;
    int n = 0;
    // general gathers first, contiguous jobs after them, jobs marked late last
    for (int pass = 0; pass < 3; ++pass)
        for (int i = 0; i < njobs; ++i) {
            if (jobs[i].rows * jobs[i].cols == 0) continue;
            const bool v8 = pack_vec8_ok(jobs[i]);
            if (jobs[i].late ? pass != 2 : (pass == 2 || v8 != (pass == 1))) continue;
            const bool tl = !v8 && pack_tiled_ok(jobs[i]);
            // the untransposed copy is written by the tiled path only
            if (jobs[i].st0 != nullptr && (!tl || jobs[i].rdiv != 1 || (jobs[i].st_ld % 2) != 0))
                return cudaErrorInvalidValue;
            PackJob& j = L.inline_jobs[n++];
            j = jobs[i];
            pack_prepare(j);
            j.vec8 = v8 ? 1 : 0;
            j.tiled = tl ? 1 : 0;
            if (v8) {
                const int64_t per_row = j.cols / 8;
                j.fast8 = (j.rows * per_row < (int64_t(1) << 31)) ? 1 : 0;
                if (j.fast8) div_magic(per_row, j.m_u8, j.s_u8);
            }
            if (tl) {
                const int64_t rpo = j.rows_per_op < j.rows ? j.rows_per_op : j.rows;
                j.t_hrows = rpo / j.rdiv;
                const int64_t ht = (j.t_hrows + kTile - 1) / kTile, ct = (j.cols + kTile - 1) / kTile;
                const int64_t hc = ht * ct, pg = int64_t(j.rdiv) * hc;
                if (pg >= (int64_t(1) << 31) || pack_tiles_host(j) >= (int64_t(1) << 31))
                    return cudaErrorInvalidConfiguration;
                j.t_ct = int32_t(ct);
                j.t_hc = int32_t(hc);
                j.t_pg = int32_t(pg);
                div_magic(ct, j.m_ct, j.s_ct);
                div_magic(hc, j.m_hc, j.s_hc);
                div_magic(pg, j.m_pg, j.s_pg);
            }
            j.block_start = blocks;
            blocks += v8 ? (j.rows * (j.cols / 8) + kPackThreads * kVec8Units - 1) / (kPackThreads * kVec8Units)
                    : tl ? pack_tiles_host(j)
                    : j.mode == kPackZero ? (j.rows * j.cols + kPackThreads * 8 - 1) / (kPackThreads * 8)
                                          : pack_blocks_for(j);
        }
    if (n == 0 || blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    L.table = nullptr;
    L.njobs = n;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(blocks), 1, 1);
    cfg.blockDim = dim3(kPackThreads, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, pack_mixed_kernel, L);
}

cudaError_t pack_grouped_launch(const PackJob* jobs_dev, int njobs, int64_t total_blocks,
                                const void* const srcs[2], void* ws_base, int src1_f64,
                                cudaStream_t s) {
    if (njobs <= 0 || total_blocks <= 0) return cudaSuccess;
    if (total_blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    PackLaunch L{};
    L.table = jobs_dev;
    L.njobs = njobs;
    L.srcs[0] = srcs[0];
    L.srcs[1] = srcs[1];
    L.ws_base = static_cast<char*>(ws_base);
    L.src1_f64 = src1_f64;
    pack_kernel<<<unsigned(total_blocks), kPackThreads, 0, s>>>(L);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- host helpers
namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
}

// Looks up cuTensorMapEncodeTiled once (through the runtime: no driver library link).
static bool have_encode() {
    if (g_encode == nullptr) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || fn == nullptr)
            return false;
        g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    return true;
}

bool encode_operand_map(CUtensorMap* map, const void* base, bool fp32, int64_t rows, int64_t cols,
                        int64_t ld, int box_rows, int64_t nbatch, int64_t batch_stride,
                        int row_bytes) {
    if (!have_encode()) return false;
    const int esize = fp32 ? 4 : 2;
    if (nbatch < 1) nbatch = 1;
    if (nbatch == 1) batch_stride = rows * ld;
    cuuint64_t gdim[3] = {cuuint64_t(cols), cuuint64_t(rows), cuuint64_t(nbatch)};
    cuuint64_t gstride[2] = {cuuint64_t(ld) * esize, cuuint64_t(std::max<int64_t>(batch_stride, 1)) * esize};
    if (nbatch == 1) gstride[1] = (gstride[1] + 15) / 16 * 16;
    cuuint32_t box[3] = {cuuint32_t(row_bytes / esize), cuuint32_t(box_rows), 1};
    cuuint32_t estride[3] = {1, 1, 1};
    CUresult r = g_encode(map, fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                          3, const_cast<void*>(base), gdim, gstride, box, estride,
                          CU_TENSOR_MAP_INTERLEAVE_NONE,
                          row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool encode_store_map(CUtensorMap* map, void* base, int64_t nx, int64_t ny, int64_t nz, int64_t ld,
                      int bx, int by, int swizzle, bool fp32) {
    const int es = fp32 ? 4 : 2;
    if ((ld * es) % 16 != 0 || nx > ld || (reinterpret_cast<uintptr_t>(base) & 15) ||
        (bx * es) % 16 != 0 || (swizzle != 0 && swizzle != es * bx) ||
        (swizzle != 0 && swizzle != 32 && swizzle != 64))
        return false;
    if (!have_encode()) return false;
    cuuint64_t gdim[3] = {cuuint64_t(nx), cuuint64_t(ny), cuuint64_t(nz)};
    cuuint64_t gstride[2] = {cuuint64_t(ld) * es, cuuint64_t(ny * ld) * es};
    cuuint32_t box[3] = {cuuint32_t(bx), cuuint32_t(by), 1};
    cuuint32_t estride[3] = {1, 1, 1};
    CUresult r = g_encode(map, fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                          3, base, gdim, gstride, box, estride,
                          CU_TENSOR_MAP_INTERLEAVE_NONE,
                          swizzle == 64   ? CU_TENSOR_MAP_SWIZZLE_64B
                          : swizzle == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                                          : CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// N tile width: tiles of equal width when there are few of them (a narrow last tile
// would leave its wave short), the widest tile when there are many, whose wider MMAs
// do more work per instruction (measured at N = 1600: 256-wide tiles 3 % faster than
// seven of 240; at N = 400, 256 + 144 3 % slower than 208 + 192).
constexpr int64_t kWideTilesFrom = 6;

int choose_tile_n(int64_t N, int tile_n_max) {
    const int64_t ntiles = (N + tile_n_max - 1) / tile_n_max;
    int64_t t = ntiles >= kWideTilesFrom ? tile_n_max : (N + ntiles - 1) / ntiles;
    t = (t + 15) / 16 * 16;
    if (t > tile_n_max) t = tile_n_max;
    if (t < 16) t = 16;
    return int(t);
}

bool make_problem(TcProblem& p, TcMode mode, const TcOperand& A, const TcOperand& B,
                  int tile_n_max, int k_splits, int row_bytes, int pair_form) {
    const bool f32 = (mode == TC_TF32);
    const bool split = (mode == TC_BF16X3);
    if (row_bytes != 64) row_bytes = 128;
    const int elems = row_bytes / (f32 ? 4 : 2);
    if (A.cols != B.cols || A.nbatch != B.nbatch) return false;
    // CTA pairs: 256-row M tiles, each CTA stages half of the N tile (at least 16 rows)
    if (pair_form != 0 && pair_form != 1) return false;
    const bool pair = pair_form == 1;
    const int tile_n = pair ? std::max(32, choose_tile_n(B.rows, tile_n_max)) : choose_tile_n(B.rows, tile_n_max);
    const int b_box = pair ? tile_n / 2 : tile_n;
    const int a_box = kBM;
    const int bm = pair ? 2 * kBM : kBM;
    // An FP32 source for A (CTA pairs, 128-byte rows): boxes of 32 floats x 128 rows
    // that the converter warps turn into the operand in place.
    if (A.f32_source && (!pair || row_bytes != 128 || (A.ld & 3) != 0 ||
                         (reinterpret_cast<uintptr_t>(A.hi) & 15) != 0))
        return false;
    // MN-major operands (CTA pairs, BF16, 128-byte rows): boxes of 64 rows of the operand
    // (its contiguous index) by one 64-element k-block, two per CTA's share of the tile.
    auto mn_ok = [&](const TcOperand& X) {
        return pair && !f32 && row_bytes == 128 && !X.f32_source && (X.ld & 7) == 0 &&
               (reinterpret_cast<uintptr_t>(X.hi) & 15) == 0 &&
               (X.lo == nullptr || (reinterpret_cast<uintptr_t>(X.lo) & 15) == 0);
    };
    if ((A.mn_major && !mn_ok(A)) || (B.mn_major && !mn_ok(B))) return false;
    if (B.mn_major && tile_n / 2 > 2 * kMnBox) return false;
    auto encode = [&](CUtensorMap* map, const void* base, const TcOperand& X, bool fp32, int box) {
        if (X.mn_major)   // dimensions (row, reduction, slice): the row index is contiguous
            return encode_operand_map(map, base, false, X.cols, X.rows, X.ld, kMnBox, X.nbatch,
                                      X.batch_stride, row_bytes);
        return encode_operand_map(map, base, fp32, X.rows, X.cols, X.ld, box, X.nbatch,
                                  X.batch_stride, row_bytes);
    };
    for (int i = 0; i < (split ? 2 : 1); ++i) {
        const void* a = i ? A.lo : A.hi;
        const void* b = i ? B.lo : B.hi;
        if (!(A.f32_source && i == 1) && !encode(&p.tmA[i], a, A, f32 || A.f32_source, a_box))
            return false;
        if (!encode(&p.tmB[i], b, B, f32, b_box)) return false;
    }
    p.a_mn = A.mn_major ? 1 : 0;
    p.b_mn = B.mn_major ? 1 : 0;
    if (A.f32_source) p.tmA[1] = p.tmA[0];
    if (!split) {
        p.tmA[1] = p.tmA[0];
        p.tmB[1] = p.tmB[0];
    }
    p.M = int32_t(A.rows);
    p.N = int32_t(B.rows);
    p.Kred = int32_t(A.cols);
    p.nbatch = int32_t(A.nbatch);
    p.tile_n = tile_n;
    p.m_tiles = int32_t((A.rows + bm - 1) / bm);
    p.n_tiles = int32_t((B.rows + tile_n - 1) / tile_n);
    const int kb_total = int((A.cols + elems - 1) / elems) * int(A.nbatch);
    if (k_splits < 1) k_splits = 1;
    if (k_splits > kb_total) k_splits = kb_total;
    p.kb_per_split = (kb_total + k_splits - 1) / k_splits;
    p.k_splits = (kb_total + p.kb_per_split - 1) / p.kb_per_split;
    p.tile_start = 0;
    p.m_tile0 = 0;
    p.atomic = 0;
    p.sc[0] = scatter_rowmajor(B.rows);
    return true;
}

TcScatter scatter_rowmajor(int64_t ld) {
    TcScatter sc{};
    sc.out_off = 0;
    sc.rows_per_op = 1 << 30;
    sc.s_op = 0;
    sc.s_row = ld;
    sc.col_div = 1;
    sc.s_col_hi = 1;
    sc.s_col_lo = 0;
    sc.op_off = nullptr;
    return sc;
}

}  // namespace dmrg
