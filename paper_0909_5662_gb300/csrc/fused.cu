// fused.cu -- the rotation O'_k = U^T (O_k (x) I_d) U (Sec. 3.2: Z R^+ and then
// R (Z R^+)) in one tensor-core kernel that keeps the intermediate product on chip.
//
// Work unit: one operator k and one block of 128 output columns beta.  For every site
// state s and every chunk of 128 rows i of O_k the unit forms
//     T^T[beta][i]       = sum_j  U[j d + s][beta] O_k[i][j]            (TMEM, FP32)
// splits it into a BF16 hi/lo pair in shared memory, and accumulates
//     O'_k^T[beta][alpha] += sum_i T^T[beta][i] U[i d + s][alpha]        (TMEM, FP32)
// so T never reaches global memory.  The accumulator holds all m' <= 256 columns alpha;
// the two T accumulators (128 columns each) alternate, so the first product of chunk
// c + 1 runs on the tensor core while the epilogue warps convert chunk c.
//
//   warp 0   : TMA producer (64-byte-swizzled K-major tiles, one ring of 32 KB stages
//              shared by both products, in the order the MMA issuer consumes them);
//   warp 1   : MMA issuer (tcgen05.mma kind::f16, BF16x3: lo*hi + hi*lo + hi*hi);
//   warps 2-5: epilogue (T: TMEM -> BF16 hi/lo -> shared memory; O': TMEM -> global).
//
// Operands (packed by the caller): O hi/lo as K x m rows of m (row stride ld), and
// Pu hi/lo with Pu[s][x][j] = U[j d + s][x] as d x m' rows of m (row stride ld).
// Reductions longer than the accumulation chain are cut: at a chain end the epilogue
// adds the accumulator into the output (stores the first chain), in a fixed order.
//
// Opt-in (DMRG_OPT_FUSED_ROTATION): at m = 400, d = 4 it is slower than the two products
// for every m' it supports.  A unit re-streams O_k once per site state and the U panel
// once per chunk, a 32 KB stage feeds only 400 cycles of MMAs, and the tensor pipe is
// 26 % active with no other unit near its limit (latency along the chain from the first
// product through the epilogue warps to the second).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "ptx.cuh"
#include "tc_common.cuh"

namespace dmrg {
namespace {

using namespace tcdev;

constexpr int kFThreads = 192;                  // producer, MMA issuer, 4 epilogue warps
constexpr int kFStages = 4;
constexpr int kIC = 128;                        // rows i of O_k per chunk
constexpr int kKB = 32;                         // reduction elements per k-block (64 B rows)
constexpr uint32_t kSlotBytes = 32768;          // one ring stage
constexpr uint32_t kTile = 128 * 64;            // 128 rows x 64 bytes
constexpr uint32_t kB2Lo = 16384;               // offset of the lo half of a B2 stage
constexpr uint32_t kTsmBytes = 4 * 2 * kTile;   // T chunk: 4 k-blocks x (hi, lo)
constexpr uint32_t kTaccCol = 256;              // T accumulators at TMEM columns 256, 384
constexpr uint64_t kFDrainNs = 2000000000ull;

struct FusedLaunch {
    CUtensorMap tmO[2];    // O hi/lo: (j, i, k), box 32 x 128
    CUtensorMap tmUa[2];   // Pu hi/lo: (j, x, s), box 32 x 128 (first product's A)
    CUtensorMap tmUb[2];   // Pu hi/lo: (i, x, s), box 32 x slice_b (second product's B)
    float* out;            // K x m' x m' (row-major O'_k[alpha][beta])
    int K, m, d, mp, mpp, nb, chain_chunks;
    int units;                 // (operator, output block) pairs
    int slice_b;               // rows of the second product's U tile (m' rounded up to 16)
    unsigned* status;
    uint64_t timeout_ns;
};

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t e) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
                 "r"(e)
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo_elem, __nv_bfloat16 hi_elem) {
    return uint32_t(__bfloat16_as_ushort(lo_elem)) | (uint32_t(__bfloat16_as_ushort(hi_elem)) << 16);
}

__global__ void __launch_bounds__(kFThreads, 1) fused_rotate_kernel(const __grid_constant__ FusedLaunch L) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* ring = smem;
    uint8_t* tsm = smem + size_t(kFStages) * kSlotBytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(tsm + kTsmBytes);
    uint64_t* empty = full + kFStages;
    uint64_t* tacc_full = empty + kFStages;   // [2]
    uint64_t* tacc_empty = tacc_full + 2;     // [2]
    uint64_t* tsm_full = tacc_empty + 2;
    uint64_t* tsm_empty = tsm_full + 1;
    uint64_t* oacc_full = tsm_empty + 1;
    uint64_t* oacc_empty = oacc_full + 1;
    uint64_t* drain = oacc_empty + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
    int* zero_flag = abort_flag + 1;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kFStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tacc_full[a], 1);
            mbar_init(&tacc_empty[a], 4);
        }
        mbar_init(tsm_full, 4);
        mbar_init(tsm_empty, 1);
        mbar_init(oacc_full, 1);
        mbar_init(oacc_empty, 4);
        mbar_init(drain, 1);
        *abort_flag = 0;
        *zero_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc<512>(tmem_slot);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    volatile int* vabort = abort_flag;
    const uint64_t tmo = L.timeout_ns;
    griddep_wait();
    griddep_launch_dependents();

    const int m = L.m, nIC = (m + kIC - 1) / kIC, nch = L.d * nIC;
    const int nkb1 = (m + kKB - 1) / kKB;
    auto rows_in = [&](int c) { return min(kIC, m - (c % nIC) * kIC); };
    auto nkb2 = [&](int c) { return (rows_in(c) + kKB - 1) / kKB; };
    const int cc = L.chain_chunks;
    const int cta = int(blockIdx.x), ncta = int(gridDim.x);
    auto chain_first = [&](int c) { return c % cc == 0; };
    auto chain_last = [&](int c) { return c % cc == cc - 1 || c == nch - 1; };

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            for (int i = 0; i < 2; ++i) {
                tma_prefetch_desc(&L.tmO[i]);
                tma_prefetch_desc(&L.tmUa[i]);
                tma_prefetch_desc(&L.tmUb[i]);
            }
            int stage = 0;
            uint32_t phase = 0;
            uint32_t armed = 0, armed_parity = 0;
            bool ok = true;
            const uint32_t bytes1 = 4 * kTile;
            const uint32_t bytes2 = 2u * uint32_t(L.slice_b) * 64u;
            auto acquire = [&](uint32_t bytes) -> bool {
                if (!mbar_wait(&empty[stage], phase ^ 1u, tmo, L.status, vabort)) return false;
                mbar_arrive_expect_tx(&full[stage], bytes);
                return true;
            };
            auto advance = [&]() {
                armed |= 1u << stage;
                armed_parity = (armed_parity & ~(1u << stage)) | (phase << stage);
                if (++stage == kFStages) {
                    stage = 0;
                    phase ^= 1u;
                }
            };
            for (int t = cta; t < L.units && ok; t += ncta) {
                const int k = t / L.nb, b = t % L.nb;
                auto load1 = [&](int c) -> bool {
                    const int s = c / nIC, i0 = (c % nIC) * kIC;
                    for (int kb = 0; kb < nkb1; ++kb) {
                        if (!acquire(bytes1)) return false;
                        uint8_t* sl = ring + size_t(stage) * kSlotBytes;
                        const int x = kb * kKB;
                        const int ya = b * 128;
                        tma_load_3d(sl, &L.tmUa[0], &full[stage], x, ya, s);
                        tma_load_3d(sl + kTile, &L.tmUa[1], &full[stage], x, ya, s);
                        tma_load_3d(sl + 2 * kTile, &L.tmO[0], &full[stage], x, i0, k);
                        tma_load_3d(sl + 3 * kTile, &L.tmO[1], &full[stage], x, i0, k);
                        advance();
                    }
                    return true;
                };
                auto load2 = [&](int c) -> bool {
                    const int s = c / nIC, i0 = (c % nIC) * kIC;
                    for (int kb = 0; kb < nkb2(c); ++kb) {
                        if (!acquire(bytes2)) return false;
                        uint8_t* sl = ring + size_t(stage) * kSlotBytes;
                        const int x = i0 + kb * kKB;
                        tma_load_3d(sl, &L.tmUb[0], &full[stage], x, 0, s);
                        tma_load_3d(sl + kB2Lo, &L.tmUb[1], &full[stage], x, 0, s);
                        advance();
                    }
                    return true;
                };
                ok = load1(0);
                for (int c = 1; c < nch && ok; ++c) ok = load1(c) && load2(c - 1);
                if (ok) ok = load2(nch - 1);
            }
            for (int s = 0; s < kFStages; ++s)
                if (armed & (1u << s))
                    mbar_wait(&full[s], (armed_parity >> s) & 1u, kFDrainNs, L.status, zero_flag);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t g1 = 0, g2 = 0, gd = 0;   // T accumulations, T conversions used, drains
            bool ok = true;
            const uint32_t idesc2 = make_idesc(1u, uint32_t(L.mpp));
            auto release = [&]() { mma_commit(&empty[stage]); };
            auto next = [&]() {
                if (++stage == kFStages) {
                    stage = 0;
                    phase ^= 1u;
                }
            };
            auto mma1 = [&](int c) -> bool {
                // N trimmed to the chunk's rows (rounded up to 16; the columns past m are
                // zero, and the second product reads no column past the chunk's rows)
                const uint32_t idesc1 = make_idesc(1u, uint32_t((rows_in(c) + 15) & ~15));
                const uint32_t tb = g1 & 1u;
                if (!mbar_wait(&tacc_empty[tb], ((g1 >> 1) & 1u) ^ 1u, tmo, L.status, vabort))
                    return false;
                tc_fence_after();
                const uint32_t td = tmem_base + kTaccCol + tb * kIC;
                for (int kb = 0; kb < nkb1; ++kb) {
                    if (!mbar_wait(&full[stage], phase, tmo, L.status, vabort)) return false;
                    tc_fence_after();
                    const uint32_t sl = smem_u32(ring + size_t(stage) * kSlotBytes);
                    const uint64_t ah = smem_desc_kmajor<64>(sl), al = smem_desc_kmajor<64>(sl + kTile);
                    const uint64_t bh = smem_desc_kmajor<64>(sl + 2 * kTile);
                    const uint64_t bl = smem_desc_kmajor<64>(sl + 3 * kTile);
                    const int steps = min(2, (m - kb * kKB + 15) / 16);
                    for (int q = 0; q < steps; ++q) {
                        const uint64_t off = uint64_t(q) * 2;
                        mma_bf16(td, al + off, bh + off, idesc1, (kb > 0 || q > 0) ? 1u : 0u);
                        mma_bf16(td, ah + off, bl + off, idesc1, 1u);
                        mma_bf16(td, ah + off, bh + off, idesc1, 1u);
                    }
                    release();
                    next();
                }
                mma_commit(&tacc_full[tb]);
                ++g1;
                return true;
            };
            auto mma2 = [&](int c) -> bool {
                if (chain_first(c)) {
                    if (!mbar_wait(oacc_empty, (gd & 1u) ^ 1u, tmo, L.status, vabort)) return false;
                }
                if (!mbar_wait(tsm_full, g2 & 1u, tmo, L.status, vabort)) return false;
                tc_fence_after();
                const int rows = rows_in(c);
                for (int kb = 0; kb < nkb2(c); ++kb) {
                    if (!mbar_wait(&full[stage], phase, tmo, L.status, vabort)) return false;
                    tc_fence_after();
                    const uint32_t sl = smem_u32(ring + size_t(stage) * kSlotBytes);
                    const uint32_t ta = smem_u32(tsm) + uint32_t(kb) * 2 * kTile;
                    const uint64_t th = smem_desc_kmajor<64>(ta), tl = smem_desc_kmajor<64>(ta + kTile);
                    const uint64_t bh = smem_desc_kmajor<64>(sl), bl = smem_desc_kmajor<64>(sl + kB2Lo);
                    const int steps = min(2, (rows - kb * kKB + 15) / 16);
                    for (int q = 0; q < steps; ++q) {
                        const uint64_t off = uint64_t(q) * 2;
                        const uint32_t acc = (chain_first(c) && kb == 0 && q == 0) ? 0u : 1u;
                        mma_bf16(tmem_base, tl + off, bh + off, idesc2, acc);
                        mma_bf16(tmem_base, th + off, bl + off, idesc2, 1u);
                        mma_bf16(tmem_base, th + off, bh + off, idesc2, 1u);
                    }
                    release();
                    next();
                }
                mma_commit(tsm_empty);
                ++g2;
                if (chain_last(c)) {
                    mma_commit(oacc_full);
                    ++gd;
                }
                return true;
            };
            for (int t = cta; t < L.units && ok; t += ncta) {
                ok = mma1(0);
                for (int c = 1; c < nch && ok; ++c) ok = mma1(c) && mma2(c - 1);
                if (ok) ok = mma2(nch - 1);
            }
            mma_commit(drain);
            mbar_wait(drain, 0, kFDrainNs, L.status, zero_flag);
        }
    } else {
        // ------------------------------------------------------------ epilogue (warps 2..5)
        const int quad = warp & 3;                 // TMEM lanes [32 quad, 32 quad + 32)
        const int row = quad * 32 + lane;          // beta within the block
        const uint32_t lane_off = uint32_t(quad * 32) << 16;
        uint32_t g1 = 0, g2 = 0, gd = 0;
        bool ok = true;
        auto wait_warp = [&](uint64_t* bar, uint32_t parity) -> bool {
            int v = 1;
            if (lane == 0) v = mbar_wait(bar, parity, tmo, L.status, vabort) ? 1 : 0;
            return __shfl_sync(0xffffffffu, v, 0) != 0;
        };
        auto convert = [&](int c) -> bool {
            const uint32_t tb = g1 & 1u;
            if (!wait_warp(&tacc_full[tb], (g1 >> 1) & 1u)) return false;
            if (!wait_warp(tsm_empty, (g2 & 1u) ^ 1u)) return false;
            tc_fence_after();
            const uint32_t tbase = smem_u32(tsm);
            const uint32_t sw = uint32_t((row >> 1) & 3);
            for (int kb = 0; kb < nkb2(c); ++kb) {
                uint32_t r[32];
                tmem_ld_32x32b_x32(tmem_base + lane_off + kTaccCol + tb * kIC + uint32_t(kb) * 32, r);
                tmem_ld_wait();
                const uint32_t hi_tile = tbase + uint32_t(kb) * 2 * kTile + uint32_t(row) * 64;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint32_t h[4], l[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        __nv_bfloat16 h0, l0, h1, l1;
                        split_bf16(__uint_as_float(r[8 * q + 2 * e]), h0, l0);
                        split_bf16(__uint_as_float(r[8 * q + 2 * e + 1]), h1, l1);
                        h[e] = pack2(h0, h1);
                        l[e] = pack2(l0, l1);
                    }
                    const uint32_t chunk = (uint32_t(q) ^ sw) << 4;
                    st_shared_v4(hi_tile + chunk, h[0], h[1], h[2], h[3]);
                    st_shared_v4(hi_tile + kTile + chunk, l[0], l[1], l[2], l[3]);
                }
            }
            fence_proxy_async_smem();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&tacc_empty[tb]);
                mbar_arrive(tsm_full);
            }
            ++g1;
            ++g2;
            return true;
        };
        auto drain_out = [&](int k, int b, int c) -> bool {
            if (!wait_warp(oacc_full, gd & 1u)) return false;
            tc_fence_after();
            const int beta = b * 128 + row;
            const bool first = (c / cc) == 0;
            float* outk = L.out + int64_t(k) * L.mp * L.mp;
            for (int a0 = 0; a0 < L.mpp; a0 += 32) {
                uint32_t r[32];
                tmem_ld_32x32b_x32(tmem_base + lane_off + uint32_t(a0), r);
                tmem_ld_wait();
                if (beta >= L.mp) continue;
                const int amax = min(32, L.mp - a0);
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    if (q >= amax) break;
                    float* p = outk + int64_t(a0 + q) * L.mp + beta;
                    const float v = __uint_as_float(r[q]);
                    *p = first ? v : *p + v;
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(oacc_empty);
            ++gd;
            return true;
        };
        for (int t = cta; t < L.units && ok; t += ncta) {
            const int k = t / L.nb, b = t % L.nb;
            for (int c = 0; c < nch && ok; ++c) {
                ok = convert(c);
                if (ok && c >= 1 && chain_last(c - 1)) ok = drain_out(k, b, c - 1);
            }
            if (ok) ok = drain_out(k, b, nch - 1);
        }
    }

    tc_fence_before();
    __syncthreads();
    if (*vabort) {
        // After an expired wait, copies issued before it may still be landing here.
        const uint64_t t0 = globaltimer_ns();
        while (globaltimer_ns() - t0 < 1000000ull) __nanosleep(1000);
    }
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc<512>(tmem_base);
    }
}

}  // namespace

size_t fused_smem_bytes() {
    return 1024 + size_t(kFStages) * kSlotBytes + kTsmBytes + 8 * (2 * kFStages + 9) + 16;
}

cudaError_t fused_rotate_launch(const FusedArgs& a, cudaStream_t s) {
    if (a.K <= 0) return cudaSuccess;
    if (a.mp < 1 || a.mp > kFusedMaxMp || a.m < 1 || a.d < 1) return cudaErrorInvalidValue;
    FusedLaunch L{};
    const int mpp = (int(a.mp) + 15) / 16 * 16;
    L.slice_b = mpp;
    for (int i = 0; i < 2; ++i) {
        if (!encode_operand_map(&L.tmO[i], a.Op[i], false, a.m, a.m, a.ld, kIC, a.K,
                                int64_t(a.m) * a.ld, 64) ||
            !encode_operand_map(&L.tmUa[i], a.Pu[i], false, a.mp, a.m, a.ld, 128, a.d,
                                int64_t(a.mp) * a.ld, 64) ||
            !encode_operand_map(&L.tmUb[i], a.Pu[i], false, a.mp, a.m, a.ld, L.slice_b, a.d,
                                int64_t(a.mp) * a.ld, 64))
            return cudaErrorInvalidValue;
    }
    L.out = a.out;
    L.K = int(a.K);
    L.m = int(a.m);
    L.d = a.d;
    L.mp = int(a.mp);
    L.mpp = mpp;
    L.nb = (int(a.mp) + 127) / 128;
    const int64_t units = a.K * L.nb;   // (operator, output block)
    if (units > 0x7fffffffLL) return cudaErrorInvalidValue;
    L.units = int(units);
    const int nIC = (L.m + kIC - 1) / kIC;
    const int nch = L.d * nIC;
    // chains of whole chunks: at most accum_chain reduction elements each (0 = one chain)
    L.chain_chunks = a.accum_chain > 0 ? std::max(1, int(a.accum_chain / kIC)) : nch;
    L.status = a.status;
    L.timeout_ns = a.timeout_ns;
    const size_t smem = fused_smem_bytes();
    if (smem > 232448) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(fused_rotate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem));
    if (e != cudaSuccess) return e;
    const int ctas = std::max(1, std::min(a.grid, L.units));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(ctas), 1, 1);
    cfg.blockDim = dim3(kFThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fused_rotate_kernel, L);
}

}  // namespace dmrg
