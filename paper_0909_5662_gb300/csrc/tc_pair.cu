// tc_pair.cu -- tcgen05 GEMM on CTA pairs (cta_group::2), sm_103a.
//
// The same persistent pipeline as tc.cu, but two CTAs (a pair) compute one
// 256 x N tile together: each CTA stages its 128 rows of A and half of the N rows
// of B in its own shared memory, and one thread of the even ("leader") CTA issues
// tcgen05.mma.cta_group::2, which reads both CTAs' operands and accumulates each
// CTA's 128 rows in that CTA's TMEM.  Per SM this halves the shared-memory and L2
// traffic of the B operand, which bounds the one-CTA kernel.
//
// Every TMA load lands in the shared memory of the CTA that issues it; only the
// completion (the mbarrier's transaction count) is signalled in the leader.
//
// Protocol (every wait bounded, as in the one-CTA kernel):
//   * all TMA loads landing in a pair complete on its leader's full[s] barrier
//     (the leader arms it with the bytes of both CTAs);
//   * the leader's commits arrive on empty[s] of both CTAs of the pair (a stage
//     is refilled only when the MMAs that read it are done), and on the
//     accumulator-full barrier of both CTAs;
//   * the epilogue warps of both CTAs arrive on their leader's accumulator-empty
//     barrier (the peer through its shared::cluster address);
//   * cluster barriers after set-up and before teardown keep any CTA from leaving
//     while another may still reach its barriers, its shared memory or TMEM.
//
// Converting form (CONV): the A operand arrives as an unconverted FP32 matrix (the
// operators O as the caller stores them).  Each CTA's A tile lands, 128-byte
// swizzled, on that CTA's own afull[s] barrier; four converter warps then turn it
// into the MMA operand in place, one row per lane: BF16X3 reads the 64 floats of
// its row from the two 32-float boxes and writes the row's BF16 hi part over the
// first box and the lo part over the second (the layout the MMA reads); TF32 rounds
// the 32 floats of its row to TF32 where they are.  A lane touches only its own
// row, so no other lane's data is overwritten before it is read.  Each converter
// warp then makes its writes visible to the tensor core (proxy fence) and arrives on
// the leader's full[s], which in this form counts the B bytes of both CTAs and eight
// converter arrivals.  This replaces a separate packing pass over O in global
// memory (a read and a write of the whole operator batch).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <vector>

#include "internal.h"
#include "ptx.cuh"
#include "tc_common.cuh"

namespace dmrg {
namespace {

using namespace tcdev;

constexpr int kThreads = 320;         // producer, MMA issuer, 8 epilogue warps (per CTA)
constexpr int kThreadsConv = 448;     // ... and 4 converter warps (converting form)
constexpr int kConvWarp0 = 10;
constexpr int kEpiWarps = 8;
constexpr int kBM = 128;              // rows per CTA (TMEM lanes)
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccStride = 256;
constexpr uint64_t kDrainTimeoutNs = 2000000000ull;

// MMA width of an N tile with `left` columns remaining: a multiple of 16 (each CTA
// then holds whole 8-row swizzle atoms of B), at least 32.
__device__ __forceinline__ int pair_n(int tile_n, int left) {
    const int n = min(tile_n, left);
    return max(32, (n + 15) & ~15);
}

__device__ __forceinline__ void ld_shared_v4(uint32_t addr, float4& v) {
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr)
                 : "memory");
}

__device__ __forceinline__ void st_shared_v4u(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                              uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
                 "r"(d)
                 : "memory");
}

// BF16 hi/lo of two floats as packed pairs: hi = bf16(x), lo = bf16(x - hi).
__device__ __forceinline__ void split2(float x, float y, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(x - hf.x, y - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ void fence_proxy_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void st_shared_v2u(uint32_t addr, uint32_t a, uint32_t b) {
    asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(a), "r"(b) : "memory");
}
__device__ __forceinline__ void st_shared_u32(uint32_t addr, uint32_t a) {
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"(a) : "memory");
}

__device__ __forceinline__ void st_shared_u16(uint32_t addr, uint16_t a) {
    asm volatile("st.shared.b16 [%0], %1;" ::"r"(addr), "h"(a) : "memory");
}

// TMA-store epilogue, site-interleaved layout (TcLaunch::t_store = kStoreSiteInterleaved,
// t_store_d = d): one 32-column chunk of this warp's 32 rows, split into BF16 hi/lo,
// staged in the warp's 4 KB of shared memory `stg` and sent out by lane 0 as up to four
// bulk tensor stores.  The chunk covers 32 / d values of b
// and the warp's rows are two groups of 16 consecutive rows i (each inside one operator,
// rows_per_op being a multiple of 16): the staging holds one store box per (group, half):
// hi at stg + group * 1024, lo 2048 further, each box 32 / d rows b of 16 d elements
// (i * d + s).  Lane l's values of (b, s = 0..d-1) land in row b of its group's box at
// element (l % 16) * d.  x[g], z[g]: the box coordinates of group g (valid[g] = 0: the
// group lies past the last row); y = the chunk's first b.  A lane's r[] need not hold
// data when its group is not stored.
__device__ __forceinline__ void store_chunk_tma(const TcLaunch& L, const uint32_t (&r)[32],
                                                uint32_t stg, int lane, int d, const int (&x)[2],
                                                int y, const int (&z)[2], const bool (&valid)[2]) {
    if (lane == 0) bulk_wait_group_read0();   // the previous chunk's stores have read stg
    __syncwarp();
    const uint32_t box = stg + uint32_t(lane >> 4) * 1024u + uint32_t(lane & 15) * uint32_t(2 * d);
    if (d == 4) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {   // row b = j: columns 4j .. 4j+3
            uint32_t h0, l0, h1, l1;
            split2(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]), h0, l0);
            split2(__uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]), h1, l1);
            st_shared_v2u(box + uint32_t(j) * 128u, h0, h1);
            st_shared_v2u(box + 2048u + uint32_t(j) * 128u, l0, l1);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {   // d = 2, row b = j: columns 2j, 2j+1
            uint32_t h0, l0;
            split2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]), h0, l0);
            st_shared_u32(box + uint32_t(j) * 64u, h0);
            st_shared_u32(box + 2048u + uint32_t(j) * 64u, l0);
        }
    }
    fence_proxy_async_shared();   // the staging writes, before the tensor stores read them
    __syncwarp();
    if (lane == 0) {
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            if (!valid[g]) continue;
            tma_store_3d(&L.t_store_map[0], stg + uint32_t(g) * 1024u, x[g], y, z[g]);
            tma_store_3d(&L.t_store_map[1], stg + 2048u + uint32_t(g) * 1024u, x[g], y, z[g]);
        }
        bulk_commit_group();
    }
}

// TMA-store epilogue, row-contiguous layout (TcLaunch::t_store = kStoreRowContiguous):
// column n = s * cdiv + j of row (k, i) goes to W[k][j][s * sch + i], so a lane's values
// run down a column of W.  The chunk is columns n .. n + 31 (16-aligned, cmax of them
// valid, a multiple of 16), in two halves h of 16 columns, each inside one s.  When the
// warp's 32 rows lie in one operator, half h is one box of 16 j x 32 i (64-byte rows)
// at stg + 1024 h (lo 2048 further), row j at 64 j bytes, lane i's element at 2 i.
// Otherwise each row group g of 16 has its own boxes of 16 j x 16 i at stg + (2 g + h) *
// 512, and at step j the upper half-warp writes column (j + 1) mod 16, so that its row
// lies 32 bytes along the banks from the lower half's.  x[g] = i of group g's first row,
// z[g] its operator.
__device__ __forceinline__ void store_chunk_tma_rows(const TcLaunch& L, const uint32_t (&r)[32],
                                                     uint32_t stg, int lane, const int (&x)[2],
                                                     const int (&z)[2], const bool (&valid)[2],
                                                     int n, int cmax, int cdiv, int64_t sch) {
    if (lane == 0) bulk_wait_group_read0();   // the previous chunk's stores have read stg
    __syncwarp();
    const bool wide = valid[0] && valid[1] && z[0] == z[1];   // the same for the whole warp
    if (wide) {
        const uint32_t base = stg + uint32_t(lane) * 2u;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float v = __uint_as_float(r[16 * h + j]);
                const __nv_bfloat16 hb = __float2bfloat16_rn(v);
                const __nv_bfloat16 lb = __float2bfloat16_rn(v - __bfloat162float(hb));
                const uint32_t a = base + uint32_t(h) * 1024u + uint32_t(j) * 64u;
                st_shared_u16(a, __bfloat16_as_ushort(hb));
                st_shared_u16(a + 2048u, __bfloat16_as_ushort(lb));
            }
        }
    } else {
        const bool up = lane >= 16;
        const uint32_t base = stg + (up ? 1024u : 0u) + uint32_t(lane & 15) * 2u;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int ju = (j + 1) & 15;
                const float v = __uint_as_float(up ? r[16 * h + ju] : r[16 * h + j]);
                const __nv_bfloat16 hb = __float2bfloat16_rn(v);
                const __nv_bfloat16 lb = __float2bfloat16_rn(v - __bfloat162float(hb));
                const uint32_t a = base + uint32_t(h) * 512u + uint32_t(up ? ju : j) * 32u;
                st_shared_u16(a, __bfloat16_as_ushort(hb));
                st_shared_u16(a + 2048u, __bfloat16_as_ushort(lb));
            }
        }
    }
    fence_proxy_async_shared();   // the staging writes, before the tensor stores read them
    __syncwarp();
    if (lane == 0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (16 * h >= cmax) continue;
            const int nh = n + 16 * h;
            const int s = nh / cdiv;
            const int y = nh - s * cdiv;
            if (wide) {
                const int xw = int(int64_t(s) * sch) + x[0];
                const uint32_t box = stg + uint32_t(h) * 1024u;
                tma_store_3d(&L.t_store_map[0], box, xw, y, z[0]);
                tma_store_3d(&L.t_store_map[1], box + 2048u, xw, y, z[0]);
                continue;
            }
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                if (!valid[g]) continue;
                const int xg = int(int64_t(s) * sch) + x[g];
                const uint32_t box = stg + uint32_t(2 * g + h) * 512u;
                tma_store_3d(&L.t_store_map[2], box, xg, y, z[g]);
                tma_store_3d(&L.t_store_map[3], box + 2048u, xg, y, z[g]);
            }
        }
        bulk_commit_group();
    }
}

// TMA-store epilogue, site-major layout (TcLaunch::t_store = kStoreSiteMajor): column
// n = s * o2_m + j of row (k, i) goes to out2_k[s * rps + i][j], so a lane's values of a
// chunk are contiguous in a row of out2_k.  The chunk is columns n .. n + 31 (16-aligned,
// cmax of them valid).  When all 32 lie in one site, each row group g of 16 has one box
// of 16 i x 32 j (64-byte rows, 64-byte swizzle: 16-byte piece q of row i at
// q ^ ((i >> 1) & 3)) at stg + 1024 g (lo 2048 further).  Otherwise each half h of 16
// columns has its own boxes of 16 i x 16 j (32-byte rows, 32-byte swizzle: piece q at
// q ^ ((i >> 2) & 1)) at stg + (2 g + h) * 512.  With either swizzle the 16-byte stores
// of any eight lanes fall in distinct banks.  x[g] = i of group g's first row, z[g] its
// operator.
__device__ __forceinline__ void store_chunk_tma_site(const TcLaunch& L, const uint32_t (&r)[32],
                                                     uint32_t stg, int lane, const int (&x)[2],
                                                     const int (&z)[2], const bool (&valid)[2],
                                                     int n, int cmax, int o2m, int rps) {
    if (lane == 0) bulk_wait_group_read0();   // the previous chunk's stores have read stg
    __syncwarp();
    const int s0 = n / o2m;
    const int j0 = n - s0 * o2m;
    const bool wide = cmax == 32 && j0 + 32 <= o2m;   // the same for the whole warp
    const int li = lane & 15;
    if (wide) {
        const uint32_t row = stg + uint32_t(lane >> 4) * 1024u + uint32_t(li) * 64u;
        const uint32_t flip = uint32_t((li >> 1) & 3);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int e = 0; e < 4; ++e)
                split2(__uint_as_float(r[8 * q + 2 * e]), __uint_as_float(r[8 * q + 2 * e + 1]),
                       hw[e], lw[e]);
            const uint32_t a = row + ((uint32_t(q) ^ flip) << 4);
            st_shared_v4u(a, hw[0], hw[1], hw[2], hw[3]);
            st_shared_v4u(a + 2048u, lw[0], lw[1], lw[2], lw[3]);
        }
    } else {
        const uint32_t row = stg + uint32_t(lane >> 4) * 1024u + uint32_t(li) * 32u;
        const uint32_t flip = uint32_t((li >> 2) & 1);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                uint32_t hw[4], lw[4];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    split2(__uint_as_float(r[16 * h + 8 * q + 2 * e]),
                           __uint_as_float(r[16 * h + 8 * q + 2 * e + 1]), hw[e], lw[e]);
                const uint32_t a = row + uint32_t(h) * 512u + ((uint32_t(q) ^ flip) << 4);
                st_shared_v4u(a, hw[0], hw[1], hw[2], hw[3]);
                st_shared_v4u(a + 2048u, lw[0], lw[1], lw[2], lw[3]);
            }
        }
    }
    fence_proxy_async_shared();   // the staging writes, before the tensor stores read them
    __syncwarp();
    if (lane == 0) {
        if (wide) {
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                if (!valid[g]) continue;
                const uint32_t box = stg + uint32_t(g) * 1024u;
                tma_store_3d(&L.t_store_map[0], box, j0, s0 * rps + x[g], z[g]);
                tma_store_3d(&L.t_store_map[1], box + 2048u, j0, s0 * rps + x[g], z[g]);
            }
        } else {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (16 * h >= cmax) continue;
                const int nh = n + 16 * h;
                const int s = nh / o2m;
                const int j = nh - s * o2m;
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    if (!valid[g]) continue;
                    const uint32_t box = stg + uint32_t(2 * g + h) * 512u;
                    tma_store_3d(&L.t_store_map[2], box, j, s * rps + x[g], z[g]);
                    tma_store_3d(&L.t_store_map[3], box + 2048u, j, s * rps + x[g], z[g]);
                }
            }
        }
        bulk_commit_group();
    }
}

// The site-interleaved layout for FP32 (TF32-rounded) output: one 4 KB staging buffer, the
// box of group g (16 d floats x 32 / d rows b) at stg + 2048 g; lane l's values of (b,
// s = 0..d-1) land in row b at float (l % 16) * d.  One map, t_store_map[0].
__device__ __forceinline__ void store_chunk_tma_f32(const TcLaunch& L, const uint32_t (&r)[32],
                                                    uint32_t stg, int lane, int d, const int (&x)[2],
                                                    int y, const int (&z)[2], const bool (&valid)[2]) {
    if (lane == 0) bulk_wait_group_read0();   // the previous chunk's stores have read stg
    __syncwarp();
    const uint32_t box = stg + uint32_t(lane >> 4) * 2048u + uint32_t(lane & 15) * uint32_t(4 * d);
    if (d == 4) {
#pragma unroll
        for (int j = 0; j < 8; ++j)   // row b = j: columns 4j .. 4j+3
            st_shared_v4u(box + uint32_t(j) * 256u, __float_as_uint(tf32_round(__uint_as_float(r[4 * j]))),
                          __float_as_uint(tf32_round(__uint_as_float(r[4 * j + 1]))),
                          __float_as_uint(tf32_round(__uint_as_float(r[4 * j + 2]))),
                          __float_as_uint(tf32_round(__uint_as_float(r[4 * j + 3]))));
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j)   // d = 2, row b = j: columns 2j, 2j+1
            st_shared_v2u(box + uint32_t(j) * 128u, __float_as_uint(tf32_round(__uint_as_float(r[2 * j]))),
                          __float_as_uint(tf32_round(__uint_as_float(r[2 * j + 1]))));
    }
    fence_proxy_async_shared();   // the staging writes, before the tensor stores read them
    __syncwarp();
    if (lane == 0) {
#pragma unroll
        for (int g = 0; g < 2; ++g)
            if (valid[g]) tma_store_3d(&L.t_store_map[0], stg + uint32_t(g) * 2048u, x[g], y, z[g]);
        bulk_commit_group();
    }
}

// TMA-store epilogue, columns layout for FP32 output (TcLaunch::t_store =
// kStoreColumnsF32): column n of row (k, i) goes to out_k[n][i], so a lane's values run
// down a column of out_k.  The chunk (columns n .. n + 31, cmax of them valid, a multiple
// of 16) is up to four boxes of 16 n x 16 i: box (g, h) for row group g and column half
// h at stg + (2 g + h) * 1024, row j (column n + 16 h + j) at 64 j bytes, lane i's value at
// 4 (i % 16) (the two half-warps' 64-byte rows share banks: two wavefronts per store,
// which costs less than the registers a rotation of the upper half's columns took).
// reduce: the boxes are added to the
// output (a tile's later chains, the parts of a split tile).  drain (the warp's first
// chunk of a chain that adds): the lane first waits until its earlier bulk operations
// have completed, so that the chain's additions follow the stores of the chain before it;
// otherwise it waits only until they have read the staging.  x[g] = i of group g's first
// row, z[g] its operator.
__device__ __forceinline__ void store_chunk_tma_cols_f32(const TcLaunch& L, const uint32_t (&r)[32],
                                                         uint32_t stg, int lane, const int (&x)[2],
                                                         const int (&z)[2], const bool (&valid)[2],
                                                         int n, int cmax, bool reduce, bool drain) {
    if (lane == 0) {
        if (drain) bulk_wait_group0();
        else bulk_wait_group_read0();   // the previous chunk's stores have read stg
    }
    __syncwarp();
    const uint32_t base = stg + uint32_t(lane >> 4) * 2048u + uint32_t(lane & 15) * 4u;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int j = 0; j < 16; ++j) st_shared_u32(base + uint32_t(h * 1024 + j * 64), r[16 * h + j]);
    }
    fence_proxy_async_shared();   // the staging writes, before the tensor stores read them
    __syncwarp();
    if (lane == 0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (16 * h >= cmax) continue;
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                if (!valid[g]) continue;
                const uint32_t box = stg + uint32_t(2 * g + h) * 1024u;
                if (reduce) tma_reduce_add_3d(&L.t_store_map[0], box, x[g], n + 16 * h, z[g]);
                else tma_store_3d(&L.t_store_map[0], box, x[g], n + 16 * h, z[g]);
            }
        }
        bulk_commit_group();
    }
}

// Converts row `row` of this CTA's A tile in place (see the converting form above).
// box0 / box1: shared addresses of the two 128 x 128-byte regions of the stage's A.
template <int MODE>
__device__ __forceinline__ void convert_a_row(uint32_t box0, uint32_t box1, int row) {
    const uint32_t r0 = box0 + uint32_t(row) * 128u;
    const uint32_t sw = uint32_t(row & 7);
    if (MODE == TC_BF16X3) {
        const uint32_t r1 = box1 + uint32_t(row) * 128u;
        float4 v[16];   // v[c] = floats 4c .. 4c+3 of the row
#pragma unroll
        for (int c = 0; c < 8; ++c) ld_shared_v4(r0 + ((uint32_t(c) ^ sw) << 4), v[c]);
#pragma unroll
        for (int c = 0; c < 8; ++c) ld_shared_v4(r1 + ((uint32_t(c) ^ sw) << 4), v[8 + c]);
#pragma unroll
        for (int q = 0; q < 8; ++q) {   // 16-byte chunk q: elements 8q .. 8q+7
            uint32_t h[4], l[4];
            split2(v[2 * q].x, v[2 * q].y, h[0], l[0]);
            split2(v[2 * q].z, v[2 * q].w, h[1], l[1]);
            split2(v[2 * q + 1].x, v[2 * q + 1].y, h[2], l[2]);
            split2(v[2 * q + 1].z, v[2 * q + 1].w, h[3], l[3]);
            const uint32_t off = (uint32_t(q) ^ sw) << 4;
            st_shared_v4u(r0 + off, h[0], h[1], h[2], h[3]);
            st_shared_v4u(r1 + off, l[0], l[1], l[2], l[3]);
        }
    } else {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            // chunk c ^ sw: the eight lanes of a quarter warp (eight consecutive rows)
            // then touch eight different 16-byte bank groups
            const uint32_t a = r0 + ((uint32_t(c) ^ sw) << 4);
            float4 v;
            ld_shared_v4(a, v);
            st_shared_v4u(a, __float_as_uint(tf32_round(v.x)), __float_as_uint(tf32_round(v.y)),
                          __float_as_uint(tf32_round(v.z)), __float_as_uint(tf32_round(v.w)));
        }
    }
}

// SITE: the launch also writes the site-major second copy (TcLaunch::out2); a separate
// instantiation, so that the other launches do not carry its registers.
// MN: the launch has problems with MN-major operands (a separate instantiation, so that
// the others carry none of their per-k-block choices).
template <int MODE, int EPI, int RB, bool CONV, bool SITE, bool MN>
__global__ void __launch_bounds__(CONV ? kThreadsConv : kThreads, 1)
    tc_gemm_pair_kernel(const __grid_constant__ TcLaunch L, int stages, int bh_smem) {
    constexpr int kRowBytes = RB;
    constexpr bool kSplit = (MODE == TC_BF16X3);
    constexpr int kElem = (MODE == TC_TF32) ? 4 : 2;
    constexpr int kElemsPerRow = kRowBytes / kElem;
    constexpr int kUmmaK = 32 / kElem;
    constexpr int kStepsPerBlock = kElemsPerRow / kUmmaK;
    constexpr uint32_t kFmt = (MODE == TC_TF32) ? 2u : 1u;
    // MN-major operands: BF16 with 128-byte rows only (the host refuses other forms)
    constexpr bool kMnOk = MN && (MODE != TC_TF32) && (RB == 128) && !CONV;
    constexpr uint32_t kMnBoxBytes = uint32_t(kMnBox) * 128u;
    // FP32 output: the chains of a tile are summed in the output itself (the first chain
    // stores, later ones add with reductions).  Only the MN-major instantiation carries the
    // scratch code for FP32 and uses it when given the scratch (the launcher picks it for
    // every FP32 launch that is: the adjoint's dU products, up to eight chains per tile,
    // and second products of more than two chains, for which the reductions measured
    // slower); elsewhere the unused scratch code alone cost 2-3 % of the second product.
    constexpr bool kF32Out = (EPI == EPI_F32 || EPI == EPI_F32_ATOMIC);
    constexpr bool kScratchCode = !kF32Out || MN;
    const bool sum_in_out = kF32Out && (!MN || L.chunk_scratch == nullptr);

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t a_bytes = kBM * kRowBytes;
    const uint32_t b_bytes = uint32_t(bh_smem) * kRowBytes;  // half of the N tile
    const uint32_t stage_bytes = (a_bytes + b_bytes) * (kSplit ? 2 : 1);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + size_t(stages) * stage_bytes);
    uint64_t* empty = full + stages;
    uint64_t* tfull = empty + stages;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint64_t* afull = drain + 1;   // converting form: this CTA's A tile landed ([stages])
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(afull + stages);
    int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
    int* zero_flag = abort_flag + 1;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();   // 0: leader, 1: its peer
    constexpr uint32_t lead = 0;                // cluster rank of the leader
    const bool leader = (rank == 0);
    const int pair = blockIdx.x / 2;            // cluster index (tile schedule)
    const int npairs = gridDim.x / 2;
    constexpr uint16_t pair_mask = 3u;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            // converting form: the leader's arming plus one arrival per converter warp of
            // both CTAs
            mbar_init(&full[s], CONV ? 1 + 2 * 4 : 1);
            mbar_init(&empty[s], 1);
            if (CONV) mbar_init(&afull[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 2 * kEpiWarps);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        *zero_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc_pair<kTmemCols>(tmem_slot);
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();
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
        // ------------------------------------------------------------ TMA producer (both CTAs)
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
            uint32_t armed = 0;
            uint32_t armed_parity = 0;
            bool ok = true;
            for (int t = pair; t < L.total_tiles && ok; t += npairs) {
                const Decoded dt = decode_tile(L, t, kElemsPerRow);
                const TcProblem* P = dt.P;
                // both CTAs' bytes: A (128 rows each; counted on afull in the converting
                // form) and the B halves (tile_n / 2 rows each)
                const bool a_mn = kMnOk && P->a_mn, b_mn = kMnOk && P->b_mn;
                const uint32_t bytes =
                    2u * ((CONV ? 0u : a_bytes) +
                          (b_mn ? 2u * kMnBoxBytes : uint32_t(P->tile_n / 2) * kRowBytes)) *
                    (kSplit ? 2u : 1u);
                // converting form: this CTA's FP32 A tile, 128 rows x 32 floats per box
                const uint32_t a_tx = kSplit ? 2u * a_bytes : a_bytes;
                const int n_eff = pair_n(P->tile_n, P->N - dt.nt * P->tile_n);
                const int ya = dt.mt * (2 * kBM) + int(rank) * kBM;
                const int yb = dt.nt * P->tile_n + int(rank) * (n_eff / 2);
                for (int kb = dt.kb_begin; kb < dt.kb_end; ++kb) {
                    if (!mbar_wait(&empty[stage], phase ^ 1u, tmo, L.status, vabort)) {
                        ok = false;
                        break;
                    }
                    if (leader) mbar_arrive_expect_tx(&full[stage], bytes);
                    const uint32_t fb = mapa_shared(smem_u32(&full[stage]), lead);
                    const int z = kb / dt.kb_per_batch;
                    const int x = (kb - z * dt.kb_per_batch) * kElemsPerRow;
                    if (CONV) {
                        mbar_arrive_expect_tx(&afull[stage], a_tx);
                        tma_load_3d(stage_a(stage, 0), &P->tmA[0], &afull[stage], x, ya, z);
                        if (kSplit)
                            tma_load_3d(stage_a(stage, 1), &P->tmA[0], &afull[stage], x + 32, ya, z);
                    }
                    for (int h = 0; h < (kSplit ? 2 : 1); ++h) {
                        // an MN-major operand: two boxes of 64 rows, coordinates (row, k)
                        if (a_mn) {
                            tma_load_3d_pair(stage_a(stage, h), &P->tmA[h], fb, ya, x, z);
                            tma_load_3d_pair(stage_a(stage, h) + kMnBoxBytes, &P->tmA[h], fb,
                                             ya + kMnBox, x, z);
                        } else if (!CONV) {
                            tma_load_3d_pair(stage_a(stage, h), &P->tmA[h], fb, x, ya, z);
                        }
                        if (b_mn) {
                            tma_load_3d_pair(stage_b(stage, h), &P->tmB[h], fb, yb, x, z);
                            tma_load_3d_pair(stage_b(stage, h) + kMnBoxBytes, &P->tmB[h], fb,
                                             yb + kMnBox, x, z);
                        } else {
                            tma_load_3d_pair(stage_b(stage, h), &P->tmB[h], fb, x, yb, z);
                        }
                    }
                    armed |= 1u << stage;
                    armed_parity = (armed_parity & ~(1u << stage)) | (phase << stage);
                    if (++stage == stages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            // Tail.  The leader's full barriers count both CTAs' copies: once the last
            // armed phase of each stage completed, no copy of either CTA is in flight.
            // Each CTA then waits for the release of its last fill of every stage, so
            // that no commit of the leader still has an arrival on its way to this CTA
            // when it leaves.  After an abort the release waits give up at once.
            if (leader)
                for (int s = 0; s < stages; ++s)
                    if (armed & (1u << s))
                        mbar_wait(&full[s], (armed_parity >> s) & 1u, kDrainTimeoutNs, L.status,
                                  zero_flag);
            if (CONV)   // this CTA's own A copies
                for (int s = 0; s < stages; ++s)
                    if (armed & (1u << s))
                        mbar_wait(&afull[s], (armed_parity >> s) & 1u, kDrainTimeoutNs, L.status,
                                  zero_flag);
            if (ok)
                for (int s = 0; s < stages; ++s)
                    if (armed & (1u << s))
                        mbar_wait(&empty[s], (armed_parity >> s) & 1u, tmo, L.status, vabort);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer (leader)
        if (lane == 0 && leader) {
            int stage = 0;
            uint32_t phase = 0;
            int it = 0;   // accumulation chains issued (one TMEM accumulator each, alternating)
            bool ok = true;
            for (int t = pair; t < L.total_tiles && ok; t += npairs) {
                const Decoded dt = decode_tile(L, t, kElemsPerRow);
                const TcProblem* P = dt.P;
                const int n_eff = pair_n(P->tile_n, P->N - dt.nt * P->tile_n);
                const bool a_mn = kMnOk && P->a_mn, b_mn = kMnOk && P->b_mn;
                // transpose bits: A (bit 15) and B (bit 16) MN-major
                const uint32_t idesc = make_idesc_pair(kFmt, uint32_t(n_eff)) |
                                       (a_mn ? 1u << 15 : 0u) | (b_mn ? 1u << 16 : 0u);
                // descriptor advance per 16-element k-step, in 16-byte units: 32 bytes along
                // a K-major row, 16 rows of 128 bytes MN-major
                const uint64_t a_step = a_mn ? 128 : 2, b_step = b_mn ? 128 : 2;
                // the descriptors' fields other than the start address, per operand order
                const uint64_t a_bits = a_mn ? smem_desc_mn128(0, kMnBoxBytes) : smem_desc_kmajor<RB>(0);
                const uint64_t b_bits = b_mn ? smem_desc_mn128(0, kMnBoxBytes) : smem_desc_kmajor<RB>(0);
                auto desc = [&](uint8_t* base, uint64_t bits) -> uint64_t {
                    return bits | uint64_t((smem_u32(base) & 0x3FFFFu) >> 4);
                };
                const int chunk = (P->kb_chunk > 0 && (kF32Out || L.chunk_scratch)) ? P->kb_chunk
                                                                        : (dt.kb_end - dt.kb_begin);
                int kb0 = dt.kb_begin;
                do {   // one chain per chunk of k-blocks (at least one, even for an empty tile)
                    const int kb1 = (dt.kb_end - kb0 > chunk) ? kb0 + chunk : dt.kb_end;
                    const int acc = it & 1;
                    const uint32_t acc_parity = uint32_t(it >> 1) & 1u;
                    if (!mbar_wait(&tempty[acc], acc_parity ^ 1u, tmo, L.status, vabort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t tmem_d = tmem_base + uint32_t(acc) * kAccStride;
                    for (int kb = kb0; kb < kb1; ++kb) {
                        // (formed before the wait, off the path from the barrier to the MMA)
                        const int rem = P->Kred - (kb % dt.kb_per_batch) * kElemsPerRow;
                        const int steps = min(kStepsPerBlock, (rem + kUmmaK - 1) / kUmmaK);
                        const uint64_t ah = desc(stage_a(stage, 0), a_bits);
                        const uint64_t bh = desc(stage_b(stage, 0), b_bits);
                        const uint64_t al = kSplit ? desc(stage_a(stage, 1), a_bits) : 0;
                        const uint64_t bl = kSplit ? desc(stage_b(stage, 1), b_bits) : 0;
                        if (!(CONV ? mbar_wait_cluster(&full[stage], phase, tmo, L.status, vabort)
                                   : mbar_wait(&full[stage], phase, tmo, L.status, vabort))) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        for (int k = 0; k < steps; ++k) {
                            const uint64_t oa = uint64_t(k) * a_step, ob = uint64_t(k) * b_step;
                            const uint32_t accum = (kb > kb0 || k > 0) ? 1u : 0u;
                            if (MODE == TC_BF16X3) {
                                mma_bf16_pair(tmem_d, al + oa, bh + ob, idesc, accum);
                                mma_bf16_pair(tmem_d, ah + oa, bl + ob, idesc, 1u);
                                mma_bf16_pair(tmem_d, ah + oa, bh + ob, idesc, 1u);
                            } else if (MODE == TC_TF32) {
                                mma_tf32_pair(tmem_d, ah + oa, bh + ob, idesc, accum);
                            } else {
                                mma_bf16_pair(tmem_d, ah + oa, bh + ob, idesc, accum);
                            }
                        }
                        // Test hook: withhold one release so that both producers' bounded
                        // waits on this stage expire (a barrier that nothing arrives on).
                        const bool withhold = L.drop_arrival && pair == 0 && it == 0 && kb == kb0;
                        if (!withhold) mma_commit_pair(&empty[stage], pair_mask);
                        if (++stage == stages) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                    if (!ok) break;
                    mma_commit_pair(&tfull[acc], pair_mask);
                    ++it;
                    kb0 = kb1;
                } while (kb0 < dt.kb_end);
            }
            mma_commit_pair(drain, uint16_t(1u << lead));
            mbar_wait(drain, 0, kDrainTimeoutNs, L.status, zero_flag);
        }
    } else if (CONV && warp >= kConvWarp0) {
        // ------------------------------------------------------------ A converters (both CTAs)
        const int row = (warp - kConvWarp0) * 32 + lane;
        const uint32_t full0_lead = mapa_shared(smem_u32(&full[0]), lead);
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        for (int t = pair; t < L.total_tiles && ok; t += npairs) {
            const Decoded dt = decode_tile(L, t, kElemsPerRow);
            for (int kb = dt.kb_begin; kb < dt.kb_end; ++kb) {
                int got = 1;
                if (lane == 0) got = mbar_wait(&afull[stage], phase, tmo, L.status, vabort) ? 1 : 0;
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) {
                    ok = false;
                    break;
                }
                // the phase has completed: every lane's own (immediately successful) wait
                // orders the tile's bytes before its reads
                mbar_try_wait(&afull[stage], phase);
                convert_a_row<MODE>(smem_u32(stage_a(stage, 0)), smem_u32(stage_a(stage, 1)), row);
                fence_proxy_async_shared();
                __syncwarp();
                if (lane == 0) {
                    if (leader) mbar_arrive(&full[stage]);
                    else mbar_arrive_cluster(full0_lead + uint32_t(stage) * 8u);
                }
                if (++stage == stages) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue (both CTAs)
        const int quad = warp & 3;
        const int half = (warp - 2) >> 2;
        const uint32_t tempty_leader0 = mapa_shared(smem_u32(&tempty[0]), lead);
        const uint32_t tempty_leader1 = mapa_shared(smem_u32(&tempty[1]), lead);
        int it = 0;   // accumulation chains consumed, in the MMA issuer's order
        bool ok = true;
        // Running sums of a tile's chains, added to in FP32 with round to nearest: this
        // CTA's 128 x 256 block of the scratch, stored lane-interleaved so that a warp's
        // 16-byte accesses are contiguous: the float4 j of 32-column chunk ci of lane l of
        // TMEM lane quadrant q sits at float4 index ((q * 8 + ci) * 8 + j) * 32 + l.
        // FP32 epilogues mostly keep the running sums in the output (sum_in_out).
        float4* scr = (kScratchCode && L.chunk_scratch)
                          ? reinterpret_cast<float4*>(L.chunk_scratch) +
                                (int64_t(blockIdx.x) * 4 + quad) * (8 * 8 * 32) + lane
                          : nullptr;
        // TMA-store epilogue: this warp's 4 KB of staging after the barriers
        constexpr bool kStoreOk = !SITE;
        const int tst = kStoreOk ? L.t_store : 0;
        const int tsd = L.t_store_d;
        const uint32_t stg = smem_u32(smem + size_t(stages) * stage_bytes + 512) +
                             uint32_t(warp - 2) * 4096u;
        for (int t = pair; t < L.total_tiles && ok; t += npairs) {
            const Decoded dt = decode_tile(L, t, kElemsPerRow);
            const TcProblem* P = dt.P;
            const int row = dt.mt * (2 * kBM) + int(rank) * kBM + quad * 32 + lane;
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
                if (S.s_split) row_base += int64_t(dt.kb_begin / P->kb_per_split) * S.s_split;
            }
            const int cdiv = S.col_div;
            const int64_t sch = S.s_col_hi, scl = S.s_col_lo;
            const bool tile_atomic = P->atomic != 0;
            // store boxes of the warp's two 16-row groups (TMA-store epilogue)
            int bx[2] = {0, 0}, bz[2] = {0, 0};
            bool bvalid[2] = {false, false};
            if (tst) {
                const int rpo = tst == kStoreSiteMajor ? L.o2_rows_per_op : S.rows_per_op;
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    const int rg = row - lane + 16 * g;
                    bvalid[g] = rg < P->M && dt.kb_begin < dt.kb_end;
                    const int op = rg / rpo;
                    const int il = rg - op * rpo;
                    bx[g] = tst == kStoreSiteInterleaved ? il * tsd : il;
                    bz[g] = P->store_z0 + op;
                }
            }
            const int chunk = (P->kb_chunk > 0 && (kF32Out || scr)) ? P->kb_chunk
                                                                       : (dt.kb_end - dt.kb_begin);
            int kb0 = dt.kb_begin;
            bool first = true;
            do {
                const int kb1 = (dt.kb_end - kb0 > chunk) ? kb0 + chunk : dt.kb_end;
                const bool last = kb1 >= dt.kb_end;
                const int acc = it & 1;
                const uint32_t acc_parity = uint32_t(it >> 1) & 1u;
                int got = 1;
                if (lane == 0) got = mbar_wait(&tfull[acc], acc_parity, tmo, L.status, vabort) ? 1 : 0;
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int c = half * 32; c < ncols; c += 64) {
                    uint32_t r[32];
                    tmem_ld_32x32b_x32(tmem_base + uint32_t(acc) * kAccStride +
                                           (uint32_t(quad * 32) << 16) + uint32_t(c),
                                       r);
                    tmem_ld_wait();
                    const int cmax = min(32, ncols - c);   // the same for the whole warp
                    // a chunk goes out by TMA unless, site-interleaved, it is short inside
                    // N (the box would spill into the next tile's columns; past N the map
                    // clips it); row-contiguous boxes are 16 columns wide, as are tiles
                    const bool tma_chunk =
                        tst && tst != kStoreColumnsF32 && last &&
                        (tst != kStoreSiteInterleaved || cmax == 32 || n0 + ncols == P->N);
                    if (sum_in_out) {
                        // the first chain stores, each later one adds into the output
                        // (the same lane, in program order: the same FP32 additions in
                        // the same order as through the scratch, subnormal sums aside,
                        // which the reductions flush to zero)
                        if constexpr (kF32Out && kStoreOk) {
                            if (tst == kStoreColumnsF32)   // warp-collective
                                store_chunk_tma_cols_f32(L, r, stg, lane, bx, bz, bvalid, n0 + c, cmax,
                                                         tile_atomic || !first,
                                                         (tile_atomic || !first) && c == half * 32);
                            else if (row_ok && L.out[0][0] != nullptr)
                                store_chunk<EPI>(L, r, row_base, n0, c, cmax, cdiv, sch, scl,
                                                 tile_atomic || !first);
                        } else if (row_ok && L.out[0][0] != nullptr) {
                            store_chunk<EPI>(L, r, row_base, n0, c, cmax, cdiv, sch, scl,
                                             tile_atomic || !first);
                        }
                    } else if constexpr (kScratchCode) {
                        if (row_ok) {
                            float4* s4 = scr ? scr + (c >> 5) * (8 * 32) : nullptr;
                            if (!first) {   // add the chains before this one
#pragma unroll
                                for (int j = 0; j < 8; ++j) {
                                    const float4 v = s4[j * 32];
                                    r[4 * j] = __float_as_uint(__uint_as_float(r[4 * j]) + v.x);
                                    r[4 * j + 1] = __float_as_uint(__uint_as_float(r[4 * j + 1]) + v.y);
                                    r[4 * j + 2] = __float_as_uint(__uint_as_float(r[4 * j + 2]) + v.z);
                                    r[4 * j + 3] = __float_as_uint(__uint_as_float(r[4 * j + 3]) + v.w);
                                }
                            }
                            if (!last) {
#pragma unroll
                                for (int j = 0; j < 8; ++j)
                                    s4[j * 32] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                                        __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
                            } else if (!tma_chunk && L.out[0][0] != nullptr) {   // (a launch may want
                                                                                 // the second copy only)
                                store_chunk<EPI>(L, r, row_base, n0, c, cmax, cdiv, sch, scl, tile_atomic);
                            }
                        }
                    }
                    if constexpr (kStoreOk && !kF32Out) {
                        if (tma_chunk) {
                            if constexpr (EPI == EPI_TF32) {   // site-interleaved only
                                store_chunk_tma_f32(L, r, stg, lane, tsd, bx, (n0 + c) / tsd, bz, bvalid);
                            } else {
                                if (tst == kStoreSiteInterleaved)
                                    store_chunk_tma(L, r, stg, lane, tsd, bx, (n0 + c) / tsd, bz, bvalid);
                                else if (tst == kStoreRowContiguous)
                                    store_chunk_tma_rows(L, r, stg, lane, bx, bz, bvalid, n0 + c, cmax,
                                                         cdiv, sch);
                                else
                                    store_chunk_tma_site(L, r, stg, lane, bx, bz, bvalid, n0 + c, cmax,
                                                         L.o2_m, L.o2_rows_per_op);
                            }
                        }
                    }
                    // the site-major copy's stores are warp-collective: every lane comes here
                    if (SITE && (EPI == EPI_SPLIT_BF16 || EPI == EPI_TF32) && last)
                        store_chunk_site_major<EPI>(L, r, row, n0 + c, cmax, row_ok);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if (leader) mbar_arrive(&tempty[acc]);
                    else mbar_arrive_cluster(acc ? tempty_leader1 : tempty_leader0);
                }
                first = false;
                ++it;
                kb0 = kb1;
            } while (kb0 < dt.kb_end);
        }
        // the TMA stores are complete before the CTA (and its shared memory) goes away
        if (tst && lane == 0) bulk_wait_group0();
    }

    tc_fence_before();
    __syncthreads();
    cluster_sync_all();
    if (*vabort) {
        // After an expired wait copies issued before it may still be landing here.
        const uint64_t t0 = globaltimer_ns();
        while (globaltimer_ns() - t0 < 1000000ull) __nanosleep(1000);
    }
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair<kTmemCols>(tmem_base);
    }
}

// Pairs of this kernel that are resident at once (0 if unknown), cached per
// device, kernel and shared-memory size.
int clusters_that_fit(const void* kernel, const cudaLaunchConfig_t& cfg) {
    struct Entry {
        int dev;
        const void* k;
        size_t smem;
        int fit;
    };
    static std::mutex mu;
    static std::vector<Entry> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lock(mu);
    for (const Entry& e : cache)
        if (e.dev == dev && e.k == kernel && e.smem == cfg.dynamicSmemBytes) return e.fit;
    int fit = 0;
    if (cudaOccupancyMaxActiveClusters(&fit, kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        fit = 0;
    }
    cache.push_back({dev, kernel, cfg.dynamicSmemBytes, fit});
    return fit;
}

template <int MODE, int EPI>
cudaError_t launch_pair(const TcLaunch& L, int stages, int grid, int bh_smem, size_t smem,
                        cudaStream_t s) {
    constexpr bool kSiteEpi = (EPI == EPI_SPLIT_BF16 || EPI == EPI_TF32);
    auto k = L.row_bytes == 64 ? tc_gemm_pair_kernel<MODE, EPI, 64, false, false, false>
                               : tc_gemm_pair_kernel<MODE, EPI, 128, false, false, false>;
    // (the converting form feeds the first product only: no FP32-output instantiation)
    if constexpr (EPI == EPI_SPLIT_BF16 || EPI == EPI_TF32)
        if (L.convert_a) k = tc_gemm_pair_kernel<MODE, EPI, 128, true, false, false>;
    // (the site-major TMA store writes the second copy itself, without the SITE code)
    if (kSiteEpi && L.out2[0] != nullptr && L.t_store != kStoreSiteMajor)
        k = tc_gemm_pair_kernel<MODE, EPI, 128, false, kSiteEpi, false>;
    if constexpr (MODE == TC_BF16X3) {
        bool mn = false;
        for (int i = 0; i < L.nprob; ++i) mn = mn || L.inline_prob[i].a_mn || L.inline_prob[i].b_mn;
        // FP32 output with the chain scratch: the MN-major instantiation is the FP32 one that
        // carries the scratch code (it takes K-major problems as well)
        const bool f32_scratch = (EPI == EPI_F32 || EPI == EPI_F32_ATOMIC) && L.chunk_scratch != nullptr &&
                                 L.row_bytes == 128 && !L.convert_a;
        if (mn || f32_scratch) k = tc_gemm_pair_kernel<MODE, EPI, 128, false, false, true>;
    }
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(grid), 1, 1);
    cfg.blockDim = dim3(L.convert_a ? kThreadsConv : kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    // A persistent grid larger than the clusters that fit at once would only queue.
    const int fit = clusters_that_fit(reinterpret_cast<const void*>(k), cfg);
    if (fit > 0 && 2 * fit < grid) cfg.gridDim.x = unsigned(2 * fit);
    return cudaLaunchKernelEx(&cfg, k, L, stages, bh_smem);
}

// Stages, barriers (within 512 bytes) and, for the TMA-store epilogue, the staging.
size_t pair_smem_bytes(TcMode mode, int stages, int bh, int rb, bool t_store = false) {
    const size_t a = size_t(kBM) * rb, b = size_t(bh) * rb;
    const size_t stage = (a + b) * (mode == TC_BF16X3 ? 2 : 1);
    const size_t bars = 8 * (3 * size_t(stages) + 5) + 32;
    return 1024 + stage * stages + (t_store ? 512 + kStoreStagingBytes : bars);
}

}  // namespace

int tc_pair_max_stages(TcMode mode, int tile_n_max, int row_bytes) {
    int s = 1;
    while (s < 8 && pair_smem_bytes(mode, s + 1, tile_n_max / 2, row_bytes) <= 232448) ++s;
    return s;
}

cudaError_t tc_gemm_launch_pair(TcMode mode, TcEpi epi, const TcLaunch& L, int stages, int grid,
                                cudaStream_t s) {
    if (L.total_tiles <= 0) return cudaSuccess;
    if (L.table != nullptr || L.nprob < 1 || L.nprob > kMaxInlineProblems) return cudaErrorInvalidValue;
    if (L.convert_a && (L.row_bytes != 128 || mode == TC_BF16 ||
                        !(epi == EPI_SPLIT_BF16 || epi == EPI_TF32)))
        return cudaErrorInvalidValue;
    if (L.out2[0] != nullptr && (L.row_bytes != 128 || L.convert_a ||
                                 !(epi == EPI_SPLIT_BF16 || epi == EPI_TF32)))
        return cudaErrorInvalidValue;
    int bn = 32;
    bool any_mn = false, b_mn = false;
    for (int i = 0; i < L.nprob; ++i) {
        const TcProblem& P = L.inline_prob[i];
        bn = std::max(bn, P.tile_n);
        any_mn = any_mn || P.a_mn || P.b_mn;
        b_mn = b_mn || P.b_mn;
        if (P.b_mn && P.tile_n / 2 > 2 * kMnBox) return cudaErrorInvalidValue;
    }
    if (any_mn && (mode == TC_TF32 || L.row_bytes != 128 || L.convert_a)) return cudaErrorInvalidValue;
    // an MN-major B share is two 64-row boxes whatever the tile width
    const int bh = b_mn ? 2 * kMnBox : bn / 2;
    size_t smem = pair_smem_bytes(mode, stages, bh, L.row_bytes);
    if (smem > 232448) return cudaErrorInvalidConfiguration;
    grid = std::max(2, std::min(grid, 2 * L.total_tiles)) / 2 * 2;
    // TMA-store epilogue: only for the BF16 split output without the second copy, and
    // only where its staging fits; otherwise the same launch stores from registers.
    const TcLaunch* Lp = &L;
    TcLaunch plain;
    if (L.t_store != 0) {
        const bool site = L.t_store == kStoreSiteInterleaved;
        const bool smaj = L.t_store == kStoreSiteMajor;
        const bool cols = L.t_store == kStoreColumnsF32;
        bool ok = (cols ? ((epi == EPI_F32 || epi == EPI_F32_ATOMIC) && L.out2[0] == nullptr &&
                           L.out[0][0] != nullptr && L.chunk_scratch == nullptr)
                        : (epi == EPI_SPLIT_BF16 || (epi == EPI_TF32 && site))) &&
                  (smaj ? (L.out2[0] != nullptr && L.out[0][0] == nullptr &&
                           L.o2_rows_per_op % 16 == 0 && L.o2_m % 16 == 0)
                        : (L.out2[0] == nullptr && L.out[0][0] != nullptr)) &&
                  (site ? (L.t_store_d == 2 || L.t_store_d == 4)
                        : (L.t_store == kStoreRowContiguous || smaj || cols));
        for (int i = 0; ok && cols && i < L.nprob; ++i) {
            const TcScatter& S = L.inline_prob[i].sc[0];
            ok = S.s_split == 0 && S.rows_per_op % 16 == 0 && S.col_div == 1 && S.s_row == 1 &&
                 S.op_off == nullptr && S.s_op == int64_t(L.inline_prob[i].N) * S.s_col_hi;
        }
        for (int i = 0; ok && !cols && i < L.nprob; ++i) {
            const TcProblem& P = L.inline_prob[i];
            const TcScatter& S = P.sc[0];
            ok = P.k_splits == 1 &&
                 (smaj ? P.N % 16 == 0
                       : (S.s_split == 0 && S.rows_per_op % 16 == 0 &&
                          (site ? S.col_div == L.t_store_d
                                : (S.col_div % 16 == 0 && S.s_row == 1 && S.s_col_hi % 8 == 0 &&
                                   P.N % 16 == 0))));
        }
        // the staging takes the place of pipeline stages where it must (TF32: 32 KB stages,
        // seven of which fill the shared memory), down to three
        int st = stages;
        while (ok && st > 3 && pair_smem_bytes(mode, st, bh, L.row_bytes, true) > 232448) --st;
        const size_t with = pair_smem_bytes(mode, st, bh, L.row_bytes, true);
        if (ok && with <= 232448) {
            smem = with;
            stages = st;
        } else {
            plain = L;
            plain.t_store = 0;
            Lp = &plain;
        }
    }
#define DMRG_TC_CASE(M, E) \
    if (mode == M && epi == E) return launch_pair<M, E>(*Lp, stages, grid, bh, smem, s);
    DMRG_TC_CASE(TC_BF16X3, EPI_SPLIT_BF16)
    DMRG_TC_CASE(TC_BF16X3, EPI_F32)
    DMRG_TC_CASE(TC_BF16X3, EPI_F32_ATOMIC)
    DMRG_TC_CASE(TC_TF32, EPI_TF32)
    DMRG_TC_CASE(TC_TF32, EPI_F32)
    DMRG_TC_CASE(TC_TF32, EPI_F32_ATOMIC)
#undef DMRG_TC_CASE
    return cudaErrorNotSupported;
}

}  // namespace dmrg
