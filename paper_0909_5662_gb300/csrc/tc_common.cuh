// tc_common.cuh -- device helpers shared by the tcgen05 GEMM kernels (one-CTA and
// CTA-pair forms) and the operand packers: tile decoding of the persistent schedule,
// BF16 hi/lo splitting, TF32 rounding and the epilogue's scatter of one 32-column
// accumulator chunk.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace dmrg {
namespace tcdev {

struct Decoded {
    const TcProblem* P;
    int mt, nt, kb_begin, kb_end, kb_per_batch;
};

__device__ __forceinline__ Decoded decode_tile(const TcLaunch& L, int t, int elems_per_row) {
    const TcProblem* P = &L.inline_prob[0];
    if (L.table != nullptr) {
        int lo = 0;
        if (L.tile_problem != nullptr) {
            lo = __ldg(L.tile_problem + t);
        } else {
            int hi = L.nprob - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (L.table[mid].tile_start <= t) lo = mid; else hi = mid - 1;
            }
        }
        P = &L.table[lo];
    } else {
        for (int i = 1; i < L.nprob; ++i)
            if (L.inline_prob[i].tile_start <= t) P = &L.inline_prob[i];
    }
    Decoded d;
    d.P = P;
    const int local = t - P->tile_start;
    const int per_split = P->m_tiles * P->n_tiles;
    const int ks = local / per_split;
    const int rem = local - ks * per_split;
    d.mt = rem / P->n_tiles;
    d.nt = rem - d.mt * P->n_tiles;
    if (L.reverse_m) d.mt = P->m_tiles - 1 - d.mt;
    d.mt += P->m_tile0;
    d.kb_per_batch = (P->Kred + elems_per_row - 1) / elems_per_row;
    const int kb_total = d.kb_per_batch * P->nbatch;
    d.kb_begin = ks * P->kb_per_split;
    d.kb_end = min(kb_total, d.kb_begin + P->kb_per_split);
    return d;
}

// BF16 pair of x: hi = bf16(x), lo = bf16(x - hi).  For an FP32 source the residual
// x - hi is exact in FP32; for an FP64 source it is formed in FP64 (one subtraction)
// and then rounded, so FP64 arithmetic stays off the per-element path otherwise.
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& h, __nv_bfloat16& l) {
    h = __float2bfloat16_rn(x);
    l = __float2bfloat16_rn(x - __bfloat162float(h));
}
__device__ __forceinline__ void split_bf16(double x, __nv_bfloat16& h, __nv_bfloat16& l) {
    h = __float2bfloat16_rn(__double2float_rn(x));
    l = __float2bfloat16_rn(__double2float_rn(x - double(__bfloat162float(h))));
}

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// out[0..3] += v0..v3 as one relaxed, GPU-scope vector reduction (16-byte aligned).
__device__ __forceinline__ void red_add_v4(float* out, float v0, float v1, float v2, float v3) {
    asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(out), "f"(v0),
                 "f"(v1), "f"(v2), "f"(v3)
                 : "memory");
}

// Stores one 32-column chunk of a finished accumulator row through scatter map S
// (row_base already includes the row part of the map).  r[] is indexed with
// constants only, so it stays in registers.
template <int EPI>
__device__ __forceinline__ void store_chunk(const TcLaunch& L, const uint32_t (&r)[32],
                                        int64_t row_base, int n0, int c, int cmax, int cdiv,
                                        int64_t sch, int64_t scl, bool tile_atomic) {
    if (EPI == EPI_SPLIT_BF16) {
        __nv_bfloat16* hi = static_cast<__nv_bfloat16*>(L.out[0][0]);
        __nv_bfloat16* lo = static_cast<__nv_bfloat16*>(L.out[0][1]);
        const bool vec4 = cdiv == 4 && scl == 1 && ((row_base & 3) == 0) &&
                          ((sch & 3) == 0) && cmax == 32;
        if (vec4) {
            // four consecutive columns (b, s = 0..3) -> four consecutive
            // elements; pairs are split with packed bf16x2 conversions
            const int64_t base = row_base + int64_t((n0 + c) >> 2) * sch;
            uint2* ph = reinterpret_cast<uint2*>(hi + base);
            uint2* pl = reinterpret_cast<uint2*>(lo + base);
            const int64_t step = sch >> 2;  // in uint2 units
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
                uint32_t hw[2], lw[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const float2 v = make_float2(__uint_as_float(r[j + 2 * q]),
                                                 __uint_as_float(r[j + 2 * q + 1]));
                    const __nv_bfloat162 h2 = __float22bfloat162_rn(v);
                    const float2 hf = __bfloat1622float2(h2);
                    const __nv_bfloat162 l2 =
                        __float22bfloat162_rn(make_float2(v.x - hf.x, v.y - hf.y));
                    hw[q] = *reinterpret_cast<const uint32_t*>(&h2);
                    lw[q] = *reinterpret_cast<const uint32_t*>(&l2);
                }
                ph[(j >> 2) * step] = make_uint2(hw[0], hw[1]);
                pl[(j >> 2) * step] = make_uint2(lw[0], lw[1]);
            }
        } else {
            // r[] is indexed with constants only (full unroll), so it stays in
            // registers; the scatter index advances column by column (one division
            // per chunk)
            const int n = n0 + c;
            int rem = n % cdiv;
            int64_t idx = row_base + int64_t(n / cdiv) * sch + int64_t(rem) * scl;
            const int64_t wrap = sch - int64_t(cdiv - 1) * scl;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (j < cmax) {
                    const float v = __uint_as_float(r[j]);
                    const __nv_bfloat16 h = __float2bfloat16_rn(v);
                    hi[idx] = h;
                    lo[idx] = __float2bfloat16_rn(v - __bfloat162float(h));
                }
                if (++rem == cdiv) {
                    rem = 0;
                    idx += wrap;
                } else {
                    idx += scl;
                }
            }
        }
    } else {
        float* out = static_cast<float*>(L.out[0][0]);
        const bool atom = (EPI == EPI_F32_ATOMIC) || tile_atomic;
        if (!atom && cdiv == 4 && scl == 1 && cmax == 32 && ((row_base & 3) == 0) &&
            ((sch & 3) == 0)) {
            // groups of four columns (b, s = 0..3) land on four consecutive words
            float4* p4 = reinterpret_cast<float4*>(out + row_base +
                                                   int64_t((n0 + c) >> 2) * sch);
            const int64_t step = sch >> 2;  // in float4 units
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
                float4 v;
                v.x = __uint_as_float(r[j]);
                v.y = __uint_as_float(r[j + 1]);
                v.z = __uint_as_float(r[j + 2]);
                v.w = __uint_as_float(r[j + 3]);
                if (EPI == EPI_TF32) {
                    v.x = tf32_round(v.x); v.y = tf32_round(v.y);
                    v.z = tf32_round(v.z); v.w = tf32_round(v.w);
                }
                p4[(j >> 2) * step] = v;
            }
        } else if (!atom && cdiv == 1 && sch == 1 && cmax == 32 &&
                   (((row_base + n0 + c) & 3) == 0)) {
            float4* o4 = reinterpret_cast<float4*>(out + row_base + n0 + c);
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
                float4 v;
                v.x = __uint_as_float(r[j]);
                v.y = __uint_as_float(r[j + 1]);
                v.z = __uint_as_float(r[j + 2]);
                v.w = __uint_as_float(r[j + 3]);
                if (EPI == EPI_TF32) {
                    v.x = tf32_round(v.x); v.y = tf32_round(v.y);
                    v.z = tf32_round(v.z); v.w = tf32_round(v.w);
                }
                o4[j >> 2] = v;
            }
        } else if (atom && cdiv == 1 && sch == 1 && cmax == 32 &&
                   ((reinterpret_cast<uintptr_t>(out + row_base + n0 + c) & 15) == 0)) {
            // a contiguous row segment accumulated with 16-byte vector reductions
            float* p = out + row_base + n0 + c;
#pragma unroll
            for (int j = 0; j < 32; j += 4)
                red_add_v4(p + j, __uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                           __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
        } else if (cdiv == 1) {
            // one stride per column (the transposed store of the second product):
            // lanes hold consecutive rows, so each store instruction is coalesced
            float* p = out + row_base + int64_t(n0 + c) * sch;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (j < cmax) {
                    const float v = __uint_as_float(r[j]);
                    if (atom) atomicAdd(p + j * sch, v);
                    else p[j * sch] = (EPI == EPI_TF32) ? tf32_round(v) : v;
                }
            }
        } else {
            const int n = n0 + c;
            int rem = n % cdiv;
            int64_t idx = row_base + int64_t(n / cdiv) * sch + int64_t(rem) * scl;
            const int64_t wrap = sch - int64_t(cdiv - 1) * scl;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (j < cmax) {
                    const float v = __uint_as_float(r[j]);
                    if (atom) atomicAdd(out + idx, v);
                    else if (EPI == EPI_TF32) out[idx] = tf32_round(v);
                    else out[idx] = v;
                }
                if (++rem == cdiv) {
                    rem = 0;
                    idx += wrap;
                } else {
                    idx += scl;
                }
            }
        }
    }
}

// out[0..3] = the 16-byte word x[sel] (sel in 0..3, chosen per lane) of four.
__device__ __forceinline__ void pick4(const uint32_t (&x)[4][4], int sel, uint32_t (&out)[4]) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const uint32_t a = (sel & 1) ? x[1][e] : x[0][e];
        const uint32_t b = (sel & 1) ? x[3][e] : x[2][e];
        out[e] = (sel & 2) ? b : a;
    }
}

// Writes the 4 x 16-byte words x[q] (elements 8q .. 8q+7 of this lane's row segment,
// 64 bytes at rowp) so that the four lanes of each aligned group of four write one
// row's 64 bytes per store instruction: the words are exchanged in a 4 x 4 transpose
// within the group (three shuffle rounds), then store i of lane 4g + t writes word t of
// row 4g + i.  All 32 lanes must take part.
__device__ __forceinline__ void store_rows64_grouped(uint4* rowp, const uint32_t (&x)[4][4]) {
    const int t = threadIdx.x & 3;
    uint32_t y[4][4];   // y[v] = word t of the row of lane (4g + (t ^ v))
#pragma unroll
    for (int e = 0; e < 4; ++e) y[0][e] = 0;
    pick4(x, t, y[0]);
#pragma unroll
    for (int v = 1; v < 4; ++v) {
        uint32_t snd[4];
        pick4(x, t ^ v, snd);
#pragma unroll
        for (int e = 0; e < 4; ++e) y[v][e] = __shfl_xor_sync(0xffffffffu, snd[e], v);
    }
    const uint64_t mine = reinterpret_cast<uint64_t>(rowp);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        // row 4g + i: its pointer comes from lane 4g + i; its word t is y[t ^ i]
        const uint64_t p = __shfl_sync(0xffffffffu, mine, (threadIdx.x & ~3) | i);
        uint32_t w[4];
        pick4(y, t ^ i, w);
        if (p != 0) reinterpret_cast<uint4*>(p)[t] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Stores one 32-column chunk (first column c0) of accumulator row `row` into the
// site-major copy described by TcLaunch::out2 (see internal.h).  A chunk that lies in
// one site state's run of columns is 32 consecutive j of one output row; when every
// lane's segment is 16-byte aligned the warp writes them as whole 64-byte row pieces
// (BF16: store_rows64_grouped; FP32: 16-byte vectors).  `active`: this lane's row
// exists (all lanes of the warp call this function).
template <int EPI>
__device__ __forceinline__ void store_chunk_site_major(const TcLaunch& L, const uint32_t (&r)[32],
                                                       int row, int c0, int cmax, bool active) {
    const int mm = L.o2_m;
    int64_t base = 0;
    if (active) {
        const int g = row / L.o2_rows_per_op;
        const int rr = row - g * L.o2_rows_per_op;
        base = int64_t(g) * L.o2_s_op + int64_t(rr) * L.o2_s_row;
    }
    const int s0 = c0 / mm;
    const int j0 = c0 - s0 * mm;
    const int64_t o0 = base + int64_t(s0) * L.o2_s_site + j0;
    // c0, cmax and the site-major layout are the same for every lane of the warp
    const bool one_run = cmax == 32 && j0 + 32 <= mm;
    if (EPI == EPI_SPLIT_BF16) {
        __nv_bfloat16* hi = static_cast<__nv_bfloat16*>(L.out2[0]);
        __nv_bfloat16* lo = static_cast<__nv_bfloat16*>(L.out2[1]);
        const bool vec = one_run && __all_sync(0xffffffffu, !active || (o0 & 7) == 0);
        if (vec) {
            uint32_t hw[4][4], lw[4][4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {   // elements 8q .. 8q + 7
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float2 v = make_float2(__uint_as_float(r[8 * q + 2 * e]),
                                                 __uint_as_float(r[8 * q + 2 * e + 1]));
                    const __nv_bfloat162 h2 = __float22bfloat162_rn(v);
                    const float2 hf = __bfloat1622float2(h2);
                    const __nv_bfloat162 l2 =
                        __float22bfloat162_rn(make_float2(v.x - hf.x, v.y - hf.y));
                    hw[q][e] = *reinterpret_cast<const uint32_t*>(&h2);
                    lw[q][e] = *reinterpret_cast<const uint32_t*>(&l2);
                }
            }
            store_rows64_grouped(active ? reinterpret_cast<uint4*>(hi + o0) : nullptr, hw);
            store_rows64_grouped(active ? reinterpret_cast<uint4*>(lo + o0) : nullptr, lw);
        } else if (active) {
            // groups of eight elements: one 16-byte store each where the group lies in one
            // run and is aligned (the tail chunk of a tile, a chunk across two runs)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (8 * q >= cmax) break;
                const int c = c0 + 8 * q;
                const int sidx = c / mm;
                const int j = c - sidx * mm;
                const int64_t o = base + int64_t(sidx) * L.o2_s_site + j;
                if (8 * q + 8 <= cmax && j + 8 <= mm && (o & 7) == 0) {
                    uint32_t hw[4], lw[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float2 v = make_float2(__uint_as_float(r[8 * q + 2 * e]),
                                                     __uint_as_float(r[8 * q + 2 * e + 1]));
                        const __nv_bfloat162 h2 = __float22bfloat162_rn(v);
                        const float2 hf = __bfloat1622float2(h2);
                        const __nv_bfloat162 l2 =
                            __float22bfloat162_rn(make_float2(v.x - hf.x, v.y - hf.y));
                        hw[e] = *reinterpret_cast<const uint32_t*>(&h2);
                        lw[e] = *reinterpret_cast<const uint32_t*>(&l2);
                    }
                    *reinterpret_cast<uint4*>(hi + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                    *reinterpret_cast<uint4*>(lo + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        if (8 * q + e < cmax) {
                            const int ce = c + e;
                            const int se = ce / mm;
                            const int64_t oe = base + int64_t(se) * L.o2_s_site + (ce - se * mm);
                            const float v = __uint_as_float(r[8 * q + e]);
                            const __nv_bfloat16 h = __float2bfloat16_rn(v);
                            hi[oe] = h;
                            lo[oe] = __float2bfloat16_rn(v - __bfloat162float(h));
                        }
                    }
                }
            }
        }
    } else if (active) {
        float* out = static_cast<float*>(L.out2[0]);
        // groups of four elements: one 16-byte store each where the group lies in one run
        // and is aligned
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (4 * q >= cmax) break;
            const int c = c0 + 4 * q;
            const int sidx = c / mm;
            const int j = c - sidx * mm;
            const int64_t o = base + int64_t(sidx) * L.o2_s_site + j;
            if (4 * q + 4 <= cmax && j + 4 <= mm && (o & 3) == 0) {
                float4 v;
                v.x = tf32_round(__uint_as_float(r[4 * q]));
                v.y = tf32_round(__uint_as_float(r[4 * q + 1]));
                v.z = tf32_round(__uint_as_float(r[4 * q + 2]));
                v.w = tf32_round(__uint_as_float(r[4 * q + 3]));
                *reinterpret_cast<float4*>(out + o) = v;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (4 * q + e < cmax) {
                        const int ce = c + e;
                        const int se = ce / mm;
                        out[base + int64_t(se) * L.o2_s_site + (ce - se * mm)] =
                            tf32_round(__uint_as_float(r[4 * q + e]));
                    }
                }
            }
        }
    }
}

}  // namespace tcdev
}  // namespace dmrg
