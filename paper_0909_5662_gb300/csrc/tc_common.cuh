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

// Stores one 32-column chunk (first column c0) of accumulator row `row` into the
// site-major copy described by TcLaunch::out2 (see internal.h).  With d = 4 and aligned
// rows the four site states' runs of eight consecutive j go out as vector stores.
template <int EPI>
__device__ __forceinline__ void store_chunk_site_major(const TcLaunch& L, const uint32_t (&r)[32],
                                                       int row, int c0, int cmax) {
    const int g = row / L.o2_rows_per_op;
    const int rr = row - g * L.o2_rows_per_op;
    const int d = L.o2_d;
    const int64_t base = int64_t(g) * L.o2_s_op + int64_t(rr) * L.o2_s_row;
    const bool fast = d == 4 && cmax == 32 && (c0 & 3) == 0 && ((base + c0 / 4) & 3) == 0 &&
                      (L.o2_s_site & 3) == 0;
    if (EPI == EPI_SPLIT_BF16) {
        __nv_bfloat16* hi = static_cast<__nv_bfloat16*>(L.out2[0]);
        __nv_bfloat16* lo = static_cast<__nv_bfloat16*>(L.out2[1]);
        if (fast) {
            const int64_t j0 = base + c0 / 4;
#pragma unroll
            for (int s = 0; s < 4; ++s) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {   // j = 4q .. 4q + 3 of the chunk: columns 4j + s
                    uint32_t hw[2], lw[2];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const float2 v = make_float2(__uint_as_float(r[4 * (4 * q + 2 * e) + s]),
                                                     __uint_as_float(r[4 * (4 * q + 2 * e + 1) + s]));
                        const __nv_bfloat162 h2 = __float22bfloat162_rn(v);
                        const float2 hf = __bfloat1622float2(h2);
                        const __nv_bfloat162 l2 =
                            __float22bfloat162_rn(make_float2(v.x - hf.x, v.y - hf.y));
                        hw[e] = *reinterpret_cast<const uint32_t*>(&h2);
                        lw[e] = *reinterpret_cast<const uint32_t*>(&l2);
                    }
                    const int64_t o = j0 + int64_t(s) * L.o2_s_site + 4 * q;
                    *reinterpret_cast<uint2*>(hi + o) = make_uint2(hw[0], hw[1]);
                    *reinterpret_cast<uint2*>(lo + o) = make_uint2(lw[0], lw[1]);
                }
            }
        } else {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
                if (jj < cmax) {
                    const int c = c0 + jj;
                    const int j = c / d;
                    const int64_t o = base + int64_t(c - j * d) * L.o2_s_site + j;
                    const float v = __uint_as_float(r[jj]);
                    const __nv_bfloat16 h = __float2bfloat16_rn(v);
                    hi[o] = h;
                    lo[o] = __float2bfloat16_rn(v - __bfloat162float(h));
                }
            }
        }
    } else {
        float* out = static_cast<float*>(L.out2[0]);
        if (fast) {
            const int64_t j0 = base + c0 / 4;
#pragma unroll
            for (int s = 0; s < 4; ++s) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    float4 v;
                    v.x = tf32_round(__uint_as_float(r[4 * (4 * q) + s]));
                    v.y = tf32_round(__uint_as_float(r[4 * (4 * q + 1) + s]));
                    v.z = tf32_round(__uint_as_float(r[4 * (4 * q + 2) + s]));
                    v.w = tf32_round(__uint_as_float(r[4 * (4 * q + 3) + s]));
                    *reinterpret_cast<float4*>(out + j0 + int64_t(s) * L.o2_s_site + 4 * q) = v;
                }
            }
        } else {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
                if (jj < cmax) {
                    const int c = c0 + jj;
                    const int j = c / d;
                    out[base + int64_t(c - j * d) * L.o2_s_site + j] = tf32_round(__uint_as_float(r[jj]));
                }
            }
        }
    }
}

}  // namespace tcdev
}  // namespace dmrg
