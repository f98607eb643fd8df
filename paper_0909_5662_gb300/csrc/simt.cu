// simt.cu -- plain-FMA kernels of the FP64 / FP32 paths and the FP64 checks.
//
// The FP64 path is the GPU reference of the rotation O'_k = U^T (O_k (x) I_d) U
// (Sec. 2 step 5): the two products of Sec. 3.2 run as strided batched GEMMs on
// the CUDA cores.  The same GEMM serves the orthonormality check ||U^T U - I||_F
// and the last step of the two-point functions <psi|O'_i O'_j|psi> (Sec. 3.2).
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace dmrg {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

enum SimtEpi { SE_STORE = 0, SE_ORTHO = 1 };

template <typename T, int EPI>
__device__ __forceinline__ void simt_gemm_tile(const SimtGemm& g, int64_t b, int tm, int tn,
                                               double* ortho_acc) {
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t i0 = int64_t(tm) * BM, j0 = int64_t(tn) * BN;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = T(0);

    const bool a_kfast = (g.sAk == 1);
    const bool b_jfast = (g.sBj == 1);
    const int64_t bb0 = g.reduce_batch ? 0 : b;
    const int64_t bb1 = g.reduce_batch ? g.batch : b + 1;
    for (int64_t bb = bb0; bb < bb1; ++bb)
    for (int64_t k0 = 0; k0 < g.K; k0 += BK) {
        const T* A = static_cast<const T*>(g.A) + (g.a_boff ? g.a_boff[bb] : bb * g.sAb);
        const T* B = static_cast<const T*>(g.B) + bb * g.sBb;
#pragma unroll
        for (int q = 0; q < (BM * BK) / NT; ++q) {
            const int e = tid + q * NT;
            int ii, kk;
            if (a_kfast) { ii = e / BK; kk = e % BK; } else { ii = e % BM; kk = e / BM; }
            const int64_t gi = i0 + ii, gk = k0 + kk;
            As[kk][ii] = (gi < g.M && gk < g.K) ? A[gi * g.sAi + gk * g.sAk] : T(0);
        }
#pragma unroll
        for (int q = 0; q < (BN * BK) / NT; ++q) {
            const int e = tid + q * NT;
            int jj, kk;
            if (b_jfast) { jj = e % BN; kk = e / BN; } else { kk = e % BK; jj = e / BK; }
            const int64_t gj = j0 + jj, gk = k0 + kk;
            Bs[kk][jj] = (gj < g.N && gk < g.K) ? B[gk * g.sBk + gj * g.sBj] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
            for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][tx + 16 * c];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[a][c] = fma(av[a], bv[c], acc[a][c]);
        }
        __syncthreads();
    }
    if (EPI == SE_STORE) {
        T* C = static_cast<T*>(g.C) + (g.c_boff ? g.c_boff[b] : b * g.sCb);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int64_t gi = i0 + ty + 16 * a;
            if (gi >= g.M) continue;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t gj = j0 + tx + 16 * c;
                if (gj >= g.N) continue;
                T* dst = C + gi * g.sCi + gj * g.sCj;
                *dst = g.accumulate ? (*dst + acc[a][c]) : acc[a][c];
            }
        }
    } else {
        // ||G - I||_F^2 contribution of this tile.
        double part = 0.0;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int64_t gi = i0 + ty + 16 * a;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t gj = j0 + tx + 16 * c;
                if (gi < g.M && gj < g.N) {
                    const double e = double(acc[a][c]) - (gi == gj ? 1.0 : 0.0);
                    part += e * e;
                }
            }
        }
        __shared__ double red[NT / 32];
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if ((tid & 31) == 0) red[tid >> 5] = part;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < NT / 32; ++w) s += red[w];
            atomicAdd(ortho_acc, s);
        }
    }
}

template <typename T, int EPI>
__global__ void __launch_bounds__(NT) simt_gemm_kernel(const SimtGemm g, double* ortho_acc) {
    const int64_t t = blockIdx.x;
    const int64_t per_b = int64_t(g.tiles_m) * g.tiles_n;
    const int64_t b = t / per_b;
    const int64_t r = t % per_b;
    const int tm = int(r / g.tiles_n), tn = int(r % g.tiles_n);
    if (g.lower && tn > tm) return;
    simt_gemm_tile<T, EPI>(g, b, tm, tn, ortho_acc);
}

// C[i][j] = C[j][i] for the entries of the tiles a `lower` launch skipped (the tile of j
// after the tile of i), through a 32 x 32 shared-memory transpose.
__global__ void mirror_lower_kernel(double* __restrict__ C, int64_t n, int64_t ldc) {
    __shared__ double t[32][33];
    const int64_t i0 = int64_t(blockIdx.y) * 32, j0 = int64_t(blockIdx.x) * 32;
    if ((j0 + 31) / BN <= i0 / BM) return;   // every entry of this block was computed
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t j = j0 + r, i = i0 + threadIdx.x;   // read C[j][i] along i
        if (j < n && i < n) t[r][threadIdx.x] = C[j * ldc + i];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = i0 + r, j = j0 + threadIdx.x;   // write C[i][j] along j
        if (i < n && j < n && j / BN > i / BM) C[i * ldc + j] = t[threadIdx.x][r];
    }
}

struct SimtBases {
    const void* p[4];
};

template <typename T>
__global__ void __launch_bounds__(NT) simt_gemm_grouped_kernel(const SimtGemm* __restrict__ probs,
                                                               int nprob, const SimtBases bases) {
    const int t = blockIdx.x;
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {  // last problem with tile_start <= t
        const int mid = (lo + hi + 1) >> 1;
        if (probs[mid].tile_start <= t) lo = mid; else hi = mid - 1;
    }
    SimtGemm g = probs[lo];
    auto rebase = [&](const void* off, int sel) -> const void* {
        if (sel < 0) return off;
        return static_cast<const T*>(bases.p[sel]) + reinterpret_cast<intptr_t>(off);
    };
    g.A = rebase(g.A, g.a_sel);
    g.B = rebase(g.B, g.b_sel);
    g.C = const_cast<void*>(rebase(g.C, g.c_sel));
    const int64_t local = t - g.tile_start;
    if (g.small) {
        // one warp per batch entry: lanes stride over the (at most 32 x 32) outputs,
        // operands read through L1 (tiny blocks, no shared-memory staging)
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int64_t b = local * kSimtSmallPerBlock + warp;
        if (b >= g.batch) return;
        const T* A = static_cast<const T*>(g.A) + (g.a_boff ? g.a_boff[b] : b * g.sAb);
        const T* B = static_cast<const T*>(g.B) + b * g.sBb;
        T* C = static_cast<T*>(g.C) + (g.c_boff ? g.c_boff[b] : b * g.sCb);
        const int n = int(g.N);
        for (int e = lane; e < int(g.M) * n; e += 32) {
            const int i = e / n, j = e - (e / n) * n;
            const T* a = A + i * g.sAi;
            const T* bp = B + j * g.sBj;
            T acc = T(0);
            for (int64_t k = 0; k < g.K; ++k) acc = fma(a[k * g.sAk], bp[k * g.sBk], acc);
            T* dst = C + i * g.sCi + j * g.sCj;
            *dst = g.accumulate ? (*dst + acc) : acc;
        }
        return;
    }
    const int64_t per_b = int64_t(g.tiles_m) * g.tiles_n;
    const int64_t b = local / per_b;
    const int64_t r = local % per_b;
    simt_gemm_tile<T, SE_STORE>(g, b, int(r / g.tiles_n), int(r % g.tiles_n), nullptr);
}

__global__ void sqrt_kernel(const double* acc, double* out) { *out = sqrt(*acc); }
__global__ void zero_double_kernel(double* p) { *p = 0.0; }

template <typename T>
__global__ void rows_dot_kernel(const T* __restrict__ Op, const double* __restrict__ psi,
                                int64_t K, int64_t mp, double* __restrict__ y) {
    // one warp per row: y[k][a] = sum_b O'_k[a][b] psi[b]
    const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= K * mp) return;
    const T* row = Op + warp * mp;
    double s = 0.0;
    for (int64_t b = lane; b < mp; b += 32) s += double(row[b]) * psi[b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[warp] = s;
}

template <typename T>
__global__ void cols_dot_kernel(const T* __restrict__ Op, const double* __restrict__ psi,
                                int64_t mp, double* __restrict__ x) {
    // x[k][b] = sum_a O'_k[a][b] psi[a]; one thread per column, coalesced rows.
    const int64_t k = blockIdx.y;
    const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= mp) return;
    const T* M = Op + k * mp * mp;
    double s = 0.0;
    for (int64_t a = 0; a < mp; ++a) s += double(M[a * mp + b]) * psi[a];
    x[k * mp + b] = s;
}

__global__ void f32_to_f64_kernel(const float* __restrict__ src, double* __restrict__ dst,
                                  int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x)
        dst[i] = double(src[i]);
}

}  // namespace

int simt_tile_m() { return BM; }
int simt_tile_n() { return BN; }

cudaError_t simt_gemm_launch(Real t, const SimtGemm& g0, cudaStream_t s) {
    SimtGemm g = g0;
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
    g.tiles_m = int((g.M + BM - 1) / BM);
    g.tiles_n = int((g.N + BN - 1) / BN);
    const int64_t blocks = int64_t(g.tiles_m) * g.tiles_n * (g.reduce_batch ? 1 : g.batch);
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (g.lower && (t != Real::F64 || g.M != g.N || g.batch != 1 || g.sCj != 1 || g.accumulate))
        return cudaErrorInvalidValue;
    if (t == Real::F64)
        simt_gemm_kernel<double, SE_STORE><<<unsigned(blocks), NT, 0, s>>>(g, nullptr);
    else
        simt_gemm_kernel<float, SE_STORE><<<unsigned(blocks), NT, 0, s>>>(g, nullptr);
    if (g.lower) {
        const unsigned nb = unsigned((g.M + 31) / 32);
        mirror_lower_kernel<<<dim3(nb, nb), dim3(32, 8), 0, s>>>(static_cast<double*>(g.C), g.M, g.sCi);
    }
    return cudaGetLastError();
}

cudaError_t simt_gemm_grouped_launch(Real t, const SimtGemm* d_problems, int nprob,
                                     int total_tiles, const void* const bases[4], cudaStream_t s) {
    if (nprob <= 0 || total_tiles <= 0) return cudaSuccess;
    SimtBases b;
    for (int i = 0; i < 4; ++i) b.p[i] = bases[i];
    if (t == Real::F64)
        simt_gemm_grouped_kernel<double><<<total_tiles, NT, 0, s>>>(d_problems, nprob, b);
    else
        simt_gemm_grouped_kernel<float><<<total_tiles, NT, 0, s>>>(d_problems, nprob, b);
    return cudaGetLastError();
}

cudaError_t ortho_error_launch(const double* U, int64_t rows, int64_t mp, double* acc, double* out,
                               cudaStream_t s) {
    zero_double_kernel<<<1, 1, 0, s>>>(acc);
    SimtGemm g{};
    g.A = U; g.B = U; g.C = nullptr;
    g.M = mp; g.N = mp; g.K = rows;
    g.sAb = 0; g.sAi = 1; g.sAk = mp;       // A(a, r) = U[r][a]
    g.sBb = 0; g.sBk = mp; g.sBj = 1;       // B(r, b) = U[r][b]
    g.batch = 1;
    g.tiles_m = int((mp + BM - 1) / BM);
    g.tiles_n = int((mp + BN - 1) / BN);
    if (mp > 0 && rows > 0)
        simt_gemm_kernel<double, SE_ORTHO><<<g.tiles_m * g.tiles_n, NT, 0, s>>>(g, acc);
    sqrt_kernel<<<1, 1, 0, s>>>(acc, out);
    return cudaGetLastError();
}

cudaError_t corr_matvec_launch(const void* Op, bool f64, const double* psi, int64_t K, int64_t mp,
                               double* x, double* y, cudaStream_t s) {
    if (K <= 0 || mp <= 0) return cudaSuccess;
    const int64_t rows = K * mp;
    const unsigned gr = unsigned((rows * 32 + 255) / 256);
    dim3 gc(unsigned((mp + 127) / 128), unsigned(K));
    if (f64) {
        rows_dot_kernel<double><<<gr, 256, 0, s>>>(static_cast<const double*>(Op), psi, K, mp, y);
        cols_dot_kernel<double><<<gc, 128, 0, s>>>(static_cast<const double*>(Op), psi, mp, x);
    } else {
        rows_dot_kernel<float><<<gr, 256, 0, s>>>(static_cast<const float*>(Op), psi, K, mp, y);
        cols_dot_kernel<float><<<gc, 128, 0, s>>>(static_cast<const float*>(Op), psi, mp, x);
    }
    return cudaGetLastError();
}

cudaError_t convert_f32_to_f64_launch(const float* src, double* dst, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    f32_to_f64_kernel<<<unsigned(blocks), 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t f32_to_f64_strided_launch(const float* src, double* dst, int64_t n, cudaStream_t s) {
    return convert_f32_to_f64_launch(src, dst, n, s);
}

cudaError_t fill_zero_launch(void* p, size_t bytes, cudaStream_t s) {
    return cudaMemsetAsync(p, 0, bytes, s);
}

}  // namespace dmrg
