// measure.cu -- the measurement stage: expectation values of stored operators in the
// superblock ground state and the structure factors built from them.
//
// The superblock ground state psi0 = sum_{a,e} Psi[a][e] |a>|e> (system basis a,
// environment basis e) is a rows x cols FP64 matrix.  Sec. 3.2 needs the one-point
// functions <Z_i> and the two-point functions <Z_i Z_j>: a product of operators of one
// block is stored and rotated as one operator, so it is a one-point function too, while
// operators of different blocks combine across the superblock.  Sec. 2 forms the charge
// and spin structure factors N(q), S^z(q) from them.  Everything here is FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "api_common.h"

using namespace dmrg;

namespace {

// Tr(rho Z_k) = sum_{a,b} Z_k[a][b] rho[a][b] (rho symmetric), in two passes so that
// every operator is read by many blocks at once: block (c, k) sums chunk c of Z_k into
// part[k * chunks + c], then trace_finish_kernel adds the chunks in order.
constexpr int kTraceThreads = 256;

__device__ __forceinline__ double block_sum(double acc) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;   // valid in thread 0
}

// FP32 -> FP64 on the integer pipe (exponent rebias, mantissa shift): the FP64 pipe of
// this part is slow, and a hardware conversion there would cost as much as the FMA it
// feeds.  Zero keeps its sign; subnormals, infinities and NaN take the hardware path.
__device__ __forceinline__ double widen(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    const bool zero = (u << 1) == 0u;
    if (!zero && (e == 0u || e == 0xffu)) return double(f);
    const unsigned hi = zero ? (u & 0x80000000u)
                             : ((u & 0x80000000u) | ((e + 896u) << 20) | ((u >> 3) & 0xfffffu));
    const unsigned lo = zero ? 0u : (u << 29);
    return __hiloint2double(int(hi), int(lo));
}

template <typename T>
__global__ void __launch_bounds__(kTraceThreads)
trace_partial_kernel(const T* __restrict__ Z, const double* __restrict__ rho, int64_t nn,
                     int64_t per, int chunks, double* __restrict__ part) {
    const int64_t k = blockIdx.y;
    const int64_t lo = int64_t(blockIdx.x) * per;
    const int64_t hi = lo + per < nn ? lo + per : nn;
    const T* Zk = Z + k * nn;
    double acc = 0.0;
    if (sizeof(T) == 4 && (nn & 3) == 0 && (per & 3) == 0 &&
        (reinterpret_cast<uintptr_t>(Z) & 15) == 0 && (reinterpret_cast<uintptr_t>(rho) & 15) == 0) {
        // four FP32 entries and the matching rho entries per step
        const float4* z4 = reinterpret_cast<const float4*>(Zk);
        const double2* r2 = reinterpret_cast<const double2*>(rho);
        for (int64_t q = lo / 4 + threadIdx.x; q < hi / 4; q += blockDim.x) {
            const float4 z = __ldcs(z4 + q);
            const double2 ra = r2[2 * q], rb = r2[2 * q + 1];
            acc = fma(widen(z.x), ra.x, acc);
            acc = fma(widen(z.y), ra.y, acc);
            acc = fma(widen(z.z), rb.x, acc);
            acc = fma(widen(z.w), rb.y, acc);
        }
    } else {
        for (int64_t x = lo + threadIdx.x; x < hi; x += blockDim.x) acc += double(Zk[x]) * rho[x];
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) part[k * chunks + blockIdx.x] = s;
}

__global__ void trace_finish_kernel(const double* __restrict__ part, int chunks, int64_t K,
                                    double* __restrict__ out) {
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= K) return;
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += part[k * chunks + c];
    out[k] = s;
}

// C[i][j] = sum_s part[s][i][j], the split reduction of the cross correlations in order.
__global__ void split_sum_kernel(const double* __restrict__ part, int nsplit, int64_t nout,
                                 double* __restrict__ C) {
    const int64_t x = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (x >= nout) return;
    double s = 0.0;
    for (int p = 0; p < nsplit; ++p) s += part[int64_t(p) * nout + x];
    C[x] = s;
}

// Chunking of Tr(rho Z_k): about 2048 blocks over all operators, chunks of at least
// 8192 entries, chunk length a multiple of 4 (vector loads).
struct TraceSplit {
    int chunks;
    int64_t per;
};
TraceSplit trace_split(int64_t K, int64_t nn) {
    TraceSplit t;
    int64_t c = std::max<int64_t>(1, (2048 + K - 1) / std::max<int64_t>(K, 1));
    c = std::min<int64_t>(c, std::max<int64_t>(1, (nn + 8191) / 8192));
    int64_t per = (nn + c - 1) / c;
    per = (per + 3) / 4 * 4;
    t.per = per;
    t.chunks = int((nn + per - 1) / per);
    return t;
}

// Split of the reduction of length Lx = cols^2 in the cross correlations into about 608
// pieces (four per SM) of a multiple of 16 entries.
struct CrossSplit {
    int64_t kc, full, tail;
    int nsplit;
};
CrossSplit cross_split(int64_t Lx) {
    CrossSplit c;
    int64_t kc = std::max<int64_t>(1024, (Lx + 607) / 608);
    kc = (kc + 15) / 16 * 16;
    c.kc = kc;
    c.full = Lx / kc;
    c.tail = Lx - c.full * kc;
    c.nsplit = int(c.full + (c.tail ? 1 : 0));
    return c;
}

// F(q_p) = (1/L) sum_{k,j} e^{i q_p (k-j)} (G[k][j] - c v[k] - c v[j] + c^2),
// q_p = 2 pi p / L, one block per p.  The phase p (k - j) is reduced modulo L in
// integers, so the angle passed to sincospi is exact to rounding.
__global__ void structure_factor_kernel(const double* __restrict__ G, const double* __restrict__ v,
                                        double c, int64_t L, double* __restrict__ Fre,
                                        double* __restrict__ Fim) {
    const int64_t p = blockIdx.x;
    double re = 0.0, im = 0.0;
    for (int64_t x = threadIdx.x; x < L * L; x += blockDim.x) {
        const int64_t k = x / L, j = x - (x / L) * L;
        double g = G[x] + c * c;
        if (v) g -= c * (v[k] + v[j]);
        int64_t r = (p * (k - j)) % L;
        if (r < 0) r += L;
        double sn, cs;
        sincospi(2.0 * double(r) / double(L), &sn, &cs);
        re += cs * g;
        im += sn * g;
    }
    __shared__ double red[2][32];
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = re;
        red[1][threadIdx.x >> 5] = im;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const bool live = threadIdx.x < (blockDim.x >> 5);
        double a = live ? red[0][threadIdx.x] : 0.0, b = live ? red[1][threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (threadIdx.x == 0) {
            Fre[p] = a / double(L);
            Fim[p] = b / double(L);
        }
    }
}

}  // namespace

namespace dmrg {

// rho = Psi Psi^T (side 0, rows x rows) or Psi^T Psi (side 1, cols x cols).  rho is
// symmetric: the tiles on and below the diagonal are computed and mirrored (the mirror
// is exact, C[i][j] and C[j][i] being the same products summed in the same order).
cudaError_t rho_launch(const double* Psi, int64_t rows, int64_t cols, int side, double* rho,
                       cudaStream_t s) {
    SimtGemm g{};
    g.A = Psi; g.B = Psi; g.C = rho; g.batch = 1; g.lower = 1;
    if (side == 0) {
        g.M = rows; g.N = rows; g.K = cols;
        g.sAi = cols; g.sAk = 1;          // A(a, e) = Psi[a][e]
        g.sBk = 1; g.sBj = cols;          // B(e, b) = Psi[b][e]
        g.sCi = rows; g.sCj = 1;
    } else {
        g.M = cols; g.N = cols; g.K = rows;
        g.sAi = 1; g.sAk = cols;          // A(e, a) = Psi[a][e]
        g.sBk = cols; g.sBj = 1;          // B(a, f) = Psi[a][f]
        g.sCi = cols; g.sCj = 1;
    }
    return simt_gemm_launch(Real::F64, g, s);
}

}  // namespace dmrg

namespace {

WsLayout cross_layout(int64_t Ks, int64_t Ke, int64_t rows, int64_t cols, int z64, int w64) {
    WsLayout W;
    W.add("Z64", z64 ? 0 : size_t(Ks) * rows * rows * 8);
    W.add("W64", w64 ? 0 : size_t(Ke) * cols * cols * 8);
    W.add("Y", size_t(Ks) * rows * cols * 8);
    W.add("M", size_t(Ks) * cols * cols * 8);
    W.add("part", size_t(cross_split(cols * cols).nsplit) * Ks * Ke * 8);
    return W;
}

}  // namespace

extern "C" {

dmrg_status dmrg_expectation_workspace(dmrg_handle h, int64_t K, int64_t rows, int64_t cols, int side,
                                       size_t* bytes) {
    if (!h || !bytes) return DMRG_ERR_INVALID_ARG;
    if (K < 0 || rows < 1 || cols < 1) return fail(h, DMRG_ERR_SHAPE, "need K >= 0, rows, cols >= 1");
    if (side != 0 && side != 1) return fail(h, DMRG_ERR_INVALID_ARG, "side must be 0 or 1");
    const int64_t n = side == 0 ? rows : cols;
    const TraceSplit t = trace_split(K, n * n);
    *bytes = align_up(size_t(n) * n * 8, 256) + size_t(K) * t.chunks * 8;
    return DMRG_OK;
}

dmrg_status dmrg_expectation(dmrg_handle h, const void* Z, int in_is_fp64, int64_t K,
                             const double* Psi, int64_t rows, int64_t cols, int side, double* out,
                             void* ws, size_t ws_bytes, dmrg_stream_t stream) {
    size_t need = 0;
    dmrg_status st = dmrg_expectation_workspace(h, K, rows, cols, side, &need);
    if (st != DMRG_OK) return st;
    if (K == 0) return DMRG_OK;
    if (!Z || !Psi || !out) return fail(h, DMRG_ERR_INVALID_ARG, "null pointer");
    st = check_ws(h, ws, ws_bytes, need);
    if (st != DMRG_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    double* rho = static_cast<double*>(ws);
    const int64_t n = side == 0 ? rows : cols;
    cudaError_t e = timed_launch(h, "measure_rho", s, [&] { return rho_launch(Psi, rows, cols, side, rho, s); });
    if (e != cudaSuccess) return cuda_fail(h, e, "reduced density matrix");
    const TraceSplit t = trace_split(K, n * n);
    double* part = reinterpret_cast<double*>(static_cast<char*>(ws) + align_up(size_t(n) * n * 8, 256));
    if (K > 65535) return fail(h, DMRG_ERR_SHAPE, "K too large");
    e = timed_launch(h, "measure_trace", s, [&] {
        const dim3 grid(unsigned(t.chunks), unsigned(K));
        if (in_is_fp64)
            trace_partial_kernel<double><<<grid, kTraceThreads, 0, s>>>(
                static_cast<const double*>(Z), rho, n * n, t.per, t.chunks, part);
        else
            trace_partial_kernel<float><<<grid, kTraceThreads, 0, s>>>(
                static_cast<const float*>(Z), rho, n * n, t.per, t.chunks, part);
        trace_finish_kernel<<<unsigned((K + 255) / 256), 256, 0, s>>>(part, t.chunks, K, out);
        return cudaGetLastError();
    });
    return cuda_fail(h, e, "expectation values");
}

dmrg_status dmrg_cross_correlations_workspace(dmrg_handle h, int64_t Ks, int64_t Ke, int64_t rows,
                                              int64_t cols, int z_is_fp64, int w_is_fp64,
                                              size_t* bytes) {
    if (!h || !bytes) return DMRG_ERR_INVALID_ARG;
    if (Ks < 0 || Ke < 0 || rows < 1 || cols < 1)
        return fail(h, DMRG_ERR_SHAPE, "need Ks, Ke >= 0 and rows, cols >= 1");
    *bytes = cross_layout(Ks, Ke, rows, cols, z_is_fp64, w_is_fp64).total;
    return DMRG_OK;
}

dmrg_status dmrg_cross_correlations(dmrg_handle h, const void* Z, int z_is_fp64, int64_t Ks,
                                    const void* W, int w_is_fp64, int64_t Ke, const double* Psi,
                                    int64_t rows, int64_t cols, double* C, void* ws,
                                    size_t ws_bytes, dmrg_stream_t stream) {
    size_t need = 0;
    dmrg_status st = dmrg_cross_correlations_workspace(h, Ks, Ke, rows, cols, z_is_fp64, w_is_fp64, &need);
    if (st != DMRG_OK) return st;
    if (Ks == 0 || Ke == 0) return DMRG_OK;
    if (!Z || !W || !Psi || !C) return fail(h, DMRG_ERR_INVALID_ARG, "null pointer");
    st = check_ws(h, ws, ws_bytes, need);
    if (st != DMRG_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const WsLayout L = cross_layout(Ks, Ke, rows, cols, z_is_fp64, w_is_fp64);
    char* base = static_cast<char*>(ws);
    const double* Z64 = static_cast<const double*>(Z);
    const double* W64 = static_cast<const double*>(W);
    cudaError_t e = cudaSuccess;
    if (!z_is_fp64) {
        double* dst = reinterpret_cast<double*>(base + L.offsets[0]);
        e = convert_f32_to_f64_launch(static_cast<const float*>(Z), dst, Ks * rows * rows, s);
        Z64 = dst;
    }
    if (e == cudaSuccess && !w_is_fp64) {
        double* dst = reinterpret_cast<double*>(base + L.offsets[1]);
        e = convert_f32_to_f64_launch(static_cast<const float*>(W), dst, Ke * cols * cols, s);
        W64 = dst;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "convert");
    double* Y = reinterpret_cast<double*>(base + L.offsets[2]);
    double* M = reinterpret_cast<double*>(base + L.offsets[3]);
    // Y_i = Z_i Psi (rows x cols)
    SimtGemm g1{};
    g1.A = Z64; g1.B = Psi; g1.C = Y; g1.batch = int32_t(Ks);
    g1.M = rows; g1.N = cols; g1.K = rows;
    g1.sAb = rows * rows; g1.sAi = rows; g1.sAk = 1;
    g1.sBb = 0; g1.sBk = cols; g1.sBj = 1;
    g1.sCb = rows * cols; g1.sCi = cols; g1.sCj = 1;
    e = timed_launch(h, "measure_Z_psi", s, [&] { return simt_gemm_launch(Real::F64, g1, s); });
    if (e != cudaSuccess) return cuda_fail(h, e, "Z Psi");
    // M_i = Psi^T Y_i (cols x cols)
    SimtGemm g2{};
    g2.A = Psi; g2.B = Y; g2.C = M; g2.batch = int32_t(Ks);
    g2.M = cols; g2.N = cols; g2.K = rows;
    g2.sAb = 0; g2.sAi = 1; g2.sAk = cols;
    g2.sBb = rows * cols; g2.sBk = cols; g2.sBj = 1;
    g2.sCb = cols * cols; g2.sCi = cols; g2.sCj = 1;
    e = timed_launch(h, "measure_psiT_Y", s, [&] { return simt_gemm_launch(Real::F64, g2, s); });
    if (e != cudaSuccess) return cuda_fail(h, e, "Psi^T Y");
    // C[i][j] = <M_i, W_j>_F: the reduction over cols^2 entries is split into pieces
    // (one batch entry each, partial C per piece), then the pieces are added in order.
    double* part = reinterpret_cast<double*>(base + L.offsets[4]);
    const int64_t Lx = cols * cols;
    const CrossSplit cs = cross_split(Lx);
    e = timed_launch(h, "measure_cross", s, [&] {
        SimtGemm g3{};
        g3.A = M; g3.B = W64; g3.C = part;
        g3.M = Ks; g3.N = Ke; g3.K = cs.kc; g3.batch = int32_t(cs.full);
        g3.sAb = cs.kc; g3.sAi = Lx; g3.sAk = 1;
        g3.sBb = cs.kc; g3.sBk = 1; g3.sBj = Lx;
        g3.sCb = Ks * Ke; g3.sCi = Ke; g3.sCj = 1;
        cudaError_t r = simt_gemm_launch(Real::F64, g3, s);
        if (r == cudaSuccess && cs.tail) {
            SimtGemm t3 = g3;
            t3.A = M + cs.full * cs.kc;
            t3.B = W64 + cs.full * cs.kc;
            t3.C = part + cs.full * Ks * Ke;
            t3.K = cs.tail;
            t3.batch = 1;
            r = simt_gemm_launch(Real::F64, t3, s);
        }
        if (r != cudaSuccess) return r;
        split_sum_kernel<<<unsigned((Ks * Ke + 255) / 256), 256, 0, s>>>(part, cs.nsplit, Ks * Ke, C);
        return cudaGetLastError();
    });
    return cuda_fail(h, e, "cross correlations");
}

dmrg_status dmrg_structure_factor(dmrg_handle h, const double* G, const double* v, double c,
                                  int64_t L, double* Fre, double* Fim, dmrg_stream_t stream) {
    if (!h) return DMRG_ERR_INVALID_ARG;
    if (L < 1) return fail(h, DMRG_ERR_SHAPE, "need L >= 1");
    if (!G || !Fre || !Fim) return fail(h, DMRG_ERR_INVALID_ARG, "null pointer");
    if (L > (int64_t(1) << 20)) return fail(h, DMRG_ERR_SHAPE, "L too large");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = timed_launch(h, "structure_factor", s, [&] {
        structure_factor_kernel<<<unsigned(L), 256, 0, s>>>(G, v, c, L, Fre, Fim);
        return cudaGetLastError();
    });
    return cuda_fail(h, e, "structure factor");
}

}  // extern "C"
