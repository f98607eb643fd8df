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

#include "api_common.h"

using namespace dmrg;

namespace {

// out[k] = sum_{a,b} Z_k[a][b] rho[a][b]  (rho symmetric: Tr(rho Z_k)), one block per k.
template <typename T>
__global__ void trace_kernel(const T* __restrict__ Z, const double* __restrict__ rho, int64_t n,
                             double* __restrict__ out) {
    const int64_t k = blockIdx.x;
    const T* Zk = Z + k * n * n;
    double acc = 0.0;
    for (int64_t x = threadIdx.x; x < n * n; x += blockDim.x) acc += double(Zk[x]) * rho[x];
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) out[k] = s;
    }
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

// rho = Psi Psi^T (side 0, rows x rows) or Psi^T Psi (side 1, cols x cols).
cudaError_t rho_launch(const double* Psi, int64_t rows, int64_t cols, int side, double* rho,
                       cudaStream_t s) {
    SimtGemm g{};
    g.A = Psi; g.B = Psi; g.C = rho; g.batch = 1;
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
    *bytes = size_t(n) * n * 8;
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
    e = timed_launch(h, "measure_trace", s, [&] {
        if (in_is_fp64)
            trace_kernel<double><<<unsigned(K), 256, 0, s>>>(static_cast<const double*>(Z), rho, n, out);
        else
            trace_kernel<float><<<unsigned(K), 256, 0, s>>>(static_cast<const float*>(Z), rho, n, out);
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
    // C[i][j] = <M_i, W_j>_F
    SimtGemm g3{};
    g3.A = M; g3.B = W64; g3.C = C; g3.batch = 1;
    g3.M = Ks; g3.N = Ke; g3.K = cols * cols;
    g3.sAi = cols * cols; g3.sAk = 1;
    g3.sBk = 1; g3.sBj = cols * cols;
    g3.sCi = Ke; g3.sCj = 1;
    e = timed_launch(h, "measure_cross", s, [&] { return simt_gemm_launch(Real::F64, g3, s); });
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
