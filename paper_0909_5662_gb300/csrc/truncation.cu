// truncation.cu -- the truncation matrix (Sec. 2, steps 3-4): the reduced density
// matrix rho = Psi Psi^T of the system (Eq. rho), its eigen-decomposition, the m'
// eigenvectors with the largest eigenvalues as the columns of U = R^+, and the
// discarded weight eps_rho (Eq. error).
//
// The eigen-decomposition is the cyclic Jacobi method in FP64.  A sweep visits every
// pair (p, q) once, in N - 1 rounds of N / 2 disjoint pairs (the round-robin "circle"
// schedule, N = n rounded up to even; pairs with the padding index are skipped).  In a
// round every pair's rotation J (the stable 2 x 2 symmetric Schur step: the angle that
// zeroes a_pq) is computed from the current matrix, then applied as A <- J^T A (a pass
// over row pairs), A <- A J and V <- V J (a pass over column pairs).  The sweeps stop
// when the off-diagonal part is below tol * ||A||_F.  Eigenvalues are ranked on the
// device, and U's columns are V's columns in decreasing eigenvalue order, each with its
// largest-magnitude component positive (the first such index on ties).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "api_common.h"

using namespace dmrg;

namespace {

constexpr int kThreads = 256;

// Pair i of round r in the circle schedule on N (even) indices: index N - 1 is fixed,
// the others turn.  Every pair of indices meets exactly once in rounds 0 .. N - 2.
__device__ __forceinline__ void round_pair(int64_t N, int64_t r, int64_t i, int64_t& p, int64_t& q) {
    const int64_t M = N - 1;
    int64_t a, b;
    if (i == 0) {
        a = M;
        b = r;
    } else {
        a = (r + i) % M;
        b = (r - i + M) % M;
    }
    p = a < b ? a : b;
    q = a < b ? b : a;
}

__global__ void identity_kernel(double* V, int64_t n) {
    const int64_t x = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (x < n * n) V[x] = (x / n == x % n) ? 1.0 : 0.0;
}

// Rotation of every pair of round r: cs[2i] = c, cs[2i+1] = s, pq[2i] = p, pq[2i+1] = q
// (p = q = -1 for a skipped pair).
__global__ void angles_kernel(const double* __restrict__ A, int64_t n, int64_t N, int64_t r,
                              double* __restrict__ cs, int64_t* __restrict__ pq) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= N / 2) return;
    int64_t p, q;
    round_pair(N, r, i, p, q);
    double c = 1.0, s = 0.0;
    if (q < n) {
        const double apq = A[p * n + q];
        if (apq != 0.0) {
            const double tau = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
            double t;
            if (fabs(tau) > 1e150) {
                t = 0.5 / tau;
            } else {
                t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            }
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
        }
    } else {
        p = q = -1;
    }
    cs[2 * i] = c;
    cs[2 * i + 1] = s;
    pq[2 * i] = p;
    pq[2 * i + 1] = q;
}

// A <- J^T A on the rows of every pair: thread per (pair, column), columns fastest.
__global__ void row_pass_kernel(double* __restrict__ A, int64_t n, int64_t npair,
                                const double* __restrict__ cs, const int64_t* __restrict__ pq) {
    const int64_t x = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (x >= npair * n) return;
    const int64_t i = x / n, j = x - (x / n) * n;
    const int64_t p = pq[2 * i], q = pq[2 * i + 1];
    if (p < 0) return;
    const double c = cs[2 * i], s = cs[2 * i + 1];
    const double a = A[p * n + j], b = A[q * n + j];
    A[p * n + j] = c * a - s * b;
    A[q * n + j] = s * a + c * b;
}

// A <- A J and V <- V J on the columns of every pair: thread per (row, pair), pairs
// fastest (one row per warp stays in L1).
__global__ void col_pass_kernel(double* __restrict__ A, double* __restrict__ V, int64_t n,
                                int64_t npair, const double* __restrict__ cs,
                                const int64_t* __restrict__ pq) {
    const int64_t x = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (x >= npair * n) return;
    const int64_t row = x / npair, i = x - (x / npair) * npair;
    const int64_t p = pq[2 * i], q = pq[2 * i + 1];
    if (p < 0) return;
    const double c = cs[2 * i], s = cs[2 * i + 1];
    double a = A[row * n + p], b = A[row * n + q];
    A[row * n + p] = c * a - s * b;
    A[row * n + q] = s * a + c * b;
    a = V[row * n + p];
    b = V[row * n + q];
    V[row * n + p] = c * a - s * b;
    V[row * n + q] = s * a + c * b;
}

// out[0] = sum_{i != j} A_ij^2, out[1] = sum A_ij^2 (one block).
__global__ void off_norm_kernel(const double* __restrict__ A, int64_t n, double* __restrict__ out) {
    double off = 0.0, all = 0.0;
    for (int64_t x = threadIdx.x; x < n * n; x += blockDim.x) {
        const double v = A[x] * A[x];
        all += v;
        if (x / n != x % n) off += v;
    }
    __shared__ double red[2][kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(0xffffffffu, off, o);
        all += __shfl_xor_sync(0xffffffffu, all, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = off;
        red[1][threadIdx.x >> 5] = all;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
            a += red[0][w];
            b += red[1][w];
        }
        out[0] = a;
        out[1] = b;
    }
}

// Rank of every eigenvalue in decreasing order (ties by index): lambda[rank] = d_i,
// col[rank] = i.
__global__ void rank_kernel(const double* __restrict__ A, int64_t n, double* __restrict__ lambda,
                            int64_t* __restrict__ col) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double di = A[i * n + i];
    int64_t rank = 0;
    for (int64_t j = 0; j < n; ++j) {
        const double dj = A[j * n + j];
        rank += (dj > di || (dj == di && j < i)) ? 1 : 0;
    }
    lambda[rank] = di;
    col[rank] = i;
}

// U[:, a] = sign * V[:, col[a]], the sign making the largest-magnitude component
// positive (first index on ties); one block per kept column.
__global__ void gather_kernel(const double* __restrict__ V, int64_t n, const int64_t* __restrict__ col,
                              int64_t mp, double* __restrict__ U) {
    const int64_t a = blockIdx.x;
    const int64_t c = col[a];
    double best = -1.0;
    int64_t bi = 0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
        const double v = fabs(V[r * n + c]);
        if (v > best) {
            best = v;
            bi = r;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
        }
    }
    __shared__ double sb[kThreads / 32];
    __shared__ int64_t si[kThreads / 32];
    __shared__ double sign;
    if ((threadIdx.x & 31) == 0) {
        sb[threadIdx.x >> 5] = best;
        si[threadIdx.x >> 5] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kThreads / 32; ++w)
            if (sb[w] > best || (sb[w] == best && si[w] < bi)) {
                best = sb[w];
                bi = si[w];
            }
        sign = V[bi * n + c] < 0.0 ? -1.0 : 1.0;
    }
    __syncthreads();
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) U[r * mp + a] = sign * V[r * n + c];
}

// eps = sum_{a >= mp} lambda[a] (one block).
__global__ void discarded_kernel(const double* __restrict__ lambda, int64_t n, int64_t mp,
                                 double* __restrict__ eps) {
    double acc = 0.0;
    for (int64_t a = mp + threadIdx.x; a < n; a += blockDim.x) acc += lambda[a];
    __shared__ double red[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += red[w];
        *eps = s;
    }
}

struct TruncDims {
    int64_t N, npair;
    WsLayout ws;
};

TruncDims trunc_dims(int64_t rows) {
    TruncDims D;
    D.N = rows + (rows & 1);
    D.npair = D.N / 2;
    D.ws.add("A", size_t(rows) * rows * 8);
    D.ws.add("V", size_t(rows) * rows * 8);
    D.ws.add("cs", size_t(D.npair) * 2 * 8);
    D.ws.add("pq", size_t(D.npair) * 2 * 8);
    D.ws.add("norms", 2 * 8);
    D.ws.add("col", size_t(rows) * 8);
    return D;
}

unsigned blocks_for(int64_t n) { return unsigned((n + kThreads - 1) / kThreads); }

}  // namespace

extern "C" {

dmrg_status dmrg_truncation_workspace(dmrg_handle h, int64_t rows, int64_t cols, size_t* bytes) {
    if (!h || !bytes) return DMRG_ERR_INVALID_ARG;
    if (rows < 1 || cols < 1) return fail(h, DMRG_ERR_SHAPE, "need rows, cols >= 1");
    *bytes = trunc_dims(rows).ws.total;
    return DMRG_OK;
}

dmrg_status dmrg_truncation(dmrg_handle h, const double* Psi, int64_t rows, int64_t cols, int64_t mp,
                            double* U, double* lambda, double* eps, double tol, int max_sweeps,
                            int* sweeps, void* ws, size_t ws_bytes, dmrg_stream_t stream) {
    size_t need = 0;
    dmrg_status st = dmrg_truncation_workspace(h, rows, cols, &need);
    if (st != DMRG_OK) return st;
    if (mp < 1 || mp > rows) return fail(h, DMRG_ERR_SHAPE, "need 1 <= mp <= rows");
    if (!Psi || !U || !lambda || !eps) return fail(h, DMRG_ERR_INVALID_ARG, "null pointer");
    if (!(tol > 0.0) || max_sweeps < 1) return fail(h, DMRG_ERR_INVALID_ARG, "need tol > 0, max_sweeps >= 1");
    if (rows * rows > (int64_t(1) << 31)) return fail(h, DMRG_ERR_SHAPE, "rows too large");
    st = check_ws(h, ws, ws_bytes, need);
    if (st != DMRG_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const TruncDims D = trunc_dims(rows);
    char* base = static_cast<char*>(ws);
    double* A = reinterpret_cast<double*>(base + D.ws.offsets[0]);
    double* V = reinterpret_cast<double*>(base + D.ws.offsets[1]);
    double* cs = reinterpret_cast<double*>(base + D.ws.offsets[2]);
    int64_t* pq = reinterpret_cast<int64_t*>(base + D.ws.offsets[3]);
    double* norms = reinterpret_cast<double*>(base + D.ws.offsets[4]);
    int64_t* col = reinterpret_cast<int64_t*>(base + D.ws.offsets[5]);
    const int64_t n = rows;
    cudaError_t e = timed_launch(h, "trunc_rho", s, [&] { return rho_launch(Psi, rows, cols, 0, A, s); });
    if (e != cudaSuccess) return cuda_fail(h, e, "reduced density matrix");
    identity_kernel<<<blocks_for(n * n), kThreads, 0, s>>>(V, n);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "identity");
    int done = -max_sweeps;
    double host_norms[2] = {0.0, 0.0};
    for (int sweep = 0; sweep < max_sweeps && n > 1; ++sweep) {
        for (int64_t r = 0; r < D.N - 1; ++r) {
            angles_kernel<<<blocks_for(D.npair), kThreads, 0, s>>>(A, n, D.N, r, cs, pq);
            row_pass_kernel<<<blocks_for(D.npair * n), kThreads, 0, s>>>(A, n, D.npair, cs, pq);
            col_pass_kernel<<<blocks_for(D.npair * n), kThreads, 0, s>>>(A, V, n, D.npair, cs, pq);
        }
        off_norm_kernel<<<1, kThreads, 0, s>>>(A, n, norms);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "Jacobi sweep");
        e = cudaMemcpyAsync(host_norms, norms, sizeof host_norms, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(h, e, "convergence test");
        if (host_norms[0] <= tol * tol * host_norms[1]) {
            done = sweep + 1;
            break;
        }
    }
    if (n == 1) done = 0;
    rank_kernel<<<blocks_for(n), kThreads, 0, s>>>(A, n, lambda, col);
    gather_kernel<<<unsigned(mp), kThreads, 0, s>>>(V, n, col, mp, U);
    discarded_kernel<<<1, kThreads, 0, s>>>(lambda, n, mp, eps);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "eigenvectors");
    if (sweeps) *sweeps = done;
    return DMRG_OK;
}

}  // extern "C"
