// tridiag.cu -- eigen-decomposition of the reduced density matrix for the truncation
// (Sec. 2, steps 3-4) by Householder tridiagonalisation, bisection and inverse iteration,
// all in FP64.
//
// FP64 runs at a small fraction of the FP32 and tensor rates on this part, so the solver
// spends as few FP64 operations as the problem allows: rho = Q T Q^T costs about 4n^3/3
// multiply-adds once (a cyclic Jacobi sweep costs 4n^3 and ~20 sweeps are needed), and
// only the m' kept eigenvectors are formed.
//   1. Tridiagonalisation (one cooperative launch, one grid barrier per column): for
//      column k, the reflector H_k = I - tau v v^T (v_0 = 1) with H_k x = beta e_1 for
//      x = A[k+1:, k]; then A22 <- H_k A22 H_k as A22 - v w^T - w v^T with
//      p = tau A22 v and w = p - (tau/2)(p^T v) v.  v is kept in row k of A.
//   2. All eigenvalues of T by multisection on Sturm counts (4, 8 or 16 threads per
//      eigenvalue), to an interval of max(2 eps max(|lo|, |hi|), eps ||T||) + pivmin.
//   3. The m' largest: inverse iteration with T - lambda I factored once (Gaussian
//      elimination with partial pivoting on the tridiagonal), four solves from a hashed
//      signed start vector, one thread per eigenvector.
//   4. Modified Gram-Schmidt over the m' vectors in decreasing eigenvalue order, twice
//      (one cooperative launch): eigenvectors of close or equal eigenvalues come out of
//      step 3 independent but not orthogonal.
//   5. Back-transformation x = H_0 H_1 ... H_{n-3} z, and the sign convention of U
//      (largest-magnitude component positive, the first such index on ties).
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>

#include "api_common.h"
#include "grid_sync.cuh"
#include "ptx.cuh"

namespace {

using dmrg::GridBarrier;
using dmrg::block_sum_all;
using dmrg::grid_barrier;
using dmrg::globaltimer_ns;
using dmrg::ld_acquire_gpu;

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
// Dynamic shared memory of the resident tridiagonalisation (227 KB per block, less the
// static shared memory of the barrier and block sums).
constexpr size_t kTridiagResidentSmem = 226 * 1024;
constexpr int kResidentPer = 8;                        // column entries per thread at most
constexpr int kResidentMaxN = kResidentPer * kThreads;
constexpr int kInvitIters = 4;

// ---------------------------------------------------------------- 1. tridiagonalisation
struct TriArgs {
    double* A;          // n x n symmetric, both triangles; row k receives v_k
    double* P;          // 2 x n: p of a column, by column parity
    double* R;          // 2 x n: the next-but-one pivot row, by row parity
    double* d;          // n: diagonal of T
    double* e;          // n: e[k] = T[k+1][k]
    double* tau;        // n
    GridBarrier* bar;
    unsigned* status;
    uint64_t timeout_ns;
    int n;
};

// Warp-wide sum over j < L of x[j] * y[j] (x read through L2), eight loads in flight per
// lane: a row is a chain of L2 round trips.
constexpr int kUnroll = 8;

__device__ __forceinline__ double warp_dot_l2(const double* __restrict__ x, const double* __restrict__ y,
                                              int L, int lane) {
    double a[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) a[u] = 0.0;
    int j = lane;
    for (; j + 32 * (kUnroll - 1) < L; j += 32 * kUnroll) {
        double xv[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) xv[u] = __ldcg(x + j + 32 * u);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) a[u] = fma(xv[u], y[j + 32 * u], a[u]);
    }
    for (; j < L; j += 32) a[0] = fma(__ldcg(x + j), y[j], a[0]);
    double acc = 0.0;
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) acc += a[u];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

// Rows are dealt to blocks first, then to warps: row r = b + g * (w + kWarps * t) belongs
// to warp w of block b for the whole launch.  First such row >= lo:
__device__ __forceinline__ int first_own_row(int lo, int b, int w, int g) {
    const int base = b + g * w, step = g * kWarps;
    if (base >= lo) return base;
    return base + ((lo - base + step - 1) / step) * step;
}

// The reflector H = I - tau v v^T with H x = beta e_1, for x = xs[0..Lx) in shared memory
// (v[0] = 1).  Every thread of the block returns tau and beta; v is complete on return.
__device__ void reflector(const double* xs, int Lx, double* v, double& tau, double& beta) {
    double ss = 0.0;
    for (int j = 1 + int(threadIdx.x); j < Lx; j += kThreads) ss = fma(xs[j], xs[j], ss);
    ss = block_sum_all(ss);
    const double alpha = xs[0];
    tau = 0.0;
    beta = alpha;
    double scale = 0.0;
    if (ss > 0.0) {
        beta = -copysign(sqrt(fma(alpha, alpha, ss)), alpha);
        tau = (beta - alpha) / beta;
        scale = 1.0 / (alpha - beta);
    }
    for (int j = threadIdx.x; j < Lx; j += kThreads) v[j] = j == 0 ? 1.0 : xs[j] * scale;
    __syncthreads();
}

// One grid barrier per column.  After the barrier of column k (p_k = tau_k A22 v_k
// complete) every block forms w_k = p_k - (tau_k / 2)(p_k^T v_k) v_k, and brings the
// next pivot row k+1 up to date itself (from the copy its owner published one column
// earlier, with the owner's arithmetic), so it has v_{k+1} without waiting for anyone.
// Then one pass over its own rows r >= k+2 applies A22 -= v_k w_k^T + w_k v_k^T and
// accumulates p_{k+1} = tau_{k+1} A v_{k+1} from the updated entries; the owner of row
// k+2 also publishes that row for the next column.
__global__ void __launch_bounds__(kThreads) tridiag_kernel(TriArgs T) {
    extern __shared__ double sm[];
    const int n = T.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nstep = gridDim.x * kWarps;
    if (n < 3) {   // already tridiagonal
        if (blockIdx.x == 0 && tid == 0) {
            T.d[0] = T.A[0];
            T.tau[0] = 0.0;
            if (n == 2) {
                T.e[0] = T.A[1];
                T.d[1] = T.A[3];
                T.tau[1] = 0.0;
            }
        }
        return;
    }
    double* vs = sm;            // v_k
    double* ws = sm + n;        // w_k
    double* xs = sm + 2 * n;    // row k+1 (columns k+1 ..) after column k
    double* vn = sm + 3 * n;    // v_{k+1}
    unsigned gen = 0;
    double tau_k, beta;
    // column 0: the reflector of row 0 and p_0 on own rows
    for (int j = tid; j < n - 1; j += kThreads) xs[j] = __ldcg(T.A + 1 + j);
    __syncthreads();
    reflector(xs, n - 1, vs, tau_k, beta);
    if (blockIdx.x == 0 && tid == 0) {
        T.d[0] = __ldcg(T.A);
        T.e[0] = beta;
        T.tau[0] = tau_k;
    }
    for (int r = first_own_row(1, blockIdx.x, warp, gridDim.x); r < n; r += nstep) {
        const double acc = warp_dot_l2(T.A + size_t(r) * n + 1, vs, n - 1, lane);
        if (lane == 0) __stcg(T.P + (r - 1), tau_k * acc);
    }
    for (int k = 0; k + 2 < n; ++k) {
        const int L = n - k - 1;   // trailing size of column k
        if (!grid_barrier(T.bar, gen, T.timeout_ns, T.status)) return;
        // row k is read by no one any more: it keeps v_k for the back-transformation
        if (blockIdx.x == 0)
            for (int j = tid; j < L; j += kThreads) __stcg(T.A + size_t(k) * n + (k + 1) + j, vs[j]);
        const double* P = T.P + (k & 1) * n;
        double pv = 0.0;
        for (int j = tid; j < L; j += kThreads) {
            const double pj = __ldcg(P + j);
            ws[j] = pj;
            pv = fma(pj, vs[j], pv);
        }
        const double half = 0.5 * tau_k * block_sum_all(pv);
        for (int j = tid; j < L; j += kThreads) ws[j] = fma(-half, vs[j], ws[j]);   // w = p - half v
        __syncthreads();
        // row k+1 after column k: its owner would compute a - v_0 w - w_0 v with v_0 = 1
        const double* xold = (k == 0) ? T.A + size_t(n) + 1 : T.R + ((k + 1) & 1) * n;
        const double w0 = ws[0];
        for (int j = tid; j < L; j += kThreads) xs[j] = fma(-1.0, ws[j], fma(-w0, vs[j], __ldcg(xold + j)));
        __syncthreads();
        const bool next = k + 3 < n;   // column k+1 has a reflector
        double tau_n = 0.0;
        if (next) {
            double beta_n;
            reflector(xs + 1, L - 1, vn, tau_n, beta_n);
            if (blockIdx.x == 0 && tid == 0) {
                T.d[k + 1] = xs[0];
                T.e[k + 1] = beta_n;
                T.tau[k + 1] = tau_n;
            }
        } else if (blockIdx.x == 0 && tid == 0) {   // k = n-3: rows n-2 and n-1 remain
            T.d[n - 2] = xs[0];
            T.e[n - 2] = xs[1];
            T.tau[n - 2] = 0.0;
            T.tau[n - 1] = 0.0;
        }
        // own rows r >= k+2: update for column k, p for column k+1 (columns k+2 .. only;
        // column k+1 of these rows is the pivot row's, already eliminated)
        double* Pn = T.P + ((k + 1) & 1) * n;
        double* Rn = T.R + (k & 1) * n;   // row k+2, columns k+2 ..
        for (int r = first_own_row(k + 2, blockIdx.x, warp, gridDim.x); r < n; r += nstep) {
            const int i = r - (k + 1);
            double* ri = T.A + size_t(r) * n + (k + 1);
            const double vi = vs[i], wi = ws[i];
            const bool pub = (r == k + 2) && next;
            double acc[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) acc[u] = 0.0;
            int j = 1 + lane;
            for (; j + 32 * (kUnroll - 1) < L; j += 32 * kUnroll) {
                double a[kUnroll];
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) a[u] = __ldcg(ri + j + 32 * u);
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    const int jj = j + 32 * u;
                    const double an = fma(-vi, ws[jj], fma(-wi, vs[jj], a[u]));
                    __stcg(ri + jj, an);
                    if (pub) __stcg(Rn + (jj - 1), an);
                    acc[u] = fma(an, vn[jj - 1], acc[u]);
                }
            }
            for (; j < L; j += 32) {
                const double an = fma(-vi, ws[j], fma(-wi, vs[j], __ldcg(ri + j)));
                __stcg(ri + j, an);
                if (pub) __stcg(Rn + (j - 1), an);
                acc[0] = fma(an, vn[j - 1], acc[0]);
                if (!next && r == n - 1) T.d[n - 1] = an;   // k = n-3: the last diagonal entry
            }
            if (next) {
                double p = 0.0;
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) p += acc[u];
                for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
                if (lane == 0) __stcg(Pn + (r - (k + 2)), tau_n * p);
            }
        }
        double* t = vs;
        vs = vn;
        vn = t;
        tau_k = tau_n;
    }
}

// The same column steps with every block's rows of A resident in shared memory for the
// whole launch (block b owns rows b + G i, G = gridDim.x; rpb rows at most).  Each
// column's update and product then read and write shared memory instead of making a
// chain of L2 round trips per row, and the block's eight warps share the entries of
// each row, so that the FP64 pipe, not memory latency, bounds the column.  Products of
// a row are summed per warp and then over the warps in a fixed order.
__global__ void __launch_bounds__(kThreads) tridiag_smem_kernel(TriArgs T, int rpb) {
    extern __shared__ double sm[];
    const int n = T.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x, b = blockIdx.x;
    double* vs = sm;                      // v_k
    double* ws = sm + n;                  // w_k
    double* xs = sm + 2 * n;              // row k+1 (columns k+1 ..) after column k
    double* vn = sm + 3 * n;              // v_{k+1}
    double* rows = sm + 4 * n;            // rpb x n: this block's rows of A
    const int nown = b < n ? (n - 1 - b) / G + 1 : 0;
    __shared__ double p0;                  // p_k[0] of the current column
    __shared__ double red[kWarps], sc[2];  // per-warp sums; tau and scale of the reflector
    for (int i = 0; i < nown; ++i)
        for (int c = tid; c < n; c += kThreads) rows[size_t(i) * n + c] = __ldcg(T.A + size_t(b + G * i) * n + c);
    unsigned gen = 0;
    double tau_k, beta;
    // column 0: the reflector of row 0 and p_0 on own rows
    for (int j = tid; j < n - 1; j += kThreads) xs[j] = __ldcg(T.A + 1 + j);
    __syncthreads();
    reflector(xs, n - 1, vs, tau_k, beta);
    if (b == 0 && tid == 0) {
        T.d[0] = __ldcg(T.A);
        T.e[0] = beta;
        T.tau[0] = tau_k;
    }
    const int i_first0 = (b >= 1) ? 0 : 1;   // own rows r >= 1
    for (int i = i_first0 + warp; i < nown; i += kWarps) {
        const double* ri = rows + size_t(i) * n + 1;
        double acc = 0.0;
        for (int j = lane; j < n - 1; j += 32) acc = fma(ri[j], vs[j], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) __stcg(T.P + (b + G * i - 1), tau_k * acc);
    }
    for (int k = 0; k + 2 < n; ++k) {
        const int L = n - k - 1;   // trailing size of column k
        if (!grid_barrier(T.bar, gen, T.timeout_ns, T.status)) return;
        // row k is read by no one any more: it keeps v_k for the back-transformation
        if (b == 0)
            for (int j = tid; j < L; j += kThreads) __stcg(T.A + size_t(k) * n + (k + 1) + j, vs[j]);
        // p_k (summed by every block over its rows) and row k+1 (published by its owner
        // one column earlier) are read together, one L2 round trip
        const double* P = T.P + (k & 1) * n;
        const double* xold = (k == 0) ? T.A + size_t(n) + 1 : T.R + ((k + 1) & 1) * n;
        double pv = 0.0;
        {   // every load in flight before the first use (L <= kResidentMaxN)
            double pr[kResidentPer], xr[kResidentPer];
#pragma unroll
            for (int u = 0; u < kResidentPer; ++u) {
                const int j = tid + u * kThreads;
                if (j < L) {
                    pr[u] = __ldcg(P + j);
                    xr[u] = __ldcg(xold + j);
                }
            }
#pragma unroll
            for (int u = 0; u < kResidentPer; ++u) {
                const int j = tid + u * kThreads;
                if (j < L) {
                    ws[j] = pr[u];
                    xs[j] = xr[u];
                    pv = fma(pr[u], vs[j], pv);
                }
            }
            if (tid == 0) p0 = pr[0];   // ws[0] is rewritten below while others still need p_0
        }
        const double half = 0.5 * tau_k * block_sum_all(pv);   // (its barriers order p0)
        // w = p - half v, row k+1 after column k: x - v_0 w - w_0 v with v_0 = 1, and the
        // squared norm of its entries 2 .. for the next reflector, in one pass
        const double w0 = fma(-half, vs[0], p0);
        double ss = 0.0;
        for (int j = tid; j < L; j += kThreads) {
            const double wj = fma(-half, vs[j], ws[j]);
            ws[j] = wj;
            const double xj = fma(-1.0, wj, fma(-w0, vs[j], xs[j]));
            xs[j] = xj;
            if (j >= 2) ss = fma(xj, xj, ss);
        }
        const bool next = k + 3 < n;   // column k+1 has a reflector
        // The sum of ss over the block, and the reflector's scalars from it, in one thread:
        // an FP64 instruction occupies the SM's FP64 pipe for a whole warp's worth of
        // lanes, so scalar work repeated by every warp costs as much as vector work.
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (lane == 0) red[warp] = ss;
        __syncthreads();   // (also completes ws and xs)
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < kWarps; ++w) t += red[w];
            // H x = beta e_1 for x = xs[1 .. L): v[0] = 1, as reflector() forms it
            const double alpha = xs[1];
            double beta_n = alpha, tau_r = 0.0, scale = 0.0;
            if (next && t > 0.0) {
                beta_n = -copysign(sqrt(fma(alpha, alpha, t)), alpha);
                tau_r = (beta_n - alpha) / beta_n;
                scale = 1.0 / (alpha - beta_n);
            }
            sc[0] = tau_r;
            sc[1] = scale;
            if (b == 0) {
                if (next) {
                    T.d[k + 1] = xs[0];
                    T.e[k + 1] = beta_n;
                    T.tau[k + 1] = tau_r;
                } else {   // k = n-3: rows n-2 and n-1 remain
                    T.d[n - 2] = xs[0];
                    T.e[n - 2] = xs[1];
                    T.tau[n - 2] = 0.0;
                    T.tau[n - 1] = 0.0;
                }
            }
        }
        __syncthreads();
        const double tau_n = sc[0];
        if (next) {
            const double scale = sc[1];
            for (int j = tid; j < L - 1; j += kThreads) vn[j] = j == 0 ? 1.0 : xs[j + 1] * scale;
            __syncthreads();
        }
        // own rows r >= k+2: update for column k, p for column k+1 (columns k+2 ..)
        double* Pn = T.P + ((k + 1) & 1) * n;
        double* Rn = T.R + (k & 1) * n;   // row k+2, columns k+2 ..
        // one warp per row (a row's product then takes one warp reduction)
        const int i0 = (k + 2 > b) ? (k + 2 - b + G - 1) / G : 0;
        for (int i = i0 + warp; i < nown; i += kWarps) {
            const int r = b + G * i;
            const int ii = r - (k + 1);
            double* ri = rows + size_t(i) * n + (k + 1);
            const double vi = vs[ii], wi = ws[ii];
            const bool pub = (r == k + 2) && next;
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
            int j = 1 + lane;
            for (; j + 96 < L; j += 128) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int jj = j + 32 * u;
                    const double an = fma(-vi, ws[jj], fma(-wi, vs[jj], ri[jj]));
                    ri[jj] = an;
                    if (pub) __stcg(Rn + (jj - 1), an);
                    acc[u] = fma(an, vn[jj - 1], acc[u]);
                }
            }
            for (; j < L; j += 32) {
                const double an = fma(-vi, ws[j], fma(-wi, vs[j], ri[j]));
                ri[j] = an;
                if (pub) __stcg(Rn + (j - 1), an);
                acc[0] = fma(an, vn[j - 1], acc[0]);
                if (!next && r == n - 1) T.d[n - 1] = an;   // k = n-3: the last diagonal entry
            }
            if (next) {
                double p = (acc[0] + acc[1]) + (acc[2] + acc[3]);
                for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
                if (lane == 0) __stcg(Pn + (r - (k + 2)), tau_n * p);
            }
        }
        double* t = vs;
        vs = vn;
        vn = t;
        tau_k = tau_n;
    }
}

// ---------------------------------------------------------------- 2. eigenvalues
// stats: [0] Gershgorin lower bound, [1] upper bound, [2] max(|lo|, |hi|) = ||T|| bound,
// [3] pivmin (smallest pivot magnitude of a Sturm count)
__global__ void tri_stats_kernel(const double* __restrict__ d, const double* __restrict__ e, int n,
                                 double* __restrict__ stats) {
    __shared__ double lo_s[kThreads], hi_s[kThreads], e2_s[kThreads];
    double lo = DBL_MAX, hi = -DBL_MAX, e2 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double r = 0.0;
        if (i > 0) r += fabs(e[i - 1]);
        if (i + 1 < n) r += fabs(e[i]);
        lo = fmin(lo, d[i] - r);
        hi = fmax(hi, d[i] + r);
        if (i + 1 < n) e2 = fmax(e2, e[i] * e[i]);
    }
    lo_s[threadIdx.x] = lo;
    hi_s[threadIdx.x] = hi;
    e2_s[threadIdx.x] = e2;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int t = 1; t < blockDim.x; ++t) {
            lo = fmin(lo, lo_s[t]);
            hi = fmax(hi, hi_s[t]);
            e2 = fmax(e2, e2_s[t]);
        }
        const double tn = fmax(fabs(lo), fabs(hi));
        const double pivmin = DBL_MIN * fmax(1.0, e2);
        const double pad = 2.0 * DBL_EPSILON * tn * n + 2.0 * pivmin;
        stats[0] = lo - pad;
        stats[1] = hi + pad;
        stats[2] = tn;
        stats[3] = pivmin;
    }
}

// 1/q by Newton-Raphson iteration for the reciprocal: the hardware's approximate
// reciprocal refined by two Newton steps r <- r + r (1 - q r), each of which doubles
// the correct bits (|q| >= pivmin keeps q normal, so the flush-to-zero form is exact
// here; for |q| > 1/DBL_MIN the result flushes to zero, which leaves a Sturm count
// unchanged because the term e2 / q it scales is then below the rounding of d - x).
// dmrg_debug_reciprocal exposes it so that a test can bound its error in ulps
// against correctly rounded division.
__device__ __forceinline__ double recip(double q) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(q));
    r = fma(r, fma(-q, r, 1.0), r);
    r = fma(r, fma(-q, r, 1.0), r);
    return r;
}

// Number of eigenvalues of T below x (Sturm sequence of the LDL^T pivots).
__device__ __forceinline__ int sturm_count(const double* d, const double* e2, int n, double x,
                                           double pivmin) {
    double q = d[0] - x;
    int c = q < 0.0 ? 1 : 0;
    for (int i = 1; i < n; ++i) {
        if (fabs(q) < pivmin) q = -pivmin;
        q = fma(-e2[i - 1], recip(q), d[i] - x);
        c += q < 0.0 ? 1 : 0;
    }
    return c;
}

// The same count in FP32 (for the coarse phase below, on T / ||T||), 1/q correctly
// rounded.
__device__ __forceinline__ int sturm_count32(const float* d, const float* e2, int n, float x,
                                             float pivmin) {
    float q = d[0] - x;
    int c = q < 0.f ? 1 : 0;
    for (int i = 1; i < n; ++i) {
        if (fabsf(q) < pivmin) q = -pivmin;
        q = fmaf(-e2[i - 1], __frcp_rn(q), d[i] - x);
        c += q < 0.f ? 1 : 0;
    }
    return c;
}

// Multisection: kSect neighbouring threads share eigenvalue j (the j-th smallest) and
// count at kSect interior points of its interval at once, so each round shrinks it
// kSect + 1 times.  Stops at width 2 eps max(|lo|, |hi|), or eps ||T|| (the absolute
// accuracy a backward-stable dense solver gives), plus pivmin.  The eigenvalue is
// stored as lambda[n - 1 - j] (decreasing order).  d and e^2 are staged in shared
// memory when they fit.  A Sturm count is a chain of dependent FP64 operations, so the
// host picks kSect (4, 8 or 16) to give every SM at least two warps: more points per
// round cost more counts in all but fewer rounds on the critical path.
constexpr int kBisectThreads = 64;

template <int kSect>
__global__ void __launch_bounds__(kBisectThreads) bisect_kernel(const double* __restrict__ d,
                                                                const double* __restrict__ e, int n,
                                                                const double* __restrict__ stats,
                                                                double* __restrict__ e2g, int staged,
                                                                double* __restrict__ lambda) {
    extern __shared__ double sm[];
    const double* dd = d;
    const double* ee = e2g;
    const float* d32 = nullptr;
    const float* e32 = nullptr;
    // staged: 0 = d and e^2 read from global memory; 1 = staged in shared memory (FP64);
    // 2 = also their FP32 copies for the coarse phase
    const double tn = stats[2];
    const bool coarse = staged == 2 && tn > 0.0;
    if (staged) {
        double* ds = sm;
        double* es = sm + n;
        float* fs = reinterpret_cast<float*>(sm + 2 * n);   // T / ||T|| in FP32
        float* gs = fs + n;
        const double inv = tn > 0.0 ? 1.0 / tn : 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            ds[i] = d[i];
            if (staged == 2) fs[i] = float(d[i] * inv);
            if (i + 1 < n) {
                es[i] = e[i] * e[i];
                const double es_i = e[i] * inv;
                if (staged == 2) gs[i] = float(es_i * es_i);
            }
        }
        __syncthreads();
        dd = ds;
        ee = es;
        d32 = fs;
        e32 = gs;
    }
    const int t = threadIdx.x % kSect;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) / kSect;
    const bool live = j < n;
    double lo = stats[0], hi = stats[1];
    const double atol = DBL_EPSILON * stats[2], pivmin = stats[3];
    const int gbase = (threadIdx.x & 31) & ~(kSect - 1);   // first lane of this group
    if (coarse) {
        // Coarse phase: the same multisection with FP32 counts on T / ||T|| (an FP32
        // operation costs a small fraction of an FP64 one here).  A computed count is the
        // exact count of a matrix within a few FP32 roundings of T, so the interval, widened
        // by 16 FP32 epsilons of ||T||, is checked with FP64 counts at its two ends and
        // used only if they bracket j; otherwise the search starts from the Gershgorin
        // interval as before.
        float flo = float(lo / tn), fhi = float(hi / tn);
        bool fdone = !live;
        for (int round = 0; round < 64; ++round) {
            const float w = fhi - flo;
            if (!fdone && w <= 0x1p-20f) fdone = true;
            if (__all_sync(0xffffffffu, fdone)) break;
            const float x = flo + w * float(t + 1) / float(kSect + 1);
            const int c = fdone ? 0 : sturm_count32(d32, e32, n, x, FLT_MIN);
            float nlo = flo, nhi = fhi;
            bool hit = false;
#pragma unroll
            for (int u = 0; u < kSect; ++u) {
                const int cu = __shfl_sync(0xffffffffu, c, gbase + u);
                const float xu = __shfl_sync(0xffffffffu, x, gbase + u);
                if (!hit) {
                    if (cu <= j) {
                        nlo = xu;
                    } else {
                        nhi = xu;
                        hit = true;
                    }
                }
            }
            if (!fdone) {
                const bool stuck = !(nlo > flo || nhi < fhi);
                flo = nlo;
                fhi = nhi;
                if (stuck) fdone = true;
            }
        }
        const double margin = 16.0 * double(FLT_EPSILON) * tn;
        const double clo = fmax(double(flo) * tn - margin, lo);
        const double chi = fmin(double(fhi) * tn + margin, hi);
        int cend = 0;
        if (live && t < 2) cend = sturm_count(dd, ee, n, t == 0 ? clo : chi, pivmin);
        const int clo_n = __shfl_sync(0xffffffffu, cend, gbase);
        const int chi_n = __shfl_sync(0xffffffffu, cend, gbase + 1);
        if (live && clo < chi && clo_n <= j && j < chi_n) {
            lo = clo;
            hi = chi;
        }
    }
    bool done = !live;
    for (int round = 0; round < 128; ++round) {
        // every group runs the same number of rounds of the warp's loop; finished or
        // absent groups keep their interval
        const double w = hi - lo;
        if (!done && (w <= fmax(2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)), atol) + pivmin)) done = true;
        if (__all_sync(0xffffffffu, done)) break;
        const double x = lo + w * double(t + 1) / double(kSect + 1);
        const int c = done ? 0 : sturm_count(dd, ee, n, x, pivmin);
        // the new interval: from the first point whose count exceeds j back to the point
        // before it (so a count that is not monotone in rounding cannot cross the bounds)
        double nlo = lo, nhi = hi;
        bool hit = false;
#pragma unroll
        for (int u = 0; u < kSect; ++u) {
            const int src = gbase + u;
            const int cu = __shfl_sync(0xffffffffu, c, src);
            const double xu = __shfl_sync(0xffffffffu, x, src);
            if (!hit) {
                if (cu <= j) {
                    nlo = xu;
                } else {
                    nhi = xu;
                    hit = true;
                }
            }
        }
        if (!done) {
            const bool stuck = !(nlo > lo || nhi < hi);
            lo = nlo;
            hi = nhi;
            if (stuck) done = true;
        }
    }
    if (live && t == 0) lambda[n - 1 - j] = 0.5 * (lo + hi);
}

__global__ void square_kernel(const double* __restrict__ e, int n, double* __restrict__ e2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i + 1 < n) e2[i] = e[i] * e[i];
}

// ---------------------------------------------------------------- 3. inverse iteration
// Signed start entry in [-1, 1) from a multiply-xorshift hash of (i, j).
__device__ __forceinline__ double start_entry(int i, int j) {
    uint32_t h = uint32_t(i) * 2654435761u + uint32_t(j) * 40503u + 12345u;
    h = (h ^ (h >> 15)) * 2246822519u;
    h ^= h >> 13;
    return double(h) * (1.0 / 2147483648.0) - 1.0;
}

// Thread j: the eigenvector of lambda[j] (j < mp, decreasing order).  Scratch arrays are
// interleaved, entry i of vector j at i * mp + j, so a warp's accesses are contiguous.
// The factorisation keeps its running row in registers (d and e are read by every thread
// of the warp at once); the solves read their operands kChunk at a time, so that the
// loads of a chunk are in flight together and only the arithmetic is sequential.
constexpr int kChunk = 8;

__global__ void __launch_bounds__(32) invit_kernel(const double* __restrict__ d,
                                                   const double* __restrict__ e, int n, int mp,
                                                   const double* __restrict__ lambda,
                                                   const double* __restrict__ stats,
                                                   double* __restrict__ u1, double* __restrict__ u2,
                                                   double* __restrict__ u3, double* __restrict__ lm,
                                                   unsigned char* __restrict__ sw,
                                                   double* __restrict__ z, double* __restrict__ Zt) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= mp) return;
    const double lam = lambda[j];
    const double small = DBL_EPSILON * fmax(stats[2], DBL_MIN);
    auto at = [&](int i) { return size_t(i) * mp + j; };
    auto guard = [&](double a) { return fabs(a) < small ? (a >= 0.0 ? small : -small) : a; };
    // T - lam I = P L U with partial pivoting; U has diagonals u1, u2 (super), u3.  u1 is
    // stored inverted: the one division per row here replaces one per row in each of the
    // solves below (a division is a long FP64 sequence, and FP64 is this kernel's bound).
    double a = d[0] - lam, s_cur = n > 1 ? e[0] : 0.0;
    for (int i = 0; i + 1 < n; ++i) {
        const double c = e[i], a_next = d[i + 1] - lam, s_next = (i + 2 < n) ? e[i + 1] : 0.0;
        if (fabs(a) >= fabs(c)) {
            const double inv = 1.0 / guard(a);
            const double l = c * inv;
            u1[at(i)] = inv;
            u2[at(i)] = s_cur;
            u3[at(i)] = 0.0;
            lm[at(i)] = l;
            sw[at(i)] = 0;
            a = a_next - l * s_cur;
            s_cur = s_next;
        } else {
            const double inv = 1.0 / guard(c);
            const double l = a * inv;
            u1[at(i)] = inv;
            u2[at(i)] = a_next;
            u3[at(i)] = s_next;
            lm[at(i)] = l;
            sw[at(i)] = 1;
            a = s_cur - l * a_next;
            s_cur = -l * s_next;
        }
    }
    u1[at(n - 1)] = 1.0 / guard(a);
    for (int i = 0; i < n; ++i) z[at(i)] = start_entry(i, j);
    for (int it = 0; it < kInvitIters; ++it) {
        double zmax = 0.0;
        for (int i0 = 0; i0 < n; i0 += kChunk) {
            double v[kChunk];
#pragma unroll
            for (int q = 0; q < kChunk; ++q) v[q] = (i0 + q < n) ? z[at(i0 + q)] : 0.0;
#pragma unroll
            for (int q = 0; q < kChunk; ++q) zmax = fmax(zmax, fabs(v[q]));
        }
        const double inv = zmax > 0.0 ? 1.0 / zmax : 1.0;
        // forward: the row interchanges and multipliers of the factorisation
        double prev = z[at(0)] * inv;
        for (int i0 = 0; i0 + 1 < n; i0 += kChunk) {
            double zc[kChunk], lc[kChunk];
            unsigned char sc[kChunk];
#pragma unroll
            for (int q = 0; q < kChunk; ++q) {
                const int i = i0 + q;
                const bool ok = i + 1 < n;
                zc[q] = ok ? z[at(i + 1)] : 0.0;
                lc[q] = ok ? lm[at(i)] : 0.0;
                sc[q] = ok ? sw[at(i)] : 0;
            }
#pragma unroll
            for (int q = 0; q < kChunk; ++q) {
                const int i = i0 + q;
                if (i + 1 < n) {
                    double cur = zc[q] * inv;
                    if (sc[q]) {
                        const double t = prev;
                        prev = cur;
                        cur = t;
                    }
                    z[at(i)] = prev;
                    prev = cur - lc[q] * prev;
                }
            }
        }
        z[at(n - 1)] = prev;
        // backward substitution
        double x1 = 0.0, x2 = 0.0;
        for (int i0 = n - 1; i0 >= 0; i0 -= kChunk) {
            double yc[kChunk], a1[kChunk], a2[kChunk], a3[kChunk];
#pragma unroll
            for (int q = 0; q < kChunk; ++q) {
                const int i = i0 - q;
                const bool ok = i >= 0;
                yc[q] = ok ? z[at(i)] : 0.0;
                a1[q] = ok ? u1[at(i)] : 1.0;
                a2[q] = (ok && i + 1 < n) ? u2[at(i)] : 0.0;
                a3[q] = (ok && i + 2 < n) ? u3[at(i)] : 0.0;
            }
#pragma unroll
            for (int q = 0; q < kChunk; ++q) {
                const int i = i0 - q;
                if (i >= 0) {
                    const double x = (yc[q] - a2[q] * x1 - a3[q] * x2) * a1[q];
                    z[at(i)] = x;
                    x2 = x1;
                    x1 = x;
                }
            }
        }
    }
    for (int i = 0; i < n; ++i) Zt[size_t(j) * n + i] = z[at(i)];
}

// ---------------------------------------------------------------- 4. Gram-Schmidt
// Warp-wide sum over i < n of x[i] * y[i], both read through L2, four of each in flight.
__device__ __forceinline__ double warp_dot_l2_both(const double* __restrict__ x,
                                                   const double* __restrict__ y, int n, int lane) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int i = lane;
    for (; i + 96 < n; i += 128) {
        const double x0 = __ldcg(x + i), x1 = __ldcg(x + i + 32), x2 = __ldcg(x + i + 64),
                     x3 = __ldcg(x + i + 96);
        const double y0 = __ldcg(y + i), y1 = __ldcg(y + i + 32), y2 = __ldcg(y + i + 64),
                     y3 = __ldcg(y + i + 96);
        a0 = fma(x0, y0, a0);
        a1 = fma(x1, y1, a1);
        a2 = fma(x2, y2, a2);
        a3 = fma(x3, y3, a3);
    }
    for (; i < n; i += 32) a0 = fma(__ldcg(x + i), __ldcg(y + i), a0);
    double acc = (a0 + a1) + (a2 + a3);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

struct MgsArgs {
    double* Zt;   // mp x n, row j = eigenvector j
    GridBarrier* bar;
    unsigned* status;
    uint64_t timeout_ns;
    int n, mp;
};

// Two passes of modified Gram-Schmidt in row order; each step projects row j out of the
// later rows (one row per warp), then every row is normalised.
__global__ void __launch_bounds__(kThreads) mgs_kernel(MgsArgs M) {
    const int n = M.n, mp = M.mp, tid = threadIdx.x, lane = tid & 31;
    const int gwarp = blockIdx.x * kWarps + (tid >> 5), nwarps = gridDim.x * kWarps;
    unsigned gen = 0;
    for (int pass = 0; pass < 2; ++pass) {
        for (int j = 0; j + 1 < mp; ++j) {
            const double* zj = M.Zt + size_t(j) * n;
            double ss = 0.0;
            for (int i = tid; i < n; i += kThreads) {
                const double x = __ldcg(zj + i);
                ss = fma(x, x, ss);
            }
            const double nn = block_sum_all(ss);
            const double inv2 = nn > 0.0 ? 1.0 / nn : 0.0;
            for (int r = first_own_row(j + 1, blockIdx.x, tid >> 5, gridDim.x); r < mp; r += nwarps) {
                double* zr = M.Zt + size_t(r) * n;
                const double c = warp_dot_l2_both(zj, zr, n, lane) * inv2;
                int i = lane;
                for (; i + 96 < n; i += 128) {
                    double a[4], b[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        a[u] = __ldcg(zr + i + 32 * u);
                        b[u] = __ldcg(zj + i + 32 * u);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) __stcg(zr + i + 32 * u, fma(-c, b[u], a[u]));
                }
                for (; i < n; i += 32) __stcg(zr + i, fma(-c, __ldcg(zj + i), __ldcg(zr + i)));
            }
            if (!grid_barrier(M.bar, gen, M.timeout_ns, M.status)) return;
        }
        for (int r = gwarp; r < mp; r += nwarps) {
            double* zr = M.Zt + size_t(r) * n;
            double ss = 0.0;
            for (int i = lane; i < n; i += 32) {
                const double x = __ldcg(zr + i);
                ss = fma(x, x, ss);
            }
            for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
            const double inv = ss > 0.0 ? 1.0 / sqrt(ss) : 0.0;
            for (int i = lane; i < n; i += 32) __stcg(zr + i, __ldcg(zr + i) * inv);
        }
        if (!grid_barrier(M.bar, gen, M.timeout_ns, M.status)) return;
    }
}

// The same two passes of modified Gram-Schmidt with the rows kept in shared memory and
// no grid-wide barrier.  Rows are dealt to blocks in groups of kMgsG consecutive rows
// (group G to block G mod gridDim); kMgsS warps share each row, every warp owning a
// contiguous slice of its entries, so a block keeps all four SM sub-partitions busy with
// FP64 work.  Each block walks the groups in order: when group J is its own it runs the
// Gram-Schmidt steps of the group's rows among themselves, publishes them and their
// squared norms, and raises the group's flag; then, if it holds rows of later groups,
// it waits for group J's flag, stages the published rows in shared memory and projects
// them, in order, out of those rows.  Each row receives the same projections in the same
// order as in mgs_kernel; a block waits only for the group it needs next, so the
// critical path is one group's hand-on per group instead of a grid barrier per row.
// Every pass publishes into its own buffer, so a block still reading a group of the first
// pass never sees the second pass's rows.  Waits are bounded: on expiry a block records
// the timeout, raises the abort word and returns, and the others return at their next
// wait.
constexpr int kMgsG = 2;                       // rows per group
constexpr int kMgsS = 2;                       // warps per row
constexpr int kMgsThreads = 32 * kMgsG * kMgsS;

struct MgsFlowArgs {
    double* Zt;           // mp x n, row j = eigenvector j (input and output)
    double* pub[2];       // per pass: published rows, mp x n
    double* norms[2];     // per pass: reciprocal squared norms of the published rows (0 for 0)
    unsigned* flags;      // [2][ngroups] publication flags, then the abort word; zeroed
    unsigned* status;
    uint64_t timeout_ns;
    int n, mp;
};

// Partial dot over this warp's slice [i0, i1) of two shared-memory rows.
__device__ __forceinline__ double slice_dot(const double* x, const double* y, int i0, int i1,
                                            int lane) {
    double a0 = 0.0, a1 = 0.0;
    int i = i0 + lane;
    for (; i + 32 < i1; i += 64) {
        a0 = fma(x[i], y[i], a0);
        a1 = fma(x[i + 32], y[i + 32], a1);
    }
    for (; i < i1; i += 32) a0 = fma(x[i], y[i], a0);
    double acc = a0 + a1;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0 waits (bounded) until *flag is set; the block follows its verdict.
__device__ bool wait_flag(unsigned* flag, unsigned* abort_word, uint64_t timeout_ns,
                          unsigned* status) {
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        if (ld_acquire_gpu(flag) == 0u) {
            const uint64_t t0 = globaltimer_ns();
            uint32_t spins = 0;
            while (ld_acquire_gpu(flag) == 0u) {
                if ((++spins & 31u) == 0) {
                    if (ld_acquire_gpu(abort_word) != 0u) {
                        ok = 0;
                        break;
                    }
                    if (globaltimer_ns() - t0 > timeout_ns) {
                        atomicOr(status, DMRG_DEV_ERR_TIMEOUT);
                        atomicExch(abort_word, 1u);
                        ok = 0;
                        break;
                    }
                }
            }
        }
    }
    __syncthreads();
    const bool r = ok != 0;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kMgsThreads) mgs_flow_kernel(MgsFlowArgs M) {
    extern __shared__ double own[];   // [owned group t][row][n], then pub[kMgsG][n]
    __shared__ double part[kMgsG][kMgsS];
    __shared__ double rinv;
    const int n = M.n, mp = M.mp, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w = warp / kMgsS;       // row of the group
    const int q = warp % kMgsS;       // slice of the row
    const int slice = (n + kMgsS - 1) / kMgsS;
    const int i0 = min(n, q * slice), i1 = min(n, i0 + slice);
    const int ngroups = (mp + kMgsG - 1) / kMgsG;
    const int nown = (ngroups - int(blockIdx.x) + int(gridDim.x) - 1) / int(gridDim.x);
    double* stage = own + size_t(nown) * kMgsG * n;
    const int last_own = int(blockIdx.x) + (nown - 1) * int(gridDim.x);
    unsigned* abort_word = M.flags + 2 * ngroups;
    // sum of the kMgsS partial dots of row w (every thread of the block calls this)
    auto row_sum = [&](double v) -> double {
        if (lane == 0) part[w][q] = v;
        __syncthreads();
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < kMgsS; ++k) t += part[w][k];
        __syncthreads();
        return t;
    };
    for (int t = 0; t < nown; ++t) {
        const int r = (int(blockIdx.x) + t * int(gridDim.x)) * kMgsG + w;
        if (r < mp)
            for (int i = i0 + lane; i < i1; i += 32) own[(size_t(t) * kMgsG + w) * n + i] = M.Zt[size_t(r) * n + i];
    }
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        double* pubz = M.pub[pass];
        double* norms = M.norms[pass];
        unsigned* flags = M.flags + pass * ngroups;
        for (int J = 0; J < ngroups; ++J) {
            const int nj = min(kMgsG, mp - J * kMgsG);
            if (J % int(gridDim.x) == int(blockIdx.x)) {
                // the group's own Gram-Schmidt steps, then publication and the flag
                double* grow = own + size_t(J / int(gridDim.x)) * kMgsG * n;
                for (int jj = 0; jj < nj; ++jj) {
                    const double* zj = grow + size_t(jj) * n;
                    double nn = 0.0;
                    {
                        const double v = (w == jj) ? slice_dot(zj, zj, i0, i1, lane) : 0.0;
                        if (lane == 0) part[w][q] = v;
                        __syncthreads();
                        for (int k = 0; k < kMgsS; ++k) nn += part[jj][k];
                        __syncthreads();
                    }
                    // the reciprocal, once: every projection of row jj multiplies by it
                    if (threadIdx.x == 0) rinv = nn > 0.0 ? 1.0 / nn : 0.0;
                    __syncthreads();
                    const double rn = rinv;
                    if (threadIdx.x == 0) __stcg(norms + J * kMgsG + jj, rn);
                    double* zr = grow + size_t(w) * n;
                    const bool mine = w > jj && w < nj;
                    const double dsum = row_sum(mine ? slice_dot(zj, zr, i0, i1, lane) : 0.0);
                    if (mine) {
                        const double c = dsum * rn;
                        for (int i = i0 + lane; i < i1; i += 32) zr[i] = fma(-c, zj[i], zr[i]);
                    }
                    __syncthreads();
                }
                if (w < nj)
                    for (int i = i0 + lane; i < i1; i += 32)
                        __stcg(pubz + size_t(J * kMgsG + w) * n + i, grow[size_t(w) * n + i]);
                __threadfence();
                __syncthreads();
                if (threadIdx.x == 0) st_release_gpu(flags + J, 1u);
            }
            if (last_own <= J) continue;   // no later rows here (block-uniform)
            if (!wait_flag(flags + J, abort_word, M.timeout_ns, M.status)) return;
            // stage the published group J in shared memory, then project it out of this
            // block's rows of later groups
            {
                const double* src = pubz + size_t(J) * kMgsG * n;
                const int total = nj * n;
                if ((n & 1) == 0) {
                    const double2* s2 = reinterpret_cast<const double2*>(src);
                    double2* d2 = reinterpret_cast<double2*>(stage);
                    for (int i = threadIdx.x; i < total / 2; i += kMgsThreads) d2[i] = __ldcg(s2 + i);
                } else {
                    for (int i = threadIdx.x; i < total; i += kMgsThreads) stage[i] = __ldcg(src + i);
                }
            }
            __syncthreads();
            for (int t = 0; t < nown; ++t) {
                const int G2 = int(blockIdx.x) + t * int(gridDim.x);
                if (G2 <= J) continue;   // block-uniform
                const int r = G2 * kMgsG + w;
                const bool live = r < mp;
                double* zr = own + (size_t(t) * kMgsG + w) * n;
                for (int jj = 0; jj < nj; ++jj) {
                    const double* zj = stage + size_t(jj) * n;
                    const double rn = __ldcg(norms + J * kMgsG + jj);   // 1 / ||z_j||^2 (0 for 0)
                    const double dsum = row_sum(live ? slice_dot(zr, zj, i0, i1, lane) : 0.0);
                    if (live) {
                        const double c = dsum * rn;
                        for (int i = i0 + lane; i < i1; i += 32) zr[i] = fma(-c, zj[i], zr[i]);
                    }
                }
            }
            __syncthreads();   // the staging buffer is refilled for the next group
        }
        // normalise this block's rows
        for (int t = 0; t < nown; ++t) {
            const int r = (int(blockIdx.x) + t * int(gridDim.x)) * kMgsG + w;
            double* zr = own + (size_t(t) * kMgsG + w) * n;
            const double ss = row_sum(r < mp ? slice_dot(zr, zr, i0, i1, lane) : 0.0);
            const double inv = ss > 0.0 ? 1.0 / sqrt(ss) : 0.0;
            if (r < mp)
                for (int i = i0 + lane; i < i1; i += 32) zr[i] *= inv;
        }
        __syncthreads();
    }
    for (int t = 0; t < nown; ++t) {
        const int r = (int(blockIdx.x) + t * int(gridDim.x)) * kMgsG + w;
        if (r < mp)
            for (int i = i0 + lane; i < i1; i += 32) M.Zt[size_t(r) * n + i] = own[(size_t(t) * kMgsG + w) * n + i];
    }
}

// ---------------------------------------------------------------- 5. back-transformation
// One block of kBackSplit warps per eigenvector.  The vector lives in shared memory and
// each warp owns a fixed set of its entries (alternate 32-entry blocks), so the warps
// meet once per reflector, to add their halves of v^T z.  The reflectors are applied from
// the last to the first; each is fetched with cp.async into one of three rotating
// shared-memory buffers while the one before it is applied.  FP64 issues per SM
// sub-partition, so the vectors are split over warps to occupy all four of them.
// Then the vector gets its sign (the largest-magnitude component positive, the first
// index on ties) and is written into U (n x mp, row-major).
constexpr int kBackSplit = 4;   // warps per eigenvector
constexpr int kBackThreads = 32 * kBackSplit;

__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dmrg::smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__global__ void __launch_bounds__(kBackThreads) back_kernel(const double* __restrict__ A,
                                                            const double* __restrict__ tau,
                                                            const double* __restrict__ Zt, int n,
                                                            int mp, double* __restrict__ U) {
    extern __shared__ double bsm[];   // the vector (n), three reflector buffers (n each)
    __shared__ double lanes[2][kBackThreads];   // every lane's part of v^T z
    __shared__ double coef[2];                  // tau v^T z
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int j = blockIdx.x;
    double* z = bsm;
    for (int i = tid; i < n; i += kBackThreads) z[i] = Zt[size_t(j) * n + i];
    auto buf = [&](int slot) { return bsm + size_t(1 + slot) * n; };
    auto fetch = [&](int k, double* dst) {   // v_k: A[k][k+1 .. n-1], one group (maybe empty)
        if (k >= 0) {
            const double* src = A + size_t(k) * n + (k + 1);
            for (int i = tid; i < n - k - 1; i += kBackThreads) cp_async8(dst + i, src + i);
        }
        cp_async_commit();
    };
    fetch(n - 3, buf(0));
    fetch(n - 4, buf(1));
    cp_async_wait_all();
    __syncthreads();
    // this warp's entries: i = 32 (kBackSplit q + w) + lane, q = 0, 1, ...
    int slot = 0;
    for (int k = n - 3; k >= 0; --k) {
        const double t = tau[k];   // uniform over the block
        const double* v = buf(slot);
        // first of this warp's 32-entry blocks that reaches past k
        const int b0 = (k + 1) >> 5;
        const int i0 = 32 * (b0 + (w - b0 % kBackSplit + kBackSplit) % kBackSplit) + lane;
        double a0 = 0.0, a1 = 0.0;
        for (int i = i0; i < n; i += 64 * kBackSplit) {
            if (i > k) a0 = fma(v[i - (k + 1)], z[i], a0);
            const int i2 = i + 32 * kBackSplit;
            if (i2 < n) a1 = fma(v[i2 - (k + 1)], z[i2], a1);
        }
        lanes[k & 1][tid] = a0 + a1;
        cp_async_wait_all();   // v_{k-1}, fetched one reflector ago
        __syncthreads();       // every lane's part of v^T z; v_{k-1} complete; v_{k+1} read
        fetch(k - 2, buf(slot == 0 ? 2 : slot - 1));   // into the buffer of v_{k+1}
        // One warp adds the parts and forms tau v^T z: an FP64 instruction holds the
        // sub-partition's FP64 pipe for a whole warp, so the sum is not repeated per warp.
        if (w == 0) {
            double sdot = 0.0;
#pragma unroll
            for (int u = 0; u < kBackSplit; ++u) sdot += lanes[k & 1][32 * u + lane];
            for (int o = 16; o > 0; o >>= 1) sdot += __shfl_xor_sync(0xffffffffu, sdot, o);
            if (lane == 0) coef[k & 1] = t * sdot;
        }
        __syncthreads();
        if (t != 0.0) {
            const double c = coef[k & 1];
            for (int i = i0; i < n; i += 32 * kBackSplit)
                if (i > k) z[i] = fma(-c, v[i - (k + 1)], z[i]);
        }
        slot = slot == 2 ? 0 : slot + 1;
    }
    cp_async_wait_all();
    __syncthreads();
    __shared__ double bv[kBackSplit];
    __shared__ int bi[kBackSplit];
    double best = -1.0;
    int idx = 0;
    for (int i = tid; i < n; i += kBackThreads) {
        const double a = fabs(z[i]);
        if (a > best) {
            best = a;
            idx = i;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ob > best || (ob == best && oi < idx)) {
            best = ob;
            idx = oi;
        }
    }
    if (lane == 0) {
        bv[w] = best;
        bi[w] = idx;
    }
    __syncthreads();
    best = bv[0];
    idx = bi[0];
    for (int u = 1; u < kBackSplit; ++u)
        if (bv[u] > best || (bv[u] == best && bi[u] < idx)) {
            best = bv[u];
            idx = bi[u];
        }
    const double sgn = z[idx] < 0.0 ? -1.0 : 1.0;
    for (int i = tid; i < n; i += kBackThreads) U[size_t(i) * mp + j] = sgn * z[i];
}

// Blocks of a cooperative launch of `kernel` with `smem` dynamic bytes, at most `cap`.
// (one block per SM at most when per_sm_cap = 1: FP64 work is bound per SM)
cudaError_t coop_grid(const void* kernel, size_t smem, int cap, int* grid, int per_sm_cap = 2) {
    int dev = 0, sms = 0, per_sm = 0, coop = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (!coop || per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    *grid = std::max(1, std::min(cap, sms * std::min(per_sm, per_sm_cap)));
    return cudaSuccess;
}

__global__ void recip_kernel(const double* __restrict__ q, double* __restrict__ out, int64_t n) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) out[i] = recip(q[i]);
}

}  // namespace

extern "C" DMRG_API dmrg_status dmrg_debug_reciprocal(const double* q, double* out, int64_t n,
                                                      dmrg_stream_t stream) {
    if (n < 0 || (n > 0 && (!q || !out))) return DMRG_ERR_INVALID_ARG;
    if (n == 0) return DMRG_OK;
    const int64_t blocks = (n + 255) / 256;
    if (blocks > 0x7fffffffLL) return DMRG_ERR_SHAPE;
    recip_kernel<<<unsigned(blocks), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(q, out, n);
    return cudaGetLastError() == cudaSuccess ? DMRG_OK : DMRG_ERR_CUDA;
}

namespace dmrg {

WsLayout tridiag_layout(int64_t n, int64_t mp) {
    WsLayout W;
    W.add("A", size_t(n) * n * 8);
    W.add("P", size_t(n) * 2 * 8);
    W.add("R", size_t(n) * 2 * 8);
    W.add("d", size_t(n) * 8);
    W.add("e", size_t(n) * 8);
    W.add("e2", size_t(n) * 8);
    W.add("tau", size_t(n) * 8);
    W.add("stats", 4 * 8);
    W.add("bar", sizeof(GridBarrier));
    W.add("Zt", size_t(mp) * n * 8);
    for (int a = 0; a < 5; ++a) W.add("lu", size_t(mp) * n * 8);   // u1, u2, u3, l, z
    W.add("sw", size_t(mp) * n);
    return W;
}

// rho (n x n, in the layout's A section) -> U (n x mp), lambda (n, decreasing), eps.
dmrg_status tridiag_eigen(dmrg_handle h, int64_t n64, int64_t mp64, char* ws, double* U,
                          double* lambda, double* eps, cudaStream_t s) {
    const int n = int(n64), mp = int(mp64);
    const WsLayout W = tridiag_layout(n, mp);
    double* A = reinterpret_cast<double*>(ws + W.offsets[0]);
    double* P = reinterpret_cast<double*>(ws + W.offsets[1]);
    double* R = reinterpret_cast<double*>(ws + W.offsets[2]);
    double* d = reinterpret_cast<double*>(ws + W.offsets[3]);
    double* e = reinterpret_cast<double*>(ws + W.offsets[4]);
    double* e2 = reinterpret_cast<double*>(ws + W.offsets[5]);
    double* tau = reinterpret_cast<double*>(ws + W.offsets[6]);
    double* stats = reinterpret_cast<double*>(ws + W.offsets[7]);
    GridBarrier* bar = reinterpret_cast<GridBarrier*>(ws + W.offsets[8]);
    double* Zt = reinterpret_cast<double*>(ws + W.offsets[9]);
    double* lu[5];
    for (int a = 0; a < 5; ++a) lu[a] = reinterpret_cast<double*>(ws + W.offsets[10 + a]);
    unsigned char* sw = reinterpret_cast<unsigned char*>(ws + W.offsets[15]);
    cudaError_t err;
    // 1. tridiagonalisation: with every block's rows in shared memory when they fit
    //    (one block per SM), else through L2
    const int g_res = std::max(1, std::min(h->num_sms, n));
    const int rpb = (n + g_res - 1) / g_res;
    const size_t smem_res = (size_t(4) * n + size_t(rpb) * n) * 8;
    bool resident = n >= 3 && n <= kResidentMaxN && smem_res <= kTridiagResidentSmem;
    if (resident) {
        int grid = 0;
        err = cudaFuncSetAttribute(tridiag_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   int(smem_res));
        if (err == cudaSuccess)
            err = coop_grid(reinterpret_cast<const void*>(tridiag_smem_kernel), smem_res, g_res, &grid, 1);
        if (err != cudaSuccess || grid != g_res) {
            cudaGetLastError();
            resident = false;
        }
    }
    if (resident) {
        err = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s);
        if (err != cudaSuccess) return cuda_fail(h, err, "tridiagonalisation set-up");
        TriArgs T{A, P, R, d, e, tau, bar, h->d_status, timeout_ns(h), n};
        int rpb_arg = rpb;
        err = timed_launch(h, "trunc_tridiag", s, [&] {
            void* args[] = {&T, &rpb_arg};
            return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(tridiag_smem_kernel),
                                               dim3(unsigned(g_res)), dim3(kThreads), args, smem_res, s);
        });
        if (err != cudaSuccess) return cuda_fail(h, err, "tridiagonalisation");
    } else {
        const size_t smem = size_t(n) * 32;
        if (smem > 200 * 1024) return fail(h, DMRG_ERR_SHAPE, "rows too large for the tridiagonal solver");
        err = cudaFuncSetAttribute(tridiag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        int grid = 1;
        if (err == cudaSuccess)
            err = coop_grid(reinterpret_cast<const void*>(tridiag_kernel), smem, std::max(1, (n + kWarps - 1) / kWarps),
                            &grid, 1);
        if (err == cudaSuccess) err = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s);
        if (err != cudaSuccess) return cuda_fail(h, err, "tridiagonalisation set-up");
        TriArgs T{A, P, R, d, e, tau, bar, h->d_status, timeout_ns(h), n};
        err = timed_launch(h, "trunc_tridiag", s, [&] {
            void* args[] = {&T};
            return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(tridiag_kernel), dim3(unsigned(grid)),
                                               dim3(kThreads), args, smem, s);
        });
        if (err != cudaSuccess) return cuda_fail(h, err, "tridiagonalisation");
    }
    // 2. eigenvalues
    {
        // d and e^2 in shared memory, with their FP32 copies for the coarse phase when
        // those fit too
        const int staged = size_t(n) * 24 <= 96 * 1024 ? 2 : size_t(n) * 16 <= 96 * 1024 ? 1 : 0;
        const size_t smem = size_t(n) * (staged == 2 ? 24 : staged == 1 ? 16 : 0);
        err = timed_launch(h, "trunc_bisect", s, [&] {
            tri_stats_kernel<<<1, kThreads, 0, s>>>(d, e, n, stats);
            if (!staged) square_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(e, n, e2);
            // at least two warps per SM where n allows it (measured at n = 1600: 4 points
            // 11.2 ms, 8 points 8.4 ms, 16 points 9.1 ms)
            const int64_t want = int64_t(h->num_sms) * 2 * 32;
            const int sect = int64_t(n) * 4 >= want ? 4 : int64_t(n) * 8 >= want ? 8 : 16;
            const int64_t threads = int64_t(n) * sect;
            const unsigned blocks = unsigned((threads + kBisectThreads - 1) / kBisectThreads);
            auto kern = sect == 4 ? bisect_kernel<4> : sect == 8 ? bisect_kernel<8> : bisect_kernel<16>;
            cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 int(std::max<size_t>(smem, 1)));
            if (r != cudaSuccess) return r;
            kern<<<blocks, kBisectThreads, smem, s>>>(d, e, n, stats, e2, staged, lambda);
            return cudaGetLastError();
        });
        if (err != cudaSuccess) return cuda_fail(h, err, "bisection");
    }
    // 3. inverse iteration
    err = timed_launch(h, "trunc_invit", s, [&] {
        // four threads per block: the vectors spread over many SM sub-partitions
        invit_kernel<<<unsigned((mp + 3) / 4), 4, 0, s>>>(d, e, n, mp, lambda, stats, lu[0], lu[1], lu[2],
                                                             lu[3], sw, lu[4], Zt);
        return cudaGetLastError();
    });
    if (err != cudaSuccess) return cuda_fail(h, err, "inverse iteration");
    // 4. Gram-Schmidt: rows in shared memory, groups handed on by flags, when every
    //    block's rows fit (else the row-per-barrier form through L2)
    bool grouped_done = false;
    {
        const int ngroups = (mp + kMgsG - 1) / kMgsG;
        int dev = 0, sms = 0, coop = 0, per_sm = 0;
        err = cudaGetDevice(&dev);
        if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (err == cudaSuccess) err = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        if (err != cudaSuccess) return cuda_fail(h, err, "orthogonalisation set-up");
        // as many blocks as groups, up to two per SM (a block holds all its groups' rows);
        // the flag waits need every block resident: a cooperative launch
        const int grid = std::max(1, std::min(ngroups, 2 * sms));
        const int nown = (ngroups + grid - 1) / grid;
        const size_t smem = size_t(nown + 1) * kMgsG * n * 8;   // own rows + the staged ones
        // buffers free once the inverse iteration is done: published rows of the two
        // passes, their squared norms, the flags
        const bool fits = size_t(2 * mp + 2 * ngroups + 1) * 8 <= size_t(mp) * n * 8;
        if (coop && smem <= 200 * 1024 && fits) {
            err = cudaFuncSetAttribute(mgs_flow_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            if (err == cudaSuccess)
                err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mgs_flow_kernel, kMgsThreads, smem);
            if (err != cudaSuccess) return cuda_fail(h, err, "orthogonalisation set-up");
            if (per_sm * sms >= grid) {
                MgsFlowArgs M{};
                M.Zt = Zt;
                M.pub[0] = lu[0];
                M.pub[1] = lu[1];
                M.norms[0] = lu[2];
                M.norms[1] = lu[2] + mp;
                M.flags = reinterpret_cast<unsigned*>(lu[3]);
                M.status = h->d_status;
                M.timeout_ns = timeout_ns(h);
                M.n = n;
                M.mp = mp;
                err = cudaMemsetAsync(M.flags, 0, size_t(2 * ngroups + 1) * sizeof(unsigned), s);
                if (err != cudaSuccess) return cuda_fail(h, err, "orthogonalisation set-up");
                err = timed_launch(h, "trunc_orthogonalise", s, [&] {
                    void* args[] = {&M};
                    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(mgs_flow_kernel),
                                                       dim3(unsigned(grid)), dim3(kMgsThreads), args, smem, s);
                });
                if (err != cudaSuccess) return cuda_fail(h, err, "orthogonalisation");
                grouped_done = true;
            }
        }
    }
    if (!grouped_done) {
        int grid = 1;
        err = coop_grid(reinterpret_cast<const void*>(mgs_kernel), 0, std::max(1, mp), &grid, 1);
        if (err == cudaSuccess) err = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s);
        if (err != cudaSuccess) return cuda_fail(h, err, "orthogonalisation set-up");
        MgsArgs M{Zt, bar, h->d_status, timeout_ns(h), n, mp};
        err = timed_launch(h, "trunc_orthogonalise", s, [&] {
            void* args[] = {&M};
            return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(mgs_kernel), dim3(unsigned(grid)),
                                               dim3(kThreads), args, 0, s);
        });
        if (err != cudaSuccess) return cuda_fail(h, err, "orthogonalisation");
    }
    // 5. back-transformation and the sign convention
    {
        const size_t smem = size_t(4) * n * 8;
        if (smem > 200 * 1024) return fail(h, DMRG_ERR_SHAPE, "rows too large for the tridiagonal solver");
        err = cudaFuncSetAttribute(back_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (err == cudaSuccess)
            err = timed_launch(h, "trunc_back", s, [&] {
                back_kernel<<<unsigned(mp), kBackThreads, smem, s>>>(A, tau, Zt, n, mp, U);
                return cudaGetLastError();
            });
        if (err != cudaSuccess) return cuda_fail(h, err, "back-transformation");
    }
    (void)eps;
    return DMRG_OK;
}

}  // namespace dmrg
