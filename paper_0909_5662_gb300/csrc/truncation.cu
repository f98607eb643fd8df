// truncation.cu -- the truncation matrix (Sec. 2, steps 3-4): the reduced density
// matrix rho = Psi Psi^T of the system (Eq. rho), its eigen-decomposition, the m'
// eigenvectors with the largest eigenvalues as the columns of U = R^+, and the
// discarded weight eps_rho (Eq. error).
//
// By default the eigen-decomposition is the tridiagonal solver of tridiag.cu; with
// DMRG_OPT_TRUNCATION_JACOBI it is the cyclic Jacobi method in FP64 below.  A sweep visits every
// pair of indices once, in N - 1 rounds of N / 2 disjoint pairs (the round-robin
// "circle" schedule, N = n rounded up to even; the padding index pairs with nobody).
// In a round every pair's rotation J (the stable 2 x 2 symmetric Schur step: the angle
// that zeroes a_ab) is computed from the current matrix, and the whole round is applied
// at once, A <- J^T A J and V <- V J.  A pair whose a_ab is below the rounding level of
// its diagonal, a_ab^2 <= eps^2 |a_aa a_bb|, is not rotated, nor (from the second sweep
// on) one at the rounding level of the whole matrix, |a_ab| <= eps ||A||_F / sqrt(n):
// the entries among eigenvectors of eigenvalues below rounding are noise of rho itself,
// and rotating them only spends sweeps (all skipped entries together perturb the
// eigenvalues by at most eps ||A||_F sqrt(n)).  The sweeps stop when
// the off-diagonal part is below tol * ||A||_F, or when a sweep rotated no pair.
// Eigenvalues are ranked on the device, and U's columns are V's columns in decreasing
// eigenvalue order, each with its largest-magnitude component positive (the first such
// index on ties).
//
// One sweep is one cooperative launch.  The rounds are separated by a grid-wide barrier
// (bounded wait), and A is double-buffered: a round reads A_in and writes A_out, so
// every block can compute the rotations it needs from A_in without waiting for anyone.
// Within a round, the pairs are cut into tiles of kPT pairs; an A work item is a tile
// pair (I <= K) and transforms its 2 x 2 blocks J_i^T A[{a_i,b_i},{a_k,b_k}] J_k, writing
// both triangles; a V work item is 64 rows of V times one tile of pairs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>

#include "api_common.h"
#include "grid_sync.cuh"
#include "ptx.cuh"

using namespace dmrg;

namespace {

constexpr int kThreads = 256;
constexpr int kPT = 16;          // pairs per tile side (kPT * kPT = kThreads)
constexpr int kVRows = 64;       // rows of V per work item
constexpr int kMaxBlocksPerSm = 3;
constexpr int64_t kTridiagMaxRows = 6144;   // the tridiagonal solver's shared-memory staging

// Slot i of round r on N (even) indices: index N - 1 stays, the others turn, and every
// pair of indices meets exactly once in rounds 0 .. N - 2.  For i >= 1 the first index
// (r + i) mod (N - 1) ascends with i and the second (r - i) mod (N - 1) descends, so a
// tile of consecutive slots reads two runs of neighbouring columns.
__device__ __forceinline__ void slot_indices(int N, int r, int i, int& a, int& b) {
    const int M = N - 1;
    if (i == 0) {
        a = M;
        b = r;
    } else {
        a = (r + i) % M;
        b = (r - i + M) % M;
    }
}

struct Rot {
    double c, s, t;   // J = [[c, s], [-s, c]], t = s / c
    int a, b;         // -1 for the padding index
};

__device__ Rot slot_rotation(const double* __restrict__ A, int n, int N, int npair, int r, int slot,
                             double abs2) {
    Rot R{1.0, 0.0, 0.0, -1, -1};
    if (slot >= npair) return R;
    int a, b;
    slot_indices(N, r, slot, a, b);
    R.a = a < n ? a : -1;
    R.b = b < n ? b : -1;
    if (R.a < 0 || R.b < 0) return R;
    const double g = __ldcg(A + size_t(a) * n + b);
    const double al = __ldcg(A + size_t(a) * n + a);
    const double be = __ldcg(A + size_t(b) * n + b);
    if (!(g * g > (DBL_EPSILON * DBL_EPSILON) * fabs(al * be)) || !(g * g > abs2)) return R;
    const double tau = (be - al) / (2.0 * g);
    double t;
    if (fabs(tau) > 1e150) {
        t = 0.5 / tau;
    } else {
        t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
    }
    R.c = 1.0 / sqrt(1.0 + t * t);
    R.s = t * R.c;
    R.t = t;
    return R;
}

// A rotation written by another block in this launch: read through L2.
__device__ __forceinline__ Rot ld_rot(const Rot* p) {
    Rot R;
    R.c = __ldcg(&p->c);
    R.s = __ldcg(&p->s);
    R.t = __ldcg(&p->t);
    R.a = __ldcg(&p->a);
    R.b = __ldcg(&p->b);
    return R;
}

// Barrier state of one sweep, zeroed before the launch; the sweep's results follow it.
struct SweepSync {
    GridBarrier bar;
    double off2, all2;              // sum of squares off the diagonal, and in total
    unsigned long long rotations;   // pairs rotated in the sweep
};

struct SweepArgs {
    double* A[2];       // the sweep reads A[cur] first; round r writes A[(cur + r + 1) & 1]
    double* V;
    double* partials;   // 3 per block: off2, all2 of its last-round entries, rotations
    Rot* rots;          // the round's rotations, npair of them
    SweepSync* sync;
    unsigned* status;
    uint64_t timeout_ns;
    double abs2;        // square of the absolute rotation threshold
    int n, N, npair, npt, n_atiles, n_vtiles, cur;
};

// Tile pair (I, K), I <= K, of linear index x over the upper triangle.
__device__ __forceinline__ void tri_index(int x, int& I, int& K) {
    int k = int((sqrtf(8.0f * float(x) + 1.0f) - 1.0f) * 0.5f);   // FP32 guess, fixed below
    while (k * (k + 1) / 2 > x) --k;
    while ((k + 1) * (k + 2) / 2 <= x) ++k;
    K = k;
    I = x - k * (k + 1) / 2;
}

__global__ void __launch_bounds__(kThreads) jacobi_sweep_kernel(SweepArgs P) {
    __shared__ Rot rot[2 * kPT];
    __shared__ double red[3][kThreads / 32];
    const int n = P.n;
    const int tid = threadIdx.x;
    unsigned gen_seen = 0;
    double off2 = 0.0, all2 = 0.0, nrot = 0.0;
    const int items = P.n_atiles + P.n_vtiles;
    for (int r = 0; r < P.N - 1; ++r) {
        const bool odd = ((P.cur + r) & 1) != 0;
        const double* __restrict__ Ain = odd ? P.A[1] : P.A[0];
        double* __restrict__ Aout = odd ? P.A[0] : P.A[1];
        const bool last = r == P.N - 2;
        // phase 1: every pair's rotation, once
        // (slot-major over blocks, so that every SM takes a few of the FP64 divide chains)
        for (int slot = tid * gridDim.x + blockIdx.x; slot < P.npair; slot += gridDim.x * kThreads) {
            const Rot R = slot_rotation(Ain, n, P.N, P.npair, r, slot, P.abs2);
            if (R.s != 0.0) nrot += 1.0;
            P.rots[slot] = R;
        }
        if (!grid_barrier(&P.sync->bar, gen_seen, P.timeout_ns, P.status)) return;
        // phase 2: A <- J^T A J and V <- V J
        for (int item = blockIdx.x; item < items; item += gridDim.x) {
            if (item < P.n_atiles) {
                int I, K;
                tri_index(item, I, K);
                if (tid < 2 * kPT) {
                    const int slot = (tid < kPT ? I : K) * kPT + (tid & (kPT - 1));
                    if (slot < P.npair) rot[tid] = ld_rot(P.rots + slot);
                }
                __syncthreads();
                const int i = tid / kPT, k = tid % kPT;
                const int si = I * kPT + i, sk = K * kPT + k;
                if (si < P.npair && sk < P.npair && !(I == K && i > k)) {
                    const Rot Ri = rot[i], Rk = rot[kPT + k];
                    auto ld = [=](int x, int y) {
                        return (x >= 0 && y >= 0) ? __ldcg(Ain + size_t(x) * n + y) : 0.0;
                    };
                    auto st = [=](int x, int y, double v) {
                        if (x >= 0 && y >= 0) __stcg(Aout + size_t(x) * n + y, v);
                    };
                    if (si == sk) {
                        double x00 = ld(Ri.a, Ri.a), x11 = ld(Ri.b, Ri.b), x01 = ld(Ri.a, Ri.b);
                        if (Ri.s != 0.0) {
                            x00 -= Ri.t * x01;
                            x11 += Ri.t * x01;
                            x01 = 0.0;
                        }
                        st(Ri.a, Ri.a, x00);
                        st(Ri.b, Ri.b, x11);
                        st(Ri.a, Ri.b, x01);
                        st(Ri.b, Ri.a, x01);
                        if (last) {
                            const double o = (Ri.a >= 0 && Ri.b >= 0) ? 2.0 * x01 * x01 : 0.0;
                            off2 += o;
                            all2 += o + (Ri.a >= 0 ? x00 * x00 : 0.0) + (Ri.b >= 0 ? x11 * x11 : 0.0);
                        }
                    } else {
                        const double x00 = ld(Ri.a, Rk.a), x01 = ld(Ri.a, Rk.b);
                        const double x10 = ld(Ri.b, Rk.a), x11 = ld(Ri.b, Rk.b);
                        // right factor J_k on the two rows, then left factor J_i^T
                        const double y00 = Rk.c * x00 - Rk.s * x01, y01 = Rk.s * x00 + Rk.c * x01;
                        const double y10 = Rk.c * x10 - Rk.s * x11, y11 = Rk.s * x10 + Rk.c * x11;
                        const double z00 = Ri.c * y00 - Ri.s * y10, z01 = Ri.c * y01 - Ri.s * y11;
                        const double z10 = Ri.s * y00 + Ri.c * y10, z11 = Ri.s * y01 + Ri.c * y11;
                        st(Ri.a, Rk.a, z00);
                        st(Ri.a, Rk.b, z01);
                        st(Ri.b, Rk.a, z10);
                        st(Ri.b, Rk.b, z11);
                        st(Rk.a, Ri.a, z00);
                        st(Rk.b, Ri.a, z01);
                        st(Rk.a, Ri.b, z10);
                        st(Rk.b, Ri.b, z11);
                        if (last) {
                            // padding entries were loaded as 0 and stay 0
                            const double o = 2.0 * (z00 * z00 + z01 * z01 + z10 * z10 + z11 * z11);
                            off2 += o;
                            all2 += o;
                        }
                    }
                }
                __syncthreads();
            } else {
                const int v = item - P.n_atiles;
                const int R = v / P.npt, K = v % P.npt;
                if (tid < kPT && K * kPT + tid < P.npair) rot[tid] = ld_rot(P.rots + K * kPT + tid);
                __syncthreads();
                const int sk = K * kPT + tid % kPT;
                const Rot Rk = rot[tid % kPT];
                if (sk < P.npair && Rk.s != 0.0) {
                    for (int j = 0; j < kVRows / (kThreads / kPT); ++j) {
                        const int row = R * kVRows + tid / kPT + j * (kThreads / kPT);
                        if (row >= n) break;
                        double* va = P.V + size_t(row) * n + Rk.a;
                        double* vb = P.V + size_t(row) * n + Rk.b;
                        const double x = __ldcg(va), y = __ldcg(vb);
                        __stcg(va, Rk.c * x - Rk.s * y);
                        __stcg(vb, Rk.s * x + Rk.c * y);
                    }
                }
                __syncthreads();
            }
        }
        if (last) {
            // per-block partial sums of the final matrix, combined in block order below
            for (int o = 16; o > 0; o >>= 1) {
                off2 += __shfl_xor_sync(0xffffffffu, off2, o);
                all2 += __shfl_xor_sync(0xffffffffu, all2, o);
                nrot += __shfl_xor_sync(0xffffffffu, nrot, o);
            }
            if ((tid & 31) == 0) {
                red[0][tid >> 5] = off2;
                red[1][tid >> 5] = all2;
                red[2][tid >> 5] = nrot;
            }
            __syncthreads();
            if (tid < 3) {
                double acc = 0.0;
                for (int w = 0; w < kThreads / 32; ++w) acc += red[tid][w];
                P.partials[3 * blockIdx.x + tid] = acc;
            }
        }
        if (!grid_barrier(&P.sync->bar, gen_seen, P.timeout_ns, P.status)) return;
    }
    if (blockIdx.x == 0 && tid == 0) {
        double o = 0.0, a = 0.0, q = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) {
            o += __ldcg(P.partials + 3 * b);
            a += __ldcg(P.partials + 3 * b + 1);
            q += __ldcg(P.partials + 3 * b + 2);
        }
        P.sync->off2 = o;
        P.sync->all2 = a;
        P.sync->rotations = static_cast<unsigned long long>(q);
    }
}

__global__ void identity_kernel(double* V, int64_t n) {
    const int64_t x = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (x < n * n) V[x] = (x / n == x % n) ? 1.0 : 0.0;
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

constexpr int kMaxSweepBlocks = 4096;

struct TruncDims {
    int N, npair, npt, n_atiles, n_vtiles;
    WsLayout ws;
};

TruncDims trunc_dims(int64_t rows) {
    TruncDims D;
    D.N = int(rows + (rows & 1));
    D.npair = D.N / 2;
    D.npt = (D.npair + kPT - 1) / kPT;
    D.n_atiles = D.npt * (D.npt + 1) / 2;
    D.n_vtiles = int((rows + kVRows - 1) / kVRows) * D.npt;
    D.ws.add("A0", size_t(rows) * rows * 8);
    D.ws.add("A1", size_t(rows) * rows * 8);
    D.ws.add("V", size_t(rows) * rows * 8);
    D.ws.add("sync", sizeof(SweepSync));
    D.ws.add("partials", size_t(kMaxSweepBlocks) * 3 * 8);
    D.ws.add("col", size_t(rows) * 8);
    D.ws.add("rots", size_t(D.npair) * sizeof(Rot));
    return D;
}

unsigned blocks_for(int64_t n) { return unsigned((n + kThreads - 1) / kThreads); }

// Blocks of one sweep launch: every block must be resident at once (cooperative launch).
cudaError_t sweep_grid(int items, int* grid) {
    int dev = 0, sms = 0, per_sm = 0, coop = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_sweep_kernel, kThreads, 0);
    if (e != cudaSuccess) return e;
    if (!coop || per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    *grid = std::min({items, sms * std::min(per_sm, kMaxBlocksPerSm), kMaxSweepBlocks});
    return cudaSuccess;
}

}  // namespace

extern "C" {

dmrg_status dmrg_truncation_workspace(dmrg_handle h, int64_t rows, int64_t cols, size_t* bytes) {
    if (!h || !bytes) return DMRG_ERR_INVALID_ARG;
    if (rows < 1 || cols < 1) return fail(h, DMRG_ERR_SHAPE, "need rows, cols >= 1");
    // either solver (the option may change after the query); mp <= rows
    *bytes = std::max(trunc_dims(rows).ws.total, tridiag_layout(rows, rows).total);
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
    if (!h->trunc_jacobi && rows <= kTridiagMaxRows) {
        char* base = static_cast<char*>(ws);
        double* rho = reinterpret_cast<double*>(base + tridiag_layout(rows, mp).offsets[0]);
        cudaError_t e = timed_launch(h, "trunc_rho", s, [&] { return rho_launch(Psi, rows, cols, 0, rho, s); });
        if (e != cudaSuccess) return cuda_fail(h, e, "reduced density matrix");
        st = tridiag_eigen(h, rows, mp, base, U, lambda, eps, s);
        if (st != DMRG_OK) return st;
        discarded_kernel<<<1, kThreads, 0, s>>>(lambda, rows, mp, eps);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "discarded weight");
        if (sweeps) *sweeps = 0;
        return DMRG_OK;
    }
    const TruncDims D = trunc_dims(rows);
    char* base = static_cast<char*>(ws);
    double* A0 = reinterpret_cast<double*>(base + D.ws.offsets[0]);
    double* A1 = reinterpret_cast<double*>(base + D.ws.offsets[1]);
    double* V = reinterpret_cast<double*>(base + D.ws.offsets[2]);
    SweepSync* sync = reinterpret_cast<SweepSync*>(base + D.ws.offsets[3]);
    double* partials = reinterpret_cast<double*>(base + D.ws.offsets[4]);
    int64_t* col = reinterpret_cast<int64_t*>(base + D.ws.offsets[5]);
    Rot* rots = reinterpret_cast<Rot*>(base + D.ws.offsets[6]);
    const int64_t n = rows;
    cudaError_t e = timed_launch(h, "trunc_rho", s, [&] { return rho_launch(Psi, rows, cols, 0, A0, s); });
    if (e != cudaSuccess) return cuda_fail(h, e, "reduced density matrix");
    identity_kernel<<<blocks_for(n * n), kThreads, 0, s>>>(V, n);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "identity");
    int grid = 0;
    if (n > 1 && (e = sweep_grid(D.n_atiles + D.n_vtiles, &grid)) != cudaSuccess)
        return cuda_fail(h, e, "cooperative launch size");
    SweepArgs P{};
    P.A[0] = A0;
    P.A[1] = A1;
    P.V = V;
    P.partials = partials;
    P.rots = rots;
    P.sync = sync;
    P.status = h->d_status;
    P.timeout_ns = timeout_ns(h);
    P.n = int(n);
    P.N = D.N;
    P.npair = D.npair;
    P.npt = D.npt;
    P.n_atiles = D.n_atiles;
    P.n_vtiles = D.n_vtiles;
    P.cur = 0;
    int done = -max_sweeps;
    SweepSync host{};
    for (int sweep = 0; sweep < max_sweeps && n > 1; ++sweep) {
        e = cudaMemsetAsync(sync, 0, sizeof(SweepSync), s);
        if (e == cudaSuccess)
            e = timed_launch(h, "trunc_sweep", s, [&] {
                void* args[] = {&P};
                return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(jacobi_sweep_kernel),
                                                   dim3(unsigned(grid)), dim3(kThreads), args, 0, s);
            });
        if (e != cudaSuccess) return cuda_fail(h, e, "Jacobi sweep");
        P.cur = (P.cur + D.N - 1) & 1;
        e = cudaMemcpyAsync(&host, sync, sizeof host, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(h, e, "convergence test");
        if (host.bar.abort) return fail(h, DMRG_ERR_TIMEOUT, "a Jacobi sweep's grid barrier timed out");
        if (host.off2 <= tol * tol * host.all2 || host.rotations == 0) {
            done = sweep + 1;
            break;
        }
        // From the second sweep on, entries at or below DBL_EPSILON ||A||_F / sqrt(n) are
        // rounding noise of rho itself and are not rotated.
        P.abs2 = DBL_EPSILON * DBL_EPSILON * host.all2 / double(n);
    }
    const double* A = P.A[P.cur];
    if (n == 1) done = 0;
    rank_kernel<<<blocks_for(n), kThreads, 0, s>>>(A, n, lambda, col);
    gather_kernel<<<unsigned(mp), kThreads, 0, s>>>(V, n, col, mp, U);
    discarded_kernel<<<1, kThreads, 0, s>>>(lambda, n, mp, eps);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "eigenvectors");
    if (sweeps) *sweeps = done;
    return DMRG_OK;
}

}  // extern "C"
