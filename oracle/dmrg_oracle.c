/*
 * dmrg_oracle.c -- plain FP64 CPU oracle for the DMRG operator rotation.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or helper with the CUDA
 * library: every layout rule it needs is re-implemented here from its written
 * definition.
 *
 * What it computes (Rincon, Garcia, Hallberg, "Improved parallelization
 * techniques for the density matrix renormalization group"):
 *
 *   Sec. 2, algorithm step 5 and the paragraph after it: every block operator
 *   Z is first blocked onto [B a] (Z -> Z (x) I_d, the added site being
 *   complete) and then rotated and decimated, Z_new = R Z R^+, where
 *   R = (|w_1> ... |w_m'>)^T holds the kept density-matrix eigenvectors
 *   (step 4).  With real data U := R^+ = R^T, an (m*d) x m' matrix, so
 *   Z_new = U^T (Z (x) I_d) U.
 *
 *   Sec. 3.2 ("Novel strategy"): the rotation is done as two matrix-matrix
 *   products, first Z R^+ and then R (Z R^+).  The oracle follows that order:
 *   T = (O (x) I_d) U, then O' = U^T T.
 *
 *   Sec. 3.2, UMD paragraph: p workers each own floor(L/p) contiguous
 *   operators and the first mod(L, p) workers own one more.  The oracle uses
 *   exactly that split over OpenMP threads.
 *
 * Index conventions (the paper does not fix them; these are the readings the
 * whole project uses):
 *   [B a] basis index r = i*d + s (block state i slow, site state s fast), so
 *   the blocked operator is kron(O, I_d).  All matrices are row-major.
 *
 * Every routine is a literal loop over the definition in FP64; none is
 * blocked, fused or reordered beyond choosing which index runs innermost.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* UMD split (Sec. 3.2): worker w of p owns operators [lo, hi). */
static void umd_range(int64_t L, int p, int w, int64_t* lo, int64_t* hi) {
    int64_t base = L / p, extra = L % p;
    int64_t start = (int64_t)w * base + (w < extra ? w : extra);
    int64_t len = base + (w < extra ? 1 : 0);
    *lo = start;
    *hi = start + len;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* One operator: T = (O (x) I_d) U, then Oout = U^T T.  (Sec. 2 step 5;
 * Sec. 3.2 order of the two products.)  T is caller scratch of m*d*mp. */
static void rotate_one(const double* U, const double* O, double* Oout, double* T,
                       int64_t m, int d, int64_t mp) {
    const int64_t md = m * (int64_t)d;
    /* T[i*d+s][b] = sum_j O[i][j] * U[j*d+s][b] */
    for (int64_t i = 0; i < m; ++i) {
        for (int s = 0; s < d; ++s) {
            double* Trow = T + (i * d + s) * mp;
            for (int64_t b = 0; b < mp; ++b) Trow[b] = 0.0;
            for (int64_t j = 0; j < m; ++j) {
                const double o = O[i * m + j];
                const double* Urow = U + (j * d + s) * mp;
                for (int64_t b = 0; b < mp; ++b) Trow[b] += o * Urow[b];
            }
        }
    }
    /* Oout[a][b] = sum_r U[r][a] * T[r][b] */
    for (int64_t a = 0; a < mp * mp; ++a) Oout[a] = 0.0;
    for (int64_t r = 0; r < md; ++r) {
        const double* Urow = U + r * mp;
        const double* Trow = T + r * mp;
        for (int64_t a = 0; a < mp; ++a) {
            const double u = Urow[a];
            double* orow = Oout + a * mp;
            for (int64_t b = 0; b < mp; ++b) orow[b] += u * Trow[b];
        }
    }
}

/* Dense rotation of K operators, O: K x m x m, U: (m*d) x mp, Oout: K x mp x mp.
 * nthreads <= 0 uses every OpenMP thread.  Returns 0 on success. */
int oracle_rotate_dense(const double* U, const double* O, double* Oout,
                        int64_t m, int d, int64_t mp, int64_t K, int nthreads) {
    if (m <= 0 || d <= 0 || mp <= 0 || K < 0) return 1;
    int p = nthreads > 0 ? nthreads : oracle_num_threads();
    if (p > K && K > 0) p = (int)K;
    if (p < 1) p = 1;
    int fail = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(p) reduction(| : fail)
#endif
    {
        int w = 0;
#ifdef _OPENMP
        w = omp_get_thread_num();
#endif
        int64_t lo, hi;
        umd_range(K, p, w, &lo, &hi);
        double* T = (double*)malloc(sizeof(double) * (size_t)(m * d * mp));
        if (!T) {
            fail = 1;
        } else {
            for (int64_t k = lo; k < hi; ++k)
                rotate_one(U, O + k * m * m, Oout + k * mp * mp, T, m, d, mp);
            free(T);
        }
    }
    return fail;
}

/* Blocked site and cross operators, then rotated (Sec. 2, the blocking that follows
 * step 5 -- operators acting on the added site, and products of a block operator
 * with a site operator, are written in the [B a] basis before R Z R^+ -- and the
 * "blocking" task (ii) of Sec. 3.2):
 *
 *   Z_k = (A_k P^{f_k}) (x) S_{c(k)},   O'_k = U^T Z_k U,
 *
 * where P = diag(parity) is the block's fermion parity (-1)^{N_B}: with the
 * Jordan-Wigner order block modes before the site's, a fermion operator of the
 * added site carries the string P on the block, and f = 1 for operators that are
 * odd on the site.  The operators come in n_class consecutive classes: class c
 * has counts[c] operators, site matrix S + c*d*d (d x d, row-major) and parity
 * flag flags[c].  A: K x m x m, U: (m*d) x mp, parity: m entries (+1/-1; unused
 * when every flag is 0).  Literal loops in the paper's order: T = Z U, then
 * O' = U^T T.  Returns 0 on success. */
int oracle_rotate_site(const double* U, const double* A, const double* S, const int64_t* counts,
                       const int32_t* flags, int n_class, const double* parity, double* Oout,
                       int64_t m, int d, int64_t mp, int64_t K) {
    if (m <= 0 || d <= 0 || mp <= 0 || K < 0 || n_class < 0) return 1;
    const int64_t md = m * d;
    double* T = (double*)malloc(sizeof(double) * (size_t)(md * mp));
    if (!T) return 1;
    int64_t k = 0;
    for (int c = 0; c < n_class; ++c) {
        const double* Sc = S + (int64_t)c * d * d;
        for (int64_t q = 0; q < counts[c]; ++q, ++k) {
            if (k >= K) { free(T); return 1; }
            const double* Ak = A + k * m * m;
            /* T[(i,s)][b] = sum_{j,t} A[i][j] P[j]^f S[s][t] U[(j,t)][b] */
            for (int64_t i = 0; i < m; ++i)
                for (int s = 0; s < d; ++s) {
                    double* Trow = T + (i * d + s) * mp;
                    for (int64_t b = 0; b < mp; ++b) Trow[b] = 0.0;
                    for (int64_t j = 0; j < m; ++j) {
                        const double a = Ak[i * m + j] * (flags[c] ? parity[j] : 1.0);
                        if (a == 0.0) continue;
                        for (int t = 0; t < d; ++t) {
                            const double z = a * Sc[s * d + t];
                            if (z == 0.0) continue;
                            const double* Urow = U + (j * d + t) * mp;
                            for (int64_t b = 0; b < mp; ++b) Trow[b] += z * Urow[b];
                        }
                    }
                }
            /* O'[a][b] = sum_r U[r][a] T[r][b] */
            double* Ok = Oout + k * mp * mp;
            for (int64_t x = 0; x < mp * mp; ++x) Ok[x] = 0.0;
            for (int64_t r = 0; r < md; ++r) {
                const double* Trow = T + r * mp;
                for (int64_t a = 0; a < mp; ++a) {
                    const double u = U[r * mp + a];
                    if (u == 0.0) continue;
                    double* orow = Ok + a * mp;
                    for (int64_t b = 0; b < mp; ++b) orow[b] += u * Trow[b];
                }
            }
        }
    }
    free(T);
    return k == K ? 0 : 1;
}

/* Measurement stage (Sec. 3.2, one- and two-point functions <psi0|Z_i|psi0>,
 * <psi0|Z_i Z_j|psi0>; Sec. 2, the structure factors).  The superblock ground state
 * is psi0 = sum_{a,e} Psi[a][e] |a>|e>, system basis a (rows), environment basis e
 * (cols), Psi row-major.
 *
 * oracle_expectation: <Z_k> = <psi0| Z_k (x) I |psi0> (side 0, Z_k rows x rows) or
 * <psi0| I (x) Z_k |psi0> (side 1, cols x cols), written out over every index.
 * Returns 0 on success. */
int oracle_expectation(const double* Z, int64_t K, const double* Psi, int64_t rows, int64_t cols,
                       int side, double* out) {
    if (K < 0 || rows <= 0 || cols <= 0 || (side != 0 && side != 1)) return 1;
    const int64_t n = side == 0 ? rows : cols;
    for (int64_t k = 0; k < K; ++k) {
        const double* Zk = Z + k * n * n;
        double acc = 0.0;
        if (side == 0) {
            /* sum_{a,b,e} Psi[a][e] Z[a][b] Psi[b][e] */
            for (int64_t a = 0; a < rows; ++a)
                for (int64_t b = 0; b < rows; ++b) {
                    const double z = Zk[a * rows + b];
                    if (z == 0.0) continue;
                    double t = 0.0;
                    for (int64_t e = 0; e < cols; ++e) t += Psi[a * cols + e] * Psi[b * cols + e];
                    acc += z * t;
                }
        } else {
            /* sum_{a,e,f} Psi[a][e] Z[e][f] Psi[a][f] */
            for (int64_t e = 0; e < cols; ++e)
                for (int64_t f = 0; f < cols; ++f) {
                    const double z = Zk[e * cols + f];
                    if (z == 0.0) continue;
                    double t = 0.0;
                    for (int64_t a = 0; a < rows; ++a) t += Psi[a * cols + e] * Psi[a * cols + f];
                    acc += z * t;
                }
        }
        out[k] = acc;
    }
    return 0;
}

/* oracle_cross_correlations: C[i][j] = <psi0| Z_i (x) W_j |psi0>
 *   = sum_{a,b,e,f} Psi[a][e] Z_i[a][b] W_j[e][f] Psi[b][f],
 * Z: Ks x rows x rows (system), W: Ke x cols x cols (environment).  The inner sum
 * over (b, f) is formed once per (i, a, e) as (Z_i Psi W_j^T)[a][e]. */
int oracle_cross_correlations(const double* Z, int64_t Ks, const double* W, int64_t Ke,
                              const double* Psi, int64_t rows, int64_t cols, double* C) {
    if (Ks < 0 || Ke < 0 || rows <= 0 || cols <= 0) return 1;
    double* Y = (double*)malloc(sizeof(double) * (size_t)(rows * cols));
    if (!Y) return 1;
    for (int64_t i = 0; i < Ks; ++i) {
        const double* Zi = Z + i * rows * rows;
        /* Y = Z_i Psi */
        for (int64_t a = 0; a < rows; ++a)
            for (int64_t f = 0; f < cols; ++f) {
                double t = 0.0;
                for (int64_t b = 0; b < rows; ++b) t += Zi[a * rows + b] * Psi[b * cols + f];
                Y[a * cols + f] = t;
            }
        for (int64_t j = 0; j < Ke; ++j) {
            const double* Wj = W + j * cols * cols;
            double acc = 0.0;
            for (int64_t a = 0; a < rows; ++a)
                for (int64_t e = 0; e < cols; ++e) {
                    double t = 0.0;
                    for (int64_t f = 0; f < cols; ++f) t += Wj[e * cols + f] * Y[a * cols + f];
                    acc += Psi[a * cols + e] * t;
                }
            C[i * Ke + j] = acc;
        }
    }
    free(Y);
    return 0;
}

/* oracle_structure_factor (Sec. 2, N(q) and S^z(q)):
 *   F(q_p) = (1/L) sum_{k,j} e^{i q_p (k - j)} <(X_k - c)(X_j - c)>,   q_p = 2 pi p / L,
 * with G[k][j] = <X_k X_j> and v[k] = <X_k> (v may be NULL when c = 0), so that
 * <(X_k - c)(X_j - c)> = G[k][j] - c v[k] - c v[j] + c^2.  Writes the real part
 * Fre[p] and the imaginary part Fim[p] for p = 0 .. L-1. */
int oracle_structure_factor(const double* G, const double* v, double c, int64_t L, double* Fre,
                            double* Fim) {
    if (L <= 0) return 1;
    const double pi = 3.14159265358979323846;
    for (int64_t p = 0; p < L; ++p) {
        const double q = 2.0 * pi * (double)p / (double)L;
        double re = 0.0, im = 0.0;
        for (int64_t k = 0; k < L; ++k)
            for (int64_t j = 0; j < L; ++j) {
                double x = G[k * L + j];
                if (v) x += -c * v[k] - c * v[j] + c * c;
                else x += c * c;
                re += cos(q * (double)(k - j)) * x;
                im += sin(q * (double)(k - j)) * x;
            }
        Fre[p] = re / (double)L;
        Fim[p] = im / (double)L;
    }
    return 0;
}

/* ||U^T U - I||_F in FP64 (U needs orthonormal columns: B is only
 * approximately complete, Sec. 2; the kept |w_alpha> are orthonormal). */
double oracle_orthonormality_error(const double* U, int64_t rows, int64_t mp) {
    double acc = 0.0;
    for (int64_t a = 0; a < mp; ++a) {
        for (int64_t b = 0; b < mp; ++b) {
            double g = 0.0;
            for (int64_t r = 0; r < rows; ++r) g += U[r * mp + a] * U[r * mp + b];
            double e = g - (a == b ? 1.0 : 0.0);
            acc += e * e;
        }
    }
    return sqrt(acc);
}

/* Two-point correlations C[i][j] = <psi| O'_i O'_j |psi> (Sec. 3.2, the
 * one- and two-point functions), for real data written as
 * (O'_i^T psi) . (O'_j psi).  Op: K x mp x mp, psi: mp, C: K x K. */
int oracle_correlations(const double* Op, const double* psi, double* C, int64_t K, int64_t mp) {
    double* x = (double*)malloc(sizeof(double) * (size_t)(K * mp)); /* O'^T psi */
    double* y = (double*)malloc(sizeof(double) * (size_t)(K * mp)); /* O' psi   */
    if (!x || !y) { free(x); free(y); return 1; }
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t k = 0; k < K; ++k) {
        const double* A = Op + k * mp * mp;
        for (int64_t g = 0; g < mp; ++g) {
            double sx = 0.0, sy = 0.0;
            for (int64_t a = 0; a < mp; ++a) {
                sx += A[a * mp + g] * psi[a];
                sy += A[g * mp + a] * psi[a];
            }
            x[k * mp + g] = sx;
            y[k * mp + g] = sy;
        }
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < K; ++i)
        for (int64_t j = 0; j < K; ++j) {
            double s = 0.0;
            for (int64_t g = 0; g < mp; ++g) s += x[i * mp + g] * y[j * mp + g];
            C[i * K + j] = s;
        }
    free(x);
    free(y);
    return 0;
}

/* Adjoint of the rotation for L = sum_k <G_k, O'_k> (chain rule applied to
 * O'_k = U^T (O_k (x) I_d) U of Sec. 2 step 5; the paper has no gradient):
 *   dO_k[i][j] = sum_s (U G_k U^T)[i*d+s][j*d+s]           (partial trace over the site)
 *   dU        = sum_k (O_k (x) I) U G_k^T + (O_k (x) I)^T U G_k
 * dU may be NULL.  Loops run straight from these formulas. */
int oracle_rotate_backward(const double* U, const double* O, const double* G,
                           double* dO, double* dU, int64_t m, int d, int64_t mp, int64_t K) {
    const int64_t md = m * (int64_t)d;
    /* dO */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t k = 0; k < K; ++k) {
        const double* Gk = G + k * mp * mp;
        double* W = (double*)malloc(sizeof(double) * (size_t)(md * mp)); /* U G_k */
        if (!W) continue;
        for (int64_t r = 0; r < md; ++r)
            for (int64_t b = 0; b < mp; ++b) {
                double s = 0.0;
                for (int64_t a = 0; a < mp; ++a) s += U[r * mp + a] * Gk[a * mp + b];
                W[r * mp + b] = s;
            }
        for (int64_t i = 0; i < m; ++i)
            for (int64_t j = 0; j < m; ++j) {
                double acc = 0.0;
                for (int s = 0; s < d; ++s)
                    for (int64_t b = 0; b < mp; ++b)
                        acc += W[(i * d + s) * mp + b] * U[(j * d + s) * mp + b];
                dO[k * m * m + i * m + j] = acc;
            }
        free(W);
    }
    if (!dU) return 0;
    /* dU[r][g] = sum_k sum_{r'} A_k[r][r'] (U G_k^T)[r'][g] + A_k[r'][r] (U G_k)[r'][g],
     * with A_k = O_k (x) I_d, i.e. A_k[i*d+s][j*d+t] = O_k[i][j] delta_{st}. */
    for (int64_t x = 0; x < md * mp; ++x) dU[x] = 0.0;
    double* UGt = (double*)malloc(sizeof(double) * (size_t)(md * mp));
    double* UG = (double*)malloc(sizeof(double) * (size_t)(md * mp));
    if (!UGt || !UG) { free(UGt); free(UG); return 1; }
    for (int64_t k = 0; k < K; ++k) {
        const double* Gk = G + k * mp * mp;
        const double* Ok = O + k * m * m;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int64_t r = 0; r < md; ++r)
            for (int64_t g = 0; g < mp; ++g) {
                double s1 = 0.0, s2 = 0.0;
                for (int64_t a = 0; a < mp; ++a) {
                    s1 += U[r * mp + a] * Gk[g * mp + a];
                    s2 += U[r * mp + a] * Gk[a * mp + g];
                }
                UGt[r * mp + g] = s1;
                UG[r * mp + g] = s2;
            }
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int64_t i = 0; i < m; ++i)
            for (int s = 0; s < d; ++s)
                for (int64_t g = 0; g < mp; ++g) {
                    double acc = 0.0;
                    for (int64_t j = 0; j < m; ++j)
                        acc += Ok[i * m + j] * UGt[(j * d + s) * mp + g] +
                               Ok[j * m + i] * UG[(j * d + s) * mp + g];
                    dU[(i * d + s) * mp + g] += acc;
                }
    }
    free(UGt);
    free(UG);
    return 0;
}

/* ------------------------------------------------------------------------
 * Block-sparse U(1)xU(1) rotation (operators labelled by quantum numbers,
 * Sec. 3.1, Eq. (hache) and the remark that the sub-blocks have dissimilar
 * dimensions).  Layout, restated from the library's public description and
 * re-implemented here on its own:
 *   block sectors q = 0..S-1 with labels (bu[q], bd[q]) and sizes bm[q];
 *   site states s = 0..d-1 with quantum-number shifts (su[s], sd[s]);
 *   kept sectors Q = 0..P-1 with labels (ku[Q], kd[Q]) and sizes km[Q];
 *   the [B a] sector of kept Q stacks, for s = 0..d-1 in order, the block
 *   sector with label Q - delta_s (if present), so U_Q has
 *   D_Q = sum_s bm[q(Q - delta_s)] rows and km[Q] columns, row-major;
 *   U blocks are stored kept-sector after kept-sector.
 *   Operator k shifts labels by (ou[k], od[k]); it stores, for every block
 *   sector q (in order) whose label plus the shift is also a block sector q2,
 *   the bm[q2] x bm[q] block O_k[q2, q]; operators are stored one after the
 *   other.  Output operator k stores, for every kept sector Q whose label plus
 *   the shift is a kept sector Q2, the km[Q2] x km[Q] block O'_k[Q2, Q].
 * The rotation is the dense definition restricted to sectors:
 *   O'_k[Q2,Q] = sum_s U_Q2[seg s]^T  O_k[Q2 - d_s, Q - d_s]  U_Q[seg s].
 * ------------------------------------------------------------------------ */
static int find_sector(const int32_t* lu, const int32_t* ld, int n, int32_t u, int32_t dn) {
    for (int q = 0; q < n; ++q)
        if (lu[q] == u && ld[q] == dn) return q;
    return -1;
}

int oracle_rotate_blocked(int S, const int32_t* bu, const int32_t* bd, const int64_t* bm,
                          int d, const int32_t* su, const int32_t* sd,
                          int P, const int32_t* ku, const int32_t* kd, const int64_t* km,
                          int64_t K, const int32_t* ou, const int32_t* od,
                          const double* Ublk, const double* Oblk, double* Outblk) {
    /* U block offsets and, per kept sector and site state, the source block
     * sector and its row offset inside U_Q. */
    int64_t* uoff = (int64_t*)calloc((size_t)P + 1, sizeof(int64_t));
    int64_t* Drows = (int64_t*)calloc((size_t)P, sizeof(int64_t));
    int* segq = (int*)malloc(sizeof(int) * (size_t)(P * d));
    int64_t* segoff = (int64_t*)malloc(sizeof(int64_t) * (size_t)(P * d));
    if (!uoff || !Drows || !segq || !segoff) return 1;
    for (int Q = 0; Q < P; ++Q) {
        int64_t rows = 0;
        for (int s = 0; s < d; ++s) {
            int q = find_sector(bu, bd, S, ku[Q] - su[s], kd[Q] - sd[s]);
            segq[Q * d + s] = q;
            segoff[Q * d + s] = rows;
            if (q >= 0) rows += bm[q];
        }
        Drows[Q] = rows;
        uoff[Q + 1] = uoff[Q] + rows * km[Q];
    }
    int64_t in_off = 0, out_off = 0;
    for (int64_t k = 0; k < K; ++k) {
        /* offsets of this operator's input blocks, indexed by source sector q */
        int64_t* ioff = (int64_t*)malloc(sizeof(int64_t) * (size_t)S);
        for (int q = 0; q < S; ++q) {
            int q2 = find_sector(bu, bd, S, bu[q] + ou[k], bd[q] + od[k]);
            ioff[q] = -1;
            if (q2 >= 0) {
                ioff[q] = in_off;
                in_off += bm[q2] * bm[q];
            }
        }
        for (int Q = 0; Q < P; ++Q) {
            int Q2 = find_sector(ku, kd, P, ku[Q] + ou[k], kd[Q] + od[k]);
            if (Q2 < 0) continue;
            double* Ob = Outblk + out_off;
            const int64_t n2 = km[Q2], n1 = km[Q];
            for (int64_t x = 0; x < n2 * n1; ++x) Ob[x] = 0.0;
            for (int s = 0; s < d; ++s) {
                int qs = segq[Q * d + s];    /* block sector Q - d_s  */
                int q2s = segq[Q2 * d + s];  /* block sector Q2 - d_s */
                if (qs < 0 || q2s < 0 || ioff[qs] < 0) continue;
                const double* Ob_in = Oblk + ioff[qs]; /* bm[q2s] x bm[qs] */
                const double* U1 = Ublk + uoff[Q] + segoff[Q * d + s] * n1;
                const double* U2 = Ublk + uoff[Q2] + segoff[Q2 * d + s] * n2;
                const int64_t r2 = bm[q2s], r1 = bm[qs];
                /* first product (Sec. 3.2 order): T = O[Q2-d_s, Q-d_s] U_Q[seg s] */
                double* T = (double*)malloc(sizeof(double) * (size_t)(r2 * n1 + 1));
                if (!T) return 1;
                for (int64_t x = 0; x < r2; ++x)
                    for (int64_t b = 0; b < n1; ++b) {
                        double acc = 0.0;
                        for (int64_t y = 0; y < r1; ++y) acc += Ob_in[x * r1 + y] * U1[y * n1 + b];
                        T[x * n1 + b] = acc;
                    }
                /* second product: Ob += U_Q2[seg s]^T T */
                for (int64_t x = 0; x < r2; ++x)
                    for (int64_t a = 0; a < n2; ++a) {
                        const double ua = U2[x * n2 + a];
                        for (int64_t b = 0; b < n1; ++b) Ob[a * n1 + b] += ua * T[x * n1 + b];
                    }
                free(T);
            }
            out_off += n2 * n1;
        }
        free(ioff);
    }
    free(uoff);
    free(Drows);
    free(segq);
    free(segoff);
    return 0;
}
