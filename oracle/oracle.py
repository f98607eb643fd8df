"""ctypes front-end of the C oracle plus two independent NumPy routes.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Nothing in the CUDA
library imports this module.

* ``rotate_dense``      -- C loops: T = (O (x) I_d) U, then O' = U^T T
                           (Sec. 2 step 5; Sec. 3.2 order of the two products).
* ``rotate_dense_kron`` -- second route: materialise kron(O, I_d) (the blocking
                           step of Sec. 2) and multiply, for small sizes.
* ``rotate_blocked``    -- C per-sector loops (Sec. 3.1 Eq. (hache) labels).
* ``rotate_blocked_assembled`` -- second route: assemble the dense U and O
                           from their blocks, rotate densely, cut the blocks.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dmrg_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_f64p = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


def library_path() -> str:
    return _LIB_PATH


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP).  Portable C only."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.oracle_rotate_dense.argtypes = [_f64p, _f64p, _f64p, ctypes.c_int64, ctypes.c_int,
                                            ctypes.c_int64, ctypes.c_int64, ctypes.c_int]
        lib.oracle_rotate_dense.restype = ctypes.c_int
        lib.oracle_orthonormality_error.argtypes = [_f64p, ctypes.c_int64, ctypes.c_int64]
        lib.oracle_orthonormality_error.restype = ctypes.c_double
        lib.oracle_correlations.argtypes = [_f64p, _f64p, _f64p, ctypes.c_int64, ctypes.c_int64]
        lib.oracle_correlations.restype = ctypes.c_int
        lib.oracle_rotate_backward.argtypes = [_f64p, _f64p, _f64p, _f64p, _f64p, ctypes.c_int64,
                                               ctypes.c_int, ctypes.c_int64, ctypes.c_int64]
        lib.oracle_rotate_backward.restype = ctypes.c_int
        lib.oracle_rotate_blocked.argtypes = [
            ctypes.c_int, _i32p, _i32p, _i64p, ctypes.c_int, _i32p, _i32p,
            ctypes.c_int, _i32p, _i32p, _i64p, ctypes.c_int64, _i32p, _i32p,
            _f64p, _f64p, _f64p]
        lib.oracle_rotate_blocked.restype = ctypes.c_int
        lib.oracle_rotate_site.argtypes = [_f64p, _f64p, _f64p, _i64p, _i32p, ctypes.c_int, _f64p,
                                           _f64p, ctypes.c_int64, ctypes.c_int, ctypes.c_int64,
                                           ctypes.c_int64]
        lib.oracle_rotate_site.restype = ctypes.c_int
        lib.oracle_expectation.argtypes = [_f64p, ctypes.c_int64, _f64p, ctypes.c_int64, ctypes.c_int64,
                                           ctypes.c_int, _f64p]
        lib.oracle_expectation.restype = ctypes.c_int
        lib.oracle_cross_correlations.argtypes = [_f64p, ctypes.c_int64, _f64p, ctypes.c_int64, _f64p,
                                                  ctypes.c_int64, ctypes.c_int64, _f64p]
        lib.oracle_cross_correlations.restype = ctypes.c_int
        lib.oracle_structure_factor.argtypes = [_f64p, _f64p, ctypes.c_double, ctypes.c_int64, _f64p,
                                                _f64p]
        lib.oracle_structure_factor.restype = ctypes.c_int
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a, ptype):
    return a.ctypes.data_as(ptype)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def rotate_dense(U, O, d: int, nthreads: int = 0) -> np.ndarray:
    """O'_k = U^T (O_k (x) I_d) U for every k (Sec. 2 step 5), FP64.

    U: (m*d) x m'; O: K x m x m (or m x m).  Returns K x m' x m'."""
    U = _c(U, np.float64)
    O = _c(O, np.float64)
    squeeze = O.ndim == 2
    if squeeze:
        O = O[None]
    K, m, m2 = O.shape
    assert m == m2 and U.shape[0] == m * d, "shape mismatch"
    mp = U.shape[1]
    out = np.empty((K, mp, mp), dtype=np.float64)
    if K:
        rc = _load().oracle_rotate_dense(_p(U, _f64p), _p(O, _f64p), _p(out, _f64p),
                                         m, d, mp, K, int(nthreads))
        if rc:
            raise RuntimeError("oracle_rotate_dense failed")
    return out[0] if squeeze else out


def rotate_dense_kron(U, O, d: int) -> np.ndarray:
    """Second route: build kron(O_k, I_d) explicitly (the blocking step) and
    form U^T Z U with library matmuls.  Small sizes only."""
    U = np.asarray(U, dtype=np.float64)
    O = np.asarray(O, dtype=np.float64)
    squeeze = O.ndim == 2
    if squeeze:
        O = O[None]
    eye = np.eye(d)
    out = np.stack([U.T @ (np.kron(Ok, eye) @ U) for Ok in O]) if len(O) else \
        np.zeros((0, U.shape[1], U.shape[1]))
    return out[0] if squeeze else out


def rotate_site(U, A, d: int, S, counts, flags, parity=None) -> np.ndarray:
    """Blocked site and cross operators, rotated (Sec. 2, blocking after step 5):
    O'_k = U^T ((A_k P^{f_c}) (x) S_c) U for the operators of class c.

    A: K x m x m; S: n_class x d x d; counts: operators per class (in order, summing
    to K); flags: 1 where the class carries the block parity P = diag(parity)."""
    U = _c(U, np.float64)
    A = _c(A, np.float64)
    S = _c(np.asarray(S, dtype=np.float64).reshape(-1, d, d), np.float64)
    counts = _c(np.asarray(counts, dtype=np.int64).reshape(-1), np.int64)
    flags = _c(np.asarray(flags, dtype=np.int32).reshape(-1), np.int32)
    K, m, m2 = A.shape
    assert m == m2 and U.shape[0] == m * d and len(counts) == len(flags) == len(S)
    par = _c(np.ones(m) if parity is None else np.asarray(parity, dtype=np.float64), np.float64)
    mp = U.shape[1]
    out = np.empty((K, mp, mp), dtype=np.float64)
    rc = _load().oracle_rotate_site(_p(U, _f64p), _p(A, _f64p), _p(S, _f64p), _p(counts, _i64p),
                                    _p(flags, _i32p), len(counts), _p(par, _f64p), _p(out, _f64p),
                                    m, d, mp, K)
    if rc:
        raise RuntimeError("oracle_rotate_site failed")
    return out


def rotate_site_kron(U, A, d: int, S, counts, flags, parity=None) -> np.ndarray:
    """Second route: build kron(A_k P^f, S_c) explicitly and form U^T Z U with
    library matmuls.  Small sizes only."""
    U = np.asarray(U, dtype=np.float64)
    A = np.asarray(A, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64).reshape(-1, d, d)
    m = A.shape[1]
    P = np.diag(np.ones(m) if parity is None else np.asarray(parity, dtype=np.float64))
    out, k = [], 0
    for c, n in enumerate(counts):
        for _ in range(int(n)):
            Ak = A[k] @ P if flags[c] else A[k]
            out.append(U.T @ np.kron(Ak, S[c]) @ U)
            k += 1
    return np.stack(out) if out else np.zeros((0, U.shape[1], U.shape[1]))


def expectation(Z, Psi, side: int = 0) -> np.ndarray:
    """<psi0| Z_k (x) I |psi0> (side 0) or <psi0| I (x) Z_k |psi0> (side 1) for the
    superblock state psi0 = sum Psi[a][e] |a>|e> (Sec. 3.2)."""
    Z = _c(Z, np.float64)
    Psi = _c(Psi, np.float64)
    if Z.ndim == 2:
        Z = Z[None]
    rows, cols = Psi.shape
    out = np.empty(len(Z))
    if _load().oracle_expectation(_p(Z, _f64p), len(Z), _p(Psi, _f64p), rows, cols, int(side),
                                  _p(out, _f64p)):
        raise RuntimeError("oracle_expectation failed")
    return out


def cross_correlations(Z, W, Psi) -> np.ndarray:
    """C[i][j] = <psi0| Z_i (x) W_j |psi0>, Z on the system, W on the environment."""
    Z = _c(Z, np.float64)
    W = _c(W, np.float64)
    Psi = _c(Psi, np.float64)
    rows, cols = Psi.shape
    C = np.empty((len(Z), len(W)))
    if _load().oracle_cross_correlations(_p(Z, _f64p), len(Z), _p(W, _f64p), len(W), _p(Psi, _f64p),
                                         rows, cols, _p(C, _f64p)):
        raise RuntimeError("oracle_cross_correlations failed")
    return C


def structure_factor(G, v=None, c: float = 0.0):
    """F(q_p) = (1/L) sum_{k,j} e^{i q_p (k-j)} <(X_k - c)(X_j - c)>, q_p = 2 pi p / L
    (Sec. 2, N(q) and S^z(q)); returns (real part, imaginary part)."""
    G = _c(G, np.float64)
    L = G.shape[0]
    vv = None if v is None else _c(v, np.float64)
    re, im = np.empty(L), np.empty(L)
    if _load().oracle_structure_factor(_p(G, _f64p), None if vv is None else _p(vv, _f64p), float(c), L,
                                       _p(re, _f64p), _p(im, _f64p)):
        raise RuntimeError("oracle_structure_factor failed")
    return re, im


def truncation(Psi, mp: int):
    """Truncation matrix (Sec. 2, steps 3-4, Eq. rho and Eq. error): the reduced
    density matrix rho[i][i'] = sum_j Psi[i][j] Psi[i'][j] of the system, its
    eigenvalues w_alpha in decreasing order, U = the mp eigenvectors |w_alpha> with
    the largest eigenvalues (columns; each with its largest-magnitude component
    positive, the first such index on ties) and the discarded weight
    eps_rho = sum_{alpha > mp} w_alpha (= 1 - sum of the kept ones for a normalized
    psi).  The eigen-decomposition is the library routine numpy.linalg.eigh.
    Returns (U, w, eps)."""
    Psi = np.asarray(Psi, dtype=np.float64)
    n, nc = Psi.shape
    rho = np.zeros((n, n))
    for i in range(n):                      # rho by its definition, row by row
        rho[i] = Psi @ Psi[i]
    w, V = np.linalg.eigh(rho)
    order = np.argsort(-w, kind="stable")
    w, V = w[order], V[:, order]
    for a in range(V.shape[1]):
        j = int(np.argmax(np.abs(V[:, a])))
        if V[j, a] < 0:
            V[:, a] = -V[:, a]
    return np.ascontiguousarray(V[:, :mp]), w, float(w[mp:].sum())


def orthonormality_error(U) -> float:
    """||U^T U - I||_F in FP64."""
    U = _c(U, np.float64)
    return float(_load().oracle_orthonormality_error(_p(U, _f64p), U.shape[0], U.shape[1]))


def correlations(Op, psi) -> np.ndarray:
    """C[i, j] = <psi| O'_i O'_j |psi> for real data (Sec. 3.2)."""
    Op = _c(Op, np.float64)
    psi = _c(psi, np.float64)
    K, mp, _ = Op.shape
    C = np.empty((K, K), dtype=np.float64)
    if _load().oracle_correlations(_p(Op, _f64p), _p(psi, _f64p), _p(C, _f64p), K, mp):
        raise RuntimeError("oracle_correlations failed")
    return C


def rotate_backward(U, O, G, d: int, want_dU: bool = True):
    """Adjoint of the rotation for L = sum_k <G_k, O'_k>.  Returns (dO, dU)."""
    U = _c(U, np.float64)
    O = _c(O, np.float64)
    G = _c(G, np.float64)
    K, m, _ = O.shape
    mp = U.shape[1]
    dO = np.empty_like(O)
    dU = np.empty_like(U) if want_dU else None
    rc = _load().oracle_rotate_backward(_p(U, _f64p), _p(O, _f64p), _p(G, _f64p), _p(dO, _f64p),
                                        _p(dU, _f64p) if want_dU else None, m, d, mp, K)
    if rc:
        raise RuntimeError("oracle_rotate_backward failed")
    return dO, dU


# ----------------------------------------------------------------------------
# Block-sparse U(1) x U(1) rotation.
# ----------------------------------------------------------------------------

def rotate_blocked(block_sectors, site_shifts, kept_sectors, op_shifts, U_blocks, O_blocks,
                   out_size: int) -> np.ndarray:
    """Per-sector C loops.  ``block_sectors`` / ``kept_sectors``: sequences of
    (N_up, N_dn, dim); ``site_shifts``: d pairs; ``op_shifts``: K pairs;
    ``U_blocks`` / ``O_blocks``: flat FP64 arrays in the library's canonical
    block order.  Returns the flat output of ``out_size`` doubles."""
    bs = np.asarray(block_sectors, dtype=np.int64).reshape(-1, 3)
    ks = np.asarray(kept_sectors, dtype=np.int64).reshape(-1, 3)
    ss = np.asarray(site_shifts, dtype=np.int64).reshape(-1, 2)
    os_ = np.asarray(op_shifts, dtype=np.int64).reshape(-1, 2)
    bu, bd, bm = (_c(bs[:, 0], np.int32), _c(bs[:, 1], np.int32), _c(bs[:, 2], np.int64))
    ku, kd, km = (_c(ks[:, 0], np.int32), _c(ks[:, 1], np.int32), _c(ks[:, 2], np.int64))
    su, sd = _c(ss[:, 0], np.int32), _c(ss[:, 1], np.int32)
    ou, od = _c(os_[:, 0], np.int32), _c(os_[:, 1], np.int32)
    Ub = _c(U_blocks, np.float64)
    Ob = _c(O_blocks, np.float64)
    out = np.zeros(max(int(out_size), 1), dtype=np.float64)
    rc = _load().oracle_rotate_blocked(
        len(bs), _p(bu, _i32p), _p(bd, _i32p), _p(bm, _i64p), len(ss), _p(su, _i32p), _p(sd, _i32p),
        len(ks), _p(ku, _i32p), _p(kd, _i32p), _p(km, _i64p), len(os_), _p(ou, _i32p), _p(od, _i32p),
        _p(Ub, _f64p), _p(Ob, _f64p), _p(out, _f64p))
    if rc:
        raise RuntimeError("oracle_rotate_blocked failed")
    return out[:int(out_size)]


def blocked_dense_assembly(block_sectors, site_shifts, kept_sectors, op_shifts, U_blocks, O_blocks):
    """Assemble dense U ((m*d) x m') and O_k (m x m) from the block storage.

    Dense block basis: block sectors in order, states in order inside each.
    Dense [B a] row of (block state i, site state s) is i*d + s.  Dense kept
    column: kept sectors in order.  Returns (U, O, index) where ``index``
    holds the block positions needed to cut blocks back out."""
    bs = [tuple(int(v) for v in x) for x in block_sectors]
    ks = [tuple(int(v) for v in x) for x in kept_sectors]
    ss = [tuple(int(v) for v in x) for x in site_shifts]
    shifts = [tuple(int(v) for v in x) for x in op_shifts]
    d = len(ss)
    boff, m = {}, 0
    for (u, dn, n) in bs:
        boff[(u, dn)] = (m, n)
        m += n
    koff, mp = {}, 0
    for (u, dn, n) in ks:
        koff[(u, dn)] = (mp, n)
        mp += n
    U = np.zeros((m * d, mp))
    pos = 0
    Ub = np.asarray(U_blocks, dtype=np.float64)
    for (u, dn, n) in ks:
        c0 = koff[(u, dn)][0]
        rows = []
        for s, (du, dd) in enumerate(ss):
            src = (u - du, dn - dd)
            if src in boff:
                o, nb = boff[src]
                rows += [(o + x) * d + s for x in range(nb)]
        blk = Ub[pos:pos + len(rows) * n].reshape(len(rows), n)
        pos += len(rows) * n
        for x, r in enumerate(rows):
            U[r, c0:c0 + n] = blk[x]
    assert pos == Ub.size, "U block storage size mismatch"
    Obf = np.asarray(O_blocks, dtype=np.float64)
    O = np.zeros((len(shifts), m, m))
    pos = 0
    for k, (du, dd) in enumerate(shifts):
        for (u, dn, n) in bs:
            dst = (u + du, dn + dd)
            if dst in boff:
                r0, nr = boff[dst]
                c0, _ = boff[(u, dn)]
                O[k, r0:r0 + nr, c0:c0 + n] = Obf[pos:pos + nr * n].reshape(nr, n)
                pos += nr * n
    assert pos == Obf.size, "O block storage size mismatch"
    return U, O, {"koff": koff, "kept": ks, "shifts": shifts, "d": d}


def rotate_blocked_assembled(block_sectors, site_shifts, kept_sectors, op_shifts, U_blocks,
                             O_blocks):
    """Second route: dense assembly, dense oracle rotation, blocks cut out.
    Returns (flat_output, dense_rotated) so callers can also check that every
    entry outside the allowed sector pairs is exactly zero."""
    U, O, idx = blocked_dense_assembly(block_sectors, site_shifts, kept_sectors, op_shifts,
                                       U_blocks, O_blocks)
    Op = rotate_dense(U, O, idx["d"]) if len(O) else np.zeros((0, U.shape[1], U.shape[1]))
    out = []
    koff = idx["koff"]
    for k, (du, dd) in enumerate(idx["shifts"]):
        for (u, dn, n) in idx["kept"]:
            dst = (u + du, dn + dd)
            if dst in koff:
                r0, nr = koff[dst]
                c0, _ = koff[(u, dn)]
                out.append(Op[k, r0:r0 + nr, c0:c0 + n].ravel())
    flat = np.concatenate(out) if out else np.zeros(0)
    return flat, Op
