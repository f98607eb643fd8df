"""Pins of the FP64 CPU oracle against facts that do not come from it.

Each test checks the oracle against a closed form, an invariant of the
rotation O' = U^T (O (x) I_d) U (Sec. 2 step 5), brute-force Jordan-Wigner
matrix elements of the Hubbard chain (Eq. HUBB), or exact finite differences,
so that a dropped term, a wrong index convention or a transposed operand in
the oracle fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

import hubbard_jw as jw
from workloads import orthonormal_columns, gaussian_sector_split, blocked_config


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


# ----------------------------------------------------------------------------
# The Jordan-Wigner fixture itself.
# ----------------------------------------------------------------------------

def test_jw_anticommutators():
    c = jw.annihilators(3)
    I = np.eye(64)
    for p, q in itertools.product(range(6), repeat=2):
        acomm = c[p] @ c[q].T + c[q].T @ c[p]
        assert np.array_equal(acomm, I if p == q else 0 * I)
        assert np.array_equal(c[p] @ c[q] + c[q] @ c[p], 0 * I)


def test_jw_two_site_hubbard_closed_form():
    # Two-site Hubbard, one up and one down electron: E0 = (U - sqrt(U^2 + 16 t^2)) / 2.
    t, U = 1.0, 8.0
    H = jw.hubbard_hamiltonian(2, t, U)
    sec = jw.sector_basis(2)
    idx = np.where((sec[:, 0] == 1) & (sec[:, 1] == 1))[0]
    e0 = np.linalg.eigvalsh(H[np.ix_(idx, idx)])[0]
    assert abs(e0 - (U - math.sqrt(U * U + 16 * t * t)) / 2) < 1e-12


def test_jw_free_fermion_spectrum():
    # U = 0 on an open chain of L sites: one-particle energies -2t cos(k pi / (L + 1)).
    L, t = 4, 1.0
    H = jw.hubbard_hamiltonian(L, t, 0.0)
    sec = jw.sector_basis(L)
    eps = np.sort(-2 * t * np.cos(np.arange(1, L + 1) * np.pi / (L + 1)))
    for nu, nd in [(1, 0), (2, 1), (2, 2), (3, 1)]:
        idx = np.where((sec[:, 0] == nu) & (sec[:, 1] == nd))[0]
        e0 = np.linalg.eigvalsh(H[np.ix_(idx, idx)])[0]
        assert abs(e0 - (eps[:nu].sum() + eps[:nd].sum())) < 1e-12


# ----------------------------------------------------------------------------
# Dense rotation.
# ----------------------------------------------------------------------------

def test_isometry_maps_identity_to_identity(oracle_lib):
    # U^T (I_m (x) I_d) U = U^T U = I_m' for any U with orthonormal columns.
    rng = np.random.default_rng(1)
    for (m, d, mp) in [(8, 4, 5), (16, 2, 16), (10, 3, 30)]:
        U = orthonormal_columns(rng, m * d, mp)
        out = oracle_lib.rotate_dense(U, np.eye(m)[None], d)
        assert np.abs(out[0] - np.eye(mp)).max() < 1e-13


def test_no_truncation_trace_and_spectrum(oracle_lib):
    # m' = m d and U orthogonal: O' is similar to O (x) I_d, so Tr O' = d Tr O and
    # the spectrum of O' is that of O with every eigenvalue repeated d times.
    rng = np.random.default_rng(2)
    m, d = 12, 4
    U = orthonormal_columns(rng, m * d, m * d)
    A = rng.standard_normal((m, m))
    O = np.stack([A + A.T, rng.standard_normal((m, m))])
    out = oracle_lib.rotate_dense(U, O, d)
    for k in range(2):
        assert abs(np.trace(out[k]) - d * np.trace(O[k])) < 1e-11
    ev = np.sort(np.linalg.eigvalsh(out[0]))
    ev_ref = np.sort(np.repeat(np.linalg.eigvalsh(O[0]), d))
    assert np.abs(ev - ev_ref).max() < 1e-11


def test_no_truncation_preserves_products(oracle_lib):
    rng = np.random.default_rng(3)
    m, d = 9, 3
    U = orthonormal_columns(rng, m * d, m * d)
    A, B = rng.standard_normal((2, m, m))
    rA, rB, rAB = oracle_lib.rotate_dense(U, np.stack([A, B, A @ B]), d)
    assert np.abs(rA @ rB - rAB).max() < 1e-12


def test_fermion_anticommutators_preserved(oracle_lib):
    # Block of 3 Hubbard sites (m = 64, d = 4), no truncation: the rotated
    # annihilators still satisfy {c'_p, c'_q^+} = delta_pq I and {c'_p, c'_q} = 0.
    rng = np.random.default_rng(4)
    c = jw.annihilators(3)
    U = orthonormal_columns(rng, 256, 256)
    cr = oracle_lib.rotate_dense(U, np.stack(c), 4)
    crd = oracle_lib.rotate_dense(U, np.stack([x.T for x in c]), 4)
    I = np.eye(256)
    for p, q in itertools.product(range(6), repeat=2):
        assert np.abs(cr[p] @ crd[q] + crd[q] @ cr[p] - (I if p == q else 0)).max() < 1e-12
        assert np.abs(cr[p] @ cr[q] + cr[q] @ cr[p]).max() < 1e-12


@pytest.mark.parametrize("mp", [64, 256])
def test_hubbard_bruteforce_matrix_elements(oracle_lib, mp):
    # 4-site Hubbard chain (t = 1, U/t = 8, open).  B = sites 1-3 (m = 64),
    # a = site 4 (d = 4); U = the lowest m' eigenvectors of the 4-site H.  The
    # rotated block operator must equal <u_a| O_full |u_b>, where O_full is
    # built independently on all 8 modes -- exact even with truncation.
    cb = jw.annihilators(3)
    cf = jw.annihilators(4)
    H = jw.hubbard_hamiltonian(4, 1.0, 8.0, cf)
    _, V = np.linalg.eigh(H)
    U = np.ascontiguousarray(V[:, :mp])
    blk, full = [], []
    for i in range(3):
        blk.append(cb[2 * i].T @ cb[2 * i] + cb[2 * i + 1].T @ cb[2 * i + 1])      # n_i
        full.append(cf[2 * i].T @ cf[2 * i] + cf[2 * i + 1].T @ cf[2 * i + 1])
    for (i, j, s) in [(0, 1, 0), (2, 0, 1), (1, 2, 1)]:
        blk.append(cb[2 * i + s].T @ cb[2 * j + s])                               # c+_is c_js
        full.append(cf[2 * i + s].T @ cf[2 * j + s])
    for p in [0, 3, 5]:
        blk.append(cb[p])                                                          # c_p (odd)
        full.append(cf[p])
    out = oracle_lib.rotate_dense(U, np.stack(blk), 4)
    for k in range(len(blk)):
        assert np.abs(out[k] - U.T @ full[k] @ U).max() < 1e-12


def test_special_cases(oracle_lib):
    rng = np.random.default_rng(5)
    O = rng.standard_normal((3, 7, 7))
    # d = 1, m' = m, U = I: O' = O.
    assert np.array_equal(oracle_lib.rotate_dense(np.eye(7), O, 1), O)
    # U a permutation: O'[a, b] = (O (x) I)[pi(a), pi(b)].
    m, d = 5, 2
    perm = rng.permutation(m * d)
    U = np.eye(m * d)[:, perm]
    O2 = rng.standard_normal((2, m, m))
    out = oracle_lib.rotate_dense(U, O2, d)
    for k in range(2):
        for a, b in itertools.product(range(m * d), repeat=2):
            ra, rb = perm[a], perm[b]
            want = O2[k, ra // d, rb // d] if ra % d == rb % d else 0.0
            assert out[k, a, b] == want


def test_thread_split_and_batch_invariance(oracle_lib):
    # The UMD split over workers (Sec. 3.2) changes nothing, bit for bit, and
    # rotating one operator alone equals rotating it inside a batch.
    rng = np.random.default_rng(6)
    m, d, mp, K = 10, 4, 13, 11
    U = orthonormal_columns(rng, m * d, mp)
    O = rng.standard_normal((K, m, m))
    a = oracle_lib.rotate_dense(U, O, d, nthreads=1)
    for p in (2, 3, 7, 11):
        assert np.array_equal(a, oracle_lib.rotate_dense(U, O, d, nthreads=p))
    assert np.array_equal(a[4], oracle_lib.rotate_dense(U, O[4], d))


def test_second_route_kron(oracle_lib):
    rng = np.random.default_rng(7)
    for (m, d, mp, K) in [(6, 4, 9, 3), (11, 3, 20, 2), (8, 1, 8, 2)]:
        U = orthonormal_columns(rng, m * d, mp)
        O = rng.standard_normal((K, m, m))
        assert rel(oracle_lib.rotate_dense(U, O, d), oracle_lib.rotate_dense_kron(U, O, d)) < 1e-14


def test_orthonormality_error_closed_form(oracle_lib):
    rng = np.random.default_rng(8)
    Q = orthonormal_columns(rng, 40, 12)
    assert oracle_lib.orthonormality_error(Q) < 1e-14
    for c in (1.001, 0.5, 2.0):
        # (cQ)^T (cQ) - I = (c^2 - 1) I  ->  |c^2 - 1| sqrt(m')
        assert abs(oracle_lib.orthonormality_error(c * Q) - abs(c * c - 1) * math.sqrt(12)) < 1e-12
    # one column scaled by c: a single diagonal entry c^2 - 1
    Q2 = Q.copy()
    Q2[:, 3] *= 1.5
    assert abs(oracle_lib.orthonormality_error(Q2) - 1.25) < 1e-13


def test_correlations_bruteforce(oracle_lib):
    # No truncation, psi = ground state u_0 expressed in the rotated basis
    # (unit vector e_0): <psi| n_i n_j |psi> must equal the full-space value.
    cb = jw.annihilators(3)
    cf = jw.annihilators(4)
    H = jw.hubbard_hamiltonian(4, 1.0, 8.0, cf)
    _, V = np.linalg.eigh(H)
    nb = [cb[2 * i].T @ cb[2 * i] + cb[2 * i + 1].T @ cb[2 * i + 1] for i in range(3)]
    nf = [cf[2 * i].T @ cf[2 * i] + cf[2 * i + 1].T @ cf[2 * i + 1] for i in range(3)]
    rot = oracle_lib.rotate_dense(V, np.stack(nb), 4)
    psi = np.zeros(256)
    psi[0] = 1.0
    C = oracle_lib.correlations(rot, psi)
    u0 = V[:, 0]
    for i, j in itertools.product(range(3), repeat=2):
        assert abs(C[i, j] - u0 @ nf[i] @ nf[j] @ u0) < 1e-12
    # Closed form: O' = I gives <psi|psi> = 1 for a unit psi.
    rng = np.random.default_rng(9)
    v = rng.standard_normal(17)
    v /= np.linalg.norm(v)
    assert abs(oracle_lib.correlations(np.eye(17)[None], v)[0, 0] - 1.0) < 1e-14


# ----------------------------------------------------------------------------
# Adjoint.
# ----------------------------------------------------------------------------

def _loss(oracle_lib, U, O, G, d):
    return float(np.sum(G * oracle_lib.rotate_dense(U, O, d)))


def test_backward_adjoint_identity(oracle_lib):
    # The rotation is linear in O, so <G, rot(O)> = <rot^*(G), O> exactly.
    rng = np.random.default_rng(10)
    m, d, mp, K = 16, 4, 16, 4
    U = orthonormal_columns(rng, m * d, mp)
    O = rng.standard_normal((K, m, m))
    G = rng.standard_normal((K, mp, mp))
    dO, _ = oracle_lib.rotate_backward(U, O, G, d, want_dU=False)
    assert abs(_loss(oracle_lib, U, O, G, d) - np.sum(dO * O)) < 1e-10


def test_backward_central_differences(oracle_lib):
    # L = sum_k <G_k, O'_k> is linear in O and quadratic in U, so the central
    # difference (L(x+hv) - L(x-hv)) / 2h has no truncation error: it matches the
    # analytic directional derivative up to rounding (step 1e-6, FP64).
    rng = np.random.default_rng(11)
    m, d, mp, K = 16, 4, 16, 4
    U = orthonormal_columns(rng, m * d, mp)
    O = rng.standard_normal((K, m, m))
    G = rng.standard_normal((K, mp, mp))
    dO, dU = oracle_lib.rotate_backward(U, O, G, d)
    h = 1e-6
    for _ in range(6):
        V = rng.standard_normal(U.shape)
        fd = (_loss(oracle_lib, U + h * V, O, G, d) - _loss(oracle_lib, U - h * V, O, G, d)) / (2 * h)
        an = np.sum(dU * V)
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an))
        W = rng.standard_normal(O.shape)
        fd = (_loss(oracle_lib, U, O + h * W, G, d) - _loss(oracle_lib, U, O - h * W, G, d)) / (2 * h)
        an = np.sum(dO * W)
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an))
    # element-wise on a tiny case
    m, d, mp, K = 3, 2, 4, 2
    U = rng.standard_normal((m * d, mp))     # unconstrained U (no Stiefel projection)
    O = rng.standard_normal((K, m, m))
    G = rng.standard_normal((K, mp, mp))
    dO, dU = oracle_lib.rotate_backward(U, O, G, d)
    for idx in np.ndindex(*U.shape):
        E = np.zeros_like(U)
        E[idx] = h
        fd = (_loss(oracle_lib, U + E, O, G, d) - _loss(oracle_lib, U - E, O, G, d)) / (2 * h)
        assert abs(fd - dU[idx]) < 1e-8
    for idx in np.ndindex(*O.shape):
        E = np.zeros_like(O)
        E[idx] = h
        fd = (_loss(oracle_lib, U, O + E, G, d) - _loss(oracle_lib, U, O - E, G, d)) / (2 * h)
        assert abs(fd - dO[idx]) < 1e-8


# ----------------------------------------------------------------------------
# Block-sparse U(1) x U(1) rotation.
# ----------------------------------------------------------------------------

def _binom_sectors(nsites):
    out = []
    for a in range(nsites + 1):
        for b in range(nsites + 1):
            out.append((a, b, math.comb(nsites, a) * math.comb(nsites, b)))
    return out


SITE = [(0, 0), (1, 0), (0, 1), (1, 1)]


def test_blocked_hubbard_bruteforce(oracle_lib):
    # Quantum-number-labelled operators (Sec. 3.1, Eq. (hache)) on the 4-site
    # Hubbard chain.  Block = sites 1-3 with sectors (N_up, N_dn); [B a] sector Q
    # stacks site states s = 0, up, down, up-down.  U_Q = lowest eigenvectors of
    # H restricted to Q.  Every rotated block must equal the full-space matrix
    # element <u^Q2_a| O_full |u^Q_b>.
    cb = jw.annihilators(3)
    cf = jw.annihilators(4)
    H = jw.hubbard_hamiltonian(4, 1.0, 8.0, cf)
    bsec = jw.sector_basis(3)
    block_sectors = _binom_sectors(3)
    states = {(u, dn): [i for i in range(64) if tuple(bsec[i]) == (u, dn)] for (u, dn, _) in block_sectors}
    # [B a] rows of kept sector Q, in storage order (s, then block state)
    def rows_of(Q):
        r = []
        for s, (du, dd) in enumerate(SITE):
            src = (Q[0] - du, Q[1] - dd)
            r += [i * 4 + s for i in states.get(src, [])]
        return r
    kept, Ublocks, Ufull = [], [], {}
    for u in range(5):
        for dn in range(5):
            r = rows_of((u, dn))
            if not r:
                continue
            keep = min(len(r), 3)          # truncate to at most 3 states per sector
            _, V = np.linalg.eigh(H[np.ix_(r, r)])
            kept.append((u, dn, keep))
            Ublocks.append(V[:, :keep].ravel())
            Ufull[(u, dn)] = (r, V[:, :keep])
    ops_b = [cb[0], cb[3].T, cb[4].T @ cb[4], cb[0].T @ cb[4], cb[2] @ cb[5]]
    ops_f = [cf[0], cf[3].T, cf[4].T @ cf[4], cf[0].T @ cf[4], cf[2] @ cf[5]]
    shifts = [(-1, 0), (0, 1), (0, 0), (0, 0), (-1, -1)]
    Oblocks = []
    bdim = {(u, dn): n for (u, dn, n) in block_sectors}
    for Ob, (du, dd) in zip(ops_b, shifts):
        for (u, dn, n) in block_sectors:
            dst = (u + du, dn + dd)
            if dst in bdim:
                Oblocks.append(Ob[np.ix_(states[dst], states[(u, dn)])].ravel())
    Ub = np.concatenate(Ublocks)
    Obl = np.concatenate(Oblocks)
    kdim = {(u, dn): n for (u, dn, n) in kept}
    expect = []
    for Of, (du, dd) in zip(ops_f, shifts):
        for (u, dn, n) in kept:
            dst = (u + du, dn + dd)
            if dst in kdim:
                r2, V2 = Ufull[dst]
                r1, V1 = Ufull[(u, dn)]
                expect.append((V2.T @ Of[np.ix_(r2, r1)] @ V1).ravel())
    expect = np.concatenate(expect)
    got = oracle_lib.rotate_blocked(block_sectors, SITE, kept, shifts, Ub, Obl, expect.size)
    assert np.abs(got - expect).max() < 1e-12
    got2, _ = oracle_lib.rotate_blocked_assembled(block_sectors, SITE, kept, shifts, Ub, Obl)
    assert np.abs(got2 - expect).max() < 1e-12


def test_blocked_selection_rule_and_routes(oracle_lib):
    # Random sector structure: the per-sector loops equal the dense route, and the
    # dense rotated operator is exactly zero outside the pairs (Q + delta_k, Q).
    rng = np.random.default_rng(12)
    sectors = [(a, b, int(rng.integers(1, 5))) for a in range(4) for b in range(3) if rng.random() < 0.8]
    kept = [(a, b, max(1, n - 1)) for (a, b, n) in sectors]
    shifts = [(0, 0), (1, 0), (0, -1), (-1, 1)]
    from workloads import blocked_layout_sizes
    ush, ish, osh = blocked_layout_sizes(sectors, SITE, kept, shifts)
    Ub = np.concatenate([orthonormal_columns(rng, r, c).ravel() for (r, c) in ush])
    Obl = rng.standard_normal(sum(r * c for s in ish for (r, c) in s))
    n_out = sum(r * c for s in osh for (r, c) in s)
    a = oracle_lib.rotate_blocked(sectors, SITE, kept, shifts, Ub, Obl, n_out)
    b, dense = oracle_lib.rotate_blocked_assembled(sectors, SITE, kept, shifts, Ub, Obl)
    assert rel(a, b) < 1e-14
    koff, off = {}, 0
    for (u, dn, n) in kept:
        koff[(u, dn)] = (off, n)
        off += n
    for k, (du, dd) in enumerate(shifts):
        mask = np.ones(dense[k].shape, dtype=bool)
        for (u, dn, n) in kept:
            if (u + du, dn + dd) in koff:
                r0, nr = koff[(u + du, dn + dd)]
                c0, _ = koff[(u, dn)]
                mask[r0:r0 + nr, c0:c0 + n] = False
        assert np.all(dense[k][mask] == 0.0)


def test_sector_split_histograms():
    # sigma = 4 literal law: 311 sectors of 1-10 states; sigma = 1.2: 45 sectors of 1-111.
    s4 = gaussian_sector_split(1000, 4.0)
    s12 = gaussian_sector_split(1000, 1.2)
    assert sum(n for *_, n in s4) == 1000 and sum(n for *_, n in s12) == 1000
    assert len(s4) == 311 and min(n for *_, n in s4) == 1 and max(n for *_, n in s4) == 10
    assert len(s12) == 45 and min(n for *_, n in s12) == 1 and max(n for *_, n in s12) == 111


# ---------------------------------------------------------------- blocked site operators
def _site_4chain(mp):
    """4-site Hubbard chain (t = 1, U/t = 8, open): block = sites 1-3, added site 4.
    Returns U (lowest mp eigenvectors), block annihilators, local annihilators, the
    block parity (-1)^{N_B} and the full-space annihilators."""
    cb = jw.annihilators(3)
    cl = jw.annihilators(1)                       # d = 4 local operators, local signs
    cf = jw.annihilators(4)
    H = jw.hubbard_hamiltonian(4, 1.0, 8.0, cf)
    _, V = np.linalg.eigh(H)
    nb = sum(cb[p].T @ cb[p] for p in range(6))
    parity = np.where(np.round(np.diag(nb)).astype(int) % 2 == 0, 1.0, -1.0)
    return np.ascontiguousarray(V[:, :mp]), cb, cl, parity, cf


@pytest.mark.parametrize("mp", [64, 256])
def test_site_operators_bruteforce(oracle_lib, mp):
    # Operators of the added site and block x site products, blocked with the
    # Jordan-Wigner string on the block (block modes first), must equal the
    # full-space matrix elements <u_a| O_full |u_b> -- built independently on all
    # 8 modes, exact even with truncation.
    U, cb, cl, parity, cf = _site_4chain(mp)
    I64 = np.eye(64)
    classes = []   # (S, flag, [(A, full operator)])
    for s in range(2):
        # c_4s = P_B (x) c_s;  c+_is c_4s = (c+_is P_B) (x) c_s
        classes.append((cl[s], 1, [(I64, cf[6 + s]),
                                   (cb[s].T, cf[s].T @ cf[6 + s]),
                                   (cb[4 + s].T, cf[4 + s].T @ cf[6 + s])]))
        # c+_4s = P_B (x) c_s^T;  c+_4s c_2s = (P_B c_2s) (x) c_s^T = (-c_2s P_B) (x) c_s^T
        classes.append((cl[s].T, 1, [(I64, cf[6 + s].T),
                                     (-cb[2 + s], cf[6 + s].T @ cf[2 + s])]))
    n_loc = cl[0].T @ cl[0] + cl[1].T @ cl[1]
    classes.append((n_loc, 0, [(I64, cf[6].T @ cf[6] + cf[7].T @ cf[7]),              # n_4
                               (cb[0].T @ cb[0], (cf[0].T @ cf[0]) @ (cf[6].T @ cf[6] + cf[7].T @ cf[7]))]))
    A = np.stack([a for _, _, ops in classes for a, _ in ops])
    S = np.stack([c[0] for c in classes])
    counts = [len(c[2]) for c in classes]
    flags = [c[1] for c in classes]
    out = oracle_lib.rotate_site(U, A, 4, S, counts, flags, parity)
    full = [f for _, _, ops in classes for _, f in ops]
    for k in range(len(full)):
        assert np.abs(out[k] - U.T @ full[k] @ U).max() < 1e-12, k


def test_site_operators_reduce_and_second_route(oracle_lib):
    rng = np.random.default_rng(31)
    m, d, mp, K = 7, 3, 12, 5
    U = orthonormal_columns(rng, m * d, mp)
    A = rng.standard_normal((K, m, m))
    # S = I without parity is the plain block rotation
    got = oracle_lib.rotate_site(U, A, d, np.eye(d)[None], [K], [0])
    assert np.abs(got - oracle_lib.rotate_dense(U, A, d)).max() < 1e-12
    # random classes against the explicit kron route
    S = rng.standard_normal((3, d, d))
    par = rng.choice([-1.0, 1.0], m)
    counts, flags = [2, 0, 3], [1, 0, 0]
    a = oracle_lib.rotate_site(U, A, d, S, counts, flags, par)
    b = oracle_lib.rotate_site_kron(U, A, d, S, counts, flags, par)
    assert np.abs(a - b).max() < 1e-12
    # parity flag: (A P) (x) S = (A (x) S)(P (x) I)
    a1 = oracle_lib.rotate_site(U, A[:1], d, S[:1], [1], [1], par)
    ref = U.T @ np.kron(A[0], S[0]) @ np.kron(np.diag(par), np.eye(d)) @ U
    assert np.abs(a1[0] - ref).max() < 1e-12



# ---------------------------------------------------------------- measurement stage
def _chain_split():
    """Ground state of the 4-site Hubbard chain (t = 1, U/t = 8) as a 16 x 16 matrix:
    system = sites 1-2 (rows), environment = sites 3-4 (cols); full-space operators."""
    cf = jw.annihilators(4)
    H = jw.hubbard_hamiltonian(4, 1.0, 8.0, cf)
    w, V = np.linalg.eigh(H)
    psi = V[:, 0]
    c2 = jw.annihilators(2)          # the local 2-site operators of either half
    return psi, psi.reshape(16, 16), cf, c2


def _n(c, i):
    return c[2 * i].T @ c[2 * i] + c[2 * i + 1].T @ c[2 * i + 1]


def _sz(c, i):
    return 0.5 * (c[2 * i].T @ c[2 * i] - c[2 * i + 1].T @ c[2 * i + 1])


def test_measurement_bruteforce_hubbard(oracle_lib):
    # <n_i>, <S^z_i> on both halves and the cross two-point functions <n_i n_j>,
    # <S^z_i S^z_j> (i in the system, j in the environment) against the full-space
    # expectation values in the exact ground state.  Number and spin operators are
    # even, so the environment's operators carry no string from the system.
    psi, Psi, cf, c2 = _chain_split()
    sys_ops = [_n(c2, 0), _n(c2, 1), _sz(c2, 0), _sz(c2, 1)]
    env_ops = sys_ops
    full_sys = [_n(cf, 0), _n(cf, 1), _sz(cf, 0), _sz(cf, 1)]
    full_env = [_n(cf, 2), _n(cf, 3), _sz(cf, 2), _sz(cf, 3)]
    e_sys = oracle_lib.expectation(np.stack(sys_ops), Psi, 0)
    e_env = oracle_lib.expectation(np.stack(env_ops), Psi, 1)
    for k in range(4):
        assert abs(e_sys[k] - psi @ full_sys[k] @ psi) < 1e-12
        assert abs(e_env[k] - psi @ full_env[k] @ psi) < 1e-12
    C = oracle_lib.cross_correlations(np.stack(sys_ops), np.stack(env_ops), Psi)
    for i in range(4):
        for j in range(4):
            assert abs(C[i, j] - psi @ full_sys[i] @ full_env[j] @ psi) < 1e-12
    # the nondegenerate ground state has a definite particle number (2 here) and the
    # open chain's reflection symmetry: <n_1> = <n_4>, <n_2> = <n_3>
    total = e_sys[0] + e_sys[1] + e_env[0] + e_env[1]
    assert abs(total - round(total)) < 1e-10 and round(total) == 2
    assert abs(e_sys[0] - e_env[1]) < 1e-10 and abs(e_sys[1] - e_env[0]) < 1e-10


def test_structure_factor_closed_forms(oracle_lib):
    L = 12
    rng = np.random.default_rng(41)
    X = rng.standard_normal((L, L))
    G = X + X.T
    v = rng.standard_normal(L)
    re, im = oracle_lib.structure_factor(G, v, 0.7)
    Gc = G - 0.7 * v[:, None] - 0.7 * v[None, :] + 0.49
    assert abs(re.sum() - np.trace(Gc)) < 1e-10               # sum rule over q
    assert abs(re[0] - Gc.sum() / L) < 1e-10                   # q = 0: total
    assert np.abs(im).max() < 1e-10                            # symmetric G: real
    re0, _ = oracle_lib.structure_factor(np.full((L, L), 0.25), np.full(L, 0.5), 0.5)
    assert np.abs(re0).max() < 1e-12                           # uncorrelated: zero
    re1, _ = oracle_lib.structure_factor(np.eye(L))
    assert np.abs(re1 - 1.0).max() < 1e-12                    # delta correlation: flat
    p0 = 3
    k = np.arange(L)
    Gcos = np.cos(2 * np.pi * p0 * (k[:, None] - k[None, :]) / L)
    re2, _ = oracle_lib.structure_factor(Gcos)
    expect = np.zeros(L)
    expect[p0] += L / 2
    expect[L - p0] += L / 2
    assert np.abs(re2 - expect).max() < 1e-10                  # a single wave vector


# ---------------------------------------------------------------- truncation matrix
def schmidt_state(rng, n, nc, weights):
    """Psi = sum_k sqrt(w_k) u_k v_k^T with orthonormal u (n) and v (nc): the reduced
    density matrix Psi Psi^T has exactly the eigenpairs (w_k, u_k)."""
    r = len(weights)
    u = orthonormal_columns(rng, n, r)
    v = orthonormal_columns(rng, nc, r)
    return (u * np.sqrt(weights)) @ v.T, u


def test_truncation_schmidt_spectrum(oracle_lib):
    rng = np.random.default_rng(71)
    n, nc, mp = 40, 30, 12
    w = np.sort(rng.uniform(0.1, 1.0, 20))[::-1] * np.exp(-0.3 * np.arange(20))
    w /= w.sum()                               # normalized psi: weights sum to 1
    Psi, u = schmidt_state(rng, n, nc, w)
    U, lam, eps = oracle_lib.truncation(Psi, mp)
    assert np.abs(lam[:20] - w).max() < 1e-14                     # the Schmidt weights
    assert np.abs(lam[20:]).max() < 1e-14                          # rank 20
    assert abs(eps - w[mp:].sum()) < 1e-14
    assert abs(eps - (1.0 - lam[:mp].sum())) < 1e-13               # Eq. error, normalized psi
    assert np.abs(np.abs(U.T @ u[:, :mp]) - np.eye(mp)).max() < 1e-12   # kept |w_alpha>
    assert np.abs(U.T @ U - np.eye(mp)).max() < 1e-13
    for a in range(mp):                                            # sign convention
        j = np.argmax(np.abs(U[:, a]))
        assert U[j, a] > 0


def test_truncation_product_state(oracle_lib):
    # A product state (rank-1 Psi) keeps everything with one state: eps = 0.
    rng = np.random.default_rng(72)
    a, b = rng.standard_normal(9), rng.standard_normal(5)
    Psi = np.outer(a, b) / (np.linalg.norm(a) * np.linalg.norm(b))
    U, lam, eps = oracle_lib.truncation(Psi, 1)
    assert abs(lam[0] - 1.0) < 1e-14 and abs(eps) < 1e-14
    assert np.abs(np.abs(U[:, 0]) - np.abs(a) / np.linalg.norm(a)).max() < 1e-14
