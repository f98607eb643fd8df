"""GPU parity of the truncation matrix (Sec. 2, steps 3-4: rho = Psi Psi^T, its kept
eigenvectors and the discarded weight) against the FP64 oracle, and its use as the
rotation U of the next step.
"""
import numpy as np
import pytest
import torch

import oracle
from workloads import orthonormal_columns

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_0909_5662_gb300 as lib
    return lib


def schmidt(rng, n, nc, w):
    u = orthonormal_columns(rng, n, len(w))
    v = orthonormal_columns(rng, nc, len(w))
    return (u * np.sqrt(w)) @ v.T


@pytest.fixture(scope="module", params=["tridiagonal", "jacobi"])
def method(request, P):
    """The default solver (tridiagonalisation, bisection, inverse iteration) and the
    cyclic Jacobi sweeps, each on its own handle."""
    h = P.Handle()
    P.dmrg_set_option("truncation_jacobi", 1 if request.param == "jacobi" else 0, handle=h)
    yield request.param, h
    h.close()


def run(P, Psi, mp, method=None):
    name, h = method if method else ("tridiagonal", None)
    U, lam, eps, sweeps = P.dmrg_truncation(torch.from_numpy(Psi).cuda(), mp, handle=h)
    torch.cuda.synchronize()
    P.dmrg_sync_status(handle=h)
    assert (sweeps >= 0) if name == "jacobi" else (sweeps == 0)   # Jacobi: 0 sweeps for one row
    return U.cpu().numpy(), lam.cpu().numpy(), float(eps.item()), sweeps


@pytest.mark.parametrize("n,nc,rank,mp", [(40, 30, 20, 12), (37, 64, 37, 10), (64, 16, 16, 16), (2, 3, 2, 1)])
def test_truncation_matches_oracle_schmidt(P, method, n, nc, rank, mp):
    # distinct Schmidt weights: every kept eigenvector is unique up to sign
    rng = np.random.default_rng(n * 100 + nc)
    w = np.exp(-0.25 * np.arange(rank)) * (1.0 + 0.05 * rng.random(rank))
    w = np.sort(w)[::-1] / w.sum()
    Psi = schmidt(rng, n, nc, w)
    U_ref, lam_ref, eps_ref = oracle.truncation(Psi, mp)
    U, lam, eps, sweeps = run(P, Psi, mp, method)
    assert np.abs(lam - lam_ref).max() < 1e-13
    assert abs(eps - eps_ref) < 1e-13
    assert np.abs(U - U_ref).max() < 1e-10
    assert np.abs(U.T @ U - np.eye(mp)).max() < 1e-12


@pytest.mark.parametrize("n,nc,mp", [(64, 50, 20), (129, 200, 40), (400, 400, 100)])
def test_truncation_random_state(P, method, n, nc, mp):
    rng = np.random.default_rng(n + nc)
    Psi = rng.standard_normal((n, nc))
    Psi /= np.linalg.norm(Psi)
    U_ref, lam_ref, eps_ref = oracle.truncation(Psi, mp)
    U, lam, eps, sweeps = run(P, Psi, mp, method)
    assert np.abs(lam - lam_ref).max() < 1e-13 * max(1.0, lam_ref[0])
    assert abs(eps - eps_ref) < 1e-12
    # the kept subspace (projector), unique when lambda[mp-1] > lambda[mp]
    assert np.abs(U @ U.T - U_ref @ U_ref.T).max() < 1e-9
    assert abs(lam.sum() - 1.0) < 1e-12                     # Tr rho = |psi|^2 = 1


def test_truncation_feeds_the_rotation(P):
    # The U of one step is the rotation of the next: orthonormal to FP64 rounding and
    # consumed by dmrg_rotate_ops (compare with the oracle's U and rotation).
    rng = np.random.default_rng(5)
    m, d, mp = 24, 4, 30
    Psi = rng.standard_normal((m * d, 50))
    Psi /= np.linalg.norm(Psi)
    U, _, _, _ = run(P, Psi, mp)
    U_ref, _, _ = oracle.truncation(Psi, mp)
    assert oracle.orthonormality_error(U) < 1e-12   # rounding of ~10 sweeps of rotations
    O = rng.standard_normal((6, m, m))
    got = P.dmrg_rotate_ops(torch.from_numpy(U).cuda(), torch.from_numpy(O).cuda(), d, "fp64").cpu().numpy()
    ref = oracle.rotate_dense(U_ref, O, d)
    assert np.abs(got - ref).max() < 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("pairs,mp", [(30, 30), (30, 31)])
def test_truncation_degenerate_pairs(P, method, pairs, mp):
    # Exactly repeated Schmidt weights: each kept pair spans an eigenspace whose basis is
    # not unique; the kept subspace (when the cut does not split a pair), the spectrum,
    # orthonormality and the residual rho U - U Lambda are what is fixed.
    rng = np.random.default_rng(pairs + mp)
    w = np.repeat(np.exp(-0.3 * np.arange(pairs)), 2)
    w /= w.sum()
    Psi = schmidt(rng, 80, 70, w)
    U_ref, lam_ref, eps_ref = oracle.truncation(Psi, mp)
    U, lam, eps, _ = run(P, Psi, mp, method)
    rho = Psi @ Psi.T
    assert np.abs(lam - lam_ref).max() < 1e-13
    assert abs(eps - eps_ref) < 1e-13
    assert np.abs(U.T @ U - np.eye(mp)).max() < 1e-12
    assert np.abs(rho @ U - U * lam[:mp]).max() < 1e-13
    if mp % 2 == 0:
        assert np.abs(U @ U.T - U_ref @ U_ref.T).max() < 1e-10


@pytest.mark.parametrize("n,mp", [(1600, 400), (1900, 100)])
def test_truncation_large_against_oracle(P, n, mp):
    # The tridiagonal solver at the benchmark's n = 1600 (every block's rows of rho held
    # in shared memory) and at n = 1900 (too many rows for that: the L2 form).  Distinct,
    # exponentially decaying Schmidt weights over 12 decades: each kept eigenvector is
    # unique up to its sign, which the convention fixes.
    rng = np.random.default_rng(n)
    w = np.exp(-np.arange(n) * (12.0 * np.log(10.0) / n))
    w /= w.sum()
    Psi = schmidt(rng, n, n, w)
    U_ref, lam_ref, eps_ref = oracle.truncation(Psi, mp)
    U, lam, eps, _ = run(P, Psi, mp)
    assert np.abs(lam - lam_ref).max() < 1e-13 * lam_ref[0]
    assert abs(eps - eps_ref) < 1e-12
    assert np.abs(U - U_ref).max() < 1e-9
    assert np.abs(U.T @ U - np.eye(mp)).max() < 1e-12


def test_truncation_tiny_sizes(P, method):
    # one and two rows (no reflector), mp = rows
    for rows in (1, 2, 3):
        Psi = np.arange(1.0, 1.0 + rows * 4).reshape(rows, 4)
        Psi /= np.linalg.norm(Psi)
        U_ref, lam_ref, eps_ref = oracle.truncation(Psi, rows)
        U, lam, eps, _ = run(P, Psi, rows, method)
        assert np.abs(lam - lam_ref).max() < 1e-14
        assert np.abs(U - U_ref).max() < 1e-12


def _ulp_distance(a, b):
    """Distance in units in the last place between same-signed finite doubles."""
    ia = a.view(np.int64)
    ib = b.view(np.int64)
    return np.abs(ia - ib)


def test_sturm_reciprocal_within_two_ulps():
    # The Sturm counts of the eigenvalue multisection divide by the pivots through a
    # Newton-Raphson reciprocal.  Over the pivot range (|q| from the pivot floor
    # DBL_MIN up to 1e300, both signs, random mantissas, exact powers of two) it must
    # stay within 2 ulps of correctly rounded division; past 1/DBL_MIN it flushes to 0.
    import ctypes
    from paper_0909_5662_gb300 import _capi
    lib = _capi.load()
    rng = np.random.default_rng(91)
    tiny = np.finfo(np.float64).tiny
    mags = np.concatenate([
        10.0 ** rng.uniform(-307.5, 300.0, 200000),
        tiny * rng.uniform(1.0, 4.0, 2000),
        2.0 ** np.arange(-1022, 997, dtype=np.float64),
        1.0 + rng.uniform(-1e-3, 1e-3, 2000),
    ])
    q = np.concatenate([mags, -mags])
    dev = torch.device("cuda")
    qd = torch.from_numpy(q).to(dev)
    out = torch.empty_like(qd)
    st = lib.dmrg_debug_reciprocal(ctypes.c_void_p(qd.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                   len(q), None)
    assert st == 0
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    exact = 1.0 / q
    assert np.all(np.sign(got) == np.sign(exact))
    assert _ulp_distance(got, exact).max() <= 2
    # beyond the range: results flush to zero instead of going subnormal
    big = torch.tensor([1e308, -1e308], dtype=torch.float64, device=dev)
    ob = torch.empty_like(big)
    assert lib.dmrg_debug_reciprocal(ctypes.c_void_p(big.data_ptr()), ctypes.c_void_p(ob.data_ptr()),
                                     2, None) == 0
    torch.cuda.synchronize()
    assert np.all(np.abs(ob.cpu().numpy()) <= tiny)
