"""GPU parity of the blocked site and cross operators against the FP64 oracle:
O'_k = U^T ((A_k P^f_c) (x) S_c) U (Sec. 2, the blocking after step 5), element by
element on the same seeded inputs, for every precision, with the 4-site Hubbard
chain's site fermion operators checked against full-space matrix elements.
"""
import numpy as np
import pytest
import torch

import hubbard_jw as jw
import oracle
from workloads import orthonormal_columns

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "bf16x3": 1e-5, "tf32": 3e-3}


@pytest.fixture(scope="module")
def P():
    import paper_0909_5662_gb300 as lib
    return lib


def rel_err(got, ref):
    num = np.linalg.norm((got - ref).reshape(len(ref), -1), axis=1)
    return num / np.maximum(np.linalg.norm(ref.reshape(len(ref), -1), axis=1), 1e-300)


def run(P, U, A, d, S, counts, flags, parity, prec, handle=None):
    dev = torch.device("cuda")
    At = torch.from_numpy(A).to(dev, torch.float64 if prec == "fp64" else torch.float32)
    par = None if parity is None else torch.from_numpy(parity.astype(np.int8)).to(dev)
    out = P.dmrg_rotate_site_ops(torch.from_numpy(U).to(dev), At, d, S, counts, flags, par, prec,
                                 handle=handle)
    torch.cuda.synchronize()
    P.dmrg_sync_status(handle=handle)
    return out.double().cpu().numpy()


CASES = [
    # (m, d, mp, counts, flags)
    (37, 3, 50, [2, 0, 3, 1], [1, 0, 0, 1]),
    (130, 2, 200, [3, 2], [0, 1]),
    (64, 4, 96, [1, 1, 1, 1, 1], [1, 1, 0, 0, 1]),
    (129, 4, 130, [4], [1]),
    # nine classes: first products in groups of four, four and one
    (100, 4, 100, [3, 1, 2, 2, 1, 3, 2, 1, 2], [1, 0, 1, 0, 1, 0, 1, 0, 1]),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3", "tf32"])
def test_site_operators_match_oracle(P, case, prec):
    m, d, mp, counts, flags = case
    rng = np.random.default_rng(900 + m + mp)
    U = orthonormal_columns(rng, m * d, mp)
    K = sum(counts)
    A = rng.standard_normal((K, m, m))
    S = rng.standard_normal((len(counts), d, d))
    parity = rng.choice([-1.0, 1.0], m)
    A_in = A if prec == "fp64" else A.astype(np.float32).astype(np.float64)
    ref = oracle.rotate_site(U, A_in, d, S, counts, flags, parity)
    got = run(P, U, A, d, S, counts, flags, parity, prec)
    assert rel_err(got, ref).max() <= TOL[prec], prec


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "tf32"])
def test_site_operators_hubbard_full_space(P, prec):
    # c_4s = P_B (x) c_s, c+_1s c_4s = (c+_1s P_B) (x) c_s, n_4 = I (x) n on the
    # 4-site Hubbard chain (t = 1, U/t = 8), U = lowest 100 eigenvectors: each must
    # equal <u_a| O_full |u_b> with O_full built on all 8 modes.
    cb, cl, cf = jw.annihilators(3), jw.annihilators(1), jw.annihilators(4)
    H = jw.hubbard_hamiltonian(4, 1.0, 8.0, cf)
    _, V = np.linalg.eigh(H)
    U = np.ascontiguousarray(V[:, :100])
    nb = sum(cb[p].T @ cb[p] for p in range(6))
    parity = np.where(np.round(np.diag(nb)).astype(int) % 2 == 0, 1.0, -1.0)
    I64 = np.eye(64)
    n_loc = cl[0].T @ cl[0] + cl[1].T @ cl[1]
    A = np.stack([I64, cb[0].T, I64, cb[1].T, I64])
    S = np.stack([cl[0], cl[1], n_loc])
    counts, flags = [2, 2, 1], [1, 1, 0]
    full = [cf[6], cf[0].T @ cf[6], cf[7], cf[1].T @ cf[7], cf[6].T @ cf[6] + cf[7].T @ cf[7]]
    got = run(P, U, A, 4, S, counts, flags, parity, prec)
    ref = np.stack([U.T @ f @ U for f in full])
    assert rel_err(got, ref).max() <= TOL[prec], prec    # per-operator relative Frobenius


def test_site_identity_equals_block_rotation_bitwise(P):
    # S = I and no parity: U_c = U exactly, so the result is the block rotation's,
    # bit for bit (deterministic mode: no atomically accumulated split tiles).
    rng = np.random.default_rng(77)
    m, d, mp, K = 96, 4, 80, 7
    U = orthonormal_columns(rng, m * d, mp)
    A = rng.standard_normal((K, m, m)).astype(np.float32)
    h = P.Handle()
    try:
        P.dmrg_set_option("deterministic", 1, handle=h)
        dev = torch.device("cuda")
        for prec in ("bf16x3", "tf32", "fp32"):
            a = run(P, U, A.astype(np.float64), d, np.eye(d)[None], [K], [0], None, prec, handle=h)
            b = P.dmrg_rotate_ops(torch.from_numpy(U).to(dev), torch.from_numpy(A).to(dev), d, prec,
                                  handle=h).double().cpu().numpy()
            assert np.array_equal(a, b), prec
    finally:
        h.close()


def test_site_argument_errors(P):
    from paper_0909_5662_gb300 import _capi
    rng = np.random.default_rng(3)
    U = orthonormal_columns(rng, 16, 8)
    A = rng.standard_normal((3, 4, 4))
    with pytest.raises(_capi.DmrgError) as ei:        # counts do not sum to K
        run(P, U, A, 4, np.eye(4)[None], [2], [0], None, "fp64")
    assert ei.value.status == 1
    with pytest.raises(_capi.DmrgError) as ei:        # parity flag without parity
        run(P, U, A, 4, np.eye(4)[None], [3], [1], None, "fp64")
    assert ei.value.status == 1
