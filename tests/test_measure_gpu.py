"""GPU parity of the measurement stage against the FP64 oracle (Sec. 3.2 one- and
two-point functions in the superblock ground state; Sec. 2 structure factors), and
the 4-site Hubbard ground state split into two halves against full-space values.
"""
import numpy as np
import pytest
import torch

import hubbard_jw as jw
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_0909_5662_gb300 as lib
    return lib


def dev(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to(torch.device("cuda"), dtype)


@pytest.mark.parametrize("shape", [(37, 50), (130, 64), (200, 17), (1, 9)])
@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("zdt", [torch.float64, torch.float32])
def test_expectation_matches_oracle(P, shape, side, zdt):
    rows, cols = shape
    rng = np.random.default_rng(rows * 7 + cols + side)
    Psi = rng.standard_normal((rows, cols))
    Psi /= np.linalg.norm(Psi)
    n = rows if side == 0 else cols
    Z = rng.standard_normal((6, n, n))
    Zin = Z if zdt == torch.float64 else Z.astype(np.float32).astype(np.float64)
    ref = oracle.expectation(Zin, Psi, side)
    got = P.dmrg_expectation(dev(Z, zdt), dev(Psi), side).cpu().numpy()
    P.dmrg_sync_status()
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("shape", [(37, 50), (64, 130), (20, 3)])
def test_cross_correlations_match_oracle(P, shape):
    rows, cols = shape
    rng = np.random.default_rng(rows + 3 * cols)
    Psi = rng.standard_normal((rows, cols))
    Psi /= np.linalg.norm(Psi)
    Z = rng.standard_normal((5, rows, rows))
    W = rng.standard_normal((7, cols, cols))
    ref = oracle.cross_correlations(Z, W, Psi)
    got = P.dmrg_cross_correlations(dev(Z), dev(W), dev(Psi)).cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    got32 = P.dmrg_cross_correlations(dev(Z, torch.float32), dev(W, torch.float32), dev(Psi)).cpu().numpy()
    ref32 = oracle.cross_correlations(Z.astype(np.float32).astype(np.float64),
                                      W.astype(np.float32).astype(np.float64), Psi)
    assert np.abs(got32 - ref32).max() <= 1e-12 * np.abs(ref32).max()
    P.dmrg_sync_status()


@pytest.mark.parametrize("L", [1, 7, 64, 300])
def test_structure_factor_matches_oracle(P, L):
    rng = np.random.default_rng(L)
    X = rng.standard_normal((L, L))
    G = X + X.T
    v = rng.standard_normal(L)
    for vv, c in ((v, 0.37), (None, 0.0)):
        re_ref, im_ref = oracle.structure_factor(G, vv, c)
        re, im = P.dmrg_structure_factor(dev(G), dev(vv) if vv is not None else None, c)
        scale = max(1.0, np.abs(re_ref).max())
        assert np.abs(re.cpu().numpy() - re_ref).max() <= 1e-12 * scale * L
        assert np.abs(im.cpu().numpy() - im_ref).max() <= 1e-12 * scale * L
    P.dmrg_sync_status()


def test_measurement_hubbard_ground_state(P):
    # 4-site Hubbard chain (t = 1, U/t = 8): the ground state as a 16 x 16 matrix
    # (system = sites 1-2, environment = sites 3-4).  All <n_i>, <n_i n_j> and the
    # charge structure factor N(q) from the GPU stage equal the full-space values.
    cf = jw.annihilators(4)
    H = jw.hubbard_hamiltonian(4, 1.0, 8.0, cf)
    _, V = np.linalg.eigh(H)
    psi = V[:, 0]
    Psi = psi.reshape(16, 16)
    c2 = jw.annihilators(2)
    n2 = [c2[2 * i].T @ c2[2 * i] + c2[2 * i + 1].T @ c2[2 * i + 1] for i in range(2)]
    nf = [cf[2 * i].T @ cf[2 * i] + cf[2 * i + 1].T @ cf[2 * i + 1] for i in range(4)]
    # one-point: single sites of either half; two-point inside a half: stored products
    sys_ops = np.stack(n2 + [n2[0] @ n2[0], n2[0] @ n2[1], n2[1] @ n2[1]])
    e_sys = P.dmrg_expectation(dev(sys_ops), dev(Psi), 0).cpu().numpy()
    e_env = P.dmrg_expectation(dev(sys_ops), dev(Psi), 1).cpu().numpy()
    C = P.dmrg_cross_correlations(dev(np.stack(n2)), dev(np.stack(n2)), dev(Psi)).cpu().numpy()
    G = np.zeros((4, 4))
    G[0, 0], G[0, 1], G[1, 1] = e_sys[2], e_sys[3], e_sys[4]
    G[2, 2], G[2, 3], G[3, 3] = e_env[2], e_env[3], e_env[4]
    G[:2, 2:] = C
    G = np.triu(G) + np.triu(G, 1).T
    G_full = np.array([[psi @ nf[i] @ nf[j] @ psi for j in range(4)] for i in range(4)])
    assert np.abs(G - G_full).max() < 1e-12
    v = np.concatenate([e_sys[:2], e_env[:2]])
    assert np.abs(v - np.array([psi @ nf[i] @ psi for i in range(4)])).max() < 1e-12
    nbar = v.mean()
    re, im = P.dmrg_structure_factor(dev(G), dev(v), nbar)
    re_ref, im_ref = oracle.structure_factor(G_full, v, nbar)
    assert np.abs(re.cpu().numpy() - re_ref).max() < 1e-12
    assert np.abs(im.cpu().numpy()).max() < 1e-12
    P.dmrg_sync_status()
