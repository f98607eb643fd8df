"""GPU parity of the adjoint (dmrg_rotate_ops_backward) and the autograd Function.

dO_k = Tr_d(U G_k U^T) and dU = sum_k (O_k (x) I) U G_k^T + (O_k (x) I)^T U G_k are
the chain rule of the rotation of Sec. 2, step 5.  Checks: central finite
differences in FP64 (torch.autograd.gradcheck through the FP64 kernels), the
oracle's analytic gradient element by element on ragged shapes, and at the full
m = 400, K = 150 size every dO_k and the whole dU of every precision against the
oracle's analytic gradient, plus exact properties of the FP64 path.

Tolerances are the forward rotation's (relative Frobenius error, per operator for
dO, over the whole matrix for dU): 1e-12 FP64, 1e-5 FP32 and BF16x3, 3e-3 TF32.
"""
import numpy as np
import pytest
import torch

import oracle
from workloads import dense_workload, backward_upstream, orthonormal_columns

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "bf16x3": 1e-5, "tf32": 3e-3}


@pytest.fixture(scope="module")
def P():
    import paper_0909_5662_gb300 as P
    return P


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def rel_per_op(a, b):
    a = np.asarray(a, dtype=np.float64)
    num = np.linalg.norm((a - b).reshape(len(b), -1), axis=1)
    return (num / np.linalg.norm(b.reshape(len(b), -1), axis=1)).max()


def test_gradcheck_fp64_central_differences(P):
    # m = 16, d = 4, m' = 16, K = 4; central differences with step 1e-6 in FP64.
    dev = torch.device("cuda")
    rng = np.random.default_rng(40)
    U = torch.from_numpy(orthonormal_columns(rng, 64, 16)).to(dev).requires_grad_(True)
    O = torch.from_numpy(rng.standard_normal((4, 16, 16))).to(dev).requires_grad_(True)
    f = lambda u, o: P.rotate(u, o, 4, "fp64")
    assert torch.autograd.gradcheck(f, (U, O), eps=1e-6, atol=1e-7, rtol=1e-7)


SHAPES = [(16, 4, 16, 4), (37, 3, 50, 5), (64, 4, 64, 8), (72, 2, 100, 3)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3", "tf32"])
def test_backward_matches_oracle(P, shape, prec):
    m, d, mp, K = shape
    rng = np.random.default_rng(500 + m + mp + K)
    U = orthonormal_columns(rng, m * d, mp)
    O = rng.standard_normal((K, m, m))
    G = rng.standard_normal((K, mp, mp))
    dev = torch.device("cuda")
    dt = torch.float64 if prec != "fp32" else torch.float32
    Oin = O if prec != "fp32" else O.astype(np.float32).astype(np.float64)
    Gin = G if prec != "fp32" else G.astype(np.float32).astype(np.float64)
    dO_ref, dU_ref = oracle.rotate_backward(U, Oin, Gin, d)
    dO, dU = P.dmrg_rotate_ops_backward(torch.from_numpy(U).to(dev), torch.from_numpy(O).to(dev, dt),
                                        torch.from_numpy(G).to(dev, dt), d, prec)
    torch.cuda.synchronize()
    P.dmrg_sync_status()
    assert rel_per_op(dO.double().cpu().numpy(), dO_ref) <= TOL[prec], "dO"
    assert rel(dU.cpu().numpy(), dU_ref) <= TOL[prec], "dU"


def test_backward_partial_requests(P):
    rng = np.random.default_rng(41)
    m, d, mp, K = 24, 4, 30, 3
    U = orthonormal_columns(rng, m * d, mp)
    O = rng.standard_normal((K, m, m))
    G = rng.standard_normal((K, mp, mp))
    dO_ref, dU_ref = oracle.rotate_backward(U, O, G, d)
    dev = torch.device("cuda")
    t = lambda x: torch.from_numpy(x).to(dev)
    for prec in ("fp64", "bf16x3"):
        dO, dU = P.dmrg_rotate_ops_backward(t(U), t(O), t(G), d, prec, want_dU=False)
        assert dU is None and rel_per_op(dO.double().cpu().numpy(), dO_ref) <= TOL[prec]
        dO, dU = P.dmrg_rotate_ops_backward(t(U), t(O), t(G), d, prec, want_dO=False)
        assert dO is None and rel(dU.cpu().numpy(), dU_ref) <= TOL[prec]


def test_autograd_function(P):
    dev = torch.device("cuda")
    rng = np.random.default_rng(42)
    m, d, mp, K = 32, 4, 40, 5
    U = torch.from_numpy(orthonormal_columns(rng, m * d, mp)).to(dev).requires_grad_(True)
    O = torch.from_numpy(rng.standard_normal((K, m, m))).to(dev, torch.float32).requires_grad_(True)
    G = rng.standard_normal((K, mp, mp))
    out = P.rotate(U, O, d, "bf16x3")
    (out * torch.from_numpy(G).to(dev, torch.float32)).sum().backward()
    dO_ref, dU_ref = oracle.rotate_backward(U.detach().cpu().numpy(),
                                            O.detach().double().cpu().numpy(),
                                            G.astype(np.float32).astype(np.float64), d)
    assert rel(U.grad.cpu().numpy(), dU_ref) <= TOL["bf16x3"]
    assert rel_per_op(O.grad.double().cpu().numpy(), dO_ref) <= TOL["bf16x3"]


def test_backward_full_size(P):
    # d = 4, m = m' = 400, K = 150, as the benchmark launches it.  The operators and the
    # upstream gradient are rounded to FP32 once, so every precision sees the same
    # values and one oracle call gives the reference gradient of all of them.
    w = dense_workload("bwd", 4042, 4, 400, 400, 150, hubbard_mix=True)
    O = w.O.astype(np.float32).astype(np.float64)
    G = backward_upstream(4043, 150, 400).astype(np.float32).astype(np.float64)
    dO_ref, dU_ref = oracle.rotate_backward(w.U, O, G, 4)
    dev = torch.device("cuda")
    U = torch.from_numpy(w.U).to(dev)
    O64 = torch.from_numpy(O).to(dev)
    G64 = torch.from_numpy(G).to(dev)
    dO64, dU64 = P.dmrg_rotate_ops_backward(U, O64, G64, 4, "fp64")
    torch.cuda.synchronize()
    # (a) every dO_k and the whole dU against the oracle's analytic gradient.
    assert rel_per_op(dO64.cpu().numpy(), dO_ref) <= TOL["fp64"]
    assert rel(dU64.cpu().numpy(), dU_ref) <= TOL["fp64"]
    # (b) adjoint identity (exact, linear in O): <G, rot(O)> = <dO, O>.
    rot = P.dmrg_rotate_ops(U, O64, 4, "fp64")
    lhs = float((G64 * rot).sum())
    rhs = float((dO64 * O64).sum())
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)
    # (c) dU along a direction: L(U) is quadratic in U, so the central difference is exact.
    V = torch.from_numpy(np.random.default_rng(7).standard_normal(w.U.shape)).to(dev)
    h = 1e-3
    Lp = float((G64 * P.dmrg_rotate_ops(U + h * V, O64, 4, "fp64")).sum())
    Lm = float((G64 * P.dmrg_rotate_ops(U - h * V, O64, 4, "fp64")).sum())
    fd = (Lp - Lm) / (2 * h)
    an = float((dU64 * V).sum())
    assert abs(fd - an) <= 1e-9 * abs(an)
    # (d) the reduced precisions, FP32 operators, against the same oracle gradient.
    O32 = O64.float()
    G32 = G64.float()
    for prec in ("bf16x3", "tf32", "fp32"):
        dO, dU = P.dmrg_rotate_ops_backward(U, O32, G32, 4, prec)
        torch.cuda.synchronize()
        P.dmrg_sync_status()
        assert rel_per_op(dO.double().cpu().numpy(), dO_ref) <= TOL[prec], (prec, "dO")
        assert rel(dU.cpu().numpy(), dU_ref) <= TOL[prec], (prec, "dU")


@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
def test_backward_reproducible_bit_for_bit(P, prec):
    # dU's reduction over every operator is split into parts with their own partial
    # sums, added in a fixed order (no atomics): two calls agree bit for bit.
    rng = np.random.default_rng(43)
    m, d, mp, K = 96, 4, 80, 24
    dev = torch.device("cuda")
    U = torch.from_numpy(orthonormal_columns(rng, m * d, mp)).to(dev)
    O = torch.from_numpy(rng.standard_normal((K, m, m))).to(dev, torch.float32)
    G = torch.from_numpy(rng.standard_normal((K, mp, mp))).to(dev, torch.float32)
    a = P.dmrg_rotate_ops_backward(U, O, G, d, prec)
    b = P.dmrg_rotate_ops_backward(U, O, G, d, prec)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
