"""GPU parity of the converting form of the first product: FP32 operators fed to the
CTA-pair kernel as they are stored, split into BF16 hi/lo (BF16x3) or rounded to TF32
in shared memory by converter warps instead of a packing pass over global memory.

The conversion produces the same operand values as the packing pass and the tensor
core then runs the same MMAs in the same order, so with the deterministic option the
two forms must agree bit for bit; both are checked against the FP64 oracle of the
rotation O'_k = U^T (O_k (x) I_d) U (Sec. 2 step 5).  Operators whose rows are not
whole 16-byte units, or whose base is not 16-byte aligned, take the packing pass.
"""
import numpy as np
import pytest
import torch

import oracle
from workloads import dense_config, orthonormal_columns

pytestmark = pytest.mark.gpu

TOL = {"bf16x3": 1e-5, "tf32": 3e-3}


@pytest.fixture(scope="module")
def P():
    import paper_0909_5662_gb300 as lib
    return lib


def rel_err(got, ref):
    num = np.linalg.norm((got - ref).reshape(len(ref), -1), axis=1)
    return num / np.linalg.norm(ref.reshape(len(ref), -1), axis=1)


def rotate(P, U, O32, d, prec, pack, deterministic=True, names=None):
    h = P.Handle()
    try:
        P.dmrg_set_option("pack_operators", pack, handle=h)
        if deterministic:
            P.dmrg_set_option("deterministic", 1, handle=h)
        if names is not None:
            P.dmrg_set_option("kernel_timing", 1, handle=h)
        out = P.dmrg_rotate_ops(U, O32, d, prec, handle=h)
        torch.cuda.synchronize()
        P.dmrg_sync_status(handle=h)
        if names is not None:
            names.extend(k["kernel"] for k in P.dmrg_kernel_timing(reset=True, handle=h))
        return out.double().cpu().numpy()
    finally:
        h.close()


SHAPES = [
    # (m, d, mp, K): m % 4 == 0; ragged 64-element k-blocks, rows past the last
    # operator, pair tiles whose second CTA is all padding, several N tiles
    (16, 1, 16, 1),
    (36, 3, 50, 5),
    (128, 2, 200, 3),
    (200, 4, 17, 7),
    (132, 4, 130, 2),
    (72, 4, 288, 4),
    (260, 4, 96, 3),
]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
def test_converting_form_matches_packing_bitwise_and_oracle(P, shape, prec):
    m, d, mp, K = shape
    rng = np.random.default_rng(9100 + m + 3 * mp + K)
    U = orthonormal_columns(rng, m * d, mp)
    O = rng.standard_normal((K, m, m)).astype(np.float32)
    dev = torch.device("cuda")
    Ud, Od = torch.from_numpy(U).to(dev), torch.from_numpy(O).to(dev)
    names = []
    conv = rotate(P, Ud, Od, d, prec, 2, names=names)
    packed = rotate(P, Ud, Od, d, prec, 1)
    assert "tc_gemm_first_product" in names and "pack_operands" not in names
    assert np.array_equal(conv, packed)
    ref = oracle.rotate_dense(U, O.astype(np.float64), d)
    assert rel_err(conv, ref).max() <= TOL[prec]


@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
def test_converting_form_full_size_sampled(P, prec):
    # the benchmark workload (d = 4, m = m' = 400, K = 150) with the default
    # (non-deterministic) second product, sampled operators against the oracle
    w = dense_config("dense_m400_k150")
    O32 = w.O.astype(np.float32)
    sample = [0, 1, 2, 74, 148, 149]
    ref = oracle.rotate_dense(w.U, O32[sample].astype(np.float64), 4)
    dev = torch.device("cuda")
    got = rotate(P, torch.from_numpy(w.U).to(dev), torch.from_numpy(O32).to(dev), 4, prec, 2,
                 deterministic=False)
    assert rel_err(got[sample], ref).max() <= TOL[prec]


def test_fallbacks_to_the_packing_pass(P):
    # rows of 37 floats (not whole 16-byte units) and a base 4 bytes past a 16-byte
    # boundary both take the packing pass; the results still match the oracle
    dev = torch.device("cuda")
    rng = np.random.default_rng(9200)
    m, d, mp, K = 37, 4, 40, 3
    U = orthonormal_columns(rng, m * d, mp)
    O = rng.standard_normal((K, m, m)).astype(np.float32)
    names = []
    got = rotate(P, torch.from_numpy(U).to(dev), torch.from_numpy(O).to(dev), d, "bf16x3", 2,
                 names=names)
    assert "pack_operands" in names
    assert rel_err(got, oracle.rotate_dense(U, O.astype(np.float64), d)).max() <= 1e-5
    m = 40
    U = orthonormal_columns(rng, m * d, mp)
    O = rng.standard_normal((K, m, m)).astype(np.float32)
    buf = torch.empty(O.size + 1, dtype=torch.float32, device=dev)
    Ov = buf[1:].view(K, m, m)
    Ov.copy_(torch.from_numpy(O))
    assert Ov.data_ptr() % 16 == 4
    names = []
    got = rotate(P, torch.from_numpy(U).to(dev), Ov, d, "bf16x3", 2, names=names)
    assert "pack_operands" in names
    assert rel_err(got, oracle.rotate_dense(U, O.astype(np.float64), d)).max() <= 1e-5


def test_automatic_choice(P):
    # default (0): BF16x3 converts when d*m' fits two N tiles, packs otherwise; TF32 packs
    dev = torch.device("cuda")
    rng = np.random.default_rng(9300)
    for (m, mp, prec, converted) in ((64, 64, "bf16x3", True), (64, 64, "tf32", False),
                                     (64, 160, "bf16x3", False)):
        U = orthonormal_columns(rng, m * 4, mp)
        O = rng.standard_normal((3, m, m)).astype(np.float32)
        names = []
        got = rotate(P, torch.from_numpy(U).to(dev), torch.from_numpy(O).to(dev), 4, prec, 0,
                     names=names)
        assert ("pack_operands" not in names) == converted, (m, mp, prec)
        assert rel_err(got, oracle.rotate_dense(U, O.astype(np.float64), 4)).max() <= TOL[prec]
    h = P.Handle()
    try:
        from paper_0909_5662_gb300._capi import DmrgError
        with pytest.raises(DmrgError):
            P.dmrg_set_option("pack_operators", 3, handle=h)
    finally:
        h.close()
