"""GPU parity of the fused rotation (both products of Sec. 3.2 in one kernel, the
intermediate (O_k (x) I_d) U kept in tensor memory and shared memory) against the FP64
CPU oracle, element by element on the same seeded inputs.

Tolerance: relative Frobenius error per operator <= 1e-5 (BF16x3), max over k.
"""
import numpy as np
import pytest
import torch

import oracle
from workloads import orthonormal_columns

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def lib():
    import paper_0909_5662_gb300 as P
    return P


@pytest.fixture
def fused(lib):
    h = lib.Handle()
    lib.dmrg_set_option("fused_rotation", 1, handle=h)
    yield h
    h.close()


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    num = np.linalg.norm((got - ref).reshape(len(ref), -1), axis=1)
    den = np.linalg.norm(ref.reshape(len(ref), -1), axis=1)
    return num / np.maximum(den, 1e-300)


def run(lib, h, U, O, d, o_dtype=torch.float64):
    dev = torch.device("cuda")
    out = lib.dmrg_rotate_ops(torch.from_numpy(U).to(dev), torch.from_numpy(O).to(dev, o_dtype), d,
                              "bf16x3", handle=h)
    torch.cuda.synchronize()
    lib.dmrg_sync_status(handle=h)
    return out.double().cpu().numpy()


def inputs(m, d, mp, K, seed):
    rng = np.random.default_rng(seed)
    return orthonormal_columns(rng, m * d, mp), rng.standard_normal((K, m, m))


SHAPES = [
    # (m, d, mp, K): ragged chunks of i (128 rows) and k-blocks (32), partial
    # output blocks (128 columns beta), one and two output blocks, mp up to 256
    (64, 4, 64, 8),
    (37, 3, 50, 5),
    (130, 2, 200, 3),
    (16, 1, 16, 1),
    (200, 4, 17, 7),
    (129, 4, 130, 2),
    (400, 4, 128, 4),
    (400, 4, 256, 2),
    (300, 2, 256, 3),
    (33, 8, 264 - 8, 2),
]


@pytest.mark.parametrize("shape", SHAPES)
def test_fused_matches_oracle(lib, fused, shape):
    m, d, mp, K = shape
    U, O = inputs(m, d, mp, K, 7000 + m + 3 * mp + K)
    ref = oracle.rotate_dense(U, O, d)
    got = run(lib, fused, U, O, d)
    assert rel_err(got, ref).max() <= TOL


def test_fused_kernel_is_the_one_that_runs(lib, fused):
    U, O = inputs(96, 4, 64, 3, 71)
    lib.dmrg_set_option("kernel_timing", 1, handle=fused)
    lib.dmrg_kernel_timing(reset=True, handle=fused)
    run(lib, fused, U, O, 4)
    names = {k["kernel"] for k in lib.dmrg_kernel_timing(reset=True, handle=fused)}
    assert "tc_fused_rotation" in names
    assert "tc_gemm_first_product" not in names and "tc_gemm_second_product" not in names


def test_wide_mp_takes_the_two_products(lib, fused):
    # mp > 256 does not fit the accumulator: the option falls back to the two products
    U, O = inputs(72, 4, 288, 2, 72)
    lib.dmrg_set_option("kernel_timing", 1, handle=fused)
    lib.dmrg_kernel_timing(reset=True, handle=fused)
    got = run(lib, fused, U, O, 4)
    names = {k["kernel"] for k in lib.dmrg_kernel_timing(reset=True, handle=fused)}
    assert "tc_fused_rotation" not in names and "tc_gemm_first_product" in names
    assert rel_err(got, oracle.rotate_dense(U, O, 4)).max() <= TOL


@pytest.mark.parametrize("chain", [128, 256, 1024])
def test_accumulation_chains(lib, fused, chain):
    # a drain after every chunk (128), chains of two chunks (256), chains of eight
    # chunks (1024: two chains over the 12 chunks of m = 300, d = 4)
    lib.dmrg_set_option("accum_chain", chain, handle=fused)
    U, O = inputs(300, 4, 160, 3, 73 + chain)
    got = run(lib, fused, U, O, 4)
    assert rel_err(got, oracle.rotate_dense(U, O, 4)).max() <= TOL


def test_fp32_operators(lib, fused):
    U, O = inputs(77, 3, 80, 6, 74)
    O32 = O.astype(np.float32)
    got = run(lib, fused, U, O32, 3, torch.float32)
    assert rel_err(got, oracle.rotate_dense(U, O32.astype(np.float64), 3)).max() <= TOL


def test_deterministic_and_batch_invariant(lib, fused):
    U, O = inputs(150, 4, 96, 5, 75)
    a = run(lib, fused, U, O, 4)
    b = run(lib, fused, U, O, 4)
    assert np.array_equal(a, b)
    one = run(lib, fused, U, O[3:4], 4)
    assert np.array_equal(a[3], one[0])


def test_identity_operator(lib, fused):
    rng = np.random.default_rng(76)
    U = orthonormal_columns(rng, 400, 100)
    O = np.eye(100)[None].repeat(2, 0)
    got = run(lib, fused, U, O, 4)
    assert np.abs(got - np.eye(100)).max() <= 10 * TOL


def test_full_size_sampled(lib, fused):
    # m = 400, d = 4, m' = 128, K = 150 in one launch; sampled operators against the oracle
    m, d, mp, K = 400, 4, 128, 150
    U, O = inputs(m, d, mp, K, 77)
    got = run(lib, fused, U, O, d, torch.float32)
    O32 = O.astype(np.float32).astype(np.float64)
    idx = [0, 1, 74, 148, 149]
    ref = oracle.rotate_dense(U, O32[idx], d)
    assert rel_err(got[idx], ref).max() <= TOL


def test_option_values(lib):
    h = lib.Handle()
    try:
        for v in (0, 1):
            lib.dmrg_set_option("fused_rotation", v, handle=h)
        from paper_0909_5662_gb300._capi import DmrgError
        for v in (2, 3, 4):
            with pytest.raises(DmrgError):
                lib.dmrg_set_option("fused_rotation", v, handle=h)
    finally:
        h.close()


def test_empty_batch(lib, fused):
    dev = torch.device("cuda")
    U = torch.from_numpy(orthonormal_columns(np.random.default_rng(78), 32, 8)).to(dev)
    O = torch.zeros((0, 8, 8), dtype=torch.float64, device=dev)
    out = lib.dmrg_rotate_ops(U, O, 4, "bf16x3", handle=fused)
    assert out.shape == (0, 8, 8)
