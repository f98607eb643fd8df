"""GPU parity of the CTA-pair (cta_group::2) tensor-core kernels against the FP64
oracle: the dense rotation O'_k = U^T (O_k (x) I_d) U (Sec. 2 step 5) with both
products forced onto the pair kernel through the tiling cache file, with one pair
per cluster and with two pairs per cluster sharing the A rows (TMA multicast).

Shapes cover a pair tile whose second CTA is wholly past the last row, N tiles
whose second half is wholly past the last column, an odd number of N tiles (the
second pair of the last cluster tile has no columns), ragged reductions, both
swizzle widths and the split tail wave of the second product.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from workloads import dense_config, orthonormal_columns

pytestmark = pytest.mark.gpu

TOL = {"bf16x3": 1e-5, "tf32": 3e-3}
PCODE = {"tf32": 2, "bf16x3": 3}


@pytest.fixture(scope="module")
def P():
    import paper_0909_5662_gb300 as lib
    return lib


def rel_err(got, ref):
    num = np.linalg.norm((got - ref).reshape(len(ref), -1), axis=1)
    return num / np.linalg.norm(ref.reshape(len(ref), -1), axis=1)


def run_pair(P, tmp_path, U, O, d, prec, tn1, tn2, rb, npc, stages=None, deterministic=False):
    K, m = O.shape[0], O.shape[1]
    mp = U.shape[1]
    key = lambda g: "%s:K%d:m%d:d%d:mp%d:p%d" % (g, K, m, d, mp, PCODE[prec])
    st = stages or 8   # reduced to the deepest pipeline that fits
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({key("g1"): [tn1, st, 0, rb, npc], key("g2"): [tn2, st, 0, rb, npc]}))
    os.environ["DMRG_AUTOTUNE_CACHE"] = str(path)
    try:
        h = P.Handle()
        try:
            if deterministic:
                P.dmrg_set_option("deterministic", 1, handle=h)
            out = P.dmrg_rotate_ops(torch.from_numpy(U).cuda(), torch.from_numpy(O).cuda(), d, prec,
                                    handle=h)
            torch.cuda.synchronize()
            P.dmrg_sync_status(handle=h)
            return out.double().cpu().numpy()
        finally:
            h.close()
    finally:
        del os.environ["DMRG_AUTOTUNE_CACHE"]


SHAPES = [
    # (m, d, mp, K)
    (16, 1, 16, 1),      # one pair tile; the second CTA's rows and B half are all padding
    (37, 3, 50, 5),
    (130, 2, 200, 3),
    (200, 4, 17, 7),
    (129, 4, 130, 2),
    (72, 4, 288, 4),
]


@pytest.mark.parametrize("npc", [1, 2])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
def test_pair_ragged(P, tmp_path, shape, prec, npc):
    m, d, mp, K = shape
    rng = np.random.default_rng(7000 + m + 3 * mp + K)
    U = orthonormal_columns(rng, m * d, mp)
    O = rng.standard_normal((K, m, m))
    ref = oracle.rotate_dense(U, O, d)
    got = run_pair(P, tmp_path, U, O, d, prec, 256, 256, 128, npc)
    assert rel_err(got, ref).max() <= TOL[prec]


@pytest.mark.parametrize("npc", [1, 2])
@pytest.mark.parametrize("tiles", [(96, 64), (160, 208), (256, 128), (224, 48)])
@pytest.mark.parametrize("rb", [128, 64])
def test_pair_tilings(P, tmp_path, tiles, rb, npc):
    m, d, mp, K = 120, 4, 150, 9
    rng = np.random.default_rng(7100 + tiles[0] + rb)
    U = orthonormal_columns(rng, m * d, mp)
    O = rng.standard_normal((K, m, m))
    ref = oracle.rotate_dense(U, O, d)
    for prec in ("bf16x3", "tf32"):
        got = run_pair(P, tmp_path, U, O, d, prec, tiles[0], tiles[1], rb, npc)
        assert rel_err(got, ref).max() <= TOL[prec], (prec, tiles, rb, npc)


@pytest.mark.parametrize("npc", [1, 2])
@pytest.mark.parametrize("deterministic", [False, True])
def test_pair_full_size_m400_sampled(P, tmp_path, deterministic, npc):
    # Full size of the benchmark workload (d=4, m=m'=400, K=150); the second product
    # has more 256-row tiles than one wave of pairs, so its tail wave is split
    # (unless the deterministic option is set).  A seeded sample of operators is
    # recomputed by the oracle.
    w = dense_config("dense_m400_k150")
    O32 = w.O.astype(np.float32)
    sample = np.unique(np.concatenate([[0, 1, 2, w.K - 1], np.random.default_rng(5).choice(w.K, 8, replace=False)]))
    ref = oracle.rotate_dense(w.U, O32[sample].astype(np.float64), 4)
    for prec in ("bf16x3", "tf32"):
        got = run_pair(P, tmp_path, w.U, O32, 4, prec, 240, 208, 128, npc, deterministic=deterministic)
        assert rel_err(got[sample], ref).max() <= TOL[prec], prec


@pytest.mark.parametrize("chain", [None, 0, 256])
def test_long_reduction_chained_accumulation(P, chain):
    # m = 800, d = 4: the second product reduces over m*d = 3200 elements.  With the
    # default chain length (1024) the tensor core sums at most 1024 of them per FP32
    # accumulator and the chains are added in FP32 registers-to-scratch with round to
    # nearest: BF16x3 stays within 1e-5 of the oracle.  chain = 0 (one chain) is
    # checked against its own, looser bound.
    m, d, mp, K = 800, 4, 800, 6
    rng = np.random.default_rng(4242)
    U = orthonormal_columns(rng, m * d, mp)
    O = rng.standard_normal((K, m, m)).astype(np.float32)
    sample = [0, 3, 5]
    ref = oracle.rotate_dense(U, O[sample].astype(np.float64), d)
    h = P.Handle()
    try:
        if chain is not None:
            P.dmrg_set_option("accum_chain", chain, handle=h)
        out = P.dmrg_rotate_ops(torch.from_numpy(U).cuda(), torch.from_numpy(O).cuda(), d, "bf16x3",
                                handle=h)
        torch.cuda.synchronize()
        P.dmrg_sync_status(handle=h)
        err = rel_err(out[sample].double().cpu().numpy(), ref).max()
        assert err <= (3e-5 if chain == 0 else 1e-5), (chain, err)
    finally:
        h.close()
