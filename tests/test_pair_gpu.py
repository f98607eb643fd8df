"""GPU parity of the CTA-pair (cta_group::2) tensor-core kernels against the FP64
oracle: the dense rotation O'_k = U^T (O_k (x) I_d) U (Sec. 2 step 5) with both
products forced onto the pair kernel through the tiling cache file.

Shapes cover a pair tile whose second CTA is wholly past the last row, N tiles
whose second half is wholly past the last column, ragged reductions, both
swizzle widths and the split tail wave of the second product.  A tiling cache
entry naming a kernel form other than 0 (one CTA) or 1 (CTA pair) is ignored.
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


def run_pair(P, tmp_path, U, O, d, prec, tn1, tn2, rb, npc=1, stages=None, deterministic=False):
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


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
def test_pair_ragged(P, tmp_path, shape, prec):
    m, d, mp, K = shape
    rng = np.random.default_rng(7000 + m + 3 * mp + K)
    U = orthonormal_columns(rng, m * d, mp)
    O = rng.standard_normal((K, m, m))
    ref = oracle.rotate_dense(U, O, d)
    got = run_pair(P, tmp_path, U, O, d, prec, 256, 256, 128)
    assert rel_err(got, ref).max() <= TOL[prec]


@pytest.mark.parametrize("tiles", [(96, 64), (160, 208), (256, 128), (224, 48)])
@pytest.mark.parametrize("rb", [128, 64])
def test_pair_tilings(P, tmp_path, tiles, rb):
    m, d, mp, K = 120, 4, 150, 9
    rng = np.random.default_rng(7100 + tiles[0] + rb)
    U = orthonormal_columns(rng, m * d, mp)
    O = rng.standard_normal((K, m, m))
    ref = oracle.rotate_dense(U, O, d)
    for prec in ("bf16x3", "tf32"):
        got = run_pair(P, tmp_path, U, O, d, prec, tiles[0], tiles[1], rb)
        assert rel_err(got, ref).max() <= TOL[prec], (prec, tiles, rb)


@pytest.mark.parametrize("deterministic", [False, True])
def test_pair_full_size_m400_sampled(P, tmp_path, deterministic):
    # Full size of the benchmark workload (d=4, m=m'=400, K=150); the second product
    # has more 256-row tiles than one wave of pairs, so its tail wave is split
    # (unless the deterministic option is set).  A seeded sample of operators is
    # recomputed by the oracle.
    w = dense_config("dense_m400_k150")
    O32 = w.O.astype(np.float32)
    sample = np.unique(np.concatenate([[0, 1, 2, w.K - 1], np.random.default_rng(5).choice(w.K, 8, replace=False)]))
    ref = oracle.rotate_dense(w.U, O32[sample].astype(np.float64), 4)
    for prec in ("bf16x3", "tf32"):
        got = run_pair(P, tmp_path, w.U, O32, 4, prec, 240, 208, 128, deterministic=deterministic)
        assert rel_err(got[sample], ref).max() <= TOL[prec], prec


@pytest.mark.parametrize("chain", [None, 1, 256, 1024])
def test_long_reduction_chained_accumulation(P, chain):
    # m = 800, d = 4: the second product reduces over m*d = 3200 elements.  With any
    # accepted chain length (at most 1024) the tensor core sums at most that many of
    # them per FP32 accumulator and the chains are added in FP32 through a scratch
    # with round to nearest: BF16x3 stays within 1e-5 of the oracle.
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
        assert err <= 1e-5, (chain, err)
    finally:
        h.close()


@pytest.mark.parametrize("chain", [0, -1, 1025, 1e6])
def test_accum_chain_values_that_break_the_bf16x3_bound_are_refused(P, chain):
    # One chain per tile (0) or chains longer than 1024 elements let the tensor core's
    # FP32 accumulation error exceed the 1e-5 bound at m*d = 4800, so they are refused.
    from paper_0909_5662_gb300._capi import DmrgError
    h = P.Handle()
    try:
        with pytest.raises(DmrgError):
            P.dmrg_set_option("accum_chain", chain, handle=h)
    finally:
        h.close()


def test_cached_one_cta_tiling_still_chains_long_reductions(P, tmp_path):
    # A tiling cache that names the one-CTA kernel (no accumulation chains) for a
    # product whose reduction is longer than one chain is overridden by the CTA-pair
    # kernel, so BF16x3 keeps its 1e-5 bound at m*d = 3200.
    m, d, mp, K = 800, 4, 800, 3
    rng = np.random.default_rng(4343)
    U = orthonormal_columns(rng, m * d, mp)
    O = rng.standard_normal((K, m, m))
    ref = oracle.rotate_dense(U, O, d)
    got = run_pair(P, tmp_path, U, O.astype(np.float32), d, "bf16x3", 256, 256, 128, npc=0)
    assert rel_err(got, ref).max() <= 1e-5


def test_cache_entry_with_unknown_kernel_form_is_ignored(P, tmp_path):
    # form 2 (two pairs per cluster) no longer exists: such an entry is skipped and
    # the untuned CTA-pair default runs.
    m, d, mp, K = 64, 4, 64, 4
    rng = np.random.default_rng(4444)
    U = orthonormal_columns(rng, m * d, mp)
    O = rng.standard_normal((K, m, m))
    ref = oracle.rotate_dense(U, O, d)
    got = run_pair(P, tmp_path, U, O, d, "bf16x3", 256, 256, 128, npc=2)
    assert rel_err(got, ref).max() <= 1e-5
