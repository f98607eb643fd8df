"""GPU parity of the BF16x3 first product's TMA-store epilogue (T = O_k U_r leaving the
CTA-pair kernel through bulk tensor stores staged in shared memory) against the same
kernel storing from registers, and of both against the FP64 oracle of the rotation
O'_k = U^T (O_k (x) I_d) U (Sec. 2 step 5).

The two epilogues write the same BF16 hi/lo values to the same places, so with the
deterministic option the rotated operators must agree bit for bit.  The shapes cover
both site dimensions the store maps take (d = 2, 4), operators that begin in the middle
of a warp's 32 rows (m = 48, 400), chunks that are short inside N (N tiles of 208 and
176 columns) and at the end of N (d * m' not a multiple of 32), rows past the last
operator, accumulation chains (m > 1024), and layouts that fall back to register stores
(d = 3, m not a multiple of 16); TF32 takes the FP32 form of the first layout.  The
second product's FP32 O' leaves through the columns layout, its second accumulation
chain and the parts of its split tail adding with TMA reductions.  The adjoint's W' product takes the row-contiguous form
of the same epilogue and is checked the same way against the oracle's adjoint.
"""
import numpy as np
import pytest
import torch

import oracle
from workloads import orthonormal_columns

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def P():
    import paper_0909_5662_gb300 as lib
    return lib


def rel_err(got, ref):
    num = np.linalg.norm((got - ref).reshape(len(ref), -1), axis=1)
    return num / np.linalg.norm(ref.reshape(len(ref), -1), axis=1)


def rotate(P, U, O, d, store, opts=(), prec="bf16x3"):
    h = P.Handle()
    try:
        P.dmrg_set_option("deterministic", 1, handle=h)
        P.dmrg_set_option("store_epilogue", store, handle=h)
        for k, v in opts:
            P.dmrg_set_option(k, v, handle=h)
        out = P.dmrg_rotate_ops(U, O, d, prec, handle=h)
        torch.cuda.synchronize()
        P.dmrg_sync_status(handle=h)
        return out.double().cpu().numpy()
    finally:
        h.close()


SHAPES = [
    # (m, d, mp, K)
    (16, 4, 8, 1),        # one 16-row group, one short chunk at the end of N
    (48, 4, 100, 7),      # operators start inside a warp's rows; rows past the last one
    (400, 4, 400, 9),     # the benchmark's m, d, m' (N tiles of 256, a short last tile)
    (64, 2, 104, 5),      # d = 2: N = 208, one 208-column tile (a 16-column chunk at N's end)
    (96, 4, 130, 3),      # N = 520: tiles of 176 (a short chunk inside N) and 168
    (1040, 4, 64, 2),     # accumulation chains over the reduction (m > 1024)
    (160, 2, 333, 4),     # d = 2, odd m': the last chunk partly past N
    (50, 4, 60, 3),       # m not a multiple of 16: register stores
    (48, 3, 70, 3),       # d = 3: register stores
    # the second product's FP32 columns layout (m' a multiple of 16):
    (64, 4, 48, 7),       # one chain, operators of 48 rows inside a warp's 32
    (300, 4, 80, 5),      # two chains (m*d = 1200): the second adds by TMA reductions
    (200, 2, 208, 3),     # one 208-column tile, its last chunk of 16 columns
]


@pytest.mark.parametrize("shape", SHAPES)
def test_tma_store_epilogue_matches_register_stores_and_oracle(P, shape):
    m, d, mp, K = shape
    rng = np.random.default_rng(9500 + m + 7 * mp + K)
    U = orthonormal_columns(rng, m * d, mp)
    O = rng.standard_normal((K, m, m)).astype(np.float32)
    dev = torch.device("cuda")
    Ud, Od = torch.from_numpy(U).to(dev), torch.from_numpy(O).to(dev)
    tma = rotate(P, Ud, Od, d, 0, opts=(("pack_operators", 1),))
    reg = rotate(P, Ud, Od, d, 1, opts=(("pack_operators", 1),))
    assert np.array_equal(tma, reg)
    ref = oracle.rotate_dense(U, O.astype(np.float64), d)
    assert rel_err(tma, ref).max() <= TOL


@pytest.mark.parametrize("shape", [(48, 4, 100, 7), (400, 4, 400, 9), (64, 2, 104, 5), (96, 4, 130, 3),
                                   (50, 4, 60, 3)])
def test_tma_store_epilogue_tf32(P, shape):
    # TF32: the first product's T is FP32 (TF32-rounded) and leaves through the same
    # site-interleaved boxes in FP32, the pipeline giving up a stage for the staging
    m, d, mp, K = shape
    rng = np.random.default_rng(9900 + m + 7 * mp + K)
    U = orthonormal_columns(rng, m * d, mp)
    O = rng.standard_normal((K, m, m)).astype(np.float32)
    dev = torch.device("cuda")
    Ud, Od = torch.from_numpy(U).to(dev), torch.from_numpy(O).to(dev)
    tma = rotate(P, Ud, Od, d, 0, opts=(("pack_operators", 1),), prec="tf32")
    reg = rotate(P, Ud, Od, d, 1, opts=(("pack_operators", 1),), prec="tf32")
    assert np.array_equal(tma, reg)
    assert rel_err(tma, oracle.rotate_dense(U, O.astype(np.float64), d)).max() <= 3e-3


@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
def test_second_product_tma_reductions_split_tail(P, prec):
    # the default (non-deterministic) second product splits its last partial wave along
    # the reduction: the parts add into O' with TMA reductions (the columns layout), as
    # does the second of its two accumulation chains (BF16x3, m*d = 1600); checked
    # against the oracle, the summation order of the split tiles being free
    m, d, mp, K = 400, 4, 400, 23
    rng = np.random.default_rng(9950)
    U = orthonormal_columns(rng, m * d, mp)
    O = rng.standard_normal((K, m, m)).astype(np.float32)
    dev = torch.device("cuda")
    h = P.Handle()
    try:
        out = P.dmrg_rotate_ops(torch.from_numpy(U).to(dev), torch.from_numpy(O).to(dev), d, prec,
                                handle=h)
        torch.cuda.synchronize()
        P.dmrg_sync_status(handle=h)
        got = out.double().cpu().numpy()
    finally:
        h.close()
    ref = oracle.rotate_dense(U, O.astype(np.float64), d)
    assert rel_err(got, ref).max() <= (TOL if prec == "bf16x3" else 3e-3)


@pytest.mark.parametrize("shape", [(64, 4, 64, 5), (48, 2, 100, 4)])
def test_tma_store_epilogue_with_converting_form(P, shape):
    # the converting first product (FP32 operators split in shared memory) keeps its
    # stage layout; the staging goes after it when it fits
    m, d, mp, K = shape
    rng = np.random.default_rng(9600 + m + mp)
    U = orthonormal_columns(rng, m * d, mp)
    O = rng.standard_normal((K, m, m)).astype(np.float32)
    dev = torch.device("cuda")
    Ud, Od = torch.from_numpy(U).to(dev), torch.from_numpy(O).to(dev)
    tma = rotate(P, Ud, Od, d, 0, opts=(("pack_operators", 2),))
    reg = rotate(P, Ud, Od, d, 1, opts=(("pack_operators", 2),))
    assert np.array_equal(tma, reg)
    assert rel_err(tma, oracle.rotate_dense(U, O.astype(np.float64), d)).max() <= TOL


def test_tma_store_epilogue_site_classes(P):
    # site operators: the first product runs as one problem per class of operators, each
    # writing its own range of T (the store maps' operator index starts at the class's k0)
    m, d, mp = 64, 4, 96
    counts, flags = [2, 1, 3, 1, 2], [1, 0, 1, 0, 1]
    rng = np.random.default_rng(9700)
    U = orthonormal_columns(rng, m * d, mp)
    K = sum(counts)
    A = rng.standard_normal((K, m, m))
    S = rng.standard_normal((len(counts), d, d))
    parity = rng.choice([-1.0, 1.0], m)
    dev = torch.device("cuda")
    par = torch.from_numpy(parity.astype(np.int8)).to(dev)
    outs = []
    for store in (0, 1):
        h = P.Handle()
        try:
            P.dmrg_set_option("deterministic", 1, handle=h)
            P.dmrg_set_option("store_epilogue", store, handle=h)
            out = P.dmrg_rotate_site_ops(torch.from_numpy(U).to(dev),
                                         torch.from_numpy(A).to(dev, torch.float32), d, S,
                                         counts, flags, par, "bf16x3", handle=h)
            torch.cuda.synchronize()
            P.dmrg_sync_status(handle=h)
            outs.append(out.double().cpu().numpy())
        finally:
            h.close()
    assert np.array_equal(outs[0], outs[1])
    ref = oracle.rotate_site(U, A.astype(np.float32).astype(np.float64), d, S, counts, flags, parity)
    assert rel_err(outs[0], ref).max() <= TOL


def test_store_epilogue_option_values(P):
    from paper_0909_5662_gb300._capi import DmrgError
    h = P.Handle()
    try:
        for v in (0, 1):
            P.dmrg_set_option("store_epilogue", v, handle=h)
        with pytest.raises(DmrgError):
            P.dmrg_set_option("store_epilogue", 2, handle=h)
    finally:
        h.close()


# The adjoint's W' product (W'_k[j d + s][a] = sum_b G_k[a][b] U[j d + s][b], stored
# row-major as W'_k[j][s m' + a]) leaves through the row-contiguous TMA-store layout:
# shapes with operators that begin inside a warp's 32 rows (m' = 48, 112), 32-column
# chunks whose two 16-column halves fall in different sites s (m = 48), N tiles of 176
# columns (a chunk with one half), and a shape that stores from registers (m = 37).
BWD_SHAPES = [(16, 4, 16, 4), (64, 4, 48, 8), (48, 2, 96, 5), (96, 4, 112, 3), (176, 2, 64, 3),
              (37, 3, 50, 5)]


@pytest.mark.parametrize("shape", BWD_SHAPES)
def test_adjoint_tma_store_matches_register_stores_and_oracle(P, shape):
    m, d, mp, K = shape
    rng = np.random.default_rng(9800 + m + 3 * mp + K)
    U = orthonormal_columns(rng, m * d, mp)
    O = rng.standard_normal((K, m, m))
    G = rng.standard_normal((K, mp, mp))
    dev = torch.device("cuda")
    outs = []
    for store in (0, 1):
        h = P.Handle()
        try:
            P.dmrg_set_option("deterministic", 1, handle=h)
            P.dmrg_set_option("store_epilogue", store, handle=h)
            dO, dU = P.dmrg_rotate_ops_backward(torch.from_numpy(U).to(dev), torch.from_numpy(O).to(dev),
                                                torch.from_numpy(G).to(dev), d, "bf16x3", handle=h)
            torch.cuda.synchronize()
            P.dmrg_sync_status(handle=h)
            outs.append((dO.cpu().numpy(), dU.cpu().numpy()))
        finally:
            h.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    dO_ref, dU_ref = oracle.rotate_backward(U, O, G, d)
    assert rel_err(outs[0][0].astype(np.float64), dO_ref).max() <= TOL
    assert np.linalg.norm(outs[0][1] - dU_ref) / np.linalg.norm(dU_ref) <= TOL
