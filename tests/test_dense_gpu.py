"""GPU parity of the dense rotation O'_k = U^T (O_k (x) I_d) U (Sec. 2 step 5)
against the FP64 CPU oracle, element by element on the same seeded inputs.

Tolerances (relative Frobenius error per operator, max over k):
FP64 1e-12, FP32 1e-5, BF16x3 1e-5, TF32 3e-3.
"""
import numpy as np
import pytest
import torch

import oracle
from workloads import dense_config, dense_workload, orthonormal_columns

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "bf16x3": 1e-5, "tf32": 3e-3}


@pytest.fixture(scope="module")
def lib():
    import paper_0909_5662_gb300 as P
    return P


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    num = np.linalg.norm((got - ref).reshape(len(ref), -1), axis=1)
    den = np.linalg.norm(ref.reshape(len(ref), -1), axis=1)
    return num / np.maximum(den, 1e-300)


def run(lib, U, O, d, prec, o_dtype=None):
    dev = torch.device("cuda")
    Ut = torch.from_numpy(U).to(dev)
    dt = o_dtype or (torch.float64 if prec == "fp64" else torch.float32)
    Ot = torch.from_numpy(O).to(dev, dt)
    out = lib.dmrg_rotate_ops(Ut, Ot, d, prec)
    torch.cuda.synchronize()
    lib.dmrg_sync_status()
    return out.double().cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3", "tf32"])
def test_config_m64(lib, prec):
    w = dense_config("dense_m64_k32")
    ref = oracle.rotate_dense(w.U, w.O, w.d)
    got = run(lib, w.U, w.O, w.d, prec, torch.float64 if prec != "fp32" else torch.float32)
    err = rel_err(got, ref)
    assert err.max() <= TOL[prec], (prec, err.max())


RAGGED = [
    # (m, d, mp, K): ragged tails in every dimension, several tiles
    (37, 3, 50, 5),
    (130, 2, 200, 3),
    (16, 1, 16, 1),
    (200, 4, 17, 7),
    (72, 4, 288, 4),
    (129, 4, 130, 2),
]


@pytest.mark.parametrize("shape", RAGGED)
@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "tf32"])
def test_ragged_shapes(lib, shape, prec):
    m, d, mp, K = shape
    rng = np.random.default_rng(1000 + m + 7 * mp + K)
    U = orthonormal_columns(rng, m * d, mp)
    O = rng.standard_normal((K, m, m))
    ref = oracle.rotate_dense(U, O, d)
    got = run(lib, U, O, d, prec, torch.float64)
    assert rel_err(got, ref).max() <= TOL[prec]


@pytest.mark.parametrize("m", [77, 96])
def test_fp32_input_for_tensor_core_paths(lib, m):
    # FP32 operators with rows that are not (m = 77) and are (m = 96) 16-byte aligned;
    # both go through the rounding (TF32) or splitting (BF16x3) of the operands
    w = dense_workload("t", 77, 3, m, 80, 6)
    ref = oracle.rotate_dense(w.U, w.O.astype(np.float32).astype(np.float64), 3)
    for prec in ("bf16x3", "tf32"):
        got = run(lib, w.U, w.O, 3, prec, torch.float32)
        assert rel_err(got, ref).max() <= TOL[prec]


def test_empty_batch_is_noop(lib):
    dev = torch.device("cuda")
    U = torch.from_numpy(orthonormal_columns(np.random.default_rng(3), 32, 8)).to(dev)
    O = torch.zeros((0, 8, 8), dtype=torch.float64, device=dev)
    for prec in ("fp64", "bf16x3"):
        out = lib.dmrg_rotate_ops(U, O, 4, prec)
        assert out.shape == (0, 8, 8)


def test_batch_invariance_fp64_bitwise(lib):
    # Operators are independent: rotating one alone equals rotating it in a batch.
    w = dense_workload("t", 5, 4, 64, 48, 9)
    full = run(lib, w.U, w.O, 4, "fp64")
    one = run(lib, w.U, w.O[4:5], 4, "fp64")
    assert np.array_equal(full[4], one[0])


def test_isometry_identity_operator(lib):
    # U^T (I (x) I) U = I for orthonormal U.
    rng = np.random.default_rng(11)
    U = orthonormal_columns(rng, 400, 100)
    O = np.eye(100)[None].repeat(2, 0)
    for prec in ("fp64", "bf16x3", "tf32"):
        got = run(lib, U, O, 4, prec, torch.float64)
        assert np.abs(got - np.eye(100)).max() <= (1e-12 if prec == "fp64" else 10 * TOL[prec])


def test_shape_and_workspace_errors(lib):
    from paper_0909_5662_gb300 import _capi
    import ctypes
    h = lib.default_handle()
    L = h.lib
    n = ctypes.c_size_t()
    assert L.dmrg_rotate_ops_workspace(h.h, 2, 4, 4, 17, 3, ctypes.byref(n)) == 2   # mp > m*d
    assert L.dmrg_rotate_ops_workspace(h.h, 2, 0, 4, 1, 3, ctypes.byref(n)) == 2
    assert L.dmrg_rotate_ops_workspace(h.h, 2, 4, 4, 4, 9, ctypes.byref(n)) == 1    # precision
    dev = torch.device("cuda")
    U = torch.zeros((16, 4), dtype=torch.float64, device=dev)
    O = torch.zeros((2, 4, 4), dtype=torch.float64, device=dev)
    out = torch.zeros((2, 4, 4), dtype=torch.float32, device=dev)
    ws = torch.zeros(16, dtype=torch.uint8, device=dev)
    st = L.dmrg_rotate_ops(h.h, ctypes.c_void_p(U.data_ptr()), 4, 4, 4, ctypes.c_void_p(O.data_ptr()), 1, 2,
                           ctypes.c_void_p(out.data_ptr()), 3, ctypes.c_void_p(ws.data_ptr()), 16, None)
    assert st == 4  # DMRG_ERR_WORKSPACE
    st = L.dmrg_rotate_ops(h.h, ctypes.c_void_p(U.data_ptr()), 4, 4, 4, ctypes.c_void_p(O.data_ptr()), 0, 2,
                           ctypes.c_void_p(out.data_ptr()), 0, ctypes.c_void_p(ws.data_ptr()), 16, None)
    assert st == 1  # FP64 path with FP32 operators


def test_orthonormality_error_gpu(lib):
    rng = np.random.default_rng(21)
    Q = orthonormal_columns(rng, 300, 77)
    for c in (1.0, 1.001, 0.5):
        got = lib.dmrg_orthonormality_error(torch.from_numpy(c * Q).cuda()).item()
        assert abs(got - oracle.orthonormality_error(c * Q)) < 1e-12


def test_correlations_gpu(lib):
    rng = np.random.default_rng(22)
    K, mp = 12, 70
    Op = rng.standard_normal((K, mp, mp))
    psi = rng.standard_normal(mp)
    psi /= np.linalg.norm(psi)
    ref = oracle.correlations(Op, psi)
    got = lib.dmrg_correlations(torch.from_numpy(Op).cuda(), torch.from_numpy(psi).cuda()).cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    got32 = lib.dmrg_correlations(torch.from_numpy(Op).cuda().float(), torch.from_numpy(psi).cuda()).cpu().numpy()
    ref32 = oracle.correlations(Op.astype(np.float32).astype(np.float64), psi)
    assert np.abs(got32 - ref32).max() <= 1e-12 * np.abs(ref32).max()


def test_correlations_gpu_chained_sweep_size(lib):
    # K = 300 operators of m' = 1200 (the chained-sweep workload's last step), FP32 and
    # FP64 operators holding the same values.  Every C_ij needs only O'_i and O'_j, so
    # the oracle recomputes the block of a seeded sample of operators (first and last
    # included) and the GPU's full K x K matrix is compared on that block.
    rng = np.random.default_rng(2300)
    K, mp = 300, 1200
    Op32 = rng.standard_normal((K, mp, mp), dtype=np.float32)
    psi = rng.standard_normal(mp)
    psi /= np.linalg.norm(psi)
    sample = np.unique(np.concatenate([[0, 1, K - 1], rng.choice(K, 21, replace=False)]))
    ref = oracle.correlations(Op32[sample].astype(np.float64), psi)
    dev = torch.device("cuda")
    O_dev = torch.from_numpy(Op32).to(dev)
    psi_dev = torch.from_numpy(psi).to(dev)
    for Ouse in (O_dev, O_dev.double()):
        got = lib.dmrg_correlations(Ouse, psi_dev).cpu().numpy()
        assert got.shape == (K, K)
        blk = got[np.ix_(sample, sample)]
        assert np.abs(blk - ref).max() <= 1e-12 * np.abs(ref).max(), Ouse.dtype
        del got


def test_full_size_m400_sampled(lib):
    # Full size of the benchmark workload (d=4, m=m'=400, K=150), launched as the
    # benchmark launches it; the oracle recomputes a seeded sample of operators.
    w = dense_config("dense_m400_k150")
    dev = torch.device("cuda")
    U = torch.from_numpy(w.U).to(dev)
    O32 = torch.from_numpy(w.O).to(dev, torch.float32)
    sample = np.random.default_rng(5).choice(w.K, 6, replace=False)
    sample = np.unique(np.concatenate([[0, 1, 2, w.K - 1], sample]))
    ref = oracle.rotate_dense(w.U, w.O[sample].astype(np.float32).astype(np.float64), 4)
    for prec in ("bf16x3", "tf32"):
        out = lib.dmrg_rotate_ops(U, O32, 4, prec)
        torch.cuda.synchronize()
        lib.dmrg_sync_status()
        got = out[torch.from_numpy(sample).to(dev)].double().cpu().numpy()
        assert rel_err(got, ref).max() <= TOL[prec], prec
    O64 = torch.from_numpy(w.O).to(dev)
    out = lib.dmrg_rotate_ops(U, O64, 4, "fp64")
    got = out[torch.from_numpy(sample).to(dev)].cpu().numpy()
    assert rel_err(got, oracle.rotate_dense(w.U, w.O[sample], 4)).max() <= TOL["fp64"]


@pytest.mark.parametrize("prec", ["bf16x3", "tf32", "fp64", "fp32"])
@pytest.mark.parametrize("chunk", [0, 1, 7, 100])
def test_host_buffer_pipeline(lib, prec, chunk):
    # dmrg_rotate_ops_host: host buffers in and out, chunked copy/compute overlap;
    # bit-identical to the device-buffer entry point on the same inputs when split
    # tiles are turned off (deterministic mode).
    w = dense_workload("host", 31, 4, 72, 64, 19)
    dt = torch.float64 if prec in ("fp64",) else torch.float32
    Uh = torch.from_numpy(w.U).pin_memory()
    Oh = torch.from_numpy(w.O).to(dt).pin_memory()
    h = lib.Handle()
    try:
        lib.dmrg_set_option("deterministic", 1, handle=h)
        out = lib.dmrg_rotate_ops_host(Uh, Oh, 4, prec, chunk=chunk, handle=h)
        ref_dev = lib.dmrg_rotate_ops(Uh.cuda(), Oh.cuda(), 4, prec, handle=h).cpu()
        lib.dmrg_sync_status(handle=h)
        assert torch.equal(out, ref_dev)
        # default mode (split tiles allowed): within the tolerance
        out2 = lib.dmrg_rotate_ops_host(Uh, Oh, 4, prec, chunk=chunk)
        lib.dmrg_sync_status()
        assert rel_err(out2.double().numpy(), out.double().numpy()).max() <= TOL[prec]
    finally:
        h.close()
    ref = oracle.rotate_dense(w.U, Oh.double().numpy(), 4)
    assert rel_err(out.double().numpy(), ref).max() <= TOL[prec]
