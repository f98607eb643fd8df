"""dmrg_rotate_ops_noalloc: the dense rotation for callers that cannot allocate.

Some callers cannot call cudaMalloc (a plug-in whose host program has already
reserved all device memory in its own pool, code under a fixed per-client
memory limit, or a loop where an allocation would synchronise the device).
This entry point takes no handle and no workspace; its scratch is a fixed
static device array inside the library.  The test calls it through the C ABI
twice in a row on different inputs and checks each result against
dmrg_rotate_ops on the same inputs and against the FP64 oracle, with the
tolerances of the other dense tests.  Two BF16x3 cases have m*d > 1024, so their
second product cuts the reduction into accumulation chains: two per tile at
m*d = 1200, summed in the output itself, and three at m*d = 2400, whose running
sums live in the static array too.  Finally an oversized problem must be refused
before any launch.  This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from workloads import dense_workload

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "bf16x3": 1e-5, "tf32": 3e-3}
PREC = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16x3": 3}


def _call_noalloc(lib, U, O, d, prec, out):
    K, m, _ = O.shape
    return lib.dmrg_rotate_ops_noalloc(
        ctypes.c_void_p(U.data_ptr()), m, d, U.shape[1], ctypes.c_void_p(O.data_ptr()),
        int(O.dtype == torch.float64), K, ctypes.c_void_p(out.data_ptr()), PREC[prec],
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    num = np.linalg.norm((a - b).reshape(len(b), -1), axis=1)
    return (num / np.linalg.norm(b.reshape(len(b), -1), axis=1)).max()


CASES = [
    # (prec, d, m, mp, K)
    ("fp64", 4, 64, 64, 32),
    ("bf16x3", 4, 64, 64, 32),
    ("tf32", 4, 64, 64, 32),
    ("fp32", 4, 64, 64, 32),
    # m*d = 1200 > 1024: two accumulation chains per tile, summed in the output
    ("bf16x3", 4, 300, 64, 8),
    # m*d = 2400: three chains, summed through the scratch in the static array (about 26 MB)
    ("bf16x3", 4, 600, 64, 2),
]


@pytest.mark.parametrize("prec,d,m,mp,K", CASES)
def test_noalloc_matches_dmrg_rotate_ops_twice(prec, d, m, mp, K):
    import paper_0909_5662_gb300 as P
    from paper_0909_5662_gb300 import _capi
    lib = _capi.load()
    dev = torch.device("cuda")
    odt = torch.float64 if prec == "fp64" else torch.float32
    for call, seed in enumerate((101, 202)):
        w = dense_workload("noalloc", seed + m, d, m, mp, K)
        U = torch.from_numpy(w.U).to(dev)
        O = torch.from_numpy(w.O).to(dev, torch.float64 if prec != "fp32" else torch.float32)
        ref = P.dmrg_rotate_ops(U, O, d, prec)
        out = torch.full((K, mp, mp), float("nan"), dtype=odt, device=dev)
        st = _call_noalloc(lib, U, O, d, prec, out)
        assert st == 0, (prec, call, _capi.STATUS.get(st))
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert _rel(out, ref) <= TOL[prec], (prec, call)
        # and against the FP64 oracle on the operators as the call saw them
        o_seen = O.double().cpu().numpy()
        exact = torch.from_numpy(oracle.rotate_dense(w.U, o_seen, d))
        assert _rel(out, exact) <= TOL[prec], (prec, call, "oracle")


def test_noalloc_refuses_problems_beyond_its_scratch():
    from paper_0909_5662_gb300 import _capi
    lib = _capi.load()
    dev = torch.device("cuda")
    # m = 400, K = 150 needs hundreds of MiB of scratch: refused with DMRG_ERR_WORKSPACE.
    U = torch.zeros((1600, 400), dtype=torch.float64, device=dev)
    O = torch.zeros((150, 400, 400), dtype=torch.float32, device=dev)
    out = torch.zeros((150, 400, 400), dtype=torch.float32, device=dev)
    assert _call_noalloc(lib, U, O, 4, "bf16x3", out) == 4
    # and an invalid shape is still refused as a shape error
    assert lib.dmrg_rotate_ops_noalloc(ctypes.c_void_p(U.data_ptr()), 4, 4, 17,
                                       ctypes.c_void_p(O.data_ptr()), 0, 1,
                                       ctypes.c_void_p(out.data_ptr()), 3, None) == 2
