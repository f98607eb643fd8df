"""Chained block-growth steps: the rotated operators of one step are the inputs of
the next (Sec. 2, algorithm steps 2-5 repeated).  Drift of the reduced precisions
against the FP64 GPU path stays bounded, and the first step of the FP64 path
matches the oracle."""
import numpy as np
import pytest
import torch

import oracle
from workloads import chained_inputs

pytestmark = pytest.mark.gpu


def test_chained_steps_drift():
    import paper_0909_5662_gb300 as P
    dev = torch.device("cuda")
    d, m, K, steps = 4, 160, 24, 8
    g = torch.Generator(device=dev)
    g.manual_seed(123)
    O0 = torch.randn(K, m, m, generator=g, dtype=torch.float64, device=dev)
    cur = {"bf16x3": O0.float(), "tf32": O0.float(), "fp64": O0.clone()}
    drift = {"bf16x3": [], "tf32": []}
    for step in range(steps):
        U = chained_inputs(step, m * d, m, dev)
        if step == 0:
            r0 = oracle.rotate_dense(U.cpu().numpy(), O0.cpu().numpy(), d)
        for p in cur:
            cur[p] = P.dmrg_rotate_ops(U, cur[p], d, p)
        if step == 0:
            got = cur["fp64"].cpu().numpy()
            err = np.linalg.norm((got - r0).reshape(K, -1), axis=1) / np.linalg.norm(r0.reshape(K, -1), axis=1)
            assert err.max() <= 1e-12
        ref = cur["fp64"]
        for p in drift:
            num = torch.linalg.vector_norm((cur[p].double() - ref).reshape(K, -1), dim=1)
            den = torch.linalg.vector_norm(ref.reshape(K, -1), dim=1)
            drift[p].append(float((num / den).max()))
    P.dmrg_sync_status()
    # single-step errors of about 1e-5 (BF16x3) and 1e-3 (TF32) accumulate at most
    # linearly in the number of steps
    assert drift["bf16x3"][0] <= 1e-5 and drift["bf16x3"][-1] <= steps * 1e-5
    assert drift["tf32"][0] <= 3e-3 and drift["tf32"][-1] <= steps * 3e-3
