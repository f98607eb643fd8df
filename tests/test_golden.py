"""Stored fixtures under tests/golden/.

- umd_partition.txt: the block sizes of the uniform matrix distribution, written out
  from the rule stated in Sec. 3.2 (floor(L/p) operators per processor, one more for
  the first mod(L, p) processors).
- rotate_h4_m2_d2.txt: an exact rotation O'_k = U^T (O_k (x) I_d) U (Sec. 2, step 5)
  with U = H_4 / 2 and integer O_k, written by tests/golden/make_golden.py from the
  oracle.  Its values are checked here against identities that do not depend on the
  oracle (no truncation: trace and spectrum of O_k (x) I_d), and every precision of
  the CUDA path must reproduce them bit for bit, since every intermediate is a small
  dyadic rational.
"""
import os

import numpy as np
import pytest

import oracle

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_rotation():
    rows = [ln.split() for ln in open(os.path.join(HERE, "rotate_h4_m2_d2.txt"))
            if ln.strip() and not ln.startswith("#")]
    d, m, mp, K = (int(x) for x in rows[0])
    vals = [list(map(float, r)) for r in rows[1:]]
    U = np.array(vals[:m * d])
    pos = m * d
    O, Op = [], []
    for _ in range(K):
        O.append(vals[pos:pos + m])
        pos += m
        Op.append(vals[pos:pos + mp])
        pos += mp
    return d, U, np.array(O), np.array(Op)


def test_umd_partition_matches_the_papers_rule():
    from paper_0909_5662_gb300 import umd_partition
    for ln in open(os.path.join(HERE, "umd_partition.txt")):
        if not ln.strip() or ln.startswith("#"):
            continue
        L, p, *sizes = (int(x) for x in ln.split())
        assert len(sizes) == p and sum(sizes) == L
        parts = [umd_partition(L, p, r) for r in range(p)]
        assert [hi - lo for lo, hi in parts] == sizes
        assert parts[0][0] == 0 and all(parts[r][1] == parts[r + 1][0] for r in range(p - 1))


def test_golden_rotation_identities():
    d, U, O, Op = read_rotation()
    assert np.abs(U.T @ U - np.eye(U.shape[1])).max() == 0.0   # exactly orthonormal
    for k in range(len(O)):
        # no truncation: O'_k is similar to O_k (x) I_d
        assert np.trace(Op[k]) == d * np.trace(O[k])
        ev = np.sort_complex(np.linalg.eigvals(Op[k]))
        ev_ref = np.sort_complex(np.repeat(np.linalg.eigvals(O[k]), d))
        assert np.allclose(ev, ev_ref, atol=1e-12)
        assert np.all(Op[k] * 4 == np.round(Op[k] * 4))           # dyadic entries


def test_golden_rotation_reproduced_by_oracle():
    d, U, O, Op = read_rotation()
    assert np.array_equal(oracle.rotate_dense(U, O, d), Op)
    assert np.array_equal(oracle.rotate_dense_kron(U, O, d), Op)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3", "tf32"])
def test_golden_rotation_exact_on_gpu(prec):
    import torch
    import paper_0909_5662_gb300 as P
    d, U, O, Op = read_rotation()
    dev = torch.device("cuda")
    Ot = torch.from_numpy(O).to(dev, torch.float64 if prec == "fp64" else torch.float32)
    out = P.dmrg_rotate_ops(torch.from_numpy(U).to(dev), Ot, d, prec)
    torch.cuda.synchronize()
    P.dmrg_sync_status()
    assert np.array_equal(out.double().cpu().numpy(), Op), prec
