"""GPU parity of the block-sparse U(1) x U(1) rotation (dmrg_rotate_ops_blocked)
against the oracle's per-sector loops (Sec. 3.1, Eq. (hache) labels)."""
import math

import numpy as np
import pytest
import torch

import oracle
from workloads import blocked_config, blocked_layout_sizes, orthonormal_columns, HUBBARD_SITE_SHIFTS

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "bf16x3": 1e-5, "tf32": 3e-3}
SITE = list(HUBBARD_SITE_SHIFTS)


@pytest.fixture(scope="module")
def P():
    import paper_0909_5662_gb300 as P
    return P


def per_op_slices(in_shapes, out_shapes):
    ins, outs, a, b = [], [], 0, 0
    for si, so in zip(in_shapes, out_shapes):
        n_in = sum(r * c for (r, c) in si)
        n_out = sum(r * c for (r, c) in so)
        ins.append((a, a + n_in))
        outs.append((b, b + n_out))
        a += n_in
        b += n_out
    return ins, outs


@pytest.fixture(scope="module")
def grouped_handle(P):
    """A handle on which every plan takes the grouped GEMM paths (the fused
    small-sector kernel switched off)."""
    h = P.Handle()
    P.dmrg_set_option("blocked_small", 0, handle=h)
    yield h
    h.close()


def run_gpu(P, w, prec, plan=None, handle=None):
    plan = plan or P.dmrg_blocked_plan_create(w.block_sectors, w.site_shifts, w.kept_sectors, w.op_shifts,
                                              handle=handle)
    dev = torch.device("cuda")
    U = torch.from_numpy(w.U_blocks).to(dev)
    O = torch.from_numpy(w.O_blocks).to(dev, torch.float64 if prec != "fp32" else torch.float32)
    out = P.dmrg_rotate_ops_blocked(plan, U, O, prec)
    torch.cuda.synchronize()
    P.dmrg_sync_status()
    return out.double().cpu().numpy(), plan


def rel_blocks(got, ref, out_shapes):
    """Maximum over operators of the relative Frobenius error of all the
    operator's blocks together (the per-operator metric of the dense tests)."""
    worst, pos = 0.0, 0
    for so in out_shapes:
        n = sum(r * c for (r, c) in so)
        g, f = got[pos:pos + n], ref[pos:pos + n]
        pos += n
        nf = np.linalg.norm(f)
        worst = max(worst, np.linalg.norm(g - f) / nf if nf > 0 else np.abs(g).max(initial=0.0))
    return worst


class W:
    def __init__(self, bs, ss, ks, os_, Ub, Ob, n_out):
        self.block_sectors, self.site_shifts, self.kept_sectors, self.op_shifts = bs, ss, ks, os_
        self.U_blocks, self.O_blocks, self.out_size = Ub, Ob, n_out


def random_structure(seed, nu=4, nd=3, maxdim=9, K=6, keep_frac=1.0):
    rng = np.random.default_rng(seed)
    sectors = [(a, b, int(rng.integers(1, maxdim + 1))) for a in range(nu) for b in range(nd)
               if rng.random() < 0.85]
    kept = [(a, b, max(1, int(math.ceil(n * keep_frac)))) for (a, b, n) in sectors]
    shifts = [[(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1), (1, -1)][k % 6] for k in range(K)]
    ush, ish, osh = blocked_layout_sizes(sectors, SITE, kept, shifts)
    Ub = np.concatenate([orthonormal_columns(rng, r, c).ravel() for (r, c) in ush])
    Ob = rng.standard_normal(sum(r * c for s in ish for (r, c) in s))
    return W(sectors, SITE, kept, shifts, Ub, Ob, sum(r * c for s in osh for (r, c) in s)), osh


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3", "tf32"])
@pytest.mark.parametrize("seed,maxdim,keep", [(1, 5, 1.0), (5, 32, 1.0), (2, 40, 0.7), (3, 130, 0.5)])
@pytest.mark.parametrize("grouped", [False, True])
def test_random_sectors(P, grouped_handle, prec, seed, maxdim, keep, grouped):
    # by default plans whose sectors all hold <= 32 states take the fused kernel (maxdim
    # 5 and 32), the others the grouped GEMMs; with the fused kernel switched off,
    # everything takes the grouped GEMMs
    w, osh = random_structure(seed, maxdim=maxdim, keep_frac=keep, K=7)
    ref = oracle.rotate_blocked(w.block_sectors, w.site_shifts, w.kept_sectors, w.op_shifts,
                                w.U_blocks, w.O_blocks if prec != "fp32" else
                                w.O_blocks.astype(np.float32).astype(np.float64), w.out_size)
    got, plan = run_gpu(P, w, prec, handle=grouped_handle if grouped else None)
    assert got.shape == ref.shape
    assert rel_blocks(got, ref, osh) <= TOL[prec]


def test_small_sector_kernel_is_fp32_accurate(P):
    # The fused small-sector kernel computes the reduced precisions in FP32: all of
    # them agree with the oracle to FP32 rounding, well inside their own bars.
    w, osh = random_structure(6, maxdim=16, K=9)
    ref = oracle.rotate_blocked(w.block_sectors, w.site_shifts, w.kept_sectors, w.op_shifts,
                                w.U_blocks, w.O_blocks.astype(np.float32).astype(np.float64), w.out_size)
    for prec in ("bf16x3", "tf32"):
        plan = P.dmrg_blocked_plan_create(w.block_sectors, w.site_shifts, w.kept_sectors, w.op_shifts)
        dev = torch.device("cuda")
        U = torch.from_numpy(w.U_blocks).to(dev)
        O = torch.from_numpy(w.O_blocks).to(dev, torch.float32)
        got = P.dmrg_rotate_ops_blocked(plan, U, O, prec).double().cpu().numpy()
        P.dmrg_sync_status()
        assert rel_blocks(got, ref, osh) <= 1e-6, prec


def test_plan_sizes_and_stats(P):
    w, osh = random_structure(4, maxdim=12, K=5)
    plan = P.dmrg_blocked_plan_create(w.block_sectors, w.site_shifts, w.kept_sectors, w.op_shifts)
    u, i, o, ws = plan.sizes("bf16x3")
    assert u == w.U_blocks.size and i == w.O_blocks.size and o == w.out_size and ws > 0
    n1, n2, flops = plan.stats()
    assert n1 > 0 and n2 > 0 and flops > 0


def test_plan_errors(P):
    from paper_0909_5662_gb300 import _capi
    with pytest.raises(_capi.DmrgError):   # repeated label
        P.dmrg_blocked_plan_create([(0, 0, 2), (0, 0, 3)], SITE, [(0, 0, 1)], [(0, 0)])
    with pytest.raises(_capi.DmrgError):   # kept sector larger than its [B a] sector
        P.dmrg_blocked_plan_create([(0, 0, 2)], SITE, [(0, 0, 5)], [(0, 0)])


@pytest.mark.parametrize("name", ["blocked_m1000_k200_s4", "blocked_m1000_k200_s1.2"])
def test_full_size_sampled(P, grouped_handle, name):
    # The full-size workloads in the launch configuration of the benchmark; the
    # oracle recomputes a sample of operators (each operator's output depends only on
    # its own blocks).
    w = blocked_config(name)
    ush, ish, osh = blocked_layout_sizes(w.block_sectors, w.site_shifts, w.kept_sectors, w.op_shifts)
    ins, outs = per_op_slices(ish, osh)
    sample = [0, 1, 2, 3, 4, 5, 6, 7, w.K - 1]
    for prec in ("bf16x3", "fp32", "fp64", "tf32"):
        got, _ = run_gpu(P, w, prec)
        # by default sigma = 4 (sectors of at most 10 states) takes the fused kernel;
        # the grouped GEMMs alone on a second handle
        got_g = run_gpu(P, w, prec, handle=grouped_handle)[0]
        for k in sample:
            (a, b), (c, e) = ins[k], outs[k]
            Ok = w.O_blocks[a:b] if prec != "fp32" else w.O_blocks[a:b].astype(np.float32).astype(np.float64)
            ref = oracle.rotate_blocked(w.block_sectors, w.site_shifts, w.kept_sectors,
                                        [w.op_shifts[k]], w.U_blocks, Ok, e - c)
            assert rel_blocks(got[c:e], ref, [osh[k]]) <= TOL[prec], (name, prec, k)
            assert rel_blocks(got_g[c:e], ref, [osh[k]]) <= TOL[prec], (name, prec, k)
