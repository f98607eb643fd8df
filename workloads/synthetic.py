"""Seeded input generators (no rotation arithmetic lives here).

Recipes (each seeded with ``SEED_BASE + config index`` through NumPy's PCG64):

``dense_m64_k32``    d=4, m=64 -> m*d=256 -> m'=64.  U = first 64 columns of
                     Q from the QR of a 256x256 N(0,1) matrix (signs fixed so
                     diag(R) >= 0); K=32 operators with N(0,1) entries.
``dense_m400_k150``  d=4, m=400 -> 1600 -> m'=400; U from the QR of a
                     1600x1600 N(0,1) matrix; K=150 operators = 50 sites x
                     {n_up-like: diagonal Bernoulli(1/2) plus 1e-3*N(0,1)
                     dense noise, and two N(0,1) dense operators}.
``blocked_*``        U(1)xU(1) sectors (N_up, N_dn) in [0, 40]^2; m=1000 block
                     states split by a discretised 2-D Gaussian centred at
                     (20, 20) with largest-remainder rounding; site shifts of
                     (0, up, down, up-down); kept sectors = block sectors
                     (m'_Q = m_Q); per-sector orthonormal U blocks; K=200
                     operators, alternately sector-diagonal and shifting by
                     (+1,0), (-1,0), (0,+1), (0,-1), with N(0,1) blocks.
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence, Tuple

import numpy as np

SEED_BASE = 0x5662 * 10

# Local site basis (0, up, down, up-down): quantum-number shift of each state.
HUBBARD_SITE_SHIFTS: Tuple[Tuple[int, int], ...] = ((0, 0), (1, 0), (0, 1), (1, 1))


def orthonormal_columns(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    """First ``cols`` columns of Q from the QR factorisation of a seeded
    ``rows`` x ``rows`` N(0,1) matrix, with column signs chosen so that
    diag(R) >= 0 (which makes the factor unique)."""
    A = rng.standard_normal((rows, rows))
    Q, R = np.linalg.qr(A[:, :cols])
    sgn = np.sign(np.diag(R))
    sgn[sgn == 0] = 1.0
    return np.ascontiguousarray(Q * sgn[None, :])


@dataclasses.dataclass
class DenseWorkload:
    name: str
    d: int
    m: int
    mp: int
    U: np.ndarray      # (m*d) x mp, FP64, orthonormal columns
    O: np.ndarray      # K x m x m, FP64

    @property
    def K(self) -> int:
        return int(self.O.shape[0])

    def flops(self) -> float:
        """Logical multiply-add flops of one rotation step (both products)."""
        return 2.0 * self.K * self.d * self.m * self.mp * (self.m + self.mp)


def dense_workload(name: str, seed: int, d: int, m: int, mp: int, K: int,
                   hubbard_mix: bool = False) -> DenseWorkload:
    rng = np.random.default_rng(seed)
    U = orthonormal_columns(rng, m * d, mp)
    if not hubbard_mix:
        O = rng.standard_normal((K, m, m))
    else:
        O = np.empty((K, m, m))
        for k in range(K):
            if k % 3 == 0:
                diag = rng.integers(0, 2, size=m).astype(np.float64)
                O[k] = 1e-3 * rng.standard_normal((m, m))
                O[k][np.arange(m), np.arange(m)] += diag
            else:
                O[k] = rng.standard_normal((m, m))
    return DenseWorkload(name, d, m, mp, U, O)


def dense_config(name: str) -> DenseWorkload:
    if name == "dense_m64_k32":
        return dense_workload(name, SEED_BASE + 1, 4, 64, 64, 32)
    if name == "dense_m400_k150":
        return dense_workload(name, SEED_BASE + 2, 4, 400, 400, 150, hubbard_mix=True)
    raise KeyError(name)


def backward_upstream(seed: int, K: int, mp: int) -> np.ndarray:
    """Seeded N(0,1) upstream gradient dO'_k (K x m' x m')."""
    return np.random.default_rng(seed).standard_normal((K, mp, mp))


# ----------------------------------------------------------------------------
# Block-sparse workloads.
# ----------------------------------------------------------------------------

def gaussian_sector_split(m: int, sigma: float, center=(20, 20), nmax: int = 40):
    """Split ``m`` states over sectors (N_up, N_dn) in [0, nmax]^2 in
    proportion to exp(-|N - center|^2 / (2 sigma^2)), largest-remainder
    rounding; sectors that receive zero states are dropped.  Returns a list of
    (N_up, N_dn, dim) in row-major (N_up, N_dn) order."""
    a = np.arange(nmax + 1)
    uu, dd = np.meshgrid(a, a, indexing="ij")
    w = np.exp(-((uu - center[0]) ** 2 + (dd - center[1]) ** 2) / (2.0 * sigma * sigma)).ravel()
    share = m * w / w.sum()
    base = np.floor(share).astype(np.int64)
    rem = m - int(base.sum())
    order = np.argsort(-(share - base), kind="stable")
    base[order[:rem]] += 1
    out = []
    for idx in range(base.size):
        if base[idx] > 0:
            out.append((int(uu.ravel()[idx]), int(dd.ravel()[idx]), int(base[idx])))
    return out


def blocked_layout_sizes(block_sectors, site_shifts, kept_sectors, op_shifts):
    """Bookkeeping of the canonical block storage (no arithmetic on values):
    returns (U block shapes, per-op input block shapes, per-op output block
    shapes) following the layout documented in ``include/dmrg_rotate.h``."""
    bdim = {(u, dn): n for (u, dn, n) in block_sectors}
    kdim = {(u, dn): n for (u, dn, n) in kept_sectors}
    u_shapes = []
    for (u, dn, n) in kept_sectors:
        rows = sum(bdim.get((u - su, dn - sd), 0) for (su, sd) in site_shifts)
        u_shapes.append((rows, n))
    in_shapes, out_shapes = [], []
    for (du, dd) in op_shifts:
        ins = [(bdim[(u + du, dn + dd)], n) for (u, dn, n) in block_sectors
               if (u + du, dn + dd) in bdim]
        outs = [(kdim[(u + du, dn + dd)], n) for (u, dn, n) in kept_sectors
                if (u + du, dn + dd) in kdim]
        in_shapes.append(ins)
        out_shapes.append(outs)
    return u_shapes, in_shapes, out_shapes


@dataclasses.dataclass
class BlockedWorkload:
    name: str
    block_sectors: List[Tuple[int, int, int]]
    site_shifts: List[Tuple[int, int]]
    kept_sectors: List[Tuple[int, int, int]]
    op_shifts: List[Tuple[int, int]]
    U_blocks: np.ndarray   # flat FP64
    O_blocks: np.ndarray   # flat FP64
    out_size: int

    @property
    def K(self) -> int:
        return len(self.op_shifts)

    @property
    def d(self) -> int:
        return len(self.site_shifts)


def blocked_workload(name: str, seed: int, block_sectors, site_shifts, kept_sectors,
                     op_shifts) -> BlockedWorkload:
    rng = np.random.default_rng(seed)
    u_shapes, in_shapes, out_shapes = blocked_layout_sizes(block_sectors, site_shifts,
                                                           kept_sectors, op_shifts)
    Ub = [orthonormal_columns(rng, r, c).ravel() for (r, c) in u_shapes]
    U_blocks = np.concatenate(Ub) if Ub else np.zeros(0)
    n_in = sum(r * c for shp in in_shapes for (r, c) in shp)
    O_blocks = rng.standard_normal(n_in)
    n_out = sum(r * c for shp in out_shapes for (r, c) in shp)
    return BlockedWorkload(name, list(block_sectors), list(site_shifts), list(kept_sectors),
                           list(op_shifts), U_blocks, O_blocks, int(n_out))


def blocked_op_shifts(K: int) -> List[Tuple[int, int]]:
    shifts = [(1, 0), (-1, 0), (0, 1), (0, -1)]
    return [(0, 0) if k % 2 == 0 else shifts[(k // 2) % 4] for k in range(K)]


def blocked_config(name: str) -> BlockedWorkload:
    """``blocked_m1000_k200_s4``: the literal sigma = 4 law (many small
    sectors); ``blocked_m1000_k200_s1.2``: sigma = 1.2, which realises block
    sizes of roughly 1-111 states."""
    if name == "blocked_m1000_k200_s4":
        sigma, seed = 4.0, SEED_BASE + 3
    elif name == "blocked_m1000_k200_s1.2":
        sigma, seed = 1.2, SEED_BASE + 33
    else:
        raise KeyError(name)
    sectors = gaussian_sector_split(1000, sigma)
    return blocked_workload(name, seed, sectors, list(HUBBARD_SITE_SHIFTS), sectors,
                            blocked_op_shifts(200))


# ----------------------------------------------------------------------------
# Chained sweep inputs (50 steps at m = 1200): generated with torch on the
# target device, because 50 QR factorisations of 4800 x 1200 on the host take
# minutes.  Only input generation uses torch's linear algebra here.
# ----------------------------------------------------------------------------

def chained_inputs(step: int, md: int, mp: int, device, seed: int = SEED_BASE + 5):
    """Orthonormal U for sweep step ``step`` (first mp columns of Q of a seeded
    md x md N(0,1) matrix, diag(R) >= 0), as an FP64 torch tensor on
    ``device``."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed * 1000 + step)
    A = torch.randn(md, mp, generator=g, dtype=torch.float64, device=device)
    Q, R = torch.linalg.qr(A)
    sgn = torch.sign(torch.diagonal(R))
    sgn[sgn == 0] = 1.0
    return (Q * sgn[None, :]).contiguous()



# ----------------------------------------------------------------------------
# Inputs of the stages around the rotation: the truncation matrix, the blocked
# site operators and the measurement stage.
# ----------------------------------------------------------------------------

def schmidt_state(seed: int, rows: int, cols: int, xi: float = 20.0) -> np.ndarray:
    """Unit-norm superblock state Psi (rows x cols) with a ground-state-like
    Schmidt spectrum: Psi = L diag(sqrt(w)) R^T with seeded orthonormal L and R
    and weights w_k proportional to exp(-k / xi), k = 0 .. min(rows, cols) - 1."""
    rng = np.random.default_rng(seed)
    r = min(rows, cols)
    w = np.exp(-np.arange(r) / xi)
    w /= w.sum()
    Lm = orthonormal_columns(rng, rows, r)
    Rm = orthonormal_columns(rng, cols, r)
    return np.ascontiguousarray((Lm * np.sqrt(w)[None, :]) @ Rm.T)


# Hubbard site operators in the local basis (0, up, down, up-down), with the up mode
# before the down mode inside the site: c_up, c_dn, their adjoints, n_up, n_dn.
_C_UP = np.array([[0, 1, 0, 0], [0, 0, 0, 0], [0, 0, 0, 1], [0, 0, 0, 0]], dtype=np.float64)
_C_DN = np.array([[0, 0, 1, 0], [0, 0, 0, -1], [0, 0, 0, 0], [0, 0, 0, 0]], dtype=np.float64)
HUBBARD_SITE_OPS = {
    "c_up": (_C_UP, 1), "c_dn": (_C_DN, 1), "cdag_up": (_C_UP.T.copy(), 1),
    "cdag_dn": (_C_DN.T.copy(), 1), "n_up": (_C_UP.T @ _C_UP, 0), "n_dn": (_C_DN.T @ _C_DN, 0),
}


@dataclasses.dataclass
class SiteWorkload:
    name: str
    d: int
    m: int
    mp: int
    U: np.ndarray        # (m*d) x mp, FP64
    A: np.ndarray        # K x m x m, FP64, ordered by class
    S: np.ndarray        # n_class x d x d, FP64
    counts: np.ndarray   # n_class, int64
    flags: np.ndarray    # n_class, int64 (1: the class carries the block parity)
    parity: np.ndarray   # m, int8 (+1 / -1)

    @property
    def K(self) -> int:
        return int(self.A.shape[0])


def site_workload(seed: int = SEED_BASE + 6, m: int = 400, mp: int = 400, per_class: int = 25) -> SiteWorkload:
    """``site_m400_k150``: d = 4, m = m' = 400, the six Hubbard site operators as
    classes of 25 block operators each (K = 150); block operators N(0,1), block
    parity of every block state Bernoulli(1/2) in {+1, -1}."""
    rng = np.random.default_rng(seed)
    d = 4
    U = orthonormal_columns(rng, m * d, mp)
    names = list(HUBBARD_SITE_OPS)
    S = np.stack([HUBBARD_SITE_OPS[k][0] for k in names])
    flags = np.array([HUBBARD_SITE_OPS[k][1] for k in names], dtype=np.int64)
    counts = np.full(len(names), per_class, dtype=np.int64)
    A = rng.standard_normal((per_class * len(names), m, m))
    parity = np.where(rng.integers(0, 2, size=m) == 1, 1, -1).astype(np.int8)
    return SiteWorkload("site_m400_k150", d, m, mp, U, A, S, counts, flags, parity)


@dataclasses.dataclass
class MeasureWorkload:
    name: str
    Psi: np.ndarray      # rows x cols, FP64, unit norm
    Z: np.ndarray        # Ks x rows x rows (system operators), FP32
    W: np.ndarray        # Ke x cols x cols (environment operators), FP32
    G: np.ndarray        # L x L two-point matrix, FP64, symmetric
    v: np.ndarray        # L one-point values


def measure_workload(seed: int = SEED_BASE + 7, n: int = 1600, Ks: int = 150, Ke: int = 50,
                     L: int = 128) -> MeasureWorkload:
    """``measure_m400``: the superblock state of the d = 4, m = 400 step as an
    n x n (n = m d = 1600) matrix with a ground-state-like Schmidt spectrum, Ks
    system operators and Ke environment operators on the [B a] bases (N(0,1), drawn
    in FP32, the operators' storage precision),
    and an L = 128 two-point matrix (symmetric N(0,1)) with one-point values
    for the structure factor."""
    Psi = schmidt_state(seed, n, n)
    rng = np.random.default_rng(seed + 1)
    Z = rng.standard_normal((Ks, n, n), dtype=np.float32)
    W = rng.standard_normal((Ke, n, n), dtype=np.float32)
    X = rng.standard_normal((L, L))
    return MeasureWorkload("measure_m400", Psi, Z, W, X + X.T, rng.standard_normal(L))
