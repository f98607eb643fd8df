"""torch-tensor front-end of the C ABI (argument marshalling only)."""
from __future__ import annotations

import ctypes
import json
from typing import Optional, Sequence, Tuple

import numpy as np
import torch

from . import _capi

PRECISIONS = tuple(_capi.PRECISION)


def _prec(p) -> int:
    if isinstance(p, int):
        return p
    try:
        return _capi.PRECISION[p.lower()]
    except KeyError:
        raise ValueError("precision must be one of %s" % (PRECISIONS,))


def _ptr(t: Optional[torch.Tensor]):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _need(t: torch.Tensor, name: str, dtypes, dims=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor" % name)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype not in dtypes:
        raise TypeError("%s must have dtype in %s, got %s" % (name, dtypes, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if dims is not None and t.dim() != dims:
        raise ValueError("%s must have %d dimensions" % (name, dims))


class Handle:
    """Owns a dmrg_handle (bound to the current device) and a growable workspace."""

    def __init__(self, device=None):
        self.lib = _capi.load()
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.device = dev
        with torch.cuda.device(dev):
            h = ctypes.c_void_p()
            _capi.check(self.lib.dmrg_create(ctypes.byref(h)), None, "dmrg_create")
        self.h = h
        self._ws = None

    def workspace(self, nbytes: int) -> torch.Tensor:
        if self._ws is None or self._ws.numel() < nbytes:
            # torch's caching allocator hands out 512-byte aligned blocks
            self._ws = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=self.device)
        return self._ws

    def close(self):
        if self.h:
            self.lib.dmrg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_handles = {}


def default_handle(device=None) -> Handle:
    idx = torch.cuda.current_device() if device is None else torch.device(device).index
    h = _handles.get(idx)
    if h is None:
        with torch.cuda.device(idx):
            h = Handle(torch.device("cuda", idx))
        _handles[idx] = h
    return h


def dmrg_set_option(option: str, value: float, handle: Optional[Handle] = None):
    h = handle or default_handle()
    _capi.check(h.lib.dmrg_set_option(h.h, _capi.OPTION[option], float(value)), h.h, option)


def dmrg_kernel_timing(reset: bool = True, handle: Optional[Handle] = None):
    h = handle or default_handle()
    buf = ctypes.create_string_buffer(1 << 16)
    _capi.check(h.lib.dmrg_kernel_timing(h.h, buf, len(buf), int(reset)), h.h, "timing")
    return json.loads(buf.value.decode())


def dmrg_sync_status(handle: Optional[Handle] = None, stream=None):
    h = handle or default_handle()
    _capi.check(h.lib.dmrg_sync_status(h.h, _stream(stream)), h.h, "dmrg_sync_status")


def dmrg_rotate_ops_workspace(K: int, m: int, d: int, mp: int, precision="bf16x3",
                              handle: Optional[Handle] = None) -> int:
    h = handle or default_handle()
    n = ctypes.c_size_t()
    _capi.check(h.lib.dmrg_rotate_ops_workspace(h.h, K, m, d, mp, _prec(precision), ctypes.byref(n)),
                h.h, "dmrg_rotate_ops_workspace")
    return n.value


def _dense_args(U, O, d, precision):
    _need(U, "U", (torch.float64,), 2)
    _need(O, "O", (torch.float64, torch.float32), 3)
    K, m, m2 = O.shape
    if m != m2:
        raise ValueError("operators must be square")
    if U.shape[0] != m * d:
        raise ValueError("U must have m*d rows")
    return K, m, U.shape[1], _prec(precision)


def dmrg_rotate_ops(U: torch.Tensor, O: torch.Tensor, d: int, precision="bf16x3",
                    out: Optional[torch.Tensor] = None, handle: Optional[Handle] = None,
                    stream=None, _entry: str = "dmrg_rotate_ops") -> torch.Tensor:
    """O'_k = U^T (O_k (x) I_d) U for every k.  U: (m*d) x m' FP64; O: K x m x m
    (FP64 or FP32).  Returns K x m' x m' (FP64 for precision fp64, else FP32)."""
    h = handle or default_handle()
    K, m, mp, p = _dense_args(U, O, d, precision)
    odt = torch.float64 if p == 0 else torch.float32
    if out is None:
        out = torch.empty((K, mp, mp), dtype=odt, device=O.device)
    _need(out, "out", (odt,), 3)
    nbytes = dmrg_rotate_ops_workspace(K, m, d, mp, p, h)
    ws = h.workspace(nbytes)
    fn = getattr(h.lib, _entry)
    _capi.check(fn(h.h, _ptr(U), m, d, mp, _ptr(O), int(O.dtype == torch.float64), K, _ptr(out),
                   p, _ptr(ws), ws.numel(), _stream(stream)), h.h, _entry)
    return out


def _need_host(t: torch.Tensor, name: str, dtypes, dims=None):
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise ValueError("%s must be a host (CPU) tensor" % name)
    if t.dtype not in dtypes:
        raise TypeError("%s must have dtype in %s, got %s" % (name, dtypes, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if dims is not None and t.dim() != dims:
        raise ValueError("%s must have %d dimensions" % (name, dims))


def dmrg_rotate_ops_host(U: torch.Tensor, O: torch.Tensor, d: int, precision="bf16x3",
                         out: Optional[torch.Tensor] = None, chunk: int = 0,
                         handle: Optional[Handle] = None, stream=None,
                         synchronize: bool = True) -> torch.Tensor:
    """The rotation with U, O and the result in host memory (pin them with
    ``tensor.pin_memory()`` for copies that overlap the kernels)."""
    h = handle or default_handle()
    _need_host(U, "U", (torch.float64,), 2)
    _need_host(O, "O", (torch.float64, torch.float32), 3)
    K, m, m2 = O.shape
    if m != m2 or U.shape[0] != m * d:
        raise ValueError("shape mismatch")
    mp = U.shape[1]
    p = _prec(precision)
    odt = torch.float64 if p == 0 else torch.float32
    if out is None:
        out = torch.empty((K, mp, mp), dtype=odt, pin_memory=True)
    _need_host(out, "out", (odt,), 3)
    f64 = int(O.dtype == torch.float64)
    n = ctypes.c_size_t()
    _capi.check(h.lib.dmrg_rotate_ops_host_workspace(h.h, K, m, d, mp, p, f64, chunk, ctypes.byref(n)),
                h.h, "dmrg_rotate_ops_host_workspace")
    ws = h.workspace(n.value)
    st = _stream(stream)
    _capi.check(h.lib.dmrg_rotate_ops_host(h.h, _ptr(U), m, d, mp, _ptr(O), f64, K, _ptr(out), p, chunk,
                                           _ptr(ws), ws.numel(), st), h.h, "dmrg_rotate_ops_host")
    if synchronize:
        (torch.cuda.current_stream() if stream is None else stream).synchronize()
    return out


def dmrg_rotate_ops_noalloc(U: torch.Tensor, O: torch.Tensor, d: int, precision="bf16x3",
                            out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """The dense rotation with no handle and no workspace: scratch is the
    library's fixed 32 MiB static device array (small problems only)."""
    lib = _capi.load()
    K, m, mp, p = _dense_args(U, O, d, precision)
    odt = torch.float64 if p == 0 else torch.float32
    if out is None:
        out = torch.empty((K, mp, mp), dtype=odt, device=O.device)
    _need(out, "out", (odt,), 3)
    _capi.check(lib.dmrg_rotate_ops_noalloc(_ptr(U), m, d, mp, _ptr(O), int(O.dtype == torch.float64),
                                            K, _ptr(out), p, _stream(stream)),
                None, "dmrg_rotate_ops_noalloc")
    return out


def dmrg_autotune_rotate_ops(U, O, d, precision="bf16x3", out=None, handle=None, stream=None):
    return dmrg_rotate_ops(U, O, d, precision, out, handle, stream, _entry="dmrg_autotune_rotate_ops")


def dmrg_rotate_ops_backward(U: torch.Tensor, O: torch.Tensor, G: torch.Tensor, d: int,
                             precision="bf16x3", want_dO: bool = True, want_dU: bool = True,
                             handle: Optional[Handle] = None, stream=None
                             ) -> Tuple[Optional[torch.Tensor], Optional[torch.Tensor]]:
    """Adjoint for dL/dO'_k = G_k: returns (dO, dU)."""
    h = handle or default_handle()
    K, m, mp, p = _dense_args(U, O, d, precision)
    _need(G, "G", (O.dtype,), 3)
    if tuple(G.shape) != (K, mp, mp):
        raise ValueError("G must be K x m' x m'")
    odt = torch.float64 if p == 0 else torch.float32
    dO = torch.empty((K, m, m), dtype=odt, device=O.device) if want_dO else None
    dU = torch.empty_like(U) if want_dU else None
    n = ctypes.c_size_t()
    _capi.check(h.lib.dmrg_rotate_ops_backward_workspace(h.h, K, m, d, mp, p, ctypes.byref(n)),
                h.h, "dmrg_rotate_ops_backward_workspace")
    ws = h.workspace(n.value)
    _capi.check(h.lib.dmrg_rotate_ops_backward(
        h.h, _ptr(U), m, d, mp, _ptr(O), _ptr(G), int(O.dtype == torch.float64), K, _ptr(dO),
        _ptr(dU), p, _ptr(ws), ws.numel(), _stream(stream)), h.h, "dmrg_rotate_ops_backward")
    return dO, dU


def dmrg_rotate_site_ops(U: torch.Tensor, A: torch.Tensor, d: int, S, counts, flags,
                         parity: Optional[torch.Tensor] = None, precision="bf16x3",
                         out: Optional[torch.Tensor] = None, handle: Optional[Handle] = None,
                         stream=None) -> torch.Tensor:
    """Blocked site and cross operators: O'_k = U^T ((A_k P^f_c) (x) S_c) U.

    A: K x m x m on the device (operators ordered by class); S: n_class x d x d site
    matrices (host data, any array-like); counts / flags: per class, host; parity:
    m entries of +-1 (int8) on the device, needed when a flag is set."""
    h = handle or default_handle()
    K, m, mp, p = _dense_args(U, A, d, precision)
    S_np = np.ascontiguousarray(np.asarray(S, dtype=np.float64).reshape(-1, d, d))
    counts_np = np.ascontiguousarray(np.asarray(counts, dtype=np.int64).reshape(-1))
    flags_np = np.ascontiguousarray(np.asarray(flags, dtype=np.int32).reshape(-1))
    if not (len(S_np) == len(counts_np) == len(flags_np)):
        raise ValueError("S, counts and flags need one entry per class")
    if parity is not None:
        _need(parity, "parity", (torch.int8,), 1)
    odt = torch.float64 if p == 0 else torch.float32
    if out is None:
        out = torch.empty((K, mp, mp), dtype=odt, device=A.device)
    n = ctypes.c_size_t()
    _capi.check(h.lib.dmrg_rotate_site_ops_workspace(h.h, K, m, d, mp, p, ctypes.byref(n)),
                h.h, "dmrg_rotate_site_ops_workspace")
    ws = h.workspace(n.value)
    _capi.check(h.lib.dmrg_rotate_site_ops(
        h.h, _ptr(U), m, d, mp, _ptr(A), int(A.dtype == torch.float64), K, len(counts_np),
        S_np.ctypes.data_as(ctypes.c_void_p), counts_np.ctypes.data_as(ctypes.c_void_p),
        flags_np.ctypes.data_as(ctypes.c_void_p), _ptr(parity) if parity is not None else None,
        _ptr(out), p, _ptr(ws), ws.numel(), _stream(stream)), h.h, "dmrg_rotate_site_ops")
    return out


def dmrg_expectation(Z: torch.Tensor, Psi: torch.Tensor, side: int = 0,
                     handle: Optional[Handle] = None, stream=None) -> torch.Tensor:
    """<psi0| Z_k (x) I |psi0> (side 0) or <psi0| I (x) Z_k |psi0> (side 1) for the
    superblock state psi0 = sum Psi[a][e] |a>|e>; K FP64 values."""
    h = handle or default_handle()
    _need(Z, "Z", (torch.float64, torch.float32), 3)
    _need(Psi, "Psi", (torch.float64,), 2)
    rows, cols = Psi.shape
    K = Z.shape[0]
    out = torch.empty(K, dtype=torch.float64, device=Z.device)
    n = ctypes.c_size_t()
    _capi.check(h.lib.dmrg_expectation_workspace(h.h, K, rows, cols, int(side), ctypes.byref(n)),
                h.h, "dmrg_expectation_workspace")
    ws = h.workspace(n.value)
    _capi.check(h.lib.dmrg_expectation(h.h, _ptr(Z), int(Z.dtype == torch.float64), K, _ptr(Psi), rows,
                                       cols, int(side), _ptr(out), _ptr(ws), ws.numel(), _stream(stream)),
                h.h, "dmrg_expectation")
    return out


def dmrg_cross_correlations(Z: torch.Tensor, W: torch.Tensor, Psi: torch.Tensor,
                            handle: Optional[Handle] = None, stream=None) -> torch.Tensor:
    """C[i][j] = <psi0| Z_i (x) W_j |psi0>: Z on the system, W on the environment."""
    h = handle or default_handle()
    _need(Z, "Z", (torch.float64, torch.float32), 3)
    _need(W, "W", (torch.float64, torch.float32), 3)
    _need(Psi, "Psi", (torch.float64,), 2)
    rows, cols = Psi.shape
    Ks, Ke = Z.shape[0], W.shape[0]
    C = torch.empty((Ks, Ke), dtype=torch.float64, device=Z.device)
    z64, w64 = int(Z.dtype == torch.float64), int(W.dtype == torch.float64)
    n = ctypes.c_size_t()
    _capi.check(h.lib.dmrg_cross_correlations_workspace(h.h, Ks, Ke, rows, cols, z64, w64,
                                                        ctypes.byref(n)),
                h.h, "dmrg_cross_correlations_workspace")
    ws = h.workspace(n.value)
    _capi.check(h.lib.dmrg_cross_correlations(h.h, _ptr(Z), z64, Ks, _ptr(W), w64, Ke, _ptr(Psi), rows,
                                              cols, _ptr(C), _ptr(ws), ws.numel(), _stream(stream)),
                h.h, "dmrg_cross_correlations")
    return C


def dmrg_structure_factor(G: torch.Tensor, v: Optional[torch.Tensor] = None, c: float = 0.0,
                          handle: Optional[Handle] = None, stream=None):
    """F(q_p) = (1/L) sum_{k,j} e^{i q_p (k-j)} <(X_k - c)(X_j - c)> for q_p = 2 pi p / L,
    from G = <X_k X_j> (L x L) and v = <X_k>; returns (real part, imaginary part)."""
    h = handle or default_handle()
    _need(G, "G", (torch.float64,), 2)
    L = G.shape[0]
    if v is not None:
        _need(v, "v", (torch.float64,), 1)
    re = torch.empty(L, dtype=torch.float64, device=G.device)
    im = torch.empty(L, dtype=torch.float64, device=G.device)
    _capi.check(h.lib.dmrg_structure_factor(h.h, _ptr(G), _ptr(v) if v is not None else None, float(c), L,
                                            _ptr(re), _ptr(im), _stream(stream)),
                h.h, "dmrg_structure_factor")
    return re, im


def dmrg_truncation(Psi: torch.Tensor, mp: int, tol: float = 1e-14, max_sweeps: int = 30,
                    handle: Optional[Handle] = None, stream=None):
    """Truncation matrix from the superblock state Psi (rows x cols, FP64): returns
    (U rows x mp, all eigenvalues of rho = Psi Psi^T in decreasing order, the discarded
    weight eps as a 1-element tensor, sweeps done)."""
    h = handle or default_handle()
    _need(Psi, "Psi", (torch.float64,), 2)
    rows, cols = Psi.shape
    U = torch.empty((rows, mp), dtype=torch.float64, device=Psi.device)
    lam = torch.empty(rows, dtype=torch.float64, device=Psi.device)
    eps = torch.empty(1, dtype=torch.float64, device=Psi.device)
    n = ctypes.c_size_t()
    _capi.check(h.lib.dmrg_truncation_workspace(h.h, rows, cols, ctypes.byref(n)), h.h,
                "dmrg_truncation_workspace")
    ws = h.workspace(n.value)
    sweeps = ctypes.c_int()
    _capi.check(h.lib.dmrg_truncation(h.h, _ptr(Psi), rows, cols, int(mp), _ptr(U), _ptr(lam), _ptr(eps),
                                      float(tol), int(max_sweeps), ctypes.byref(sweeps), _ptr(ws),
                                      ws.numel(), _stream(stream)), h.h, "dmrg_truncation")
    return U, lam, eps, sweeps.value


def dmrg_orthonormality_error(U: torch.Tensor, handle: Optional[Handle] = None, stream=None
                              ) -> torch.Tensor:
    """||U^T U - I||_F in FP64 as a 1-element device tensor."""
    h = handle or default_handle()
    _need(U, "U", (torch.float64,), 2)
    out = torch.empty(1, dtype=torch.float64, device=U.device)
    n = ctypes.c_size_t()
    _capi.check(h.lib.dmrg_orthonormality_error_workspace(h.h, U.shape[0], U.shape[1], ctypes.byref(n)),
                h.h, "workspace")
    ws = h.workspace(n.value)
    _capi.check(h.lib.dmrg_orthonormality_error(h.h, _ptr(U), U.shape[0], U.shape[1], _ptr(out),
                                                _ptr(ws), ws.numel(), _stream(stream)),
                h.h, "dmrg_orthonormality_error")
    return out


def dmrg_correlations(Op: torch.Tensor, psi: torch.Tensor, handle: Optional[Handle] = None,
                      stream=None) -> torch.Tensor:
    """C[i, j] = <psi| O'_i O'_j |psi> in FP64."""
    h = handle or default_handle()
    _need(Op, "Op", (torch.float64, torch.float32), 3)
    _need(psi, "psi", (torch.float64,), 1)
    K, mp, _ = Op.shape
    C = torch.empty((K, K), dtype=torch.float64, device=Op.device)
    n = ctypes.c_size_t()
    _capi.check(h.lib.dmrg_correlations_workspace(h.h, K, mp, ctypes.byref(n)), h.h, "workspace")
    ws = h.workspace(n.value)
    _capi.check(h.lib.dmrg_correlations(h.h, _ptr(Op), int(Op.dtype == torch.float64), _ptr(psi),
                                        K, mp, _ptr(C), _ptr(ws), ws.numel(), _stream(stream)),
                h.h, "dmrg_correlations")
    return C


# ---------------------------------------------------------------------------- blocked
class BlockedPlan:
    """Owns a dmrg_blocked_plan: the grouped problem lists of a fixed sector structure."""

    def __init__(self, block_sectors, site_shifts, kept_sectors, op_shifts,
                 handle: Optional[Handle] = None):
        self.handle = handle or default_handle()
        lib = self.handle.lib
        bs = (_capi.DmrgQnSector * max(1, len(block_sectors)))(*[_capi.DmrgQnSector(*s) for s in block_sectors])
        ss = (_capi.DmrgQnShift * max(1, len(site_shifts)))(*[_capi.DmrgQnShift(*s) for s in site_shifts])
        ks = (_capi.DmrgQnSector * max(1, len(kept_sectors)))(*[_capi.DmrgQnSector(*s) for s in kept_sectors])
        os_ = (_capi.DmrgQnShift * max(1, len(op_shifts)))(*[_capi.DmrgQnShift(*s) for s in op_shifts])
        p = ctypes.c_void_p()
        _capi.check(lib.dmrg_blocked_plan_create(self.handle.h, bs, len(block_sectors), ss,
                                                 len(site_shifts), ks, len(kept_sectors), os_,
                                                 len(op_shifts), ctypes.byref(p)),
                    self.handle.h, "dmrg_blocked_plan_create")
        self.p = p
        self.K = len(op_shifts)

    def sizes(self, precision="bf16x3"):
        u, i, o = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        w = ctypes.c_size_t()
        _capi.check(self.handle.lib.dmrg_blocked_plan_sizes(self.p, _prec(precision), ctypes.byref(u),
                                                            ctypes.byref(i), ctypes.byref(o),
                                                            ctypes.byref(w)),
                    self.handle.h, "dmrg_blocked_plan_sizes")
        return u.value, i.value, o.value, w.value

    def stats(self):
        a, b, f = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        _capi.check(self.handle.lib.dmrg_blocked_plan_stats(self.p, ctypes.byref(a), ctypes.byref(b),
                                                            ctypes.byref(f)),
                    self.handle.h, "dmrg_blocked_plan_stats")
        return a.value, b.value, f.value

    def close(self):
        if getattr(self, "p", None):
            self.handle.lib.dmrg_blocked_plan_destroy(self.p)
            self.p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dmrg_blocked_plan_create(block_sectors, site_shifts, kept_sectors, op_shifts,
                             handle: Optional[Handle] = None) -> BlockedPlan:
    return BlockedPlan(block_sectors, site_shifts, kept_sectors, op_shifts, handle)


def dmrg_rotate_ops_blocked(plan: BlockedPlan, U_blocks: torch.Tensor, O_blocks: torch.Tensor,
                            precision="bf16x3", out: Optional[torch.Tensor] = None,
                            stream=None) -> torch.Tensor:
    h = plan.handle
    p = _prec(precision)
    _need(U_blocks, "U_blocks", (torch.float64,), 1)
    _need(O_blocks, "O_blocks", (torch.float64, torch.float32), 1)
    nu, ni, no, nws = plan.sizes(p)
    if U_blocks.numel() != nu or O_blocks.numel() != ni:
        raise ValueError("block storage sizes do not match the plan (U %d vs %d, O %d vs %d)"
                         % (U_blocks.numel(), nu, O_blocks.numel(), ni))
    odt = torch.float64 if p == 0 else torch.float32
    if out is None:
        out = torch.empty(max(no, 1), dtype=odt, device=O_blocks.device)
    ws = h.workspace(nws)
    _capi.check(h.lib.dmrg_rotate_ops_blocked(h.h, plan.p, _ptr(U_blocks), _ptr(O_blocks),
                                              int(O_blocks.dtype == torch.float64), _ptr(out), p,
                                              _ptr(ws), ws.numel(), _stream(stream)),
                h.h, "dmrg_rotate_ops_blocked")
    return out[:no]
