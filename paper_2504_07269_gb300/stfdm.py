"""Thin Python binding of the stfdm C ABI (include/stfdm.h), same entry-point names.

Argument marshalling only: torch tensors provide device memory and the current
CUDA stream; every step of the solver runs in the library's CUDA kernels.
Space-time arrays are (n_t, n_x) contiguous complex tensors on the handle's
device (complex128 for "fp64"/"mixed", complex64 for "fp32").
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import check, lib

PREC = {"fp64": _lib.ST_FP64, "fp32": _lib.ST_FP32, "mixed": _lib.ST_MIXED}
XFORM = {"Y": _lib.ST_XFORM_Y, "X": _lib.ST_XFORM_X, "XT": _lib.ST_XFORM_XT, "YT": _lib.ST_XFORM_YT}


class _Handle:
    _destroy = None

    def __init__(self, ptr):
        self.ptr = ptr

    def close(self):
        """Destroy the library object now (its device memory is released); the handle is unusable after."""
        if self.ptr and self._destroy:
            try:
                getattr(lib(), self._destroy)(self.ptr)
            except Exception:
                pass
        self.ptr = None

    def __del__(self):
        self.close()


class TimeHandle(_Handle):
    _destroy = "st_destroy_time"


class SpaceHandle(_Handle):
    _destroy = "st_destroy_space"


class FdmHandle(_Handle):
    _destroy = "st_destroy_fdm"

    def __init__(self, ptr, time, space, device):
        super().__init__(ptr)
        self.time = time
        self.space = space
        self.device = device      # CUDA ordinal the handle's device data live on
        n_t, n_x, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        kap, mni = ctypes.c_double(), ctypes.c_double()
        check(lib().st_fdm_get(ptr, ctypes.byref(n_t), ctypes.byref(n_x), ctypes.byref(m), ctypes.byref(kap),
                               ctypes.byref(mni)), "st_fdm_get")
        self.n_t, self.n_x, self.m = n_t.value, n_x.value, m.value
        self.kappa = kap.value
        self.min_neg_im_shift = mni.value


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _check_device(h: FdmHandle, t, name):
    # the library launches on the handle's device: a tensor elsewhere would be read through a
    # pointer that is not valid there
    if t.device.index != h.device:
        raise ValueError(f"{name}: tensor on {t.device}, but the handle lives on cuda:{h.device}")


def _check_st(h: FdmHandle, t, dtype, name):
    if t is None:
        return
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous() or tuple(t.shape) != (h.n_t, h.n_x):
        raise ValueError(f"{name}: expected a contiguous CUDA {dtype} tensor of shape {(h.n_t, h.n_x)}, "
                         f"got {t.dtype} {tuple(t.shape)} on {t.device}")
    _check_device(h, t, name)


def _check_vec(h: FdmHandle, t, dtype, name):
    if t is None:
        return
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous() or tuple(t.shape) != (h.n_x,):
        raise ValueError(f"{name}: expected a contiguous CUDA {dtype} tensor of shape {(h.n_x,)}")
    _check_device(h, t, name)


def _check_no_alias(R, others, name="R"):
    """R is written while other threads still read stencil neighbours of psi and psi0."""
    if R is None:
        return
    for o in others:
        if o is not None and o.data_ptr() == R.data_ptr():
            raise ValueError(f"{name} must not alias psi or psi0")


def _check_with_info(status, where, info):
    """Raise on error; the exception carries the solve info (filled on NOT_CONVERGED too)."""
    if status != _lib.ST_OK:
        err = _lib.StfdmError(status, where)
        err.info = _info_dict(info) if info is not None else None
        raise err


def _dtype(precision):
    return torch.complex64 if precision == "fp32" else torch.complex128


REFINE = {"gmres": _lib.ST_REFINE_GMRES, "classic": _lib.ST_REFINE_CLASSIC}


def _opts(precision="fp64", tol=0.0, max_sweeps=0, keep_factors=-1, fixed_sweeps=0, method="gmres", err_tol=0.0):
    if precision not in PREC:
        raise ValueError(f"unknown precision {precision!r}")
    return _lib.st_solve_opts(PREC[precision], float(tol), int(max_sweeps), int(keep_factors), int(fixed_sweeps),
                              REFINE[method], float(err_tol))


def _info_dict(info: _lib.st_solve_info):
    return dict(sweeps=info.sweeps, factors_kept=info.factors_kept, rel_residual=info.rel_residual,
                residual_history=[v for v in info.residual_history if v >= 0], kappa_x=info.kappa_x,
                min_neg_im_shift=info.min_neg_im_shift, setup_seconds=info.setup_seconds,
                tensor_cores=info.tensor_cores, kernel_launches=info.kernel_launches, restart=info.restart,
                kept_systems=info.kept_systems, rel_error_estimate=info.rel_error_estimate,
                reorth_steps=info.reorth_steps)


# ------------------------------------------------------------------ assembly / setup
def st_assemble_time(p_t: int, t_nodes) -> TimeHandle:
    t = np.ascontiguousarray(np.asarray(t_nodes, dtype=np.float64))
    out = ctypes.c_void_p()
    check(lib().st_assemble_time(int(p_t), len(t) - 1, t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 ctypes.byref(out)), "st_assemble_time")
    return TimeHandle(out)


def st_time_get(t: TimeHandle):
    n = ctypes.c_int()
    check(lib().st_time_get(t.ptr, ctypes.byref(n), None, None, None, None), "st_time_get")
    n = n.value
    M = np.zeros((n, n))
    B = np.zeros((n, n))
    m = np.zeros(n)
    tt = np.zeros(n)
    check(lib().st_time_get(t.ptr, None, M.ctypes.data, B.ctypes.data, m.ctypes.data, tt.ctypes.data),
          "st_time_get")
    return dict(M_t=M, B_t=B, m_t=m, times=tt)


def st_assemble_space(n_squares: int, Lx: float = 1.0, Ly: float = 1.0) -> SpaceHandle:
    out = ctypes.c_void_p()
    check(lib().st_assemble_space(int(n_squares), float(Lx), float(Ly), ctypes.byref(out)), "st_assemble_space")
    return SpaceHandle(out)


def st_space_get(s: SpaceHandle):
    m, n_x = ctypes.c_int(), ctypes.c_int()
    coeffs = np.zeros(8)
    check(lib().st_space_get(s.ptr, ctypes.byref(m), ctypes.byref(n_x), coeffs.ctypes.data), "st_space_get")
    return m.value, n_x.value, coeffs


def st_time_decompose(t: TimeHandle, host_threads: int = 0):
    n = st_time_get(t)["M_t"].shape[0]
    X = np.zeros((n, n), dtype=np.complex128)
    Y = np.zeros((n, n), dtype=np.complex128)
    s = np.zeros(n, dtype=np.complex128)
    k = ctypes.c_double()
    check(lib().st_time_decompose(t.ptr, int(host_threads), X.ctypes.data, s.ctypes.data, Y.ctypes.data,
                                  ctypes.byref(k)), "st_time_decompose")
    return X, s, Y, k.value


SPATIAL = {"auto": _lib.ST_SPATIAL_AUTO, "banded": _lib.ST_SPATIAL_BANDED,
           "multifrontal": _lib.ST_SPATIAL_MULTIFRONTAL}


def st_assemble_mesh(dim: int, p_x: int, coords, cells) -> SpaceHandle:
    """Spatial P1/P2 matrices on a triangle (dim 2) or tetrahedron (dim 3) mesh; coords (V, dim)
    floats, cells (C, dim + 1) vertex indices."""
    c = np.ascontiguousarray(np.asarray(coords, dtype=np.float64))
    e = np.ascontiguousarray(np.asarray(cells, dtype=np.int32))
    if c.ndim != 2 or c.shape[1] != dim or e.ndim != 2 or e.shape[1] != dim + 1:
        raise ValueError("coords must be (V, dim) and cells (C, dim + 1)")
    out = ctypes.c_void_p()
    check(lib().st_assemble_mesh(int(dim), int(p_x), c.shape[0], c.ctypes.data_as(ctypes.c_void_p), e.shape[0],
                                 e.ctypes.data_as(ctypes.c_void_p), ctypes.byref(out)), "st_assemble_mesh")
    return SpaceHandle(out)


def st_space_get_mesh(s: SpaceHandle):
    """CSR (rowptr, col, M, A) of the interior DOFs and their coordinates xyz (n_x, dim)."""
    dim, p, n, nnz = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
    check(lib().st_space_get_mesh(s.ptr, ctypes.byref(dim), ctypes.byref(p), ctypes.byref(n), ctypes.byref(nnz),
                                  None, None, None, None, None), "st_space_get_mesh")
    rp = np.zeros(n.value + 1, dtype=np.int32)
    col = np.zeros(nnz.value, dtype=np.int32)
    M = np.zeros(nnz.value)
    A = np.zeros(nnz.value)
    xyz = np.zeros((n.value, dim.value))
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)   # noqa: E731
    check(lib().st_space_get_mesh(s.ptr, None, None, None, None, ptr(rp), ptr(col), ptr(M), ptr(A), ptr(xyz)),
          "st_space_get_mesh")
    return dict(dim=dim.value, p_x=p.value, n_x=n.value, rowptr=rp, col=col, M=M, A=A, xyz=xyz)


def st_space_mf_plan(s: SpaceHandle, leaf: int = 0):
    """Statistics and structure of the sparse-direct solver's plan for a space."""
    nf, nl, mf = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    fe, fl = ctypes.c_longlong(), ctypes.c_double()
    check(lib().st_space_mf_plan(s.ptr, int(leaf), ctypes.byref(nf), ctypes.byref(nl), ctypes.byref(mf),
                                 ctypes.byref(fe), ctypes.byref(fl), None, None, None, None, None), "st_space_mf_plan")
    F = nf.value
    info = st_space_get_mesh(s)
    perm = np.zeros(info["n_x"], dtype=np.int32)
    first, npv, nu = (np.zeros(F, dtype=np.int32) for _ in range(3))
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)   # noqa: E731
    check(lib().st_space_mf_plan(s.ptr, int(leaf), None, None, None, None, None, ptr(perm), ptr(first), ptr(npv),
                                 ptr(nu), None), "st_space_mf_plan")
    urows = np.zeros(int(nu.sum()), dtype=np.int32)
    check(lib().st_space_mf_plan(s.ptr, int(leaf), None, None, None, None, None, None, None, None, None, ptr(urows)),
          "st_space_mf_plan")
    return dict(fronts=F, levels=nl.value, max_front=mf.value, factor_entries=fe.value, flops=fl.value, perm=perm,
                first=first, np=npv, nu=nu, urows=urows)


def st_fdm_setup(t: TimeHandle, s: SpaceHandle, kappa_max: float = 0.0, device: int = -1,
                 host_threads: int = 0, spatial_solver: str = "auto") -> FdmHandle:
    opts = _lib.st_setup_opts(float(kappa_max), int(device), int(host_threads), SPATIAL[spatial_solver])
    out = ctypes.c_void_p()
    check(lib().st_fdm_setup(t.ptr, s.ptr, ctypes.byref(opts), ctypes.byref(out)), "st_fdm_setup")
    return FdmHandle(out, t, s, int(device) if device >= 0 else torch.cuda.current_device())


# ------------------------------------------------------------------ solves
def st_fdm_solve(h: FdmHandle, F, psi0=None, psi=None, precision="fp64", tol=0.0, max_sweeps=0,
                 keep_factors=-1, fixed_sweeps=0, stream=None, want_info=True, method="gmres", err_tol=0.0):
    dt = _dtype(precision)
    _check_st(h, F, dt, "F")
    _check_vec(h, psi0, dt, "psi0")
    if psi is None:
        psi = torch.empty_like(F)
    _check_st(h, psi, dt, "psi")
    opts = _opts(precision, tol, max_sweeps, keep_factors, fixed_sweeps, method, err_tol)
    info = _lib.st_solve_info()
    st = lib().st_fdm_solve(h.ptr, _ptr(F), _ptr(psi0), _ptr(psi), ctypes.byref(opts),
                            ctypes.byref(info) if want_info else None, _stream(stream))
    _check_with_info(st, "st_fdm_solve", info if want_info else None)
    return psi, (_info_dict(info) if want_info else None)


def st_bs_solve(h: FdmHandle, F, psi0=None, psi=None, stream=None, want_info=True):
    """FP64 Bartels-Stewart solve (Schur choice of step 1): same arrays as st_fdm_solve(fp64)."""
    _check_st(h, F, torch.complex128, "F")
    _check_vec(h, psi0, torch.complex128, "psi0")
    if psi is None:
        psi = torch.empty_like(F)
    _check_st(h, psi, torch.complex128, "psi")
    info = _lib.st_solve_info()
    st = lib().st_bs_solve(h.ptr, _ptr(F), _ptr(psi0), _ptr(psi), ctypes.byref(info) if want_info else None,
                           _stream(stream))
    _check_with_info(st, "st_bs_solve", info if want_info else None)
    return psi, (_info_dict(info) if want_info else None)


def st_residual(h: FdmHandle, F, psi0, psi, R=None, want_norm=True, stream=None):
    _check_st(h, F, torch.complex128, "F")
    _check_st(h, psi, torch.complex128, "psi")
    _check_vec(h, psi0, torch.complex128, "psi0")
    _check_st(h, R, torch.complex128, "R")
    _check_no_alias(R, (psi, psi0))
    rel = ctypes.c_double(-1.0)
    check(lib().st_residual(h.ptr, _ptr(F), _ptr(psi0), _ptr(psi), _ptr(R), ctypes.byref(rel) if want_norm else None,
                            _stream(stream)), "st_residual")
    return rel.value, R


def st_adjoint_solve(h: FdmHandle, G, lam=None, precision="fp64", tol=0.0, max_sweeps=0, keep_factors=-1,
                     fixed_sweeps=0, stream=None, want_info=True, method="gmres", err_tol=0.0):
    dt = _dtype(precision)
    _check_st(h, G, dt, "G")
    if lam is None:
        lam = torch.empty_like(G)
    _check_st(h, lam, dt, "lambda")
    opts = _opts(precision, tol, max_sweeps, keep_factors, fixed_sweeps, method, err_tol)
    info = _lib.st_solve_info()
    st = lib().st_adjoint_solve(h.ptr, _ptr(G), _ptr(lam), ctypes.byref(opts),
                                ctypes.byref(info) if want_info else None, _stream(stream))
    _check_with_info(st, "st_adjoint_solve", info if want_info else None)
    return lam, (_info_dict(info) if want_info else None)


def st_adjoint_lift(h: FdmHandle, grad_psi, grad_F, grad_psi0=None, stream=None):
    _check_st(h, grad_psi, torch.complex128, "grad_psi")
    _check_st(h, grad_F, torch.complex128, "grad_F")
    if grad_psi0 is None:
        grad_psi0 = torch.empty(h.n_x, dtype=torch.complex128, device=grad_psi.device)
    _check_vec(h, grad_psi0, torch.complex128, "grad_psi0")
    check(lib().st_adjoint_lift(h.ptr, _ptr(grad_psi), _ptr(grad_F), _ptr(grad_psi0), _stream(stream)),
          "st_adjoint_lift")
    return grad_psi0


def _ptr_array(ts):
    return (ctypes.c_void_p * len(ts))(*[(t.data_ptr() if t is not None else None) for t in ts])


def _check_list_with_info(status, where, infos, n):
    if status != _lib.ST_OK:
        err = _lib.StfdmError(status, where)
        err.info = [_info_dict(infos[i]) for i in range(n)] if infos is not None else None
        raise err


def st_fdm_solve_batched(hs, Fs, psi0s=None, psis=None, precision="fp64", tol=0.0, max_sweeps=0,
                         keep_factors=-1, fixed_sweeps=0, stream=None, want_info=True, method="gmres"):
    n = len(hs)
    dt = _dtype(precision)
    if psis is None:
        psis = [torch.empty_like(F) for F in Fs]
    for h, F, p in zip(hs, Fs, psis):
        _check_st(h, F, dt, "F")
        _check_st(h, p, dt, "psi")
    if psi0s is not None:
        for h, p0 in zip(hs, psi0s):
            _check_vec(h, p0, dt, "psi0")
    H = (ctypes.c_void_p * n)(*[h.ptr for h in hs])
    P0 = _ptr_array(psi0s) if psi0s else None
    opts = _opts(precision, tol, max_sweeps, keep_factors, fixed_sweeps, method)
    infos = (_lib.st_solve_info * n)() if want_info else None
    st = lib().st_fdm_solve_batched(H, n, _ptr_array(Fs), P0, _ptr_array(psis), ctypes.byref(opts), infos,
                                    _stream(stream))
    _check_list_with_info(st, "st_fdm_solve_batched", infos, n)
    return psis, ([_info_dict(i) for i in infos] if want_info else None)


class BatchHandle(_Handle):
    _destroy = "st_destroy_batch"

    def __init__(self, ptr, hs):
        super().__init__(ptr)
        self.hs = list(hs)   # the problem handles must outlive the plan


def st_batch_create(hs, tol=0.0, max_sweeps=0, restart=0, no_graph=False, no_tune=False, no_keep=False) -> BatchHandle:
    """Batched mixed-precision plan over FdmHandles of any mixture of sizes (see st_batch_create)."""
    n = len(hs)
    H = (ctypes.c_void_p * n)(*[h.ptr for h in hs])
    o = _lib.st_batch_opts(float(tol), int(max_sweeps), int(restart), int(bool(no_graph)), int(bool(no_tune)),
                           int(bool(no_keep)))
    out = ctypes.c_void_p()
    check(lib().st_batch_create(H, n, ctypes.byref(o), ctypes.byref(out)), "st_batch_create")
    return BatchHandle(out, hs)


def st_batch_solve(b: BatchHandle, Fs, psi0s=None, psis=None, stream=None, want_info=True):
    n = len(b.hs)
    if len(Fs) != n or (psi0s is not None and len(psi0s) != n):
        raise ValueError("st_batch_solve: one right-hand side (and psi0) per problem")
    if psis is None:
        psis = [torch.empty_like(F) for F in Fs]
    for h, F, p in zip(b.hs, Fs, psis):
        _check_st(h, F, torch.complex128, "F")
        _check_st(h, p, torch.complex128, "psi")
    if psi0s is not None:
        for h, p0 in zip(b.hs, psi0s):
            _check_vec(h, p0, torch.complex128, "psi0")
    infos = (_lib.st_solve_info * n)() if want_info else None
    st = lib().st_batch_solve(b.ptr, _ptr_array(Fs), _ptr_array(psi0s) if psi0s is not None else None,
                              _ptr_array(psis), infos, _stream(stream))
    _check_list_with_info(st, "st_batch_solve", infos, n)
    return psis, ([_info_dict(i) for i in infos] if want_info else None)


def st_batch_spatial_solve(b: BatchHandle, stream=None):
    check(lib().st_batch_spatial_solve(b.ptr, _stream(stream)), "st_batch_spatial_solve")


def st_batch_spatial_get(b: BatchHandle, p: int, G, to_plan: bool, stream=None):
    h = b.hs[p]
    _check_st(h, G, torch.complex64, "G")
    check(lib().st_batch_spatial_get(b.ptr, int(p), _ptr(G), int(bool(to_plan)), _stream(stream)),
          "st_batch_spatial_get")
    return G


def st_batch_stats_get(b: BatchHandle) -> dict:
    s = _lib.st_batch_stats()
    check(lib().st_batch_stats_get(b.ptr, ctypes.byref(s)), "st_batch_stats_get")
    return {name: getattr(s, name) for name, _ in s._fields_}


def st_destroy_batch(b: BatchHandle):
    if b.ptr:
        lib().st_destroy_batch(b.ptr)
        b.ptr = None


def st_time_transform(h: FdmHandle, which: str, precision: str, inp, out=None, stream=None):
    """precision: "fp64" (c128), "fp32" (c64, SIMT) or "mixed" (c64 on the tensor cores, 3xTF32)."""
    dt = torch.complex64 if precision in ("fp32", "mixed") else torch.complex128
    _check_st(h, inp, dt, "in")
    if out is None:
        out = torch.empty_like(inp)
    _check_st(h, out, dt, "out")
    check(lib().st_time_transform(h.ptr, XFORM[which], PREC[precision], _ptr(inp), _ptr(out), _stream(stream)),
          "st_time_transform")
    return out


def st_spatial_solve(h: FdmHandle, precision: str, G, W=None, stream=None):
    dt = _dtype(precision)
    _check_st(h, G, dt, "G")
    if W is None:
        W = torch.empty_like(G)
    _check_st(h, W, dt, "W")
    check(lib().st_spatial_solve(h.ptr, PREC[precision], _ptr(G), _ptr(W), _stream(stream)), "st_spatial_solve")
    return W


def st_spatial_factor(h: FdmHandle, precision: str, stream=None):
    """Factorise all n_t spatial matrices and keep the factors in the handle."""
    if precision not in ("fp64", "fp32"):
        raise ValueError("precision must be fp64 or fp32")
    check(lib().st_spatial_factor(h.ptr, PREC[precision], _stream(stream)), "st_spatial_factor")


def st_spatial_substitute(h: FdmHandle, precision: str, G, W=None, stream=None):
    """W[k,:] = C_k^{-1} G[k,:] with the factors kept by st_spatial_factor."""
    dt = _dtype(precision)
    _check_st(h, G, dt, "G")
    if W is None:
        W = torch.empty_like(G)
    _check_st(h, W, dt, "W")
    check(lib().st_spatial_substitute(h.ptr, PREC[precision], _ptr(G), _ptr(W), _stream(stream)),
          "st_spatial_substitute")
    return W


def st_load_nodal(h: FdmHandle, f_nodal, F=None, stream=None):
    if not f_nodal.is_cuda or f_nodal.dtype != torch.complex128 or tuple(f_nodal.shape) != (h.n_t + 1, h.n_x):
        raise ValueError("f_nodal: expected a CUDA complex128 tensor of shape (n_t + 1, n_x)")
    f_nodal = f_nodal.contiguous()
    if F is None:
        F = torch.empty((h.n_t, h.n_x), dtype=torch.complex128, device=f_nodal.device)
    check(lib().st_load_nodal(h.ptr, _ptr(f_nodal), _ptr(F), _stream(stream)), "st_load_nodal")
    return F


EXACT = {"c1": _lib.ST_EXACT_C1, "paper": _lib.ST_EXACT_PAPER}


def st_error_norms(h: FdmHandle, exact: str, psi, psi0=None, q_t: int = 0, q_x: int = 0, stream=None):
    """(L2(Q) error, H1(Q) seminorm error) of the trial-space function with nodal values psi0 (t_0)
    and psi (t_1..) against the manufactured solution `exact` ("c1" or "paper")."""
    _check_st(h, psi, torch.complex128, "psi")
    _check_vec(h, psi0, torch.complex128, "psi0")
    out = (ctypes.c_double * 2)()
    check(lib().st_error_norms(h.ptr, EXACT[exact], _ptr(psi), _ptr(psi0), int(q_t), int(q_x), out, _stream(stream)),
          "st_error_norms")
    return out[0], out[1]


def st_load_quadrature(h: FdmHandle, exact: str, F=None, q_t: int = 0, q_x: int = 0, stream=None):
    if F is None:
        F = torch.empty((h.n_t, h.n_x), dtype=torch.complex128, device=torch.device("cuda", torch.cuda.current_device()))
    _check_st(h, F, torch.complex128, "F")
    check(lib().st_load_quadrature(h.ptr, EXACT[exact], int(q_t), int(q_x), _ptr(F), _stream(stream)),
          "st_load_quadrature")
    return F


def st_residual_noalloc(h: FdmHandle, F, psi0, psi, R, norms, stream=None):
    """Allocation-free residual: writes R (or nothing if R is None) and norms[0:2] =
    (||R||^2, ||F~||^2) into caller-provided device tensors; never synchronises."""
    _check_st(h, F, torch.complex128, "F")
    _check_st(h, psi, torch.complex128, "psi")
    _check_vec(h, psi0, torch.complex128, "psi0")
    _check_st(h, R, torch.complex128, "R")
    _check_no_alias(R, (psi, psi0))
    if not norms.is_cuda or norms.dtype != torch.float64 or norms.numel() < 2 or not norms.is_contiguous():
        raise ValueError("norms: expected a contiguous CUDA float64 tensor with 2 entries")
    _check_device(h, norms, "norms")
    check(lib().st_residual_noalloc(h.ptr, _ptr(F), _ptr(psi0), _ptr(psi), _ptr(R), _ptr(norms), _stream(stream)),
          "st_residual_noalloc")
    return norms


def st_set_wait_probe(h: FdmHandle, seconds: float):
    """Test hook: later substitution launches first wait `seconds` on a barrier nothing completes
    (the bounded-wait exit, ST_ERR_TIMEOUT); 0 turns it off."""
    check(lib().st_set_wait_probe(h.ptr, float(seconds)), "st_set_wait_probe")


def setup_problem(n_squares: int, p_t: int, t_nodes, Lx: float = 1.0, Ly: float = 1.0, **kw) -> FdmHandle:
    """assemble_time + assemble_space + fdm_setup in one call."""
    t = st_assemble_time(p_t, t_nodes)
    s = st_assemble_space(n_squares, Lx, Ly)
    return st_fdm_setup(t, s, **kw)


def setup_mesh_problem(dim: int, p_x: int, coords, cells, p_t: int, t_nodes, **kw) -> FdmHandle:
    """assemble_time + assemble_mesh + fdm_setup in one call (general meshes)."""
    t = st_assemble_time(p_t, t_nodes)
    s = st_assemble_mesh(dim, p_x, coords, cells)
    return st_fdm_setup(t, s, **kw)


def setup_problems(specs, workers: int = 0, **kw):
    """setup_problem for many (n_squares, p_t, t_nodes, Lx, Ly) tuples, concurrently on host
    threads (one host thread per decomposition); returns the handles in order."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    workers = workers or min(len(specs), os.cpu_count() or 1)
    kw = dict(kw, host_threads=1)
    with ThreadPoolExecutor(max_workers=max(1, workers)) as ex:
        futs = [ex.submit(setup_problem, n, p, t, Lx, Ly, **kw) for (n, p, t, Lx, Ly) in specs]
        return [f.result() for f in futs]
