"""Independent CPU FP64 fast diagonalisation (oracle; test infrastructure only).

Mirrors the paper's own CPU method (Section 4): eigen-decomposition of
(i B_t)^{-1} M_t, then the n_t spatial problems (M_x + s_k A_x) w_k = g_k of
eq. (LGS_x) solved by a sparse direct solver, in parallel over a process pool
(one solve per worker, one BLAS thread per worker), then the back transform.
Used for sizes beyond the explicit-K oracle and as the timed CPU baseline.
Validated against the explicit oracle at small sizes (tests).

cpu_fdm_refined adds classical FP64 iterative refinement: the same FDM applied
to the FP64 residual of eq. (LGS) (Kronecker form, oracle's solve.kron_apply),
x <- x + FDM(F~ - K x).  The FP64 FDM contracts the error by about
kappa_2(X_t) eps per sweep, so one sweep brings the residual to the FP64 floor;
it is the tight reference at sizes beyond the explicit oracle.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import time

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fe_space import assemble_space
from .fe_time import assemble_time
from .solve import kron_apply
from .timedec import fdm_decomposition

_W = {}


def _init(n, Lx, Ly):
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    Mx, Ax = assemble_space(n, Lx, Ly)
    _W["Mx"] = sp.csc_matrix(Mx, dtype=np.complex128)
    _W["Ax"] = sp.csc_matrix(Ax, dtype=np.complex128)


def _solve_one(args):
    s, g = args
    lu = spla.splu(_W["Mx"] + s * _W["Ax"])
    return lu.solve(g)


def spatial_solves(n, s, G, Lx=1.0, Ly=1.0, workers=None):
    """w_k = (M_x + s_k A_x)^{-1} g_k for all k, over a 'spawn' process pool."""
    workers = workers or os.cpu_count()
    ctx = mp.get_context("spawn")
    # one BLAS thread per worker: the children read these when they import numpy/scipy
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with ctx.Pool(workers, initializer=_init, initargs=(n, Lx, Ly)) as pool:
            out = pool.map(_solve_one, [(s[k], G[k]) for k in range(len(s))], chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return np.stack(out)


def cpu_fdm(n, p, t_nodes, F, psi0=None, Lx=1.0, Ly=1.0, workers=None, timings=None):
    """Full FP64 FDM on the CPU.  F: (n_t, n_x) load (before lifting); psi0: interior
    nodal values or None.  Returns psi_h at t_1..t_{n_t} (lifting added back)."""
    t0 = time.perf_counter()
    M_t, B_t, m_t, _ = assemble_time(p, t_nodes)
    Mx, Ax = assemble_space(n, Lx, Ly)
    t1 = time.perf_counter()
    X, s, Y, kappa = fdm_decomposition(M_t, B_t)
    t2 = time.perf_counter()
    Ft = F.copy()
    if psi0 is not None:
        Ft = Ft - np.outer(m_t, Ax @ psi0)
    G = Y @ Ft
    W = spatial_solves(n, s, G, Lx, Ly, workers)
    U = X @ W
    if psi0 is not None:
        U = U + psi0[None, :]
    t3 = time.perf_counter()
    if timings is not None:
        timings.update(assemble=t1 - t0, setup=t2 - t1, solve=t3 - t2, kappa=kappa,
                       workers=workers or os.cpu_count())
    return U


def cpu_fdm_refined(n, p, t_nodes, F, psi0=None, sweeps=1, Lx=1.0, Ly=1.0, workers=None, report=None):
    """cpu_fdm followed by `sweeps` classical FP64 refinement sweeps on the residual of eq. (LGS).
    Returns psi_h at t_1..t_{n_t} (lifting added back).  `report` (a dict, optional) receives the
    relative residual before every sweep and at the end, and the unrefined solution."""
    M_t, B_t, m_t, _ = assemble_time(p, t_nodes)
    Mx, Ax = assemble_space(n, Lx, Ly)
    X, s, Y, _ = fdm_decomposition(M_t, B_t)
    Ft = F.copy() if psi0 is None else F - np.outer(m_t, Ax @ psi0)
    fnorm = np.linalg.norm(Ft)

    def fdm_apply(R):
        return X @ spatial_solves(n, s, Y @ R, Lx, Ly, workers)

    U = fdm_apply(Ft)
    hist = []
    if report is not None:
        report["unrefined"] = U if psi0 is None else U + psi0[None, :]
    for _ in range(sweeps):
        R = Ft - kron_apply(M_t, B_t, Mx, Ax, U)
        hist.append(np.linalg.norm(R) / fnorm)
        U = U + fdm_apply(R)
        del R
    hist.append(np.linalg.norm(Ft - kron_apply(M_t, B_t, Mx, Ax, U)) / fnorm)
    if report is not None:
        report["residuals"] = hist
    return U if psi0 is None else U + psi0[None, :]
