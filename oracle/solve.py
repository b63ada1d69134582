"""Reference solvers for eq. (LGS) (oracle; test infrastructure only).

All in FP64 complex.  Arrays of space-time unknowns are (n_t, n_x), row =
time DOF, so that (B (x) M) vec(U) = B U M^T (time-outer Kronecker order).

  solve_explicit      SuperLU on the explicit K (the primary oracle).
  solve_dense         dense LU on tiny K (brute force).
  solve_space_eig     independent cross-check: generalized symmetric eig of
                      (A_x, M_x) decouples K into n_x banded time systems.
  bartels_stewart     Section 3, Schur choice: coupled spatial solves, eq. (LGS_x).
  fdm                 Section 3, eig choice: n_t independent spatial solves.
  kron_apply          K U (eq. LGS) without forming K.
  residual            F - K U and its relative 2-norm.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .timedec import fdm_decomposition, schur_decomposition


def solve_explicit(K, F):
    """u = K^{-1} F by SuperLU; F, u as (n_t, n_x)."""
    shape = F.shape
    lu = spla.splu(sp.csc_matrix(K), permc_spec="MMD_AT_PLUS_A")
    return lu.solve(np.ascontiguousarray(F).reshape(-1)).reshape(shape)


def solve_dense(K, F):
    shape = F.shape
    Kd = K.toarray() if sp.issparse(K) else np.asarray(K)
    return np.linalg.solve(Kd, F.reshape(-1)).reshape(shape)


def kron_apply(M_t, B_t, M_x, A_x, U):
    """(i B_t (x) M_x + M_t (x) A_x) vec(U) = i B_t U M_x^T + M_t U A_x^T."""
    UM = (M_x @ U.T).T
    UA = (A_x @ U.T).T
    return 1j * (np.asarray(B_t) @ UM) + np.asarray(M_t) @ UA


def kron_apply_adjoint(M_t, B_t, M_x, A_x, U):
    """K^H vec(U) = (-i B_t^T (x) M_x + M_t^T (x) A_x) vec(U) (real, symmetric M_x, A_x)."""
    UM = (M_x @ U.T).T
    UA = (A_x @ U.T).T
    return -1j * (np.asarray(B_t).T @ UM) + np.asarray(M_t).T @ UA


def residual(M_t, B_t, M_x, A_x, U, F):
    R = F - kron_apply(M_t, B_t, M_x, A_x, U)
    return R, np.linalg.norm(R) / np.linalg.norm(F)


def solve_space_eig(M_t, B_t, M_x, A_x, F):
    """Diagonalise in space: A_x V = M_x V Lambda, V^T M_x V = I.  Then
    (i B_t + lambda_j M_t) y_j = (F V)[:, j] for every spatial mode j, and U = Y V^T."""
    lam, V = sla.eigh(A_x.toarray(), M_x.toarray())
    G = F @ V
    B = np.asarray(B_t)
    Mt = np.asarray(M_t)
    n_t = B.shape[0]
    # half bandwidth of the time matrices
    nz = np.nonzero(np.abs(B) + np.abs(Mt))
    bw = int(np.max(np.abs(nz[0] - nz[1])))
    Yc = np.empty_like(G)
    for j in range(len(lam)):
        C = 1j * B + lam[j] * Mt
        ab = np.zeros((2 * bw + 1, n_t), dtype=np.complex128)
        for d in range(-bw, bw + 1):
            diag = np.diagonal(C, d)
            if d >= 0:
                ab[bw - d, d:] = diag
            else:
                ab[bw - d, :d] = diag
        Yc[:, j] = sla.solve_banded((bw, bw), ab, G[:, j])
    return Yc @ V.T


def _spatial_lu(M_x, A_x, shift):
    return spla.splu(sp.csc_matrix(M_x + shift * A_x, dtype=np.complex128))


def fdm(M_t, B_t, M_x, A_x, F, decomposition=None):
    """Fast diagonalisation (Section 3, steps 1-4 with the eig choice)."""
    X, s, Y, _ = decomposition if decomposition is not None else fdm_decomposition(M_t, B_t)
    G = Y @ F                                        # step 2
    W = np.empty_like(G)
    for k in range(len(s)):                          # step 3: independent solves
        W[k] = _spatial_lu(M_x, A_x, s[k]).solve(G[k])
    return X @ W                                     # step 4


def bartels_stewart(M_t, B_t, M_x, A_x, F):
    """Bartels-Stewart (Section 3, steps 1-4 with the Schur choice, eq. (LGS_x))."""
    X, S, Y = schur_decomposition(M_t, B_t)
    G = Y @ F
    n_t = G.shape[0]
    W = np.zeros_like(G)
    acc = np.zeros_like(G)                           # sum_{k > l} S[l,k] w_k, built as w_k arrive
    for l in range(n_t - 1, -1, -1):
        rhs = G[l] - A_x @ acc[l]
        W[l] = _spatial_lu(M_x, A_x, S[l, l]).solve(rhs)
        acc[:l] += np.outer(S[:l, l], W[l])
    return X @ W
