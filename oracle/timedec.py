"""Step 1 of the Kronecker solver (oracle; test infrastructure only).

Section 3: (i B_t)^{-1} M_t = X_t S_t X_t^{-1} and Y_t = X_t^{-1} (i B_t)^{-1}.
  * fast diagonalisation: X_t = eigenvectors (unit 2-norm columns), S_t = diag(eigenvalues);
  * Bartels-Stewart: complex Schur form, X_t unitary, S_t upper triangular.
kappa_2(X_t) is the spectral condition number reported in Tables 2 and 3.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def pencil_matrix(M_t, B_t):
    """(i B_t)^{-1} M_t as a dense complex matrix."""
    return np.linalg.solve(1j * np.asarray(B_t, dtype=np.complex128), np.asarray(M_t, dtype=np.complex128))


def fdm_decomposition(M_t, B_t):
    """Eigen-decomposition; returns (X, s, Y, kappa2)."""
    A = pencil_matrix(M_t, B_t)
    s, X = np.linalg.eig(A)
    X = X / np.linalg.norm(X, axis=0)[None, :]
    Y = np.linalg.solve(X, np.linalg.inv(1j * np.asarray(B_t, dtype=np.complex128)))
    kappa = np.linalg.cond(X, 2)
    return X, s, Y, kappa


def schur_decomposition(M_t, B_t):
    """Complex Schur form; returns (X unitary, S upper triangular, Y = X^H (iB)^{-1})."""
    A = pencil_matrix(M_t, B_t)
    S, X = sla.schur(A, output="complex")
    Y = X.conj().T @ np.linalg.inv(1j * np.asarray(B_t, dtype=np.complex128))
    return X, S, Y
