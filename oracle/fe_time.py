"""Temporal finite element matrices (oracle; test infrastructure only).

eq. (matrix_t):  M_t[k,j] = int_0^T phi_j phi_k dt,   B_t[k,j] = int_0^T phi_j' phi_k dt
for the continuous piecewise-polynomial Lagrange basis of degree p on the
temporal mesh 0 = t_0 < ... < t_{N_t} = T (Section 3).  The trial/test space is
Q_{h,0,}: the DOF at t_0 is removed (row and column), so n_t = p N_t.

Global DOF order: by time, i.e. for P2 the nodes t_0, t_{1/2}, t_1, t_{3/2}, ...
The integrals are evaluated by Gauss-Legendre quadrature that is exact for the
polynomial integrands.
"""
from __future__ import annotations

import numpy as np

from .quadrature import gauss_interval


def lagrange_ref(p: int, s: np.ndarray):
    """Lagrange basis of degree p on [0,1] with equispaced nodes, and d/ds.
    Returns (phi[p+1, len(s)], dphi[p+1, len(s)])."""
    nodes = np.linspace(0.0, 1.0, p + 1)
    phi = np.ones((p + 1, len(s)))
    dphi = np.zeros((p + 1, len(s)))
    for a in range(p + 1):
        others = [nodes[c] for c in range(p + 1) if c != a]
        denom = np.prod([nodes[a] - o for o in others])
        for o in others:
            phi[a] *= (s - o)
        phi[a] /= denom
        # derivative of prod (s - o) / denom
        for skip in range(len(others)):
            term = np.ones_like(s)
            for c, o in enumerate(others):
                if c != skip:
                    term = term * (s - o)
            dphi[a] += term
        dphi[a] /= denom
    return phi, dphi


def element_matrices(p: int, tau: float):
    """Local M (int phi_j phi_k) and B (int phi_j' phi_k) on an element of length tau,
    rows = test index k, columns = trial index j."""
    s, w = gauss_interval(p + 2, 0.0, 1.0)
    phi, dphi = lagrange_ref(p, s)
    M = tau * (phi * w) @ phi.T                    # M[k, j] = tau int phi_k phi_j ds
    B = (phi * w) @ dphi.T                         # B[k, j] = int phi_k (dphi_j/ds) ds
    return M, B


def assemble_time_full(p: int, t_nodes: np.ndarray):
    """Full (t_0 included) dense M, B of size (p N_t + 1)^2, and the DOF times."""
    t = np.asarray(t_nodes, dtype=np.float64)
    N = len(t) - 1
    nfull = p * N + 1
    M = np.zeros((nfull, nfull))
    B = np.zeros((nfull, nfull))
    times = np.zeros(nfull)
    for e in range(N):
        tau = t[e + 1] - t[e]
        Ml, Bl = element_matrices(p, tau)
        idx = [p * e + a for a in range(p + 1)]
        for a in range(p + 1):
            times[idx[a]] = t[e] + tau * a / p
            for c in range(p + 1):
                M[idx[a], idx[c]] += Ml[a, c]
                B[idx[a], idx[c]] += Bl[a, c]
    return M, B, times


def assemble_time(p: int, t_nodes: np.ndarray):
    """Reduced (t_0 DOF removed) M_t, B_t (n_t x n_t, dense), the lifting weights
    m_t[k] = int_0^T phi_k dt, and the DOF times t_1..."""
    M, B, times = assemble_time_full(p, t_nodes)
    t = np.asarray(t_nodes, dtype=np.float64)
    N = len(t) - 1
    m_t = np.zeros(M.shape[0])
    s, w = gauss_interval(p + 2, 0.0, 1.0)
    phi, _ = lagrange_ref(p, s)
    for e in range(N):
        tau = t[e + 1] - t[e]
        for a in range(p + 1):
            m_t[p * e + a] += tau * np.sum(w * phi[a])
    return M[1:, 1:].copy(), B[1:, 1:].copy(), m_t[1:].copy(), times[1:].copy()
