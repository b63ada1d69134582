"""Spatial P1 finite element matrices (oracle; test infrastructure only).

eq. (matrix_x):  M_x[k,j] = int_Omega phi_j phi_k dx,  A_x[k,j] = int_Omega grad phi_j . grad phi_k dx
on a structured triangulation of (0,Lx) x (0,Ly): n x n rectangles, each split
along its SW-NE diagonal into two triangles (the paper's Figure 1 is not
available; this is the reading of its printed DOF counts).  Interior nodes are
numbered lexicographically with x1 fastest.  Integrals by quadrature on each
triangle (exact for the polynomial integrands).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .quadrature import triangle_rule


def structured_mesh(n: int, Lx: float = 1.0, Ly: float = 1.0):
    """Nodes (all (n+1)^2, index i + (n+1) j) and triangles (vertex index triples,
    counter-clockwise) of the SW-NE split grid."""
    i, j = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy")
    nodes = np.stack([i.ravel() * (Lx / n), j.ravel() * (Ly / n)], axis=1)
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    sw = (ii + (n + 1) * jj).ravel()
    se = sw + 1
    nw = sw + (n + 1)
    ne = nw + 1
    lower = np.stack([sw, se, ne], axis=1)    # lower-right triangle
    upper = np.stack([sw, ne, nw], axis=1)    # upper-left triangle
    tris = np.stack([lower, upper], axis=1).reshape(-1, 3)
    return nodes, tris.astype(np.int64)


def interior_map(n: int):
    """Full node index -> interior DOF index (-1 on the boundary), x1 fastest."""
    full = -np.ones((n + 1) * (n + 1), dtype=np.int64)
    m = n - 1
    jj, ii = np.meshgrid(np.arange(1, n), np.arange(1, n), indexing="ij")
    full[(ii + (n + 1) * jj).ravel()] = ((ii - 1) + m * (jj - 1)).ravel()
    return full


def p1_element(vertices: np.ndarray):
    """P1 local mass and stiffness on one triangle from the integral definitions.
    vertices: (3, 2).  Returns (M_loc, A_loc, area, grads[3,2])."""
    v0, v1, v2 = vertices
    J = np.array([v1 - v0, v2 - v0]).T            # x = v0 + J (xi, eta)
    detJ = np.linalg.det(J)
    area = 0.5 * abs(detJ)
    xi, eta, w = triangle_rule(3)
    lam = np.stack([1.0 - xi - eta, xi, eta])     # barycentric = P1 basis on reference
    M = (lam * w) @ lam.T * abs(detJ)
    dref = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])
    grads = dref @ np.linalg.inv(J)               # rows: grad lambda_a in x
    A = area * grads @ grads.T
    return M, A, area, grads


def p1_elements(vertices: np.ndarray):
    """Vectorised p1_element over many triangles; vertices: (T, 3, 2).
    Returns (M_loc[T,3,3], A_loc[T,3,3])."""
    v0 = vertices[:, 0]
    J = np.stack([vertices[:, 1] - v0, vertices[:, 2] - v0], axis=2)   # (T, 2, 2) columns
    detJ = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
    xi, eta, w = triangle_rule(3)
    lam = np.stack([1.0 - xi - eta, xi, eta])
    Mref = (lam * w) @ lam.T
    M = Mref[None] * np.abs(detJ)[:, None, None]
    Jinv = np.empty_like(J)
    Jinv[:, 0, 0] = J[:, 1, 1] / detJ
    Jinv[:, 1, 1] = J[:, 0, 0] / detJ
    Jinv[:, 0, 1] = -J[:, 0, 1] / detJ
    Jinv[:, 1, 0] = -J[:, 1, 0] / detJ
    dref = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])
    grads = np.einsum("ar,trc->tac", dref, Jinv)
    A = 0.5 * np.abs(detJ)[:, None, None] * np.einsum("tac,tbc->tab", grads, grads)
    return M, A


def assemble_space_full(n: int, Lx: float = 1.0, Ly: float = 1.0):
    """Full (boundary included) sparse M, A of size (n+1)^2."""
    nodes, tris = structured_mesh(n, Lx, Ly)
    N = len(nodes)
    Ml, Al = p1_elements(nodes[tris])
    rows = np.repeat(tris, 3, axis=1).ravel()
    cols = np.tile(tris, (1, 3)).ravel()
    M = sp.csr_matrix((Ml.ravel(), (rows, cols)), shape=(N, N))
    A = sp.csr_matrix((Al.ravel(), (rows, cols)), shape=(N, N))
    return M, A


def assemble_space(n: int, Lx: float = 1.0, Ly: float = 1.0):
    """Interior (Dirichlet) sparse CSR M_x, A_x of size (n-1)^2."""
    M, A = assemble_space_full(n, Lx, Ly)
    imap = interior_map(n)
    keep = np.nonzero(imap >= 0)[0]
    order = keep[np.argsort(imap[keep])]
    Mx = M[order][:, order].tocsr()
    Ax = A[order][:, order].tocsr()
    Mx.eliminate_zeros()
    Ax.eliminate_zeros()
    return Mx, Ax


def interior_node_coords(n: int, Lx: float = 1.0, Ly: float = 1.0):
    nodes, _ = structured_mesh(n, Lx, Ly)
    imap = interior_map(n)
    keep = np.nonzero(imap >= 0)[0]
    order = keep[np.argsort(imap[keep])]
    return nodes[order, 0].copy(), nodes[order, 1].copy()
