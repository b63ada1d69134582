"""Spatial Lagrange finite element matrices on general simplicial meshes (oracle; test
infrastructure only).

eq. (matrix_x) for the spaces S^p_hx of Section 2 on any conforming triangulation: triangles
(d = 2) or tetrahedra (d = 3), continuous piecewise polynomials of degree p = 1 or 2, zero on
the boundary (Dirichlet):

    M_x[k, j] = int_Omega phi_j phi_k dx,    A_x[k, j] = int_Omega grad phi_j . grad phi_k dx.

Everything is written from the definitions: barycentric coordinates lambda_0..lambda_d of each
cell, the Lagrange basis in them (p = 1: lambda_a; p = 2: lambda_a (2 lambda_a - 1) at the
vertices and 4 lambda_a lambda_b at the edge midpoints), and collapsed (Duffy) Gauss rules on
the reference simplex that integrate the polynomial integrands exactly.

DOF numbering (an interface convention shared with the library, which implements it on its
own): global DOFs are the vertices in input order, then for p = 2 one DOF per edge, edges
ordered by their (smaller vertex, larger vertex) pair.  A DOF is on the boundary when it lies on
a boundary facet (an edge of d = 2, or a triangle of d = 3, that belongs to exactly one cell).
The interior DOFs keep the global order.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from .quadrature import gauss_interval


def simplex_rule(d: int, n: int):
    """Collapsed Gauss rule on the reference simplex {x >= 0, sum x <= 1} of dimension d = 2, 3:
    the unit cube (u, v[, w]) maps to (u, v (1 - u)[, w (1 - u)(1 - v)]), Jacobian (1 - u)
    [(1 - u)^2 (1 - v)]; n points per direction, exact for total degree 2n - d.
    Returns (points[Q, d], weights[Q]) with sum(weights) = 1 / d!."""
    g, wg = gauss_interval(n, 0.0, 1.0)
    if d == 2:
        U, V = np.meshgrid(g, g, indexing="ij")
        WU, WV = np.meshgrid(wg, wg, indexing="ij")
        pts = np.stack([U, V * (1 - U)], axis=-1).reshape(-1, 2)
        w = (WU * WV * (1 - U)).ravel()
        return pts, w
    if d == 3:
        U, V, W = np.meshgrid(g, g, g, indexing="ij")
        WU, WV, WW = np.meshgrid(wg, wg, wg, indexing="ij")
        pts = np.stack([U, V * (1 - U), W * (1 - U) * (1 - V)], axis=-1).reshape(-1, 3)
        w = (WU * WV * WW * (1 - U) ** 2 * (1 - V)).ravel()
        return pts, w
    raise ValueError("d must be 2 or 3")


def local_dofs(d: int, p: int):
    """Local DOFs of one cell: p = 1 the d + 1 vertices; p = 2 then the edges (a, b), a < b, in
    lexicographic order.  Returns a list of tuples of local vertex indices."""
    verts = [(a,) for a in range(d + 1)]
    if p == 1:
        return verts
    if p == 2:
        return verts + list(itertools.combinations(range(d + 1), 2))
    raise ValueError("p must be 1 or 2")


def basis_on_reference(d: int, p: int, pts: np.ndarray):
    """Values phi[a, q] and reference gradients dphi[a, q, r] (r = d/dx_r of the reference
    coordinates) of the local basis at the points, from the barycentric coordinates
    lambda_0 = 1 - sum x, lambda_r = x_{r-1}."""
    Q = pts.shape[0]
    lam = np.concatenate([1.0 - pts.sum(axis=1, keepdims=True), pts], axis=1).T   # (d+1, Q)
    dlam = np.zeros((d + 1, d))
    dlam[0, :] = -1.0
    dlam[1:, :] = np.eye(d)
    dofs = local_dofs(d, p)
    phi = np.zeros((len(dofs), Q))
    dphi = np.zeros((len(dofs), Q, d))
    for i, dof in enumerate(dofs):
        if len(dof) == 1:
            a = dof[0]
            if p == 1:
                phi[i] = lam[a]
                dphi[i] = np.broadcast_to(dlam[a], (Q, d))
            else:
                phi[i] = lam[a] * (2 * lam[a] - 1)
                dphi[i] = (4 * lam[a] - 1)[:, None] * dlam[a][None, :]
        else:
            a, b = dof
            phi[i] = 4 * lam[a] * lam[b]
            dphi[i] = 4 * (lam[b][:, None] * dlam[a][None, :] + lam[a][:, None] * dlam[b][None, :])
    return phi, dphi


def element_matrices(cells_xyz: np.ndarray, p: int):
    """Local mass and stiffness matrices of every cell.  cells_xyz: (C, d+1, d) vertex
    coordinates.  Returns (M_loc[C, nl, nl], A_loc[C, nl, nl], volumes[C])."""
    C, nv, d = cells_xyz.shape
    pts, w = simplex_rule(d, p + 2)
    phi, dphi = basis_on_reference(d, p, pts)
    J = np.transpose(cells_xyz[:, 1:, :] - cells_xyz[:, :1, :], (0, 2, 1))   # x = v0 + J xi
    detJ = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    adet = np.abs(detJ)
    Mref = (phi * w) @ phi.T
    M = Mref[None] * adet[:, None, None]
    # physical gradients: grad_x phi = J^{-T} grad_xi phi
    gx = np.einsum("aqr,crs->caqs", dphi, Jinv)
    A = np.einsum("caqs,cbqs,q->cab", gx, gx, w) * adet[:, None, None]
    vol = adet * (0.5 if d == 2 else 1.0 / 6.0)
    return M, A, vol


def global_dofs(cells: np.ndarray, n_vertices: int, p: int):
    """Cell -> global DOF map (C, nl), the number of global DOFs, and the DOFs of each edge.
    Global DOFs: vertices, then (p = 2) edges sorted by (min vertex, max vertex)."""
    C, nv = cells.shape
    d = nv - 1
    if p == 1:
        return cells.astype(np.int64), n_vertices, None
    pairs = list(itertools.combinations(range(d + 1), 2))
    ev = np.concatenate([np.sort(cells[:, [a, b]], axis=1) for a, b in pairs], axis=0)
    edges, inv = np.unique(ev, axis=0, return_inverse=True)
    inv = inv.reshape(len(pairs), C).T
    dofmap = np.concatenate([cells.astype(np.int64), n_vertices + inv], axis=1)
    return dofmap, n_vertices + len(edges), edges


def boundary_dofs(cells: np.ndarray, n_vertices: int, p: int):
    """Boolean mask of global DOFs on the boundary (on a facet that belongs to one cell)."""
    C, nv = cells.shape
    d = nv - 1
    facets = np.concatenate([np.sort(np.delete(cells, a, axis=1), axis=1) for a in range(d + 1)], axis=0)
    uniq, counts = np.unique(facets, axis=0, return_counts=True)
    bfac = uniq[counts == 1]
    dofmap, ndof, edges = global_dofs(cells, n_vertices, p)
    mask = np.zeros(ndof, dtype=bool)
    mask[np.unique(bfac)] = True
    if p == 2:
        # an edge is on the boundary when both its vertices lie on one boundary facet
        bedges = set()
        for f in bfac:
            for a, b in itertools.combinations(sorted(f), 2):
                bedges.add((a, b))
        for e, (a, b) in enumerate(edges):
            if (a, b) in bedges:
                mask[n_vertices + e] = True
    return mask


def dof_coords(coords: np.ndarray, cells: np.ndarray, p: int):
    """Coordinates of every global DOF (vertices, then edge midpoints)."""
    dofmap, ndof, edges = global_dofs(cells, len(coords), p)
    if p == 1:
        return coords.copy()
    return np.concatenate([coords, 0.5 * (coords[edges[:, 0]] + coords[edges[:, 1]])], axis=0)


def assemble_mesh_full(coords: np.ndarray, cells: np.ndarray, p: int):
    """Full (boundary included) CSR M, A of all global DOFs."""
    dofmap, ndof, _ = global_dofs(cells, len(coords), p)
    Ml, Al, _ = element_matrices(coords[cells], p)
    nl = dofmap.shape[1]
    rows = np.repeat(dofmap, nl, axis=1).ravel()
    cols = np.tile(dofmap, (1, nl)).ravel()
    M = sp.csr_matrix((Ml.ravel(), (rows, cols)), shape=(ndof, ndof))
    A = sp.csr_matrix((Al.ravel(), (rows, cols)), shape=(ndof, ndof))
    return M, A


def assemble_mesh(coords: np.ndarray, cells: np.ndarray, p: int):
    """Interior (Dirichlet) CSR M_x, A_x and the interior DOFs' coordinates (n_x, d)."""
    M, A = assemble_mesh_full(coords, cells, p)
    inner = np.nonzero(~boundary_dofs(cells, len(coords), p))[0]
    Mx = M[inner][:, inner].tocsr()
    Ax = A[inner][:, inner].tocsr()
    return Mx, Ax, dof_coords(coords, cells, p)[inner]
