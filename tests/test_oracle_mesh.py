"""Pins of the oracle's general-mesh spatial matrices (oracle/fe_mesh.py), CPU only.

Each pin ties the assembly to something other than itself: the independent structured-grid
assembly of oracle/fe_space.py, the textbook closed form of the P2 triangle mass matrix,
identities that the exact integrals satisfy on any mesh (partition of unity, the measure of the
domain, the stiffness of polynomials the space reproduces), and the convergence orders of the
space-time method on unstructured meshes.
"""
import math

import numpy as np
import pytest

import synth
from oracle import fe_mesh, fe_space, fe_time, solve


def test_structured_mesh_equals_stencil_assembly():
    """The SW-NE split grid through the general assembly equals the structured P1 matrices."""
    n = 7
    nodes, tris = fe_space.structured_mesh(n)
    Mx, Ax, xy = fe_mesh.assemble_mesh(nodes, tris, 1)
    # fe_mesh keeps the global (vertex) order among interior DOFs; fe_space numbers the interior
    # lexicographically with x1 fastest, which is the same order for this vertex numbering
    Ms, As = fe_space.assemble_space(n)
    assert abs(Mx - Ms).max() < 1e-15 and abs(Ax - As).max() < 1e-14
    x1, x2 = synth.interior_coords(n)
    np.testing.assert_allclose(xy, np.stack([x1, x2], axis=1), atol=1e-15)


def test_p2_triangle_mass_closed_form():
    """|T|/180 times: 6 on the vertex diagonal, -1 between vertices, 0 between a vertex and an edge
    through it, -4 to the opposite edge, 32 on the edge diagonal, 16 between edges."""
    xyz = np.array([[[0.1, 0.2], [1.3, 0.4], [0.5, 1.7]]])
    M, A, vol = fe_mesh.element_matrices(xyz, 2)
    dofs = fe_mesh.local_dofs(2, 2)
    for a, da in enumerate(dofs):
        for b, db in enumerate(dofs):
            if len(da) == 1 and len(db) == 1:
                ref = 6 if a == b else -1
            elif len(da) == 2 and len(db) == 2:
                ref = 32 if a == b else 16
            else:
                v, e = (da[0], db) if len(da) == 1 else (db[0], da)
                ref = 0 if v in e else -4
            assert abs(M[0, a, b] - ref * vol[0] / 180) < 1e-15
    # the P2 stiffness annihilates constants
    assert np.abs(A[0].sum(axis=1)).max() < 1e-13


def _meshes():
    return [("tri", *synth.square_delaunay_mesh(6, seed=3)), ("tet", *synth.cube_tet_mesh(3, seed=4))]


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("kind", ["tri", "tet"])
def test_mesh_identities(kind, p):
    name, coords, cells = [m for m in _meshes() if m[0] == kind][0]
    d = coords.shape[1]
    M, A = fe_mesh.assemble_mesh_full(coords, cells, p)
    X = fe_mesh.dof_coords(coords, cells, p)
    one = np.ones(M.shape[0])
    bnd = fe_mesh.boundary_dofs(cells, len(coords), p)
    assert abs(one @ M @ one - 1.0) < 1e-13                       # measure of the unit square / cube
    assert np.abs(A @ one).max() < 1e-12                          # constants have no gradient
    for r in range(d):                                            # linear functions: -Laplace = 0
        assert np.abs((A @ X[:, r])[~bnd]).max() < 1e-12
    x = X[:, 0]
    assert abs(x @ M @ x - 1.0 / 3.0) < 1e-13                     # int x^2 (linear x is in the space)
    if p == 2:
        q = x * x                                                 # quadratics are in the space
        assert abs(q @ M @ q - 0.2) < 1e-13                       # int x^4
        mrow = M @ one                                            # int phi_i
        assert np.abs((A @ q + 2.0 * mrow)[~bnd]).max() < 1e-12   # -Laplace x^2 = -2
        y = X[:, 1]
        assert np.abs((A @ (x * y))[~bnd]).max() < 1e-12          # Laplace(xy) = 0
    # interior DOFs lie strictly inside, boundary DOFs on the boundary
    on = np.any((X < 1e-12) | (X > 1 - 1e-12), axis=1)
    assert np.array_equal(on, bnd)


def _st_l2_error(coords, cells, p_x, t_nodes, p_t, U_full, psi):
    """Space-time L2(Q) error of the discrete solution with nodal values U_full (all time DOFs
    including t_0, all spatial DOFs including the boundary) against psi(x, t), by tensor quadrature
    on every cell x time element."""
    d = coords.shape[1]
    pts, w = fe_mesh.simplex_rule(d, p_x + 3)
    phi, _ = fe_mesh.basis_on_reference(d, p_x, pts)
    dofmap, _, _ = fe_mesh.global_dofs(cells, len(coords), p_x)
    X = coords[cells]
    J = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))
    adet = np.abs(np.linalg.det(J))
    xq = X[:, :1, :] + np.einsum("crs,qs->cqr", J, pts)           # (C, Q, d)
    ts, tw = fe_mesh.gauss_interval(p_t + 3, 0.0, 1.0)
    phit, _ = fe_time.lagrange_ref(p_t, ts)
    err2 = 0.0
    for e in range(len(t_nodes) - 1):
        t0, t1 = t_nodes[e], t_nodes[e + 1]
        Ue = U_full[p_t * e: p_t * e + p_t + 1]                    # (p_t+1, ndof)
        for it, tq in enumerate(t0 + (t1 - t0) * ts):
            u_t = phit[:, it] @ Ue                                 # nodal values at time tq
            uh = u_t[dofmap] @ phi                                 # (C, Q)
            ex = psi(xq, tq)
            err2 += (t1 - t0) * tw[it] * np.sum(adet[:, None] * w[None, :] * np.abs(ex - uh) ** 2)
    return math.sqrt(err2)


def _solve_on_mesh(coords, cells, p_x, p_t, N_t, T=1.0):
    """Space-time solve of the manufactured psi = prod sin(pi x_r) (1 + t) e^{-it} on a mesh: the
    interpolated load of f = i psi_t - Laplace psi, psi0 = psi(., 0), the oracle's space-eigenbasis
    solver; returns the L2(Q) error."""
    d = coords.shape[1]
    t = synth.uniform_time_nodes(N_t, T)

    def S(x):
        return np.prod(np.sin(np.pi * x), axis=-1)

    def psi(x, tt):
        return S(x) * (1 + tt) * np.exp(-1j * tt)

    def f(x, tt):
        return S(x) * np.exp(-1j * tt) * ((1 + d * np.pi ** 2) * (1 + tt) + 1j)

    Mx, Ax, xin = fe_mesh.assemble_mesh(coords, cells, p_x)
    M_t, B_t, m_t, _ = fe_time.assemble_time(p_t, t)
    Mf, _, tfull = fe_time.assemble_time_full(p_t, t)
    fn = f(xin[None, :, :], tfull[:, None])
    F = Mf[1:] @ (Mx @ fn.T).T
    psi0 = psi(xin, 0.0)
    U = solve.solve_space_eig(M_t, B_t, Mx, Ax, F - np.outer(m_t, Ax @ psi0)) + psi0[None, :]
    bnd = fe_mesh.boundary_dofs(cells, len(coords), p_x)
    ndof = len(bnd)
    U_full = np.zeros((len(tfull), ndof), dtype=np.complex128)
    U_full[0, ~bnd] = psi0
    U_full[1:, ~bnd] = U
    return _st_l2_error(coords, cells, p_x, t, p_t, U_full, psi)


@pytest.mark.slow
@pytest.mark.parametrize("p", [1, 2])
def test_unstructured_convergence_orders(p):
    """On unstructured Delaunay meshes refined with the time mesh (h and tau halved), the L2(Q)
    error of the space-time solution decreases at the rate p + 1 (P1: 2, P2 in space and time: 3)."""
    errs = []
    for n, N in ((4, 4), (8, 8), (16, 16)):
        coords, tri = synth.square_delaunay_mesh(n, jitter=0.25, seed=11)
        errs.append(_solve_on_mesh(coords, tri, p, p, N))
    eoc = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert abs(eoc[-1] - (p + 1)) < 0.35, (errs, eoc)


@pytest.mark.slow
def test_tetrahedral_convergence_order():
    """The same on jittered tetrahedral cube meshes, P1 in space and time: rate 2."""
    errs, ns = [], (4, 8, 12)
    for n in ns:
        coords, tets = synth.cube_tet_mesh(n, jitter=0.15, seed=12)
        errs.append(_solve_on_mesh(coords, tets, 1, 1, n))
    eoc = [math.log(errs[i] / errs[i + 1]) / math.log(ns[i + 1] / ns[i]) for i in range(2)]
    assert eoc[0] < eoc[1] and 1.8 < eoc[1] < 2.3, (errs, eoc)      # approaching 2 from below
