"""Pins of the oracle's quadrature and finite element matrices (CPU only).

Each oracle function is checked against something other than itself: exact
integrals of monomials, a library quadrature routine, hand-derived closed-form
element matrices (tests/golden/closed_forms.txt), and identities that the
basis functions must satisfy (partition of unity, integration by parts).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import assemble, fe_space, fe_time, quadrature


# ------------------------------------------------------------------ quadrature
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12])
def test_gauss_legendre_matches_library(n):
    x, w = quadrature.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, xr, atol=1e-14)
    np.testing.assert_allclose(w, wr, atol=1e-14)


@pytest.mark.parametrize("n", [2, 4, 6])
def test_gauss_exact_degree(n):
    x, w = quadrature.gauss_interval(n, 0.3, 1.7)
    for d in range(2 * n):
        exact = (1.7 ** (d + 1) - 0.3 ** (d + 1)) / (d + 1)
        assert abs(np.sum(w * x ** d) - exact) < 1e-13 * max(1, abs(exact))


@pytest.mark.parametrize("n", [2, 3, 6])
def test_triangle_rule_exact(n):
    xi, eta, w = quadrature.triangle_rule(n)
    assert abs(w.sum() - 0.5) < 1e-15
    for a in range(2 * n - 1):
        for b in range(2 * n - 1 - a):
            exact = quadrature.monomial_triangle_integral(a, b)
            assert abs(np.sum(w * xi ** a * eta ** b) - exact) < 1e-14


# ------------------------------------------------------------------ time matrices
def test_time_p1_closed_form():
    tau = 0.37
    M, B = fe_time.element_matrices(1, tau)
    np.testing.assert_allclose(M, tau / 6 * np.array([[2, 1], [1, 2]]), atol=1e-15)
    np.testing.assert_allclose(B, np.array([[-0.5, 0.5], [-0.5, 0.5]]), atol=1e-15)


def test_time_p2_closed_form():
    tau = 0.61
    M, B = fe_time.element_matrices(2, tau)
    np.testing.assert_allclose(M, tau / 30 * np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]), atol=1e-15)
    Bx = np.array([[-1 / 2, 2 / 3, -1 / 6], [-2 / 3, 0, 2 / 3], [1 / 6, -2 / 3, 1 / 2]])
    np.testing.assert_allclose(B, Bx, atol=1e-15)


def test_time_p1_uniform_global():
    N, T = 6, 2.0
    tau = T / N
    M, B, m, times = fe_time.assemble_time(1, synth.uniform_time_nodes(N, T))
    Mx = np.diag(np.full(N, 2 * tau / 3)) + np.diag(np.full(N - 1, tau / 6), 1) + np.diag(np.full(N - 1, tau / 6), -1)
    Mx[-1, -1] = tau / 3
    Bx = np.diag(np.full(N - 1, 0.5), 1) - np.diag(np.full(N - 1, 0.5), -1)
    Bx[-1, -1] = 0.5
    np.testing.assert_allclose(M, Mx, atol=1e-15)
    np.testing.assert_allclose(B, Bx, atol=1e-15)
    np.testing.assert_allclose(m, np.r_[np.full(N - 1, tau), tau / 2], atol=1e-15)
    np.testing.assert_allclose(times, tau * np.arange(1, N + 1), atol=1e-15)


@pytest.mark.parametrize("p", [1, 2])
def test_time_identities(p):
    t = synth.graded_time_nodes(1.7, 1.5, N0=7, levels=1)
    Mf, Bf, times = fe_time.assemble_time_full(p, t)
    # partition of unity: sum_j phi_j' = 0  ->  zero row sums of the full B
    np.testing.assert_allclose(Bf.sum(axis=1), 0.0, atol=1e-14)
    # integration by parts: B + B^T = [phi_j phi_k]_0^T = diag(-1, 0, ..., 0, 1)
    D = np.zeros_like(Bf)
    D[0, 0], D[-1, -1] = -1.0, 1.0
    np.testing.assert_allclose(Bf + Bf.T, D, atol=1e-14)
    # 1^T M 1 = T, M symmetric positive definite
    assert abs(Mf.sum() - t[-1]) < 1e-14
    np.testing.assert_allclose(Mf, Mf.T, atol=1e-16)
    assert np.linalg.eigvalsh(Mf).min() > 0
    # lifting weights m_t[k] = int phi_k = row sums of the full M (reduced rows)
    _, _, m, _ = fe_time.assemble_time(p, t)
    np.testing.assert_allclose(m, Mf.sum(axis=1)[1:], atol=1e-15)
    # DOF times strictly increasing and inside (0, T]
    assert np.all(np.diff(times) > 0) and times[0] == 0.0 and abs(times[-1] - t[-1]) < 1e-15


# ------------------------------------------------------------------ space matrices
@pytest.mark.parametrize("Lx,Ly", [(1.0, 1.0), (1.0, 0.6)])
def test_space_stencil_closed_form(Lx, Ly):
    n = 7
    h1, h2 = Lx / n, Ly / n
    Mx, Ax = fe_space.assemble_space(n, Lx, Ly)
    m = n - 1
    A, M = Ax.toarray(), Mx.toarray()
    i = 2 + m * 3                                   # an interior node away from the boundary
    assert abs(A[i, i] - 2 * (h2 / h1 + h1 / h2)) < 1e-14
    assert abs(A[i, i - 1] + h2 / h1) < 1e-14 and abs(A[i, i + 1] + h2 / h1) < 1e-14
    assert abs(A[i, i - m] + h1 / h2) < 1e-14 and abs(A[i, i + m] + h1 / h2) < 1e-14
    assert abs(A[i, i - m - 1]) < 1e-14 and abs(A[i, i + m + 1]) < 1e-14
    assert abs(A[i, i - m + 1]) < 1e-14 and abs(A[i, i + m - 1]) < 1e-14
    assert abs(M[i, i] - h1 * h2 / 2) < 1e-15
    for o in (1, m, m + 1):
        assert abs(M[i, i - o] - h1 * h2 / 12) < 1e-15 and abs(M[i, i + o] - h1 * h2 / 12) < 1e-15
    assert abs(M[i, i - m + 1]) < 1e-16 and abs(M[i, i + m - 1]) < 1e-16
    # half bandwidth m+1 under x1-fastest lexicographic order
    nz = np.nonzero(A + M)
    assert np.max(nz[0] - nz[1]) == m + 1


def test_space_kron_structure():
    """A_x = (h2/h1) I (x) T + (h1/h2) T (x) I with T = tridiag(-1, 2, -1) (library kron)."""
    n, Lx, Ly = 9, 1.3, 0.8
    h1, h2 = Lx / n, Ly / n
    m = n - 1
    _, Ax = fe_space.assemble_space(n, Lx, Ly)
    T = sp.diags([-np.ones(m - 1), 2 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1])
    I = sp.identity(m)
    ref = (h2 / h1) * sp.kron(I, T) + (h1 / h2) * sp.kron(T, I)
    assert abs(Ax - ref).max() < 1e-14


def test_space_identities():
    n, Lx, Ly = 6, 1.0, 2.0
    M, A = fe_space.assemble_space_full(n, Lx, Ly)
    np.testing.assert_allclose(np.asarray(A.sum(axis=1)).ravel(), 0.0, atol=1e-13)
    assert abs(M.sum() - Lx * Ly) < 1e-13
    x1, x2 = fe_space.interior_node_coords(n, Lx, Ly)
    y1, y2 = synth.interior_coords(n, Lx, Ly)
    np.testing.assert_allclose(x1, y1, atol=1e-15)
    np.testing.assert_allclose(x2, y2, atol=1e-15)


# ------------------------------------------------------------------ space-time assembly
@pytest.mark.parametrize("p,graded,Lx,Ly", [(1, False, 1.0, 1.0), (2, False, 1.0, 1.0),
                                             (1, True, 1.2, 0.7), (2, True, 1.0, 1.0)])
def test_explicit_equals_kron(p, graded, Lx, Ly):
    n = 5
    t = synth.graded_time_nodes(1.3, 1.5, N0=4, levels=0) if graded else synth.uniform_time_nodes(4, 1.3)
    K = assemble.explicit_system(n, p, t, Lx, Ly)
    M_t, B_t, _, _ = fe_time.assemble_time(p, t)
    M_x, A_x = fe_space.assemble_space(n, Lx, Ly)
    Kk = assemble.kron_system(M_t, B_t, M_x, A_x)
    assert K.shape == Kk.shape
    assert abs(K - Kk).max() < 1e-14


def test_load_vector_exact_for_nodal_polynomial():
    """For f = 1 the load is int phi_k * int varphi_alpha = m_t (x) (M_x_full row sums)."""
    n, p = 5, 2
    t = synth.uniform_time_nodes(3, 0.9)
    F = assemble.load_vector(n, p, t, lambda x1, x2, tt: np.ones_like(x1) + 0j)
    _, _, m_t, _ = fe_time.assemble_time(p, t)
    Mf, _ = fe_space.assemble_space_full(n)
    imap = fe_space.interior_map(n)
    keep = np.nonzero(imap >= 0)[0]
    rows = np.asarray(Mf.sum(axis=1)).ravel()[keep[np.argsort(imap[keep])]]
    np.testing.assert_allclose(F, np.outer(m_t, rows), atol=1e-15)
