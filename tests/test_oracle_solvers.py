"""Pins of the oracle's solvers, time decomposition, lifting and norms (CPU only)."""
import numpy as np
import pytest

import synth
from conftest import read_golden
from oracle import assemble, fe_space, fe_time, norms, solve, timedec


def _mats(n, p, t, Lx=1.0, Ly=1.0):
    M_t, B_t, m_t, _ = fe_time.assemble_time(p, t)
    M_x, A_x = fe_space.assemble_space(n, Lx, Ly)
    return M_t, B_t, m_t, M_x, A_x


@pytest.mark.parametrize("p", [1, 2])
def test_dense_brute_force_equals_superlu(p):
    n, t = 4, synth.uniform_time_nodes(3, 0.8)
    K = assemble.explicit_system(n, p, t)
    F = synth.cn01((p * 3, 9), seed=11)
    np.testing.assert_allclose(solve.solve_explicit(K, F), solve.solve_dense(K, F), rtol=0, atol=1e-12)


@pytest.mark.parametrize("p,graded", [(1, False), (2, False), (1, True)])
def test_discrete_manufactured_solution(p, graded):
    """F = K u* for a random u*; every solver must return u*."""
    n = 8
    t = synth.graded_time_nodes(1.0, 1.5, N0=6) if graded else synth.uniform_time_nodes(6, 1.0)
    K = assemble.explicit_system(n, p, t)
    M_t, B_t, _, M_x, A_x = _mats(n, p, t)
    u = synth.cn01((p * 6, 49), seed=3)
    F = (K @ u.reshape(-1)).reshape(u.shape)
    np.testing.assert_allclose(solve.kron_apply(M_t, B_t, M_x, A_x, u), F, atol=1e-14)
    for name, fn in [("explicit", lambda: solve.solve_explicit(K, F)),
                     ("space_eig", lambda: solve.solve_space_eig(M_t, B_t, M_x, A_x, F)),
                     ("fdm", lambda: solve.fdm(M_t, B_t, M_x, A_x, F)),
                     ("bs", lambda: solve.bartels_stewart(M_t, B_t, M_x, A_x, F))]:
        U = fn()
        err = np.linalg.norm(U - u) / np.linalg.norm(u)
        assert err < 1e-11, (name, err)
    R, rel = solve.residual(M_t, B_t, M_x, A_x, solve.solve_explicit(K, F), F)
    assert rel < 1e-14


def test_adjoint_apply_is_conjugate_transpose():
    n, p, t = 5, 2, synth.uniform_time_nodes(3, 1.0)
    K = assemble.explicit_system(n, p, t)
    M_t, B_t, _, M_x, A_x = _mats(n, p, t)
    u = synth.cn01((6, 16), seed=5)
    ref = (K.conj().T @ u.reshape(-1)).reshape(u.shape)
    np.testing.assert_allclose(solve.kron_apply_adjoint(M_t, B_t, M_x, A_x, u), ref, atol=1e-14)


@pytest.mark.parametrize("p", [1, 2])
def test_time_decomposition(p):
    t = synth.uniform_time_nodes(20, 1.5)
    M_t, B_t, _, _ = fe_time.assemble_time(p, t)
    X, s, Y, kappa = timedec.fdm_decomposition(M_t, B_t)
    A = np.linalg.solve(1j * B_t, M_t)
    np.testing.assert_allclose(A @ X, X * s[None, :], atol=1e-12)
    np.testing.assert_allclose(np.linalg.norm(X, axis=0), 1.0, atol=1e-14)
    np.testing.assert_allclose(Y @ (1j * B_t) @ X, np.eye(len(s)), atol=1e-10)
    # every shifted spatial matrix has a negative definite imaginary part: Im s_k < 0
    assert np.max(s.imag) < 0
    Xs, S, Ys = timedec.schur_decomposition(M_t, B_t)
    np.testing.assert_allclose(Xs.conj().T @ Xs, np.eye(len(s)), atol=1e-13)
    np.testing.assert_allclose(np.tril(S, -1), 0.0, atol=0)
    np.testing.assert_allclose(np.sort_complex(np.diag(S)), np.sort_complex(s), atol=1e-12)


def test_kappa_independent_of_T():
    """Section 4: kappa_2(X_t) depends only on n_t for a uniform mesh; s_k scales with T."""
    a = timedec.fdm_decomposition(*fe_time.assemble_time(1, synth.uniform_time_nodes(32, 1.0))[:2])
    b = timedec.fdm_decomposition(*fe_time.assemble_time(1, synth.uniform_time_nodes(32, 5.0))[:2])
    assert abs(a[3] / b[3] - 1) < 1e-10
    np.testing.assert_allclose(np.sort_complex(5.0 * a[1]), np.sort_complex(b[1]), rtol=1e-10)


def _fmt2(x):
    return "%.1e" % x


@pytest.mark.parametrize("J", [0, 1, 2, 3, 4])
def test_kappa_table2_uniform(J):
    """kappa_2(X_t) column of Table 2 (unit 2-norm eigenvector columns), 2 significant digits."""
    row = read_golden("table2_fdm_uniform.txt")[J]
    M_t, B_t, _, _ = fe_time.assemble_time(1, synth.uniform_time_nodes(64 * 2 ** J, 5.0))
    kappa = timedec.fdm_decomposition(M_t, B_t)[3]
    assert _fmt2(kappa) == "%.1e" % float(row[8]), (kappa, row[8])


@pytest.mark.parametrize("J", [0, 1, 2, 3, 4])
def test_kappa_table3_graded(J):
    """kappa_2(X_t) column of Table 3 (graded mesh q=1.5, bisection refinement)."""
    row = read_golden("table3_fdm_graded.txt")[J]
    M_t, B_t, _, _ = fe_time.assemble_time(1, synth.graded_time_nodes(5.0, 1.5, 64, J))
    kappa = timedec.fdm_decomposition(M_t, B_t)[3]
    assert _fmt2(kappa) == "%.1e" % float(row[8]), (kappa, row[8])


def test_graded_mesh_ratio():
    """Section 4: h_t ~ 12 h_t,min for the graded meshes."""
    t = synth.graded_time_nodes(5.0, 1.5, 64, 0)
    h = np.diff(t)
    assert 11.5 < h.max() / h.min() < 12.5
    assert abs(h.max() - 1.2e-1) < 0.05e-1   # printed h_t of Table 3, J=0


@pytest.mark.parametrize("p", [1, 2])
def test_lifting_equivalence(p):
    """Three readings of the psi0 lifting agree: prism quadrature of a(psi0_h, v),
    m_t (x) A_x psi0, and eliminating the t_0 trial DOFs of the full system."""
    n, t = 6, synth.uniform_time_nodes(5, 1.2)
    M_t, B_t, m_t, M_x, A_x = _mats(n, p, t)
    x1, x2 = synth.interior_coords(n)
    psi0 = synth.packet_values(synth.packet_params(7, 2), x1, x2)
    L = assemble.lifting_vector(n, p, t, psi0)
    np.testing.assert_allclose(L, np.outer(m_t, A_x @ psi0), atol=1e-14)
    F = synth.cn01((p * 5, 25), seed=2)
    K = assemble.explicit_system(n, p, t)
    Kf = assemble.explicit_system(n, p, t, keep_t0=True)
    n_x = 25
    u_hat = solve.solve_explicit(K, F - L)
    rhs = F.reshape(-1) - Kf[:, :n_x] @ psi0
    u_nodal = solve.solve_explicit(K, rhs.reshape(F.shape))
    np.testing.assert_allclose(u_hat + psi0[None, :], u_nodal, atol=1e-12)


def test_norms_closed_form():
    """||psi||_{L2(Q)}^2 = (1/4) int (1+t)^2 and |psi|_{H1(Q)}^2 = (1/4) int 1+(1+t)^2 + (pi^2/2) int (1+t)^2
    for psi_c1 on (0,1)^2 x (0,1): errors of psi_h = 0."""
    n, p, T = 12, 1, 1.0
    t = synth.uniform_time_nodes(4, T)
    U0 = np.zeros((5, (n - 1) ** 2), dtype=np.complex128)
    l2, h1 = norms.errors(n, p, t, U0, synth.psi_c1, synth.psi_c1_derivs, t_order=5, x_order=7)
    I2 = ((1 + T) ** 3 - 1) / 3
    assert abs(l2 ** 2 - 0.25 * I2) < 1e-9
    assert abs(h1 ** 2 - (0.25 * (T + I2) + np.pi ** 2 / 2 * I2)) < 1e-7


def test_norms_vanish_on_discrete_function():
    """psi_h reproduces any function of Q^p_h exactly: e = 0 for psi = bilinear in (x-separable, t)."""
    n, p = 4, 1
    t = synth.uniform_time_nodes(3, 1.0)
    x1, x2 = synth.interior_coords(n)
    tt = np.r_[0.0, fe_time.assemble_time(p, t)[3]]
    # psi = x1 (1-x1)... is not piecewise linear; use the P1 interpolant of g(x) h(t) with g
    # piecewise linear: g = 0 except one hat at an interior node, h(t) = t.
    g = np.zeros((n - 1) ** 2)
    g[4] = 1.0
    U = np.outer(tt, g).astype(np.complex128)
    hx, hy = 1.0 / n, 1.0 / n
    cx, cy = x1[4], x2[4]

    def hat(a, b):
        # P1 hat of the SW-NE split mesh at (cx, cy): max(0, 1 - max(|dx|,|dy|,|dx-dy|)) in grid units
        dx, dy = (a - cx) / hx, (b - cy) / hy
        return np.maximum(0.0, 1.0 - np.maximum(np.maximum(np.abs(dx), np.abs(dy)), np.abs(dx - dy)))

    def psi(a, b, s):
        return hat(a, b) * s + 0j

    def dpsi(a, b, s):
        eps = 1e-7
        return (hat(a, b) + 0j, (hat(a + eps, b) - hat(a - eps, b)) / (2 * eps) * s,
                (hat(a, b + eps) - hat(a, b - eps)) / (2 * eps) * s)

    l2, h1 = norms.errors(n, p, t, U, psi, dpsi)
    assert l2 < 1e-14
    assert h1 < 1e-6
