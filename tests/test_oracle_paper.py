"""Pins of the oracle against the paper's printed results and the model problem (CPU only)."""
import numpy as np
import pytest

import synth
from conftest import read_golden
from oracle import assemble, cpu_fdm, fe_space, fe_time, norms, solve


def test_manufactured_rhs_symbolic():
    """f = i d_t psi - Laplace_x psi (eq. SchroedingerBeschraenkt) for both manufactured solutions,
    checked symbolically with sympy against synth's closed forms at random points."""
    sympy = pytest.importorskip("sympy")
    x1, x2, t = sympy.symbols("x1 x2 t", real=True)
    I = sympy.I
    cases = [
        (sympy.sin(sympy.pi * x1) * sympy.sin(sympy.pi * x2) * (1 + t) * sympy.exp(-I * t),
         synth.f_c1, synth.psi_c1_derivs),
        (sympy.exp(I * t) * sympy.sin(sympy.pi * x1) * sympy.sin(sympy.pi * x2) * sympy.sin(t * x1 * x2),
         synth.f_paper, synth.psi_paper_derivs),
    ]
    rng = np.random.default_rng(0)
    pts = rng.uniform(0, 1, size=(6, 3)) * np.array([1, 1, 3])
    for psi, fnum, dnum in cases:
        f = I * sympy.diff(psi, t) - sympy.diff(psi, x1, 2) - sympy.diff(psi, x2, 2)
        fl = sympy.lambdify((x1, x2, t), f, "numpy")
        dl = [sympy.lambdify((x1, x2, t), sympy.diff(psi, v), "numpy") for v in (t, x1, x2)]
        for a, b, c in pts:
            assert abs(complex(fl(a, b, c)) - complex(fnum(a, b, c))) < 1e-11
            got = dnum(a, b, c)
            for k in range(3):
                assert abs(complex(dl[k](a, b, c)) - complex(got[k])) < 1e-11


@pytest.mark.slow
def test_paper_errors_and_eoc():
    """Tables 1-2, J = 0, 1: errors of the explicit oracle (J=0) and of the CPU FDM (J=1, checked
    against the explicit oracle at J=0) within 25 % of the printed values (the paper's mesh figure
    is missing, so the absolute values are a soft pin) and convergence orders ~2 (L2) and ~1 (H1)."""
    rows = read_golden("table2_fdm_uniform.txt")
    errs = []
    for J in (0, 1):
        pr = synth.config_problem(f"paperJ{J}")
        assert pr.unknowns == int(rows[J][0])
        F = assemble.load_vector(pr.n, 1, pr.t_nodes, synth.f_paper)
        M_t, B_t, _, _ = fe_time.assemble_time(1, pr.t_nodes)
        M_x, A_x = fe_space.assemble_space(pr.n)
        U = solve.fdm(M_t, B_t, M_x, A_x, F)
        if J == 0:
            K = assemble.explicit_system(pr.n, 1, pr.t_nodes)
            Ue = solve.solve_explicit(K, F)
            assert np.linalg.norm(U - Ue) / np.linalg.norm(Ue) < 1e-11
        Ufull = np.vstack([np.zeros((1, U.shape[1])), U])
        l2, h1 = norms.errors(pr.n, 1, pr.t_nodes, Ufull, synth.psi_paper, synth.psi_paper_derivs)
        assert abs(l2 / float(rows[J][3]) - 1) < 0.25, (J, l2)
        assert abs(h1 / float(rows[J][5]) - 1) < 0.25, (J, h1)
        errs.append((l2, h1))
    eoc_l2 = np.log2(errs[0][0] / errs[1][0])
    eoc_h1 = np.log2(errs[0][1] / errs[1][1])
    assert 1.8 < eoc_l2 < 2.2 and abs(eoc_l2 - float(rows[1][4])) < 0.1
    assert 0.9 < eoc_h1 < 1.1 and abs(eoc_h1 - float(rows[1][6])) < 0.1


@pytest.mark.slow
def test_cpu_fdm_pool_matches_explicit():
    """The process-pool CPU FDM (the timed CPU baseline) equals the explicit oracle, with lifting."""
    pr = synth.config_problem("c1")
    x1, x2 = synth.interior_coords(pr.n)
    psi0 = synth.psi0_c1(x1, x2)
    F = assemble.load_vector(pr.n, 1, pr.t_nodes, synth.f_c1)
    K = assemble.explicit_system(pr.n, 1, pr.t_nodes)
    L = assemble.lifting_vector(pr.n, 1, pr.t_nodes, psi0)
    U_ref = solve.solve_explicit(K, F - L) + psi0[None, :]
    tm = {}
    U = cpu_fdm.cpu_fdm(pr.n, 1, pr.t_nodes, F, psi0, workers=2, timings=tm)
    assert np.linalg.norm(U - U_ref) / np.linalg.norm(U_ref) < 1e-12
    assert tm["workers"] == 2 and tm["solve"] > 0
    # the discrete solution converges to the manufactured one: nodal error small at C1
    tt = fe_time.assemble_time(1, pr.t_nodes)[3]
    exact = synth.psi_c1(x1[None, :], x2[None, :], tt[:, None])
    assert np.abs(U - exact).max() < 2e-2


@pytest.mark.slow
def test_cpu_fdm_refined_reaches_the_residual_floor():
    """One classical FP64 refinement sweep of the process-pool CPU FDM: the residual drops to the
    FP64 floor (well below the unrefined FDM's, whose rounding grows with kappa_2(X_t)), and the
    refined solution equals the explicit oracle's; psi0 enters through the lifting."""
    n, p, t = 10, 2, synth.uniform_time_nodes(40, 2.0)
    M_t, B_t, m_t, _ = fe_time.assemble_time(p, t)
    M_x, A_x = fe_space.assemble_space(n)
    x1, x2 = synth.interior_coords(n)
    psi0 = synth.packet_values(synth.packet_params(3), x1, x2)
    u = synth.cn01((p * 40, (n - 1) ** 2), seed=5)
    F = solve.kron_apply(M_t, B_t, M_x, A_x, u) + np.outer(m_t, A_x @ psi0)
    rep = {}
    U = cpu_fdm.cpu_fdm_refined(n, p, t, F, psi0, sweeps=1, workers=2, report=rep)
    r0, r1 = rep["residuals"]
    assert r1 < 1e-14 and r1 < 0.1 * r0
    ref = solve.solve_explicit(assemble.explicit_system(n, p, t), F - np.outer(m_t, A_x @ psi0)) + psi0[None, :]
    assert np.linalg.norm(U - ref) / np.linalg.norm(ref) < 1e-13
    assert np.linalg.norm(U - u - psi0[None, :]) / np.linalg.norm(u) < 1e-12
    assert np.linalg.norm(rep["unrefined"] - ref) / np.linalg.norm(ref) < 1e-10
