"""Element-wise parity against the oracle at the sizes the configurations name for it, and at
spatial bands wider than 256 (the 384x384 configuration's kernel variants), through the C ABI.

  * 64x64 squares, P1 time on 128 elements, T = 1 (508,032 unknowns): the 256x256 workload's
    error-check size.  Reference: the oracle's space-eigenbasis solve (dense generalized eig of
    (A_x, M_x), then one banded time system per spatial mode): independent of the time
    diagonalisation the GPU path uses.
  * 260x260 squares (b = 260) with P2 time on 4 elements (n_t = 8) and 384x384 squares (b = 384,
    the 384^2 configuration's band) with P1 time on 4 elements: discrete manufactured solutions
    with a packet psi0; reference: the oracle's FP64 FDM with one FP64 refinement sweep (the
    explicit system is too large for SuperLU here; kappa_2(X_t) is small at these n_t).
Bars: FP64 <= 1e-11 relative l2, mixed precision <= 1e-9.
"""
import numpy as np
import pytest

import synth
from oracle import cpu_fdm, fe_space, fe_time, solve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_07269_gb300 import build

    build.build()
    return torch.device("cuda:0")


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("solver", ["banded", "multifrontal"])
def test_c2_check_size_vs_space_eig_oracle(dev, solver):
    from paper_2504_07269_gb300 import stfdm

    pr = synth.config_problem("c2check")
    M_t, B_t, m_t, times = fe_time.assemble_time(pr.p_t, pr.t_nodes)
    Mf, _, tfull = fe_time.assemble_time_full(pr.p_t, pr.t_nodes)
    M_x, A_x = fe_space.assemble_space(pr.n)
    x1, x2 = synth.interior_coords(pr.n)
    f = synth.f_c1(x1[None, :], x2[None, :], tfull[:, None])
    F = Mf[1:] @ (M_x @ f.T).T                    # interpolated load (M_t,full (x) M_x) f
    psi0 = synth.psi0_c1(x1, x2)
    ref = solve.solve_space_eig(M_t, B_t, M_x, A_x, F - np.outer(m_t, A_x @ psi0)) + psi0[None, :]
    _, r_ref = solve.residual(M_t, B_t, M_x, A_x, ref - psi0[None, :], F - np.outer(m_t, A_x @ psi0))
    h = stfdm.setup_problem(pr.n, pr.p_t, pr.t_nodes, device=0, spatial_solver=solver)
    Fd, p0 = torch.from_numpy(F).to(dev), torch.from_numpy(psi0).to(dev)
    psi64, _ = stfdm.st_fdm_solve(h, Fd, p0, precision="fp64")
    psim, info = stfdm.st_fdm_solve(h, Fd, p0, precision="mixed")
    e64, em = rel(psi64.cpu().numpy(), ref), rel(psim.cpu().numpy(), ref)
    print(f"64x64/128 {solver} ({pr.unknowns} unknowns): oracle residual {r_ref:.1e}; fp64 {e64:.2e}, mixed {em:.2e} "
          f"({info['sweeps']} FP32 applications, residual {info['rel_residual']:.1e})")
    assert e64 <= 1e-11
    assert em <= 1e-9
    exact = synth.psi_c1(x1[None, :], x2[None, :], times[:, None])
    assert np.abs(psim.cpu().numpy() - exact).max() < 2e-3     # discretisation error at this mesh


@pytest.mark.parametrize("n,p,N,solver", [(260, 2, 4, "banded"), (384, 1, 4, "banded"), (384, 1, 4, "multifrontal")])
def test_wide_band_vs_refined_cpu_fdm(dev, n, p, N, solver):
    from paper_2504_07269_gb300 import stfdm

    t = synth.uniform_time_nodes(N, 1.0)
    M_t, B_t, m_t, _ = fe_time.assemble_time(p, t)
    M_x, A_x = fe_space.assemble_space(n)
    x1, x2 = synth.interior_coords(n)
    psi0 = synth.packet_values(synth.packet_params(n), x1, x2)
    u = synth.cn01((p * N, (n - 1) ** 2), seed=n + p)
    F = solve.kron_apply(M_t, B_t, M_x, A_x, u) + np.outer(m_t, A_x @ psi0)   # psi = u + psi0
    rep = {}
    ref = cpu_fdm.cpu_fdm_refined(n, p, t, F, psi0, sweeps=1, report=rep)
    h = stfdm.setup_problem(n, p, t, device=0, spatial_solver=solver)
    assert h.m + 1 == n and h.m + 1 > 256
    Fd, p0 = torch.from_numpy(F).to(dev), torch.from_numpy(psi0).to(dev)
    psi64, _ = stfdm.st_fdm_solve(h, Fd, p0, precision="fp64")
    # the discrete manufactured solution is white noise, with as much weight on the operator's small
    # singular directions as on any other, so the error/residual ratio approaches cond(K) (~1e5 at
    # these bands): refine to 1e-13
    psim, info = stfdm.st_fdm_solve(h, Fd, p0, precision="mixed", tol=1e-13, max_sweeps=60)
    e64, em = rel(psi64.cpu().numpy(), ref), rel(psim.cpu().numpy(), ref)
    exact = u + psi0[None, :]
    print(f"b={n} P{p} n_t={p * N} {solver} ({u.size} unknowns): oracle residuals {rep['residuals']}, oracle vs u* "
          f"{rel(ref, exact):.1e}; fp64 {e64:.2e}, mixed {em:.2e} ({info['sweeps']} FP32 applications); "
          f"fp64 vs u* {rel(psi64.cpu().numpy(), exact):.1e}")
    assert rep["residuals"][-1] <= 1e-14
    assert e64 <= 1e-11
    assert em <= 1e-9
