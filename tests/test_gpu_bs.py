"""GPU Bartels-Stewart solve (Schur choice of step 1, eq. LGS_x) through the C ABI, against the
oracle: the explicit space-time system solved by SuperLU, and the oracle's own Bartels-Stewart.

Bar: FP64 <= 1e-11 relative l2.  Where kappa_2(X_t) is large (P2 on a graded temporal mesh), the
FDM's FP64 result carries that conditioning's rounding while Bartels-Stewart, whose Z is unitary,
does not: both errors are printed, and Bartels-Stewart's is asserted to be no larger."""
import numpy as np
import pytest

import synth
from oracle import assemble, fe_mesh, fe_space, fe_time, solve

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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("n,p,N,graded,solver", [
    (17, 1, 12, False, "banded"),
    (14, 2, 7, True, "banded"),
    (17, 1, 12, False, "multifrontal"),
    (2, 1, 1, False, "banded"),          # one node, one element
])
def test_bs_vs_explicit_oracle(dev, n, p, N, graded, solver):
    from paper_2504_07269_gb300 import stfdm

    t = synth.graded_time_nodes(1.0, 1.5, N0=N) if graded else synth.uniform_time_nodes(N, 1.0)
    K = assemble.explicit_system(n, p, t)
    M_t, B_t, m_t, _ = fe_time.assemble_time(p, t)
    M_x, A_x = fe_space.assemble_space(n)
    x1, x2 = synth.interior_coords(n)
    psi0 = synth.packet_values(synth.packet_params(4), x1, x2)
    F = synth.cn01((M_t.shape[0], M_x.shape[0]), seed=80 + n)
    Ft = F - np.outer(m_t, A_x @ psi0)
    ref = solve.solve_explicit(K, Ft) + psi0[None, :]
    ref_bs = solve.bartels_stewart(M_t, B_t, M_x, A_x, Ft) + psi0[None, :]
    assert rel(ref_bs, ref) <= 1e-12                      # the oracle's two paths agree
    h = stfdm.setup_problem(n, p, t, device=0, spatial_solver=solver)
    psi, info = stfdm.st_bs_solve(h, torch.from_numpy(F).to(dev), torch.from_numpy(psi0).to(dev))
    e = rel(psi.cpu().numpy(), ref)
    print(f"BS n={n} P{p} N={N} graded={graded} {solver}: {e:.2e} ({info['kernel_launches']} launches)")
    assert e <= 1e-11
    # the handle still solves with the FDM afterwards (the kept Schur-shift factors were dropped)
    psim, _ = stfdm.st_fdm_solve(h, torch.from_numpy(F).to(dev), torch.from_numpy(psi0).to(dev), precision="mixed")
    assert rel(psim.cpu().numpy(), ref) <= 1e-9


def test_bs_robust_where_kappa_is_large(dev):
    """P2 time on a graded mesh with 1000 elements (n_t = 2000) over a small spatial mesh: kappa_2(X_t)
    is large.  Against the discrete manufactured solution u* (F = K u*), the FDM's FP64 error carries
    the rounding of X_t; Bartels-Stewart's unitary Z does not (both printed)."""
    from paper_2504_07269_gb300 import stfdm

    n, p = 6, 2
    t = synth.graded_time_nodes(2.0, 1.5, N0=1000)
    M_t, B_t, m_t, _ = fe_time.assemble_time(p, t)
    M_x, A_x = fe_space.assemble_space(n)
    u = synth.cn01((M_t.shape[0], (n - 1) ** 2), seed=91)
    F = solve.kron_apply(M_t, B_t, M_x, A_x, u)
    h = stfdm.setup_problem(n, p, t, device=0)
    Fd = torch.from_numpy(F).to(dev)
    psi_bs, _ = stfdm.st_bs_solve(h, Fd)
    psi_fdm, _ = stfdm.st_fdm_solve(h, Fd, precision="fp64")
    e_bs, e_fdm = rel(psi_bs.cpu().numpy(), u), rel(psi_fdm.cpu().numpy(), u)
    print(f"n_t = {M_t.shape[0]}, kappa_2(X_t) = {h.kappa:.2e}: Bartels-Stewart {e_bs:.2e}, FDM (FP64) {e_fdm:.2e}")
    assert h.kappa > 1e3
    assert e_bs <= 1e-11
    assert e_bs <= e_fdm


def test_bs_on_a_tetrahedral_mesh(dev):
    from paper_2504_07269_gb300 import stfdm

    coords, cells = synth.cube_tet_mesh(5, jitter=0.2, seed=33)
    t = synth.uniform_time_nodes(6, 1.0)
    Mx, Ax, xin = fe_mesh.assemble_mesh(coords, cells, 1)
    M_t, B_t, m_t, _ = fe_time.assemble_time(1, t)
    psi0 = synth.packet_values_nd(synth.packet_params(9), xin)
    F = synth.cn01((M_t.shape[0], Mx.shape[0]), seed=92)
    Ft = F - np.outer(m_t, Ax @ psi0)
    ref = solve.solve_explicit(assemble.kron_system(M_t, B_t, Mx, Ax), Ft) + psi0[None, :]
    h = stfdm.setup_mesh_problem(3, 1, coords, cells, 1, t, device=0)
    psi, _ = stfdm.st_bs_solve(h, torch.from_numpy(F).to(dev), torch.from_numpy(psi0).to(dev))
    assert rel(psi.cpu().numpy(), ref) <= 1e-11
