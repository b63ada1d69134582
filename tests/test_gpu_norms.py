"""GPU error norms and quadrature loads (manufactured solutions of Section 4) against the oracle,
and the paper's Tables 2 and 3 (fast diagonalisation, P1, uniform and graded temporal meshes,
T = 5) reproduced with the GPU solver for J = 0..3: errors within the soft +-25% of the printed
values (reading S3), kappa_2(X_t) within 5%, convergence orders 2 (L2) and 1 (H1)."""
import numpy as np
import pytest

import synth
from oracle import assemble, norms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_07269_gb300 import build

    build.build()
    return torch.device("cuda:0")


EXACT = {"c1": (synth.psi_c1, synth.psi_c1_derivs, synth.f_c1),
         "paper": (synth.psi_paper, synth.psi_paper_derivs, synth.f_paper)}


@pytest.mark.parametrize("exact,n,p,N,T,graded,Lx", [
    ("c1", 8, 1, 6, 1.0, False, 1.0),
    ("paper", 7, 2, 4, 1.3, False, 1.0),
    ("paper", 9, 1, 5, 2.0, True, 1.2),
])
def test_error_norms_match_oracle(dev, exact, n, p, N, T, graded, Lx):
    """Both norms of a seeded nodal field against the oracle's prism quadrature (same rules)."""
    from paper_2504_07269_gb300 import stfdm

    t = synth.graded_time_nodes(T, 1.5, N0=N) if graded else synth.uniform_time_nodes(N, T)
    h = stfdm.setup_problem(n, p, t, Lx, 1.0, device=0)
    U = synth.cn01((h.n_t + 1, h.n_x), seed=60 + n)
    psi, dpsi, _ = EXACT[exact]
    ref = norms.errors(n, p, t, U, psi, dpsi, Lx, 1.0, t_order=4, x_order=4)
    got = stfdm.st_error_norms(h, exact, torch.from_numpy(U[1:]).to(dev), torch.from_numpy(U[0]).to(dev), 4, 4)
    print(exact, n, p, N, "oracle", ref, "gpu", got)
    assert abs(got[0] - ref[0]) <= 1e-12 * ref[0]
    assert abs(got[1] - ref[1]) <= 1e-12 * ref[1]


@pytest.mark.parametrize("exact,n,p,N,T,graded", [("c1", 8, 1, 6, 1.0, False), ("paper", 7, 2, 4, 1.3, True)])
def test_load_quadrature_matches_oracle(dev, exact, n, p, N, T, graded):
    from paper_2504_07269_gb300 import stfdm

    t = synth.graded_time_nodes(T, 1.5, N0=N) if graded else synth.uniform_time_nodes(N, T)
    h = stfdm.setup_problem(n, p, t, device=0)
    ref = assemble.load_vector(n, p, t, EXACT[exact][2], t_order=6, x_order=6)
    F = stfdm.st_load_quadrature(h, exact, q_t=6, q_x=6).cpu().numpy()
    assert np.abs(F - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("table", ["table2_fdm_uniform", "table3_fdm_graded"])
def test_paper_tables_on_gpu(dev, table):
    """J = 0..3 of Tables 2 (uniform temporal mesh) and 3 (graded initial mesh t_l = T (l/64)^1.5,
    bisected J times): n = 32 2^J squares, T = 5, psi = e^{it} sin(pi x1) sin(pi x2) sin(t x1 x2)
    (psi0 = 0); load by quadrature, mixed-precision solve, GPU norms; kappa_2(X_t) from the setup."""
    import time

    from paper_2504_07269_gb300 import stfdm

    rows = [l.split() for l in open(__file__.replace("test_gpu_norms.py", f"golden/{table}.txt"))
            if l.strip() and not l.startswith("#")]
    errs = []
    for J in range(4):
        n = 32 * 2 ** J
        if table.startswith("table2"):
            t = synth.uniform_time_nodes(64 * 2 ** J, 5.0)
        else:
            t = synth.graded_time_nodes(5.0, 1.5, N0=64, levels=J)
        h = stfdm.setup_problem(n, 1, t, device=0)
        F = stfdm.st_load_quadrature(h, "paper", q_t=6, q_x=6)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        psi, info = stfdm.st_fdm_solve(h, F, None, precision="mixed")
        torch.cuda.synchronize()
        ts = time.perf_counter() - t0
        l2, h1 = stfdm.st_error_norms(h, "paper", psi, None, 4, 4)
        errs.append((l2, h1))
        pl2, ph1, pk = float(rows[J][3]), float(rows[J][5]), float(rows[J][8])
        print(f"{table} J={J}: {h.n_t * h.n_x} unknowns, L2 {l2:.3e} (paper {pl2:.1e}), H1 {h1:.3e} (paper "
              f"{ph1:.1e}), kappa {h.kappa:.2e} (paper {pk:.1e}), solve {ts:.2f} s (paper {rows[J][7]} s on 24 CPU "
              f"cores), sweeps {info['sweeps']}")
        assert abs(l2 / pl2 - 1) <= 0.25 and abs(h1 / ph1 - 1) <= 0.25
        assert abs(h.kappa / pk - 1) <= 0.05
        del psi, F
    for J in range(1, 4):
        eoc_l2 = np.log2(errs[J - 1][0] / errs[J][0])
        eoc_h1 = np.log2(errs[J - 1][1] / errs[J][1])
        print(f"{table} J={J}: eoc L2 {eoc_l2:.2f}, H1 {eoc_h1:.2f}")
        assert 1.8 <= eoc_l2 <= 2.2 and 0.9 <= eoc_h1 <= 1.1
