"""GPU parity of the general-mesh path (unstructured triangles, tetrahedra, P1 and P2 in space)
through the C ABI: the sparse-direct multifrontal spatial solver, the CSR residual and lifting,
against the oracle (its own mesh assembly, Kronecker system, SuperLU).

Bars: FP64 <= 1e-11 relative l2, mixed precision after refinement <= 1e-9; spatial solves
against SuperLU: FP64 <= 1e-11, FP32 <= 1e-3 (cond(C_k) u_32)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

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


MESHES = {
    "tri": lambda: synth.square_delaunay_mesh(14, jitter=0.3, seed=31),
    "tet": lambda: synth.cube_tet_mesh(6, jitter=0.2, seed=32),
    "tet8": lambda: synth.cube_tet_mesh(8, jitter=0.2, seed=34),
    "tri40": lambda: synth.square_delaunay_mesh(40, jitter=0.3, seed=35),
}

CASES = [
    # mesh, p_x, p_t, N_t, T
    ("tri", 1, 1, 9, 1.0),
    ("tri", 2, 2, 5, 0.8),
    ("tet", 1, 1, 7, 1.0),
    ("tet", 2, 1, 4, 0.5),
    ("tet8", 2, 1, 3, 0.5),      # fronts of every size class (one warp, up to 64, larger)
    ("tri40", 2, 1, 5, 1.0),
]


@pytest.mark.parametrize("kind,p_x,p_t,N,T", CASES)
def test_mesh_solve_vs_oracle(dev, kind, p_x, p_t, N, T):
    from paper_2504_07269_gb300 import stfdm

    coords, cells = MESHES[kind]()
    dim = coords.shape[1]
    t = synth.uniform_time_nodes(N, T)
    Mx, Ax, xin = fe_mesh.assemble_mesh(coords, cells, p_x)
    M_t, B_t, m_t, _ = fe_time.assemble_time(p_t, t)
    K = assemble.kron_system(M_t, B_t, Mx, Ax)
    n_t, n_x = M_t.shape[0], Mx.shape[0]
    psi0 = synth.packet_values_nd(synth.packet_params(7), xin)
    F = synth.cn01((n_t, n_x), seed=40 + dim + p_x)
    ref = solve.solve_explicit(K, F - np.outer(m_t, Ax @ psi0)) + psi0[None, :]
    h = stfdm.setup_mesh_problem(dim, p_x, coords, cells, p_t, t, device=0)
    assert (h.n_t, h.n_x) == (n_t, n_x)
    Fd, p0 = torch.from_numpy(F).to(dev), torch.from_numpy(psi0).to(dev)
    psi64, _ = stfdm.st_fdm_solve(h, Fd, p0, precision="fp64")
    psim, info = stfdm.st_fdm_solve(h, Fd, p0, precision="mixed")
    psi32, _ = stfdm.st_fdm_solve(h, Fd.to(torch.complex64), p0.to(torch.complex64), precision="fp32")
    e64, em, e32 = rel(psi64.cpu().numpy(), ref), rel(psim.cpu().numpy(), ref), rel(psi32.cpu().numpy(), ref)
    print(f"{kind} P{p_x}/P{p_t} (n_x {n_x}, n_t {n_t}): fp64 {e64:.2e}, mixed {em:.2e} ({info['sweeps']} FP32 "
          f"applications, kept {info['kept_systems']}), fp32 {e32:.2e}")
    assert e64 <= 1e-11
    assert em <= 1e-9
    assert e32 <= 1e-3
    # the FP64 residual through the CSR operators equals the oracle's, at an iterate that is not a solution
    U = synth.cn01((n_t, n_x), seed=45)
    Ud = torch.from_numpy(U).to(dev)
    R = torch.empty_like(psim)
    r_lib, _ = stfdm.st_residual(h, Fd, p0, Ud, R)
    Ro, r_or = solve.residual(M_t, B_t, Mx, Ax, U - psi0[None, :], F - np.outer(m_t, Ax @ psi0))
    assert abs(r_lib - r_or) <= 1e-12 * r_or
    assert np.abs(R.cpu().numpy() - Ro).max() <= 1e-12 * np.abs(Ro).max()


@pytest.mark.parametrize("kind,p_x", [("tri", 2), ("tet", 1)])
def test_mesh_spatial_solves_vs_superlu(dev, kind, p_x):
    """Step 3 alone, every eigen-index k, FP64 and FP32, against SuperLU on M_x + s_k A_x."""
    from paper_2504_07269_gb300 import stfdm

    coords, cells = MESHES[kind]()
    dim = coords.shape[1]
    t = synth.uniform_time_nodes(12, 1.0)
    h = stfdm.setup_mesh_problem(dim, p_x, coords, cells, 1, t, device=0)
    Mx, Ax, _ = fe_mesh.assemble_mesh(coords, cells, p_x)
    _, s, _, _ = stfdm.st_time_decompose(h.time)
    G = synth.cn01((h.n_t, h.n_x), seed=51)
    W64 = stfdm.st_spatial_solve(h, "fp64", torch.from_numpy(G).to(dev)).cpu().numpy()
    W32 = stfdm.st_spatial_solve(h, "fp32", torch.from_numpy(G).to(dev).to(torch.complex64)).cpu().numpy()
    for k in range(h.n_t):
        ref = spla.splu(sp.csc_matrix(Mx + s[k] * Ax, dtype=np.complex128)).solve(G[k])
        assert rel(W64[k], ref) <= 1e-11, k
        assert rel(W32[k], ref) <= 1e-3, k


def test_structured_grid_multifrontal_equals_banded(dev):
    """The structured grid solved by the multifrontal solver and by the banded one: both agree with
    the oracle's explicit prism-assembled system (ragged sizes, P2 time)."""
    from paper_2504_07269_gb300 import stfdm

    n, p, t = 23, 2, synth.uniform_time_nodes(6, 0.9)
    K = assemble.explicit_system(n, p, t)
    M_t, B_t, m_t, _ = fe_time.assemble_time(p, t)
    M_x, A_x = fe_space.assemble_space(n)
    x1, x2 = synth.interior_coords(n)
    psi0 = synth.packet_values(synth.packet_params(2), x1, x2)
    F = synth.cn01((M_t.shape[0], M_x.shape[0]), seed=60)
    ref = solve.solve_explicit(K, F - np.outer(m_t, A_x @ psi0)) + psi0[None, :]
    Fd, p0 = torch.from_numpy(F).to(dev), torch.from_numpy(psi0).to(dev)
    out = {}
    for solver in ("banded", "multifrontal"):
        h = stfdm.setup_problem(n, p, t, device=0, spatial_solver=solver)
        for prec in ("fp64", "mixed"):
            psi, _ = stfdm.st_fdm_solve(h, Fd, p0, precision=prec)
            out[(solver, prec)] = rel(psi.cpu().numpy(), ref)
    print("structured grid:", out)
    assert out[("banded", "fp64")] <= 1e-11 and out[("multifrontal", "fp64")] <= 1e-11
    assert out[("banded", "mixed")] <= 1e-9 and out[("multifrontal", "mixed")] <= 1e-9


def test_mesh_adjoint_vs_explicit(dev):
    """K^H lambda = G on a tetrahedral P1 mesh against SuperLU on the explicit K^H."""
    from paper_2504_07269_gb300 import stfdm

    coords, cells = MESHES["tet"]()
    t = synth.uniform_time_nodes(5, 1.0)
    Mx, Ax, _ = fe_mesh.assemble_mesh(coords, cells, 1)
    M_t, B_t, _, _ = fe_time.assemble_time(1, t)
    KH = assemble.kron_system(M_t, B_t, Mx, Ax).conj().T.tocsc()
    h = stfdm.setup_mesh_problem(3, 1, coords, cells, 1, t, device=0)
    G = synth.cn01((h.n_t, h.n_x), seed=70)
    ref = spla.splu(KH).solve(G.reshape(-1)).reshape(G.shape)
    for prec, bar in (("fp64", 1e-11), ("mixed", 1e-9)):
        lam, _ = stfdm.st_adjoint_solve(h, torch.from_numpy(G).to(dev), precision=prec)
        assert rel(lam.cpu().numpy(), ref) <= bar, prec


def test_mesh_handle_rejects_structured_only_calls(dev):
    from paper_2504_07269_gb300 import _lib, stfdm

    coords, cells = MESHES["tri"]()
    h = stfdm.setup_mesh_problem(2, 1, coords, cells, 1, synth.uniform_time_nodes(4, 1.0), device=0)
    psi = torch.zeros((h.n_t, h.n_x), dtype=torch.complex128, device=dev)
    with pytest.raises(_lib.StfdmError) as e:
        stfdm.st_error_norms(h, "c1", psi)
    assert e.value.status == _lib.ST_ERR_UNSUPPORTED
    with pytest.raises(_lib.StfdmError) as e:
        stfdm.st_batch_create([h])
    assert e.value.status == _lib.ST_ERR_UNSUPPORTED
    with pytest.raises(_lib.StfdmError) as e:
        stfdm.setup_mesh_problem(2, 1, coords, cells, 1, synth.uniform_time_nodes(4, 1.0), device=0,
                                 spatial_solver="banded")
    assert e.value.status == _lib.ST_ERR_UNSUPPORTED


@pytest.mark.parametrize("solver", ["banded", "multifrontal"])
def test_factor_then_substitute_equals_spatial_solve(dev, solver):
    """st_spatial_factor + st_spatial_substitute (the kept factors applied twice to different right-hand
    sides) give what st_spatial_solve gives, FP32 and FP64."""
    from paper_2504_07269_gb300 import _lib, stfdm

    h = stfdm.setup_problem(37, 2, synth.uniform_time_nodes(5, 0.7), device=0, spatial_solver=solver)
    for prec, dt, bar in (("fp32", torch.complex64, 1e-6), ("fp64", torch.complex128, 1e-13)):
        with pytest.raises(_lib.StfdmError):
            stfdm.st_spatial_substitute(h, prec, torch.zeros((h.n_t, h.n_x), dtype=dt, device=dev))
        stfdm.st_spatial_factor(h, prec)
        for seed in (1, 2):
            G = torch.from_numpy(synth.cn01((h.n_t, h.n_x), seed=seed)).to(dev).to(dt)
            W1 = stfdm.st_spatial_substitute(h, prec, G)
            W2 = stfdm.st_spatial_solve(h, prec, G.clone())
            stfdm.st_spatial_factor(h, prec)   # st_spatial_solve's transient factors replaced the kept ones
            assert rel(W1.cpu().numpy(), W2.cpu().numpy()) <= bar, (prec, seed)
