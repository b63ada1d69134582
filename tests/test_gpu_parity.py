"""GPU parity of the CUDA path against the CPU oracle, through the C ABI.

Bars: FP64 <= 1e-11 relative l2, mixed precision after refinement <= 1e-9, plain
FP32 error stated with a loose bound.  Sizes span several panels of the banded
factorisation (panel width 16) with ragged tails, P1 and P2 in time, uniform and
graded temporal meshes, rectangles, and the degenerate sizes (one spatial node,
one time element).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import assemble, fe_space, fe_time, solve

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


def _problem(n, p, N, T=1.0, graded=False, Lx=1.0, Ly=1.0):
    t = synth.graded_time_nodes(T, 1.5, N0=N) if graded else synth.uniform_time_nodes(N, T)
    return t


def _handle(n, p, t, Lx=1.0, Ly=1.0):
    from paper_2504_07269_gb300 import stfdm

    return stfdm.setup_problem(n, p, t, Lx, Ly, device=0)


def _oracle_K(n, p, t, Lx=1.0, Ly=1.0):
    return assemble.explicit_system(n, p, t, Lx, Ly)


# ------------------------------------------------------------------ full solves
def test_c1_manufactured(dev):
    """C1: 16x16 squares, P1 time on 16 elements, psi = S(x)(1+t)e^{-it}, psi0 = S."""
    from paper_2504_07269_gb300 import stfdm

    pr = synth.config_problem("c1")
    x1, x2 = synth.interior_coords(pr.n)
    psi0 = synth.psi0_c1(x1, x2)
    F = assemble.load_vector(pr.n, 1, pr.t_nodes, synth.f_c1)
    K = _oracle_K(pr.n, 1, pr.t_nodes)
    L = assemble.lifting_vector(pr.n, 1, pr.t_nodes, psi0)
    ref = solve.solve_explicit(K, F - L) + psi0[None, :]
    h = _handle(pr.n, 1, pr.t_nodes)
    Fd, p0 = torch.from_numpy(F).to(dev), torch.from_numpy(psi0).to(dev)
    psi, info = stfdm.st_fdm_solve(h, Fd, p0, precision="fp64")
    assert rel(psi.cpu().numpy(), ref) <= 1e-11
    psi, info = stfdm.st_fdm_solve(h, Fd, p0, precision="mixed")
    assert rel(psi.cpu().numpy(), ref) <= 1e-9, info
    assert info["rel_residual"] <= 1e-12 and info["sweeps"] >= 1
    assert info["tensor_cores"] == 1   # the FP32 transforms ran on tcgen05
    assert info["kernel_launches"] >= 10 * info["sweeps"]   # counted by the library's launchers
    psi32, _ = stfdm.st_fdm_solve(h, Fd.to(torch.complex64), p0.to(torch.complex64), precision="fp32")
    e32 = rel(psi32.cpu().numpy(), ref)
    print(f"c1 fp32 rel. error {e32:.2e}")
    assert e32 <= 1e-4


CASES = [
    # n, p, N_t, T, graded, Lx, Ly
    (2, 1, 1, 1.0, False, 1.0, 1.0),     # one spatial node, one element
    (3, 2, 1, 0.7, False, 1.0, 1.0),     # P2, one element
    (7, 1, 5, 1.0, False, 1.0, 1.0),
    (18, 1, 9, 1.0, False, 1.0, 1.0),    # b = 18: one panel + ragged tail per grid row
    (18, 2, 6, 2.0, False, 1.3, 0.8),    # rectangle, P2
    (21, 1, 12, 1.5, True, 1.0, 1.0),    # graded time mesh
    (33, 1, 17, 1.0, False, 1.0, 1.0),   # n_x = 1024, b = 33
    (34, 2, 8, 1.0, False, 1.0, 1.0),
]


@pytest.mark.parametrize("n,p,N,T,graded,Lx,Ly", CASES)
def test_discrete_manufactured(dev, n, p, N, T, graded, Lx, Ly):
    """F = K u* for a seeded random u*; FP64, mixed and FP32 solves against the oracle's explicit solve."""
    from paper_2504_07269_gb300 import stfdm

    t = _problem(n, p, N, T, graded)
    K = _oracle_K(n, p, t, Lx, Ly)
    n_t, n_x = p * N, (n - 1) ** 2
    u = synth.cn01((n_t, n_x), seed=100 + n + N)
    F = (K @ u.reshape(-1)).reshape(u.shape)
    ref = solve.solve_explicit(K, F)
    assert rel(ref, u) < 1e-9
    h = _handle(n, p, t, Lx, Ly)
    Fd = torch.from_numpy(F).to(dev)
    psi, _ = stfdm.st_fdm_solve(h, Fd, precision="fp64")
    assert rel(psi.cpu().numpy(), ref) <= 1e-11
    psi, info = stfdm.st_fdm_solve(h, Fd, precision="mixed")
    assert rel(psi.cpu().numpy(), ref) <= 1e-9, info
    psi32, _ = stfdm.st_fdm_solve(h, Fd.to(torch.complex64), precision="fp32")
    e32 = rel(psi32.cpu().numpy(), ref)
    print(f"n={n} p={p} N={N}: fp32 rel. error {e32:.2e}, mixed sweeps {info['sweeps']}")
    assert e32 <= 1e-2


def test_lifting_with_psi0(dev):
    from paper_2504_07269_gb300 import stfdm

    n, p, t = 19, 2, synth.uniform_time_nodes(7, 1.1)
    x1, x2 = synth.interior_coords(n)
    psi0 = synth.packet_values(synth.packet_params(3), x1, x2)
    F = synth.cn01((p * 7, (n - 1) ** 2), seed=9)
    K = _oracle_K(n, p, t)
    L = assemble.lifting_vector(n, p, t, psi0)
    ref = solve.solve_explicit(K, F - L) + psi0[None, :]
    h = _handle(n, p, t)
    Fd, p0 = torch.from_numpy(F).to(dev), torch.from_numpy(psi0).to(dev)
    for prec, bound in (("fp64", 1e-11), ("mixed", 1e-9)):
        psi, _ = stfdm.st_fdm_solve(h, Fd, p0, precision=prec)
        assert rel(psi.cpu().numpy(), ref) <= bound, prec
    # residual of the solution (st_residual) against the oracle's
    psi, _ = stfdm.st_fdm_solve(h, Fd, p0, precision="fp64")
    R = torch.empty_like(Fd)
    r, _ = stfdm.st_residual(h, Fd, p0, psi, R)
    M_t, B_t, m_t, _ = fe_time.assemble_time(p, t)
    M_x, A_x = fe_space.assemble_space(n)
    Ft = F - np.outer(m_t, A_x @ psi0)
    Ro, ro = solve.residual(M_t, B_t, M_x, A_x, psi.cpu().numpy() - psi0[None, :], Ft)
    np.testing.assert_allclose(R.cpu().numpy(), Ro, atol=1e-13 * np.abs(Ft).max())
    assert r < 1e-12


# ------------------------------------------------------------------ single steps
@pytest.mark.parametrize("n,p,N", [(9, 1, 70), (12, 2, 33)])
def test_time_transform_step(dev, n, p, N):
    """Steps 2 / 4 (and the adjoint transforms): out = T in, against the plain matrix product
    with the library's own T (checked against the oracle's decomposition on the CPU); FP64 and
    FP32 SIMT kernels and the tensor-core kernel (n_t not a multiple of the 128-row tile, ragged
    column tiles)."""
    from paper_2504_07269_gb300 import stfdm

    t = synth.uniform_time_nodes(N, 1.0)
    h = _handle(n, p, t)
    X, s, Y, _ = stfdm.st_time_decompose(h.time)
    mats = {"Y": Y, "X": X, "XT": X.T, "YT": Y.T}
    inp = synth.cn01((p * N, (n - 1) ** 2), seed=5)
    di = torch.from_numpy(inp).to(dev)
    for w, T in mats.items():
        ref = T @ inp
        out = stfdm.st_time_transform(h, w, "fp64", di)
        assert rel(out.cpu().numpy(), ref) <= 1e-13, w
        out32 = stfdm.st_time_transform(h, w, "fp32", di.to(torch.complex64))
        assert rel(out32.cpu().numpy(), ref) <= 1e-5, w
        # tensor cores (tcgen05, 3xTF32 split of both operands)
        outtc = stfdm.st_time_transform(h, w, "mixed", di.to(torch.complex64))
        etc = rel(outtc.cpu().numpy(), ref)
        assert etc <= 1e-5, (w, etc)


@pytest.mark.parametrize("n,p,N,Lx", [(17, 1, 6, 1.0), (40, 2, 3, 1.4)])
def test_spatial_solve_step(dev, n, p, N, Lx):
    """Step 3: W[k] = (M_x + s_k A_x)^{-1} G[k] for every k against SuperLU on the oracle's matrices."""
    from paper_2504_07269_gb300 import stfdm

    t = synth.uniform_time_nodes(N, 1.0)
    h = _handle(n, p, t, Lx, 1.0)
    _, s, _, _ = stfdm.st_time_decompose(h.time)
    M_x, A_x = fe_space.assemble_space(n, Lx, 1.0)
    G = synth.cn01((p * N, (n - 1) ** 2), seed=8)
    ref = np.stack([spla.splu(sp.csc_matrix(M_x + s[k] * A_x, dtype=np.complex128)).solve(G[k])
                    for k in range(len(s))])
    W = stfdm.st_spatial_solve(h, "fp64", torch.from_numpy(G).to(dev))
    assert rel(W.cpu().numpy(), ref) <= 1e-11
    W32 = stfdm.st_spatial_solve(h, "fp32", torch.from_numpy(G).to(dev).to(torch.complex64))
    e32 = rel(W32.cpu().numpy(), ref)
    print(f"spatial fp32 rel. error {e32:.2e}")
    assert e32 <= 1e-3


def test_load_nodal(dev):
    from paper_2504_07269_gb300 import stfdm

    n, p, t = 11, 2, synth.graded_time_nodes(1.0, 1.5, N0=5)
    h = _handle(n, p, t)
    f = synth.cn01((p * 5 + 1, (n - 1) ** 2), seed=4)
    Mf, _, _ = fe_time.assemble_time_full(p, t)
    M_x, _ = fe_space.assemble_space(n)
    ref = Mf[1:] @ (M_x @ f.T).T
    F = stfdm.st_load_nodal(h, torch.from_numpy(f).to(dev))
    assert rel(F.cpu().numpy(), ref) <= 1e-14


# ------------------------------------------------------------------ adjoint / autograd
@pytest.mark.parametrize("p", [1, 2])
def test_adjoint(dev, p):
    from paper_2504_07269_gb300 import stfdm

    n, N = 15, 9
    t = synth.uniform_time_nodes(N, 1.0)
    K = _oracle_K(n, p, t)
    g = synth.cn01((p * N, (n - 1) ** 2), seed=21)
    ref = spla.splu(sp.csc_matrix(K.conj().T), permc_spec="MMD_AT_PLUS_A").solve(g.reshape(-1)).reshape(g.shape)
    h = _handle(n, p, t)
    gd = torch.from_numpy(g).to(dev)
    lam, _ = stfdm.st_adjoint_solve(h, gd, precision="fp64")
    assert rel(lam.cpu().numpy(), ref) <= 1e-11
    lam, info = stfdm.st_adjoint_solve(h, gd, precision="mixed")
    assert rel(lam.cpu().numpy(), ref) <= 1e-9, info
    # dot-product identity <K^{-1} a, b> = <a, K^{-H} b>
    a = synth.cn01(g.shape, seed=22)
    x, _ = stfdm.st_fdm_solve(h, torch.from_numpy(a).to(dev), precision="fp64")
    y, _ = stfdm.st_adjoint_solve(h, gd, precision="fp64")
    lhs = np.vdot(g, x.cpu().numpy())
    rhs = np.vdot(y.cpu().numpy(), a)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_autograd_matches_finite_differences(dev):
    """J(F, psi0) = 1/2 ||psi_h - target||^2_{M_t (x) M_x} + alpha/2 ||F||^2: the autograd gradient
    (adjoint solve + adjoint lift) against central differences along random complex directions and
    against the oracle's dense adjoint."""
    from paper_2504_07269_gb300 import stfdm
    from paper_2504_07269_gb300.autograd import st_solve

    n, p, N = 9, 1, 6
    t = synth.uniform_time_nodes(N, 1.0)
    h = _handle(n, p, t)
    n_t, n_x = p * N, (n - 1) ** 2
    M_t, B_t, m_t, _ = fe_time.assemble_time(p, t)
    M_x, A_x = fe_space.assemble_space(n)
    Wt = torch.from_numpy(M_t).to(dev)
    Wx = torch.from_numpy(M_x.toarray()).to(dev)
    x1, x2 = synth.interior_coords(n)
    target = torch.from_numpy(np.tile(synth.packet_values(synth.packet_params(1, 1), x1, x2), (n_t, 1))).to(dev)
    alpha = 1e-3

    def J(F, psi0):
        psi = st_solve(F, psi0, h, "fp64")
        e = psi - target
        q = (Wt.to(e.dtype) @ e @ Wx.to(e.dtype).T)
        return 0.5 * torch.real(torch.sum(e.conj() * q)) + 0.5 * alpha * torch.real(torch.sum(F.conj() * F))

    F = torch.from_numpy(synth.cn01((n_t, n_x), seed=30)).to(dev).requires_grad_(True)
    p0 = torch.from_numpy(synth.cn01((n_x,), seed=31)).to(dev).requires_grad_(True)
    val = J(F, p0)
    val.backward()
    gF, gp = F.grad.detach().clone(), p0.grad.detach().clone()
    hstep = 1e-6
    for d in range(4):
        dF = torch.from_numpy(synth.cn01((n_t, n_x), seed=40 + d)).to(dev)
        dp = torch.from_numpy(synth.cn01((n_x,), seed=50 + d)).to(dev)
        with torch.no_grad():
            fd = (J(F + hstep * dF, p0 + hstep * dp) - J(F - hstep * dF, p0 - hstep * dp)) / (2 * hstep)
        # directional derivative of a real function of complex inputs: 2 Re <grad, d> with PyTorch's grad
        ad = torch.real(torch.sum(gF.conj() * dF) + torch.sum(gp.conj() * dp))
        assert abs(float(fd) - float(ad)) <= 1e-6 * max(1.0, abs(float(ad))), (float(fd), float(ad))
    # oracle dense adjoint: dJ/dconj(F) = K^{-H} W e (+ alpha F) with W = M_t (x) M_x, e = psi - target
    K = _oracle_K(n, p, t)
    Fn = F.detach().cpu().numpy()
    L = np.outer(m_t, A_x @ p0.detach().cpu().numpy())
    psi = solve.solve_dense(K, Fn - L) + p0.detach().cpu().numpy()[None, :]
    e = psi - target.cpu().numpy()
    We = M_t @ (M_x @ e.T).T
    gref = solve.solve_dense(K.conj().T, We) + alpha * Fn
    assert rel(gF.cpu().numpy(), gref) <= 1e-10


# ------------------------------------------------------------------ failure reporting (host side)
def test_failures_are_reported(dev):
    from paper_2504_07269_gb300 import _lib, stfdm

    n, p, t = 10, 1, synth.uniform_time_nodes(20, 1.0)
    with pytest.raises(_lib.StfdmError) as e:
        stfdm.setup_problem(n, p, t, kappa_max=2.0, device=0)
    assert e.value.status == _lib.ST_ERR_ILL_CONDITIONED
    h = _handle(n, p, t)
    F = torch.from_numpy(synth.cn01((20, 81), seed=1)).to(dev)
    with pytest.raises(_lib.StfdmError) as e:
        stfdm.st_fdm_solve(h, F, precision="mixed", tol=1e-30, max_sweeps=1)
    assert e.value.status == _lib.ST_ERR_NOT_CONVERGED
    with pytest.raises(ValueError):
        stfdm.st_fdm_solve(h, F.to(torch.complex64), precision="fp64")


def test_bounded_wait_times_out_and_handle_recovers(dev):
    """Failure detection without a GPU fault: the wait probe makes the substitution kernel's copy
    issuer wait on an mbarrier that receives neither a copy nor an arrival.  The bounded wait runs
    out (1 ms), the CTA takes its timeout exit (no copy was issued, so none is in flight), the
    entry point returns ST_ERR_TIMEOUT, and after the probe is turned off the same handle solves
    correctly again (spatial solve vs SuperLU, full mixed solve vs the oracle)."""
    import time

    from paper_2504_07269_gb300 import _lib, stfdm

    n, p, t = 23, 1, synth.uniform_time_nodes(12, 1.0)
    h = _handle(n, p, t)
    G = synth.cn01((h.n_t, h.n_x), seed=21)
    Gd = torch.from_numpy(G).to(dev).to(torch.complex64)
    stfdm.st_set_wait_probe(h, 1e-3)
    t0 = time.perf_counter()
    with pytest.raises(_lib.StfdmError) as e:
        stfdm.st_spatial_solve(h, "fp32", Gd)
    waited = time.perf_counter() - t0
    assert e.value.status == _lib.ST_ERR_TIMEOUT
    print(f"wait probe: ST_ERR_TIMEOUT after {waited * 1e3:.1f} ms")
    assert waited < 1.5            # the consumers abort with the producer instead of waiting 2 s
    with pytest.raises(_lib.StfdmError) as e:
        stfdm.st_set_wait_probe(h, 2.0)
    assert e.value.status == _lib.ST_ERR_ARG
    stfdm.st_set_wait_probe(h, 0.0)
    W = stfdm.st_spatial_solve(h, "fp32", Gd).cpu().numpy()
    M_t, B_t, m_t, _ = fe_time.assemble_time(p, t)
    M_x, A_x = fe_space.assemble_space(n)
    _, s, _, _ = stfdm.st_time_decompose(h.time)
    for k in range(h.n_t):
        ref = spla.splu(sp.csc_matrix(M_x + s[k] * A_x, dtype=np.complex128)).solve(G[k])
        assert rel(W[k], ref) <= 1e-3          # FP32: cond(C_k) u_32
    F = synth.cn01((h.n_t, h.n_x), seed=22)
    ref = solve.solve_explicit(_oracle_K(n, p, t), F)
    psi, _ = stfdm.st_fdm_solve(h, torch.from_numpy(F).to(dev), precision="mixed")
    assert rel(psi.cpu().numpy(), ref) <= 1e-9
