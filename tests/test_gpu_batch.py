"""Batched plans (st_batch_create / st_batch_solve): problems of uneven spatial mesh, n_t and
temporal degree solved together by grouped launches, the spatial systems of all problems in one
persistent launch, one restart cycle captured in a CUDA graph, tile shapes from the autotuner.

Bars: every problem against the oracle's explicit solve <= 1e-9 relative l2 (the mixed-precision
bar); graph replay and direct launches give identical results; the tuner's choice does not change
the arithmetic; at the full 64-problem size every final FP64 residual meets the tolerance.
"""
import time

import numpy as np
import pytest

import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import assemble, fe_space, solve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# n, p_t, N_t, T, graded, Lx, Ly, with psi0
UNEVEN = [
    (3, 1, 2, 1.0, False, 1.0, 1.0, False),    # one element per grid row, 4 unknowns per time row
    (7, 2, 5, 0.8, False, 1.0, 1.0, True),     # P2
    (18, 1, 9, 1.0, False, 1.3, 0.8, True),    # rectangle
    (21, 1, 12, 1.5, True, 1.0, 1.0, False),   # graded time mesh
    (33, 2, 6, 1.0, False, 1.0, 1.0, True),    # b = 33: two 32-row blocks + a tail
    (12, 1, 33, 2.0, False, 1.0, 1.0, False),  # n_t > n_x
]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_07269_gb300 import build

    build.build()
    return torch.device("cuda:0")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def uneven(dev):
    """Handles, inputs and oracle solutions of the uneven batch (discrete manufactured u*)."""
    from paper_2504_07269_gb300 import stfdm

    hs, Fs, P0, refs = [], [], [], []
    for i, (n, p, N, T, graded, Lx, Ly, with_psi0) in enumerate(UNEVEN):
        t = synth.graded_time_nodes(T, 1.5, N0=N) if graded else synth.uniform_time_nodes(N, T)
        K = assemble.explicit_system(n, p, t, Lx, Ly)
        n_t, n_x = p * (len(t) - 1), (n - 1) ** 2
        u = synth.cn01((n_t, n_x), seed=300 + i)
        F = (K @ u.reshape(-1)).reshape(u.shape)
        psi0 = None
        if with_psi0:
            x1, x2 = synth.interior_coords(n, Lx, Ly)
            psi0 = synth.packet_values(synth.packet_params(40 + i), x1, x2)
            F = F + assemble.lifting_vector(n, p, t, psi0, Lx, Ly)
            ref = u + psi0[None, :]
        else:
            ref = u
        Ft = F - assemble.lifting_vector(n, p, t, psi0, Lx, Ly) if with_psi0 else F
        assert rel(solve.solve_explicit(K, Ft) + (psi0[None, :] if with_psi0 else 0), ref) < 1e-9
        hs.append(stfdm.setup_problem(n, p, t, Lx, Ly, device=0))
        Fs.append(torch.from_numpy(F).to(dev))
        P0.append(torch.from_numpy(psi0).to(dev) if with_psi0 else None)
        refs.append(ref)
    return hs, Fs, P0, refs


def test_batch_matches_oracle(dev, uneven):
    from paper_2504_07269_gb300 import stfdm

    hs, Fs, P0, refs = uneven
    b = stfdm.st_batch_create(hs, tol=1e-12)
    outs, infos = stfdm.st_batch_solve(b, Fs, P0)
    st = stfdm.st_batch_stats_get(b)
    for o, ref, info in zip(outs, refs, infos):
        assert rel(o.cpu().numpy(), ref) <= 1e-9, info
        assert info["rel_residual"] <= 1e-12 and info["sweeps"] >= 1
    assert st["count"] == len(hs) and st["items"] == sum(h.n_t for h in hs)
    assert st["graph_nodes"] > 0 and st["cycles"] >= 1 and st["tuned"] in (1, 2)
    assert (st["xform_tile_m"], st["xform_tile_n"]) in ((64, 64), (32, 128), (128, 32))
    assert st["solve_ctas_per_sm"] in (1, 2)
    print("batch stats", st)


def test_batch_spatial_solve_matches_oracle(dev, uneven):
    """The persistent factor-and-solve launch over all (problem, k) systems against SuperLU on
    the oracle's matrices (every k of every problem; same bar as the single-problem FP32 step)."""
    from paper_2504_07269_gb300 import stfdm

    hs = uneven[0]
    b = stfdm.st_batch_create(hs, no_tune=True)
    Gs = []
    for i, h in enumerate(hs):
        G = synth.cn01((h.n_t, h.n_x), seed=500 + i)
        Gs.append(G)
        stfdm.st_batch_spatial_get(b, i, torch.from_numpy(G).to(dev).to(torch.complex64), to_plan=True)
    stfdm.st_batch_spatial_solve(b)
    for i, (h, G, spec) in enumerate(zip(hs, Gs, UNEVEN)):
        n, Lx, Ly = spec[0], spec[5], spec[6]
        _, s, _, _ = stfdm.st_time_decompose(h.time)
        M_x, A_x = fe_space.assemble_space(n, Lx, Ly)
        ref = np.stack([spla.splu(sp.csc_matrix(M_x + s[k] * A_x, dtype=np.complex128)).solve(G[k])
                        for k in range(len(s))])
        W = stfdm.st_batch_spatial_get(b, i, torch.empty((h.n_t, h.n_x), dtype=torch.complex64, device=dev),
                                       to_plan=False)
        e = rel(W.cpu().numpy(), ref)
        print(f"batch spatial solve, problem {i}: fp32 rel. error {e:.2e}")
        assert e <= 1e-3


def test_batch_graph_and_direct_launches_agree(dev, uneven):
    """The captured cycle and the same launches issued directly give bit-identical results."""
    from paper_2504_07269_gb300 import stfdm

    hs, Fs, P0, _ = uneven
    b1 = stfdm.st_batch_create(hs, tol=1e-12)
    b2 = stfdm.st_batch_create(hs, tol=1e-12, no_graph=True)
    o1, i1 = stfdm.st_batch_solve(b1, Fs, P0)
    o2, i2 = stfdm.st_batch_solve(b2, Fs, P0)
    assert stfdm.st_batch_stats_get(b2)["graph_nodes"] == 0
    for a, c, x, y in zip(o1, o2, i1, i2):
        assert torch.equal(a, c)
        assert x["sweeps"] == y["sweeps"]
    # a second solve on the same plan (graph replayed with new inputs) gives the same answer
    o3, _ = stfdm.st_batch_solve(b1, Fs, P0)
    for a, c in zip(o1, o3):
        assert torch.equal(a, c)


def test_batch_kept_factors(dev, uneven):
    """With memory to spare every problem keeps its factors (later applications only stream them
    through the grouped substitutions); without, every application refactorises.  Both meet the
    oracle."""
    from paper_2504_07269_gb300 import stfdm

    hs, Fs, P0, refs = uneven
    bk = stfdm.st_batch_create(hs, tol=1e-12)
    bn = stfdm.st_batch_create(hs, tol=1e-12, no_keep=True)
    sk, sn = stfdm.st_batch_stats_get(bk), stfdm.st_batch_stats_get(bn)
    assert sk["kept_problems"] == len(hs) and sk["kept_factor_bytes"] > 0
    assert sn["kept_problems"] == 0 and sn["kept_factor_bytes"] == 0
    for b in (bk, bn):
        outs, infos = stfdm.st_batch_solve(b, Fs, P0)
        for o, ref, info in zip(outs, refs, infos):
            assert rel(o.cpu().numpy(), ref) <= 1e-9, info
    # a second solve on the kept plan refactorises for its new right-hand sides as well
    outs2, _ = stfdm.st_batch_solve(bk, [2.0 * F for F in Fs], [None if p is None else 2.0 * p for p in P0])
    for o, ref in zip(outs2, refs):
        assert rel(o.cpu().numpy(), 2.0 * ref) <= 1e-9


def test_batch_untuned_defaults_agree(dev, uneven):
    from paper_2504_07269_gb300 import stfdm

    hs, Fs, P0, _ = uneven
    o1, _ = stfdm.st_batch_solve(stfdm.st_batch_create(hs, tol=1e-12), Fs, P0)
    b0 = stfdm.st_batch_create(hs, tol=1e-12, no_tune=True)
    assert stfdm.st_batch_stats_get(b0)["tuned"] == 0
    o0, _ = stfdm.st_batch_solve(b0, Fs, P0)
    for a, c in zip(o1, o0):
        assert rel(a.cpu().numpy(), c.cpu().numpy()) <= 1e-12


def test_batch_short_restart_and_limit(dev, uneven):
    """A restart length of 2 still converges (more cycles); a sweep limit of 1 is reported as
    not converged with every problem's info filled."""
    from paper_2504_07269_gb300 import _lib, stfdm

    hs, Fs, P0, refs = uneven
    b = stfdm.st_batch_create(hs, tol=1e-12, restart=2)
    outs, infos = stfdm.st_batch_solve(b, Fs, P0)
    assert stfdm.st_batch_stats_get(b)["restart"] == 2
    for o, ref in zip(outs, refs):
        assert rel(o.cpu().numpy(), ref) <= 1e-9
    b1 = stfdm.st_batch_create(hs, tol=1e-14, max_sweeps=1)
    with pytest.raises(_lib.StfdmError) as e:
        stfdm.st_batch_solve(b1, Fs, P0)
    assert e.value.status == _lib.ST_ERR_NOT_CONVERGED
    assert len(e.value.info) == len(hs) and all(i["sweeps"] == 1 for i in e.value.info)


def test_batched_entry_point_uses_the_plan(dev, uneven):
    """st_fdm_solve_batched with mixed precision agrees with one-at-a-time solves."""
    from paper_2504_07269_gb300 import stfdm

    hs, Fs, P0, refs = uneven
    outs, infos = stfdm.st_fdm_solve_batched(hs, Fs, P0, precision="mixed")
    for h, F, p0, o, ref in zip(hs, Fs, P0, outs, refs):
        single, _ = stfdm.st_fdm_solve(h, F, p0, precision="mixed")
        # two different GMRES iterates, each with a relative residual <= 1e-12: their errors lie
        # along the operator's small singular directions and can reach cond(K) times the residual
        # (about 1e3 here), so they agree to about 1e-9 in the worst case; 1e-10 is the bound
        assert rel(o.cpu().numpy(), single.cpu().numpy()) <= 1e-10
        assert rel(o.cpu().numpy(), ref) <= 1e-9


def make_batch_inputs(hs, probs, dev):
    """F = (M_t,full (x) M_x) f_nodal on the device (f separable, from synth), psi0 packets."""
    from paper_2504_07269_gb300 import stfdm

    Fs, P0 = [], []
    for h, pr in zip(hs, probs):
        psi0, a, bx = synth.batch_inputs(pr)
        P0.append(torch.from_numpy(psi0).to(dev))
        if a is None:
            Fs.append(torch.zeros((pr.n_t, pr.n_x), dtype=torch.complex128, device=dev))
        else:
            f = torch.outer(torch.from_numpy(a).to(dev), torch.from_numpy(bx).to(dev))
            Fs.append(stfdm.st_load_nodal(h, f))
            del f
    return Fs, P0


def test_batch_full_size_64_problems(dev):
    """The 64-problem uneven batch (n in {32,...,192}, P1/P2, N_t in [32, 512], T in [0.5, 2],
    packets, half forced) refined to 1e-12: every problem's FP64 residual (st_residual, separate
    kernel) meets it (the configuration asks for 1e-10), and three problems agree with a tightly
    refined reference to 1e-9.  A GMRES solution's error lies mostly along the operator's small
    singular directions, so its error/residual ratio approaches cond(K) (about 1e3 here): 1e-10
    alone leaves errors near 1e-8."""
    from paper_2504_07269_gb300 import stfdm

    probs = synth.batch_problems(64, 5)
    t0 = time.perf_counter()
    hs = stfdm.setup_problems([(pr.n, pr.p_t, pr.t_nodes, pr.Lx, pr.Ly) for pr in probs], device=0)
    print(f"C5 setup of 64 problems: {time.perf_counter() - t0:.1f} s")
    Fs, P0 = make_batch_inputs(hs, probs, dev)
    t0 = time.perf_counter()
    b = stfdm.st_batch_create(hs, tol=1e-12)
    t1 = time.perf_counter()
    outs, infos = stfdm.st_batch_solve(b, Fs, P0)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    st = stfdm.st_batch_stats_get(b)
    print(f"C5 batch: plan {t1 - t0:.1f} s, solve {t2 - t1:.1f} s, {st['unknowns'] / (t2 - t1):.3e} unknowns/s, "
          f"stats {st}, sweeps {[i['sweeps'] for i in infos]}")
    worst = 0.0
    for h, F, p0, o in zip(hs, Fs, P0, outs):
        r, _ = stfdm.st_residual(h, F, p0, o)
        worst = max(worst, r)
    assert worst <= 1.01e-12, worst
    del b
    # the largest, the smallest and the worst-conditioned P2 problem against a tightly refined
    # single solve (FP64 GMRES to 1e-13); the FP64 FDM's own error is printed beside it
    sizes = [pr.unknowns for pr in probs]
    p2 = [i for i, pr in enumerate(probs) if pr.p_t == 2]
    pick = {int(np.argmax(sizes)), int(np.argmin(sizes)), max(p2, key=lambda i: hs[i].kappa)}
    for i in sorted(pick):
        acc, ia = stfdm.st_fdm_solve(hs[i], Fs[i], P0[i], precision="mixed", tol=1e-13, max_sweeps=80)
        f64, _ = stfdm.st_fdm_solve(hs[i], Fs[i], P0[i], precision="fp64")
        r64, _ = stfdm.st_residual(hs[i], Fs[i], P0[i], f64)
        e = rel(outs[i].cpu().numpy(), acc.cpu().numpy())
        e64 = rel(f64.cpu().numpy(), acc.cpu().numpy())
        print(f"problem {i} (n={probs[i].n}, p_t={probs[i].p_t}, n_t={probs[i].n_t}, kappa_X={hs[i].kappa:.1e}): "
              f"batch error {e:.2e} (residual {infos[i]['rel_residual']:.2e}); FP64 FDM error {e64:.2e} "
              f"(residual {r64:.2e}); reference residual {ia['rel_residual']:.2e}")
        assert e <= 1e-9
