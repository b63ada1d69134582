"""Host side of the general-mesh path, CPU only: the library's mesh assembly against the oracle's
(two independent implementations: exact barycentric-monomial integrals in C++, collapsed Gauss
quadrature in NumPy), and the sparse-direct solver's symbolic plan against a plain elimination of
the permuted sparsity pattern."""
import numpy as np
import pytest

import synth
from oracle import fe_mesh, fe_space


def _lib():
    from paper_2504_07269_gb300 import build

    build.build()
    from paper_2504_07269_gb300 import stfdm

    return stfdm


MESHES = {
    "tri": lambda: synth.square_delaunay_mesh(7, jitter=0.3, seed=21),
    "tet": lambda: synth.cube_tet_mesh(3, jitter=0.2, seed=22),
    "tet5": lambda: synth.cube_tet_mesh(5, jitter=0.2, seed=23),
}


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("kind", ["tri", "tet"])
def test_mesh_assembly_matches_oracle(kind, p):
    stfdm = _lib()
    coords, cells = MESHES[kind]()
    dim = coords.shape[1]
    s = stfdm.st_assemble_mesh(dim, p, coords, cells)
    got = stfdm.st_space_get_mesh(s)
    Mx, Ax, xin = fe_mesh.assemble_mesh(coords, cells, p)
    import scipy.sparse as sp

    n = got["n_x"]
    assert n == Mx.shape[0] and got["p_x"] == p and got["dim"] == dim
    Mg = sp.csr_matrix((got["M"], got["col"], got["rowptr"]), shape=(n, n))
    Ag = sp.csr_matrix((got["A"], got["col"], got["rowptr"]), shape=(n, n))
    assert abs(Mg - Mx).max() <= 1e-15 * max(1.0, abs(Mx).max()) * 10
    assert abs(Ag - Ax).max() <= 1e-13 * abs(Ax).max()
    np.testing.assert_allclose(got["xyz"], xin, atol=1e-15)
    # columns sorted within every row
    for r in range(n):
        c = got["col"][got["rowptr"][r]:got["rowptr"][r + 1]]
        assert np.all(np.diff(c) > 0)


def test_structured_grid_as_mesh_matches_oracle():
    stfdm = _lib()
    n = 9
    s = stfdm.st_assemble_space(n)
    got = stfdm.st_space_get_mesh(s)
    import scipy.sparse as sp

    nx = got["n_x"]
    Mg = sp.csr_matrix((got["M"], got["col"], got["rowptr"]), shape=(nx, nx))
    Ag = sp.csr_matrix((got["A"], got["col"], got["rowptr"]), shape=(nx, nx))
    Ms, As = fe_space.assemble_space(n)
    assert abs(Mg - Ms).max() < 1e-15 and abs(Ag - As).max() < 1e-13
    x1, x2 = synth.interior_coords(n)
    np.testing.assert_allclose(got["xyz"], np.stack([x1, x2], axis=1), atol=1e-15)


def test_mesh_rejects_bad_input():
    from paper_2504_07269_gb300 import _lib as L

    stfdm = _lib()
    coords, cells = MESHES["tri"]()
    with pytest.raises(L.StfdmError) as e:
        stfdm.st_assemble_mesh(2, 3, coords, cells)
    assert e.value.status == L.ST_ERR_ARG
    bad = cells.copy()
    bad[0, 0] = len(coords)
    with pytest.raises(L.StfdmError):
        stfdm.st_assemble_mesh(2, 1, coords, bad)
    flat = cells.copy()
    flat[0, 2] = flat[0, 1]
    with pytest.raises(L.StfdmError):
        stfdm.st_assemble_mesh(2, 2, coords, flat)


def _symbolic_L(n, rowptr, col, perm):
    """Sparsity of L for the pattern permuted by perm (new -> old), by plain elimination:
    struct(L[:, j]) = (rows i > j of the permuted column j) U struct(L[:, k]) \\ {j} over the columns
    k < j whose first off-diagonal row is j (the elimination tree's children)."""
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    cols = []
    for j in range(n):
        jo = perm[j]
        s = {int(iperm[c]) for c in col[rowptr[jo]:rowptr[jo + 1]] if iperm[c] > j}
        cols.append(s)
    parent_children = [[] for _ in range(n)]
    for j in range(n):
        for k in parent_children[j]:
            cols[j] |= {i for i in cols[k] if i > j}
        if cols[j]:
            parent_children[min(cols[j])].append(j)
    return cols


@pytest.mark.parametrize("kind,p,leaf", [("grid", 1, 16), ("tri", 2, 24), ("tet5", 1, 16), ("tet", 2, 32)])
def test_multifrontal_plan_covers_the_fill(kind, p, leaf):
    """Every fill position L(i, j) of the ordering lies in the front that eliminates j (i is one of
    its pivots or update rows); the fronts' pivot ranges tile 0..n-1; perm is a permutation."""
    stfdm = _lib()
    if kind == "grid":
        s = stfdm.st_assemble_space(13)
    else:
        coords, cells = MESHES[kind]()
        s = stfdm.st_assemble_mesh(coords.shape[1], p, coords, cells)
    info = stfdm.st_space_get_mesh(s)
    plan = stfdm.st_space_mf_plan(s, leaf)
    n = info["n_x"]
    perm = plan["perm"]
    assert sorted(perm.tolist()) == list(range(n))
    first, npv, nu = plan["first"], plan["np"], plan["nu"]
    order = np.argsort(first)
    assert first[order[0]] == 0 and np.all(first[order][1:] == (first + npv)[order][:-1])
    assert (first + npv)[order][-1] == n
    assert np.all(npv[order] <= max(leaf, npv.max()))
    offs = np.concatenate([[0], np.cumsum(nu)])
    front_of = np.empty(n, dtype=np.int64)
    for f in range(plan["fronts"]):
        front_of[first[f]:first[f] + npv[f]] = f
    L = _symbolic_L(n, info["rowptr"], info["col"], perm)
    fe = 0
    for f in range(plan["fronts"]):
        rows = set(range(first[f], first[f] + npv[f])) | set(plan["urows"][offs[f]:offs[f + 1]].tolist())
        ur = plan["urows"][offs[f]:offs[f + 1]]
        assert np.all(np.diff(ur) > 0) and (len(ur) == 0 or ur[0] >= first[f] + npv[f])
        fe += (npv[f] + nu[f]) * npv[f]
        for j in range(first[f], first[f] + npv[f]):
            assert L[j] <= rows, (f, j)
    assert fe == plan["factor_entries"]
    nnzL = sum(len(c) for c in L)
    print(f"{kind} P{p}: n={n}, fronts {plan['fronts']}, levels {plan['levels']}, max front {plan['max_front']}, "
          f"nnz(L) {nnzL}, stored {fe}")
