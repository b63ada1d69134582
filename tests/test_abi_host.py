"""The C-ABI library on the CPU: it builds, loads, exports every symbol of
include/stfdm.h, and its host-only entry points (assembly and the FP64 time
decomposition) agree with the oracle.  No device compute is called here."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth
from conftest import ROOT
from oracle import fe_space, fe_time, timedec


@pytest.fixture(scope="module")
def L():
    from paper_2504_07269_gb300 import _lib, build

    build.build()
    return _lib.lib()


def _declared_functions():
    with open(os.path.join(ROOT, "include", "stfdm.h")) as fh:
        src = fh.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(st_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    from paper_2504_07269_gb300 import _lib

    names = _declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(L, name), name
        assert name in _lib.SIGNATURES, f"{name} has no binding"
    assert L.st_abi_version() == 8
    assert L.st_status_string(-5).decode() == "zero or non-finite pivot"


def test_python_binding_names_match_abi():
    from paper_2504_07269_gb300 import stfdm

    for name in _declared_functions():
        if name.startswith(("st_destroy", "st_status_string", "st_last_error", "st_abi", "st_fdm_get")):
            continue
        assert hasattr(stfdm, name), name


@pytest.mark.parametrize("p,graded", [(1, False), (2, False), (1, True), (2, True)])
def test_host_time_matrices_match_oracle(L, p, graded):
    from paper_2504_07269_gb300 import stfdm

    t = synth.graded_time_nodes(1.7, 1.5, N0=9, levels=1) if graded else synth.uniform_time_nodes(11, 2.3)
    h = stfdm.st_assemble_time(p, t)
    got = stfdm.st_time_get(h)
    M, B, m, tt = fe_time.assemble_time(p, t)
    np.testing.assert_allclose(got["M_t"], M, atol=1e-15)
    np.testing.assert_allclose(got["B_t"], B, atol=1e-15)
    np.testing.assert_allclose(got["m_t"], m, atol=1e-15)
    np.testing.assert_allclose(got["times"], tt, atol=1e-15)


@pytest.mark.parametrize("n,Lx,Ly", [(2, 1.0, 1.0), (5, 1.0, 1.0), (8, 1.3, 0.7)])
def test_host_space_stencil_matches_oracle(L, n, Lx, Ly):
    from paper_2504_07269_gb300 import stfdm

    s = stfdm.st_assemble_space(n, Lx, Ly)
    m, n_x, c = stfdm.st_space_get(s)
    assert m == n - 1 and n_x == (n - 1) ** 2
    Mx, Ax = fe_space.assemble_space(n, Lx, Ly)
    M, A = Mx.toarray(), Ax.toarray()
    # rebuild the matrices from the library's stencil coefficients
    Mc, Mw, Ms, Md, Ac, Aw, As, Ad = c
    Mr = np.zeros_like(M)
    Ar = np.zeros_like(A)
    for j in range(m):
        for i in range(m):
            r = i + m * j
            Mr[r, r], Ar[r, r] = Mc, Ac
            for di, dj, mv, av in ((1, 0, Mw, Aw), (-1, 0, Mw, Aw), (0, 1, Ms, As), (0, -1, Ms, As),
                                   (1, 1, Md, Ad), (-1, -1, Md, Ad)):
                ii, jj = i + di, j + dj
                if 0 <= ii < m and 0 <= jj < m:
                    Mr[r, ii + m * jj] = mv
                    Ar[r, ii + m * jj] = av
    np.testing.assert_allclose(Mr, M, atol=1e-15)
    np.testing.assert_allclose(Ar, A, atol=1e-14)


@pytest.mark.parametrize("p,N,T,graded", [(1, 16, 1.0, False), (2, 12, 1.5, False), (1, 64, 5.0, False),
                                          (1, 30, 2.0, True), (2, 40, 2.0, False)])
def test_host_time_decomposition(L, p, N, T, graded):
    """The library's FP64 eigen-decomposition (own Hessenberg QR) against the oracle's (LAPACK via numpy):
    same spectrum, A X = X S, Y (i B) X = I, unit columns, same kappa_2 (phase-invariant)."""
    from paper_2504_07269_gb300 import stfdm

    t = synth.graded_time_nodes(T, 1.5, N0=N) if graded else synth.uniform_time_nodes(N, T)
    h = stfdm.st_assemble_time(p, t)
    X, s, Y, kappa = stfdm.st_time_decompose(h, host_threads=2)
    M, B, _, _ = fe_time.assemble_time(p, t)
    A = np.linalg.solve(1j * B, M)
    Xo, so, Yo, ko = timedec.fdm_decomposition(M, B)
    scale = np.abs(so).max()
    assert np.abs(np.sort_complex(s) - np.sort_complex(so)).max() < 1e-12 * scale * len(s)
    assert np.abs(A @ X - X * s[None, :]).max() < 1e-12 * scale
    np.testing.assert_allclose(np.linalg.norm(X, axis=0), 1.0, atol=1e-13)
    assert np.abs(Y @ (1j * B) @ X - np.eye(len(s))).max() < 1e-12 * kappa
    assert abs(kappa / ko - 1) < 1e-8
    assert np.all(np.abs(s[:-1]) >= np.abs(s[1:]))          # ordered by decreasing modulus
    # Im s_k < 0 in exact arithmetic; at rounding level for eigenvectors with v_N ~ 0 (graded meshes)
    assert np.max(s.imag) <= 1e-12 * scale


def test_paper_kappa_column_from_library(L):
    """Table 2, J=0..2: the library's kappa_2(X_t) reproduces the printed column."""
    from conftest import read_golden
    from paper_2504_07269_gb300 import stfdm

    rows = read_golden("table2_fdm_uniform.txt")
    for J in range(3):
        h = stfdm.st_assemble_time(1, synth.uniform_time_nodes(64 * 2 ** J, 5.0))
        kappa = stfdm.st_time_decompose(h)[3]
        assert "%.1e" % kappa == "%.1e" % float(rows[J][8])


def test_bad_arguments(L):
    from paper_2504_07269_gb300 import _lib, stfdm

    with pytest.raises(_lib.StfdmError) as e:
        stfdm.st_assemble_time(3, [0.0, 1.0])
    assert e.value.status == _lib.ST_ERR_ARG
    with pytest.raises(_lib.StfdmError) as e:
        stfdm.st_assemble_time(1, [0.0, 0.5, 0.5, 1.0])
    assert e.value.status == _lib.ST_ERR_ARG
    with pytest.raises(_lib.StfdmError) as e:
        stfdm.st_assemble_time(1, [0.1, 0.5])
    assert e.value.status == _lib.ST_ERR_ARG
    with pytest.raises(_lib.StfdmError) as e:
        stfdm.st_assemble_space(1)
    assert e.value.status == _lib.ST_ERR_ARG
    with pytest.raises(_lib.StfdmError) as e:
        stfdm.st_assemble_space(8, -1.0, 1.0)
    assert e.value.status == _lib.ST_ERR_ARG
    out = ctypes.c_void_p()
    assert L.st_fdm_setup(None, None, None, ctypes.byref(out)) == _lib.ST_ERR_ARG
    assert L.st_fdm_solve(None, None, None, None, None, None, None) == _lib.ST_ERR_ARG
    assert L.st_fdm_setup(None, None, None, None) == _lib.ST_ERR_ARG
