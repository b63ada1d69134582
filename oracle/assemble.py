"""Explicit space-time assembly (oracle; test infrastructure only).

The Galerkin system of eq. (VF_FEM) is assembled straight from the
sesquilinear form of eq. (VF_inhomogen),

    a(u, v) = i <d_t u, v>_{L2(Q)} + <grad_x u, grad_x v>_{L2(Q)},

on each space-time prism (time element x triangle) with the tensor-product
basis phi_k(t) varphi_alpha(x) of Q^p_h (Section 3), by quadrature on the
prism.  Test index = row.  Real basis functions, so the conjugation of the
L2 inner product does not act on them.  No Kronecker product is used here;
`kron_system` builds eq. (LGS) the other way for the comparison test.

Unknown ordering: time-outer, i.e. index = time_dof * n_x + space_dof, with
time DOFs t_1..t_{n_t} (t_0 removed) and interior space DOFs x1-fastest.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .fe_space import interior_map, structured_mesh
from .fe_time import lagrange_ref
from .quadrature import gauss_interval, triangle_rule


def _space_quadrature(nodes, tris, order):
    """Physical quadrature points, weights and P1 basis values/gradients per triangle."""
    xi, eta, w = triangle_rule(order)
    lam = np.stack([1.0 - xi - eta, xi, eta])            # (3, R)
    V = nodes[tris]                                     # (T, 3, 2)
    v0 = V[:, 0]
    J = np.stack([V[:, 1] - v0, V[:, 2] - v0], axis=2)  # (T, 2, 2)
    detJ = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
    X = v0[:, None, :] + np.einsum("tij,rj->tri", J, np.stack([xi, eta], 1))  # (T, R, 2)
    W = np.abs(detJ)[:, None] * w[None, :]              # (T, R)
    Jinv = np.empty_like(J)
    Jinv[:, 0, 0] = J[:, 1, 1] / detJ
    Jinv[:, 1, 1] = J[:, 0, 0] / detJ
    Jinv[:, 0, 1] = -J[:, 0, 1] / detJ
    Jinv[:, 1, 0] = -J[:, 1, 0] / detJ
    dref = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])
    G = np.einsum("ar,trc->tac", dref, Jinv)            # (T, 3, 2) gradient of basis a
    return X, W, lam, G


def explicit_system(n: int, p: int, t_nodes, Lx=1.0, Ly=1.0, keep_t0=False):
    """Sparse complex K of eq. (LGS) assembled prism by prism from a(.,.).

    keep_t0=False: rows/cols of Q_{h,0,} only (n_t = p N_t time DOFs).
    keep_t0=True : trial columns include the t_0 DOFs (shape n_t n_x x (n_t+1) n_x),
                   rows are still the test space Q_{h,0,}.
    """
    t = np.asarray(t_nodes, dtype=np.float64)
    N_t = len(t) - 1
    nodes, tris = structured_mesh(n, Lx, Ly)
    imap = interior_map(n)
    n_x = (n - 1) ** 2
    n_t = p * N_t
    X, W, lam, G = _space_quadrature(nodes, tris, 2)
    sq, sw = gauss_interval(p + 2, 0.0, 1.0)
    phi, dphi = lagrange_ref(p, sq)                     # (p+1, Q)
    # local space index pairs
    ncol_t = n_t + 1 if keep_t0 else n_t
    rows_all, cols_all, vals_all = [], [], []
    sidx = imap[tris]                                   # (T, 3) interior index or -1
    # spatial integrals per triangle that appear in the prism quadrature:
    # int varphi_b varphi_a  and int grad varphi_b . grad varphi_a, by quadrature
    Mloc = np.einsum("ar,br,tr->tab", lam, lam, W)      # (T, 3, 3) [test a, trial b]
    Aloc = np.einsum("tac,tbc,tr->tab", G, G, W)
    for e in range(N_t):
        tau = t[e + 1] - t[e]
        wt = tau * sw                                   # time weights
        # time factors of the prism integrals, test k (row) / trial j (col)
        tm = np.einsum("kq,jq,q->kj", phi, phi, wt)                 # int phi_j phi_k
        tb = np.einsum("kq,jq,q->kj", phi, dphi / tau, wt)          # int phi_j' phi_k
        # prism integral: a(phi_j varphi_b, phi_k varphi_a) =
        #   i int int (d_t phi_j) varphi_b phi_k varphi_a + int int phi_j grad varphi_b . phi_k grad varphi_a
        # the double integral over the prism is the product of the time and space quadratures
        loc = (1j * tb[None, :, None, :, None] * Mloc[:, None, :, None, :]
               + tm[None, :, None, :, None] * Aloc[:, None, :, None, :])   # (T, k, a, j, b)
        gt = p * e + np.arange(p + 1)                   # full time DOF indices of the element
        for kk in range(p + 1):
            if gt[kk] == 0:
                continue                                # t_0 is not a test DOF
            rt = gt[kk] - 1
            for jj in range(p + 1):
                if gt[jj] == 0 and not keep_t0:
                    continue
                ct = gt[jj] if keep_t0 else gt[jj] - 1
                for a in range(3):
                    ra = sidx[:, a]
                    for b in range(3):
                        cb = sidx[:, b]
                        ok = (ra >= 0) & (cb >= 0)
                        rows_all.append(rt * n_x + ra[ok])
                        cols_all.append(ct * n_x + cb[ok])
                        vals_all.append(loc[ok, kk, a, jj, b])
    rows = np.concatenate(rows_all)
    cols = np.concatenate(cols_all)
    vals = np.concatenate(vals_all)
    K = sp.csr_matrix((vals, (rows, cols)), shape=(n_t * n_x, ncol_t * n_x))
    K.sum_duplicates()
    return K


def kron_system(M_t, B_t, M_x, A_x):
    """eq. (LGS) the Kronecker way: i B_t (x) M_x + M_t (x) A_x."""
    return (1j * sp.kron(sp.csr_matrix(B_t), M_x) + sp.kron(sp.csr_matrix(M_t), A_x)).tocsr()


def load_vector(n: int, p: int, t_nodes, f, Lx=1.0, Ly=1.0, t_order=6, x_order=6):
    """F[k, alpha] = int_Q f phi_k varphi_alpha, by prism quadrature (Gauss in t x
    collapsed Gauss on triangles).  Returns an (n_t, n_x) complex array."""
    t = np.asarray(t_nodes, dtype=np.float64)
    N_t = len(t) - 1
    nodes, tris = structured_mesh(n, Lx, Ly)
    imap = interior_map(n)
    n_x = (n - 1) ** 2
    X, W, lam, _ = _space_quadrature(nodes, tris, x_order)
    sq, sw = gauss_interval(t_order, 0.0, 1.0)
    phi, _ = lagrange_ref(p, sq)
    sidx = imap[tris]
    F = np.zeros((p * N_t + 1, n_x), dtype=np.complex128)
    for e in range(N_t):
        tau = t[e + 1] - t[e]
        for q in range(len(sq)):
            tq = t[e] + tau * sq[q]
            fv = f(X[..., 0], X[..., 1], tq)            # (T, R)
            # int over triangles of f varphi_a at this time point
            sa = np.einsum("tr,ar,tr->ta", fv, lam, W)  # (T, 3)
            for kk in range(p + 1):
                wk = tau * sw[q] * phi[kk, q]
                row = p * e + kk
                for a in range(3):
                    ok = sidx[:, a] >= 0
                    np.add.at(F[row], sidx[ok, a], wk * sa[ok, a])
    return F[1:]


def lifting_vector(n: int, p: int, t_nodes, psi0_nodal, Lx=1.0, Ly=1.0):
    """a(psi0_h, phi_k varphi_alpha) for psi0_h = sum_beta psi0_beta varphi_beta(x),
    constant in time (Section 3: psi-hat = psi - psi0), by prism quadrature.
    psi0_nodal: interior nodal values (boundary values are zero).  Returns (n_t, n_x)."""
    t = np.asarray(t_nodes, dtype=np.float64)
    N_t = len(t) - 1
    nodes, tris = structured_mesh(n, Lx, Ly)
    imap = interior_map(n)
    n_x = (n - 1) ** 2
    X, W, lam, G = _space_quadrature(nodes, tris, 2)
    sq, sw = gauss_interval(p + 2, 0.0, 1.0)
    phi, _ = lagrange_ref(p, sq)
    sidx = imap[tris]
    vals = np.where(sidx >= 0, np.asarray(psi0_nodal)[np.maximum(sidx, 0)], 0.0)   # (T, 3)
    grad_psi0 = np.einsum("tb,tbc->tc", vals, G)                 # constant per triangle
    dt_psi0 = 0.0                                                # psi0_h does not depend on t
    area_w = W.sum(axis=1)                                       # (T,)
    space_term = np.einsum("tc,tac->ta", grad_psi0, G) * area_w[:, None]   # int grad psi0 . grad varphi_a
    space_mass = np.einsum("tb,ar,br,tr->ta", vals, lam, lam, W)           # int psi0 varphi_a
    L = np.zeros((p * N_t + 1, n_x), dtype=np.complex128)
    for e in range(N_t):
        tau = t[e + 1] - t[e]
        for kk in range(p + 1):
            row = p * e + kk
            wk = tau * np.sum(sw * phi[kk])                          # int phi_k over the element
            contrib = 1j * dt_psi0 * wk * space_mass + wk * space_term
            for a in range(3):
                ok = sidx[:, a] >= 0
                np.add.at(L[row], sidx[ok, a], contrib[ok, a])
    return L[1:]
