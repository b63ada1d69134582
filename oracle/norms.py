"""Space-time error norms (oracle; test infrastructure only).

Section 4:  ||e||_{L2(Q)}  and  |e|_{H1(Q)} = (||d_t e||^2_{L2(Q)} + ||grad_x e||^2_{L2(Q)})^{1/2}
for e = psi - psi_h, psi_h in Q^p_h given by its nodal values at all time DOFs
(t_0 included) and interior space nodes (zero on the boundary).  Tensor
quadrature on every prism.
"""
from __future__ import annotations

import numpy as np

from .assemble import _space_quadrature
from .fe_space import interior_map, structured_mesh
from .fe_time import lagrange_ref
from .quadrature import gauss_interval


def errors(n, p, t_nodes, U_full, psi, dpsi, Lx=1.0, Ly=1.0, t_order=4, x_order=4):
    """Return (L2 error, H1-seminorm error).

    U_full: (p N_t + 1, n_x) nodal values including the t_0 row.
    psi(x1, x2, t), dpsi(x1, x2, t) -> (d_t, d_x1, d_x2): exact solution.
    """
    t = np.asarray(t_nodes, dtype=np.float64)
    N_t = len(t) - 1
    nodes, tris = structured_mesh(n, Lx, Ly)
    imap = interior_map(n)
    X, W, lam, G = _space_quadrature(nodes, tris, x_order)
    sq, sw = gauss_interval(t_order, 0.0, 1.0)
    phi, dphi = lagrange_ref(p, sq)
    sidx = imap[tris]
    e2 = 0.0
    h2 = 0.0
    for e in range(N_t):
        tau = t[e + 1] - t[e]
        rows = p * e + np.arange(p + 1)
        # nodal values on the prism: (p+1, T, 3)
        vals = np.where(sidx[None] >= 0, U_full[rows][:, np.maximum(sidx, 0)], 0.0)
        for q in range(len(sq)):
            tq = t[e] + tau * sq[q]
            wq = tau * sw[q]
            v_t = np.einsum("k,kta->ta", phi[:, q], vals)            # value in time at tq
            d_t = np.einsum("k,kta->ta", dphi[:, q] / tau, vals)     # time derivative
            uh = np.einsum("ta,ar->tr", v_t, lam)
            uh_t = np.einsum("ta,ar->tr", d_t, lam)
            gx = np.einsum("ta,tac->tc", v_t, G)                      # constant in space per triangle
            ex = psi(X[..., 0], X[..., 1], tq)
            ddt, dx1, dx2 = dpsi(X[..., 0], X[..., 1], tq)
            e2 += wq * np.sum(W * np.abs(ex - uh) ** 2)
            h2 += wq * np.sum(W * (np.abs(ddt - uh_t) ** 2 + np.abs(dx1 - gx[:, None, 0]) ** 2
                                   + np.abs(dx2 - gx[:, None, 1]) ** 2))
    return float(np.sqrt(e2)), float(np.sqrt(h2))
