// Spatial matrices of eq. (matrix_x) on a general simplicial mesh (the spaces S^p_hx of
// Section 2 for d = 2, 3 and p = 1, 2; Dirichlet boundary):
//
//     M_x[k, j] = int phi_j phi_k dx,      A_x[k, j] = int grad phi_j . grad phi_k dx.
//
// The Lagrange basis of a cell is written in its barycentric coordinates lambda_0..lambda_d
// (p = 1: lambda_a; p = 2: lambda_a (2 lambda_a - 1) at the vertices, 4 lambda_a lambda_b at the
// edges), so every integrand is a polynomial in the lambdas, integrated exactly by
//
//     int_T lambda_0^{a_0} ... lambda_d^{a_d} dx = |T| d! a_0! ... a_d! / (a_0 + ... + a_d + d)!.
//
// Gradients: grad phi = sum_c (d phi / d lambda_c) grad lambda_c with constant grad lambda_c per
// cell, so A_loc = |T| sum_{c,e} G_ce I[a][b][c][e] with G_ce = grad lambda_c . grad lambda_e.
//
// DOFs: the vertices in input order, then (p = 2) the edges ordered by their (smaller vertex,
// larger vertex) pair.  A DOF is on the boundary when it lies on a boundary facet (a facet of
// exactly one cell); the interior DOFs keep the global order.  The matrices are stored in CSR
// over the interior DOFs on the union pattern of M_x and A_x (sorted columns).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "internal.h"

namespace stfdm {
namespace {

// a polynomial in the d + 1 barycentric coordinates: terms coef * prod lambda_c^{e_c}
struct Term {
    double c;
    std::array<int, 4> e;
};
using Poly = std::vector<Term>;

Poly mul(const Poly& a, const Poly& b) {
    Poly out;
    for (const Term& x : a)
        for (const Term& y : b) {
            Term t;
            t.c = x.c * y.c;
            for (int i = 0; i < 4; ++i) t.e[i] = x.e[i] + y.e[i];
            out.push_back(t);
        }
    return out;
}

// d/d lambda_c
Poly diff(const Poly& a, int c) {
    Poly out;
    for (const Term& x : a)
        if (x.e[c] > 0) {
            Term t = x;
            t.c *= x.e[c];
            t.e[c] -= 1;
            out.push_back(t);
        }
    return out;
}

double fact(int n) {
    double f = 1;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

// int over a cell of unit measure
double integrate(const Poly& a, int d) {
    double s = 0;
    for (const Term& x : a) {
        int deg = 0;
        double num = fact(d);
        for (int i = 0; i <= d; ++i) {
            num *= fact(x.e[i]);
            deg += x.e[i];
        }
        s += x.c * num / fact(deg + d);
    }
    return s;
}

Term mono(double c, int i = -1, int j = -1) {
    Term t{c, {0, 0, 0, 0}};
    if (i >= 0) t.e[i] += 1;
    if (j >= 0) t.e[j] += 1;
    return t;
}

// local basis: vertices 0..d, then (p = 2) edges (a, b), a < b, lexicographic
struct LocalBasis {
    int d = 0, p = 0, nl = 0;
    std::vector<std::pair<int, int>> dof;   // (a, -1) vertex, (a, b) edge
    std::vector<double> IM;                 // [nl][nl]       int phi_a phi_b / |T|
    std::vector<double> IA;                 // [nl][nl][d+1][d+1]
};

LocalBasis make_basis(int d, int p) {
    LocalBasis B;
    B.d = d;
    B.p = p;
    for (int a = 0; a <= d; ++a) B.dof.push_back({a, -1});
    if (p == 2)
        for (int a = 0; a <= d; ++a)
            for (int b = a + 1; b <= d; ++b) B.dof.push_back({a, b});
    B.nl = (int)B.dof.size();
    std::vector<Poly> phi(B.nl);
    for (int i = 0; i < B.nl; ++i) {
        const int a = B.dof[i].first, b = B.dof[i].second;
        if (b >= 0) phi[i] = {mono(4.0, a, b)};
        else if (p == 1) phi[i] = {mono(1.0, a)};
        else phi[i] = {mono(2.0, a, a), mono(-1.0, a)};
    }
    const int nc = d + 1;
    B.IM.assign((size_t)B.nl * B.nl, 0.0);
    B.IA.assign((size_t)B.nl * B.nl * nc * nc, 0.0);
    for (int i = 0; i < B.nl; ++i)
        for (int j = 0; j < B.nl; ++j) {
            B.IM[(size_t)i * B.nl + j] = integrate(mul(phi[i], phi[j]), d);
            for (int c = 0; c < nc; ++c)
                for (int e = 0; e < nc; ++e)
                    B.IA[(((size_t)i * B.nl + j) * nc + c) * nc + e] = integrate(mul(diff(phi[i], c), diff(phi[j], e)), d);
        }
    return B;
}

// inverse of a d x d matrix (d = 2, 3) and its determinant; false if singular
bool invert(int d, const double* J, double* Ji, double& det) {
    if (d == 2) {
        det = J[0] * J[3] - J[1] * J[2];
        if (det == 0.0 || !std::isfinite(det)) return false;
        Ji[0] = J[3] / det;
        Ji[1] = -J[1] / det;
        Ji[2] = -J[2] / det;
        Ji[3] = J[0] / det;
        return true;
    }
    const double a = J[0], b = J[1], c = J[2], dd = J[3], e = J[4], f = J[5], g = J[6], h = J[7], i = J[8];
    const double A = e * i - f * h, Bc = -(dd * i - f * g), Cc = dd * h - e * g;
    det = a * A + b * Bc + c * Cc;
    if (det == 0.0 || !std::isfinite(det)) return false;
    Ji[0] = A / det;
    Ji[1] = -(b * i - c * h) / det;
    Ji[2] = (b * f - c * e) / det;
    Ji[3] = Bc / det;
    Ji[4] = (a * i - c * g) / det;
    Ji[5] = -(a * f - c * dd) / det;
    Ji[6] = Cc / det;
    Ji[7] = -(a * h - b * g) / det;
    Ji[8] = (a * e - b * dd) / det;
    return true;
}

}  // namespace

st_status assemble_mesh(int dim, int p, int nv, const double* coords, int nc, const int* cells, MeshSpace& out) {
    const int npc = dim + 1;
    for (size_t q = 0; q < (size_t)nc * npc; ++q)
        if (cells[q] < 0 || cells[q] >= nv) return fail(ST_ERR_ARG, "st_assemble_mesh: cell vertex index out of range");
    // edges (p = 2): sorted unique (min, max) pairs
    std::vector<std::pair<int, int>> edges;
    if (p == 2) {
        edges.reserve((size_t)nc * npc * (npc - 1) / 2);
        for (int c = 0; c < nc; ++c)
            for (int a = 0; a < npc; ++a)
                for (int b = a + 1; b < npc; ++b) {
                    int u = cells[(size_t)c * npc + a], v = cells[(size_t)c * npc + b];
                    if (u == v) return fail(ST_ERR_ARG, "st_assemble_mesh: repeated vertex in a cell");
                    edges.push_back({std::min(u, v), std::max(u, v)});
                }
        std::sort(edges.begin(), edges.end());
        edges.erase(std::unique(edges.begin(), edges.end()), edges.end());
    }
    auto edge_id = [&](int u, int v) {
        std::pair<int, int> key{std::min(u, v), std::max(u, v)};
        return (int)(std::lower_bound(edges.begin(), edges.end(), key) - edges.begin());
    };
    const int ndof = nv + (int)edges.size();
    // boundary: facets (sorted vertex tuples) that belong to exactly one cell
    std::vector<std::array<int, 3>> facets;
    facets.reserve((size_t)nc * npc);
    for (int c = 0; c < nc; ++c)
        for (int drop = 0; drop < npc; ++drop) {
            std::array<int, 3> f{-1, -1, -1};
            int k = 0;
            for (int a = 0; a < npc; ++a)
                if (a != drop) f[k++] = cells[(size_t)c * npc + a];
            std::sort(f.begin(), f.begin() + dim);
            facets.push_back(f);
        }
    std::sort(facets.begin(), facets.end());
    std::vector<char> bnd(ndof, 0);
    for (size_t i = 0; i < facets.size();) {
        size_t j = i + 1;
        while (j < facets.size() && facets[j] == facets[i]) ++j;
        if (j - i == 1) {
            const auto& f = facets[i];
            for (int a = 0; a < dim; ++a) bnd[f[a]] = 1;
            if (p == 2)
                for (int a = 0; a < dim; ++a)
                    for (int b = a + 1; b < dim; ++b) bnd[nv + edge_id(f[a], f[b])] = 1;
        } else if (j - i > 2) {
            return fail(ST_ERR_ARG, "st_assemble_mesh: a facet is shared by more than two cells");
        }
        i = j;
    }
    std::vector<int> inner(ndof, -1);
    int n_x = 0;
    for (int g = 0; g < ndof; ++g)
        if (!bnd[g]) inner[g] = n_x++;
    if (n_x == 0) return fail(ST_ERR_ARG, "st_assemble_mesh: no interior DOF");
    // element matrices, scattered as COO over interior DOFs
    const LocalBasis B = make_basis(dim, p);
    const int nl = B.nl;
    struct Entry {
        int r, c;
        double m, a;
    };
    std::vector<Entry> coo;
    coo.reserve((size_t)nc * nl * nl);
    std::vector<int> gd(nl);
    for (int c = 0; c < nc; ++c) {
        const int* cv = cells + (size_t)c * npc;
        double J[9], Ji[9], det = 0;
        for (int r = 0; r < dim; ++r)
            for (int s = 0; s < dim; ++s) J[r * dim + s] = coords[(size_t)cv[s + 1] * dim + r] - coords[(size_t)cv[0] * dim + r];
        if (!invert(dim, J, Ji, det)) return fail(ST_ERR_ARG, "st_assemble_mesh: degenerate cell");
        const double vol = std::fabs(det) / (dim == 2 ? 2.0 : 6.0);
        // grad lambda_r (r >= 1) = row r-1 of J^{-1}; grad lambda_0 = -sum
        double gl[4][3] = {};
        for (int r = 1; r <= dim; ++r)
            for (int s = 0; s < dim; ++s) {
                gl[r][s] = Ji[(r - 1) * dim + s];
                gl[0][s] -= gl[r][s];
            }
        double G[4][4];
        for (int a = 0; a <= dim; ++a)
            for (int b = 0; b <= dim; ++b) {
                double t = 0;
                for (int s = 0; s < dim; ++s) t += gl[a][s] * gl[b][s];
                G[a][b] = t;
            }
        for (int i = 0; i < nl; ++i) {
            const auto& dd = B.dof[i];
            gd[i] = dd.second < 0 ? cv[dd.first] : nv + edge_id(cv[dd.first], cv[dd.second]);
        }
        for (int i = 0; i < nl; ++i) {
            const int ri = inner[gd[i]];
            if (ri < 0) continue;
            for (int j = 0; j < nl; ++j) {
                const int cj = inner[gd[j]];
                if (cj < 0) continue;
                double a = 0;
                for (int u = 0; u <= dim; ++u)
                    for (int v = 0; v <= dim; ++v) a += G[u][v] * B.IA[(((size_t)i * nl + j) * (dim + 1) + u) * (dim + 1) + v];
                coo.push_back({ri, cj, vol * B.IM[(size_t)i * nl + j], vol * a});
            }
        }
    }
    std::sort(coo.begin(), coo.end(), [](const Entry& x, const Entry& y) { return x.r != y.r ? x.r < y.r : x.c < y.c; });
    out = MeshSpace{};
    out.dim = dim;
    out.p = p;
    out.n_x = n_x;
    out.rowptr.assign(n_x + 1, 0);
    for (size_t i = 0; i < coo.size();) {
        size_t j = i;
        double m = 0, a = 0;
        while (j < coo.size() && coo[j].r == coo[i].r && coo[j].c == coo[i].c) {
            m += coo[j].m;
            a += coo[j].a;
            ++j;
        }
        out.col.push_back(coo[i].c);
        out.Mv.push_back(m);
        out.Av.push_back(a);
        out.rowptr[coo[i].r + 1] += 1;
        i = j;
    }
    for (int r = 0; r < n_x; ++r) out.rowptr[r + 1] += out.rowptr[r];
    out.xyz.resize((size_t)n_x * dim);
    for (int g = 0; g < ndof; ++g) {
        const int r = inner[g];
        if (r < 0) continue;
        for (int s = 0; s < dim; ++s) {
            double x;
            if (g < nv) x = coords[(size_t)g * dim + s];
            else {
                const auto& e = edges[g - nv];
                x = 0.5 * (coords[(size_t)e.first * dim + s] + coords[(size_t)e.second * dim + s]);
            }
            out.xyz[(size_t)r * dim + s] = x;
        }
    }
    return ST_OK;
}

// The structured grid as a mesh (CSR of its 7-point stencils, node coordinates), so that the
// sparse-direct spatial solver can also run on it.
void structured_as_mesh(const SpaceMats& sm, MeshSpace& out) {
    const int m = sm.m;
    out = MeshSpace{};
    out.dim = 2;
    out.p = 1;
    out.n_x = sm.n_x;
    out.rowptr.assign(sm.n_x + 1, 0);
    const int di[7] = {-m - 1, -m, -1, 0, 1, m, m + 1};
    for (int x = 0; x < sm.n_x; ++x) {
        const int xi = x % m, yj = x / m;
        for (int t = 0; t < 7; ++t) {
            const int ox = (t == 0 || t == 2) ? -1 : (t == 4 || t == 6) ? 1 : 0;
            const int oy = (t <= 1) ? -1 : (t >= 5) ? 1 : 0;
            if (xi + ox < 0 || xi + ox >= m || yj + oy < 0 || yj + oy >= m) continue;
            double mv, av;
            if (t == 3) mv = sm.Mc, av = sm.Ac;
            else if (t == 2 || t == 4) mv = sm.Mw, av = sm.Aw;
            else if (t == 1 || t == 5) mv = sm.Ms, av = sm.As;
            else mv = sm.Md, av = sm.Ad;
            out.col.push_back(x + di[t]);
            out.Mv.push_back(mv);
            out.Av.push_back(av);
            out.rowptr[x + 1] += 1;
        }
    }
    for (int r = 0; r < sm.n_x; ++r) out.rowptr[r + 1] += out.rowptr[r];
    out.xyz.resize((size_t)sm.n_x * 2);
    for (int x = 0; x < sm.n_x; ++x) {
        out.xyz[2 * x] = (x % m + 1) * (sm.Lx / sm.n);
        out.xyz[2 * x + 1] = (x / m + 1) * (sm.Ly / sm.n);
    }
}

}  // namespace stfdm

using namespace stfdm;

extern "C" st_status st_assemble_mesh(int dim, int p_x, int n_vertices, const double* coords, int n_cells,
                                      const int* cells, st_space** out) {
    if (!out || !coords || !cells) return fail(ST_ERR_ARG, "st_assemble_mesh: NULL argument");
    *out = nullptr;
    if (dim != 2 && dim != 3) return fail(ST_ERR_ARG, "st_assemble_mesh: dim must be 2 or 3");
    if (p_x != 1 && p_x != 2) return fail(ST_ERR_ARG, "st_assemble_mesh: p_x must be 1 or 2");
    if (n_vertices < dim + 1 || n_cells < 1) return fail(ST_ERR_ARG, "st_assemble_mesh: empty mesh");
    try {
        st_space* s = new st_space();
        s->sm.kind = 1;
        st_status st = assemble_mesh(dim, p_x, n_vertices, coords, n_cells, cells, s->sm.mesh);
        if (st != ST_OK) {
            delete s;
            return st;
        }
        s->sm.n_x = s->sm.mesh.n_x;
        *out = s;
        return ST_OK;
    } catch (const std::bad_alloc&) {
        return fail(ST_ERR_OOM, "st_assemble_mesh: host allocation");
    }
}

extern "C" st_status st_space_get_mesh(const st_space* s, int* dim, int* p_x, int* n_x, long long* nnz, int* rowptr,
                                       int* col, double* M, double* A, double* xyz) {
    if (!s) return fail(ST_ERR_ARG, "st_space_get_mesh: NULL handle");
    MeshSpace tmp;
    const MeshSpace* ms = &s->sm.mesh;
    if (s->sm.kind == 0) {
        structured_as_mesh(s->sm, tmp);
        ms = &tmp;
    }
    if (dim) *dim = ms->dim;
    if (p_x) *p_x = ms->p;
    if (n_x) *n_x = ms->n_x;
    if (nnz) *nnz = (long long)ms->col.size();
    if (rowptr) std::memcpy(rowptr, ms->rowptr.data(), ms->rowptr.size() * sizeof(int));
    if (col) std::memcpy(col, ms->col.data(), ms->col.size() * sizeof(int));
    if (M) std::memcpy(M, ms->Mv.data(), ms->Mv.size() * sizeof(double));
    if (A) std::memcpy(A, ms->Av.data(), ms->Av.size() * sizeof(double));
    if (xyz) std::memcpy(xyz, ms->xyz.data(), ms->xyz.size() * sizeof(double));
    return ST_OK;
}
