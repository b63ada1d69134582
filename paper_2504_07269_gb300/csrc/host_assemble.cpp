// Host assembly of the temporal and spatial matrices (eq. matrix_t, eq. matrix_x)
// and the status / error plumbing of the C ABI.
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "internal.h"

namespace stfdm {

static thread_local std::string g_last_error;

st_status fail(st_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

}  // namespace stfdm

using namespace stfdm;

extern "C" const char* st_status_string(st_status s) {
    switch (s) {
        case ST_OK: return "ok";
        case ST_ERR_ARG: return "invalid argument";
        case ST_ERR_OOM: return "out of memory";
        case ST_ERR_CUDA: return "CUDA error";
        case ST_ERR_ILL_CONDITIONED: return "ill-conditioned time decomposition";
        case ST_ERR_ZERO_PIVOT: return "zero or non-finite pivot";
        case ST_ERR_NOT_CONVERGED: return "not converged";
        case ST_ERR_TIMEOUT: return "device wait timed out";
        case ST_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

extern "C" const char* st_last_error_message(void) { return g_last_error.c_str(); }

extern "C" int st_abi_version(void) { return STFDM_ABI_VERSION; }

// Element matrices of eq. (matrix_t) for Lagrange elements with equispaced nodes,
// integrated by hand (rows = test index k, columns = trial index j):
//   P1: M = tau/6 [[2,1],[1,2]],  B[k][j] = int phi_j' phi_k = [[-1/2, 1/2], [-1/2, 1/2]]
//   P2: M = tau/30 [[4,2,-1],[2,16,2],[-1,2,4]],
//       B = [[-1/2, 2/3, -1/6], [-2/3, 0, 2/3], [1/6, -2/3, 1/2]]
//   int phi_k: P1 tau/2 each, P2 (tau/6, 2 tau/3, tau/6)
static void time_element(int p, double tau, double M[3][3], double B[3][3], double m[3]) {
    if (p == 1) {
        const double Mr[2][2] = {{2, 1}, {1, 2}};
        const double Br[2][2] = {{-0.5, 0.5}, {-0.5, 0.5}};
        for (int a = 0; a < 2; ++a) {
            m[a] = tau / 2;
            for (int c = 0; c < 2; ++c) {
                M[a][c] = tau / 6 * Mr[a][c];
                B[a][c] = Br[a][c];
            }
        }
    } else {
        const double Mr[3][3] = {{4, 2, -1}, {2, 16, 2}, {-1, 2, 4}};
        const double Br[3][3] = {{-0.5, 2.0 / 3, -1.0 / 6}, {-2.0 / 3, 0, 2.0 / 3}, {1.0 / 6, -2.0 / 3, 0.5}};
        const double mr[3] = {1.0 / 6, 2.0 / 3, 1.0 / 6};
        for (int a = 0; a < 3; ++a) {
            m[a] = tau * mr[a];
            for (int c = 0; c < 3; ++c) {
                M[a][c] = tau / 30 * Mr[a][c];
                B[a][c] = Br[a][c];
            }
        }
    }
}

extern "C" st_status st_assemble_time(int p_t, int N_t, const double* t_nodes, st_time** out) {
    if (!out) return fail(ST_ERR_ARG, "st_assemble_time: out is NULL");
    *out = nullptr;
    if (p_t != 1 && p_t != 2) return fail(ST_ERR_ARG, "st_assemble_time: p_t must be 1 or 2");
    if (N_t < 1 || N_t > (1 << 20)) return fail(ST_ERR_ARG, "st_assemble_time: N_t out of range");
    if (!t_nodes) return fail(ST_ERR_ARG, "st_assemble_time: t_nodes is NULL");
    if (t_nodes[0] != 0.0) return fail(ST_ERR_ARG, "st_assemble_time: t_nodes[0] must be 0");
    for (int e = 0; e < N_t; ++e)
        if (!(t_nodes[e + 1] > t_nodes[e]) || !std::isfinite(t_nodes[e + 1]))
            return fail(ST_ERR_ARG, "st_assemble_time: t_nodes must be finite and strictly increasing");
    st_time* t = new (std::nothrow) st_time();
    if (!t) return fail(ST_ERR_OOM, "st_assemble_time: host allocation");
    TimeMats& tm = t->tm;
    tm.p = p_t;
    tm.N = N_t;
    tm.n_t = p_t * N_t;
    tm.nodes.assign(t_nodes, t_nodes + N_t + 1);
    const int nf = tm.n_t + 1;  // full size including t_0
    std::vector<double> Mf((size_t)nf * 5, 0.0), Bf((size_t)nf * 5, 0.0), mf(nf, 0.0), tf(nf, 0.0);
    for (int e = 0; e < N_t; ++e) {
        double tau = t_nodes[e + 1] - t_nodes[e];
        double M[3][3], B[3][3], m[3];
        time_element(p_t, tau, M, B, m);
        for (int a = 0; a <= p_t; ++a) {
            int ga = p_t * e + a;
            tf[ga] = t_nodes[e] + tau * a / p_t;
            mf[ga] += m[a];
            for (int c = 0; c <= p_t; ++c) {
                int gc = p_t * e + c;
                Mf[(size_t)ga * 5 + (gc - ga) + 2] += M[a][c];
                Bf[(size_t)ga * 5 + (gc - ga) + 2] += B[a][c];
            }
        }
    }
    tm.Mb.assign((size_t)tm.n_t * 5, 0.0);
    tm.Bb.assign((size_t)tm.n_t * 5, 0.0);
    tm.Mfull0.assign(tm.n_t, 0.0);
    tm.m.assign(tm.n_t, 0.0);
    tm.times.assign(tm.n_t, 0.0);
    for (int l = 0; l < tm.n_t; ++l) {
        int gl = l + 1;
        for (int d = -2; d <= 2; ++d) {
            int gc = gl + d;
            if (gc < 0 || gc >= nf) continue;
            if (gc == 0) {
                tm.Mfull0[l] = Mf[(size_t)gl * 5 + d + 2];
                continue;
            }
            tm.Mb[(size_t)l * 5 + d + 2] = Mf[(size_t)gl * 5 + d + 2];
            tm.Bb[(size_t)l * 5 + d + 2] = Bf[(size_t)gl * 5 + d + 2];
        }
        tm.m[l] = mf[gl];
        tm.times[l] = tf[gl];
    }
    *out = t;
    return ST_OK;
}

extern "C" st_status st_time_get(const st_time* t, int* n_t, double* M_t, double* B_t, double* m_t,
                                 double* dof_times) {
    if (!t) return fail(ST_ERR_ARG, "st_time_get: NULL handle");
    const TimeMats& tm = t->tm;
    const int n = tm.n_t;
    if (n_t) *n_t = n;
    if (M_t) std::memset(M_t, 0, sizeof(double) * (size_t)n * n);
    if (B_t) std::memset(B_t, 0, sizeof(double) * (size_t)n * n);
    for (int l = 0; l < n; ++l) {
        for (int d = -2; d <= 2; ++d) {
            int c = l + d;
            if (c < 0 || c >= n) continue;
            if (M_t) M_t[(size_t)l * n + c] = tm.Mb[(size_t)l * 5 + d + 2];
            if (B_t) B_t[(size_t)l * n + c] = tm.Bb[(size_t)l * 5 + d + 2];
        }
        if (m_t) m_t[l] = tm.m[l];
        if (dof_times) dof_times[l] = tm.times[l];
    }
    return ST_OK;
}

// P1 on right triangles with legs h1, h2 (SW-NE split): the edge opposite a right angle
// (the diagonal) has zero stiffness coupling (cot 90 = 0); an x1-edge is opposite an angle
// with cot = h2/h1 in both adjacent triangles, an x2-edge one with cot = h1/h2; every edge
// carries mass (|T|/12) from both triangles; six triangles of area h1 h2/2 meet at a node.
extern "C" st_status st_assemble_space(int n_squares, double Lx, double Ly, st_space** out) {
    if (!out) return fail(ST_ERR_ARG, "st_assemble_space: out is NULL");
    *out = nullptr;
    if (n_squares < 2 || n_squares > 46341) return fail(ST_ERR_ARG, "st_assemble_space: n_squares out of range");
    if (!(Lx > 0) || !(Ly > 0) || !std::isfinite(Lx) || !std::isfinite(Ly))
        return fail(ST_ERR_ARG, "st_assemble_space: lengths must be positive");
    st_space* s = new (std::nothrow) st_space();
    if (!s) return fail(ST_ERR_OOM, "st_assemble_space: host allocation");
    SpaceMats& sm = s->sm;
    sm.n = n_squares;
    sm.m = n_squares - 1;
    sm.n_x = sm.m * sm.m;
    sm.Lx = Lx;
    sm.Ly = Ly;
    const double h1 = Lx / n_squares, h2 = Ly / n_squares;
    sm.Mc = h1 * h2 / 2;
    sm.Mw = h1 * h2 / 12;
    sm.Ms = h1 * h2 / 12;
    sm.Md = h1 * h2 / 12;
    sm.Ac = 2 * (h2 / h1 + h1 / h2);
    sm.Aw = -h2 / h1;
    sm.As = -h1 / h2;
    sm.Ad = 0.0;
    *out = s;
    return ST_OK;
}

extern "C" st_status st_space_get(const st_space* s, int* m, int* n_x, double* coeffs) {
    if (!s) return fail(ST_ERR_ARG, "st_space_get: NULL handle");
    const SpaceMats& sm = s->sm;
    if (sm.kind != 0) return fail(ST_ERR_ARG, "st_space_get: not a structured grid (use st_space_get_mesh)");
    if (m) *m = sm.m;
    if (n_x) *n_x = sm.n_x;
    if (coeffs) {
        double c[8] = {sm.Mc, sm.Mw, sm.Ms, sm.Md, sm.Ac, sm.Aw, sm.As, sm.Ad};
        std::memcpy(coeffs, c, sizeof(c));
    }
    return ST_OK;
}

extern "C" void st_destroy_time(st_time* t) { delete t; }
extern "C" void st_destroy_space(st_space* s) { delete s; }
