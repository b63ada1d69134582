// Internal declarations of the stfdm library (host + device).
#pragma once

#include <complex>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/stfdm.h"

namespace stfdm {

using cd = std::complex<double>;

// thread-local last error detail; returns the status for `return fail(...)`
st_status fail(st_status s, const std::string& msg);

// Reduced temporal matrices (t_0 DOF removed) in band form: row l holds entries
// (l, l + d) for d = -2..2 at band[l * 5 + d + 2].
struct TimeMats {
    int p = 1;
    int N = 0;                  // elements
    int n_t = 0;                // p N
    std::vector<double> nodes;  // N + 1
    std::vector<double> Mb, Bb; // n_t x 5 bands of the reduced M_t, B_t
    std::vector<double> Mfull0; // full mass matrix rows 1..n_t, column 0 (coupling to t_0)
    std::vector<double> m;      // m_t[k] = int phi_k
    std::vector<double> times;  // DOF times t_1..
};

// Spatial matrices on a general simplicial mesh: CSR over the interior DOFs (sorted columns, the
// union pattern of M_x and A_x) and the interior DOFs' coordinates.
struct MeshSpace {
    int dim = 0, p = 0, n_x = 0;
    std::vector<int> rowptr, col;
    std::vector<double> Mv, Av;
    std::vector<double> xyz;   // n_x * dim
};

struct SpaceMats {
    int kind = 0;      // 0 = structured grid of squares (stencils below), 1 = general mesh (CSR)
    int n = 0;         // squares per direction
    int m = 0;         // interior nodes per direction
    int n_x = 0;       // m^2 (structured) or the mesh's interior DOFs
    double Lx = 1, Ly = 1;
    // 7-point stencil coefficients
    double Mc = 0, Mw = 0, Ms = 0, Md = 0;  // centre, W/E, S/N, SW/NE
    double Ac = 0, Aw = 0, As = 0, Ad = 0;
    MeshSpace mesh;    // kind 1
    // kind 1, in a solver handle: the device copy of the CSR (set up by st_fdm_setup)
    const int* d_rowptr = nullptr;
    const int* d_col = nullptr;
    const double* d_M = nullptr;
    const double* d_A = nullptr;
};

st_status assemble_mesh(int dim, int p, int nv, const double* coords, int nc, const int* cells, MeshSpace& out);
void structured_as_mesh(const SpaceMats& sm, MeshSpace& out);

// Multifrontal plan of the spatial matrices' sparsity (nested dissection by coordinate bisection,
// assembly tree of fronts); the same for every shift s_k.  Front p eliminates the `np` pivots
// first .. first + np - 1 (new numbering) and passes an update matrix on its `nu` update rows
// (urows, new numbering, ascending) to its parent.  Per system: the factor block of front p is
// (np + nu) x np column-major at foff; its update matrix nu x nu column-major at uoff (one chunk
// slot); its update vector at uvoff.
struct MfFront {
    int first = 0, np = 0, nu = 0;
    int parent = -1, height = 0;
    long long foff = 0, uoff = 0, uvoff = 0;
    int urows_off = 0;     // urows[urows_off .. + nu)
    int relpos_off = 0;    // relpos[relpos_off .. + nu): positions of the update rows in the parent's front
    int orig_off = 0, orig_cnt = 0;   // original entries (local row, local column, CSR index)
    int child_off = 0, child_cnt = 0; // children[child_off .. + child_cnt)
};

constexpr int MF_NCLS = 4;                      // warp-per-front size classes: f <= 32, 64, 96, 128
struct MfPlan {
    int n = 0;
    std::vector<int> perm, iperm;      // new -> old, old -> new
    std::vector<MfFront> fronts;
    std::vector<int> urows, relpos, children;
    std::vector<int> orig_r, orig_c, orig_k;
    std::vector<int> level_ptr, level_fronts;   // fronts by height (leaves first); within a level by
                                                // size class: f <= 32, <= 64, <= 96, <= 128, then the rest
    std::vector<int> level_ncls;                // per level, MF_NCLS counts: fronts of each size class
                                                // that one warp factorises and solves
    long long factor_entries = 0, update_entries = 0, uvec_entries = 0;
    int max_front = 0, max_np = 0;
    double flops_cmac = 0;             // complex multiply-adds of one factorisation
};

st_status build_mf_plan(const MeshSpace& ms, int leaf, MfPlan& out);
constexpr int MF_DEFAULT_LEAF = 16;

// host FP64 dense linear algebra (column-major n x n unless stated)
namespace la {
// Schur form A = Z T Z^H (A overwritten by T, upper triangular); returns false if not converged
bool complex_schur(int n, cd* A, cd* Z, int threads);
// eigenvectors of A from its Schur form: X = Z * V, columns normalised to unit 2-norm
void schur_eigenvectors(int n, const cd* T, const cd* Z, cd* X, int threads);
// LU with partial pivoting in place (column-major); returns false if singular
bool lu_factor(int n, cd* A, int* piv);
// solve A X = B for nrhs columns (column-major B, leading dim n) with a factorisation of lu_factor
void lu_solve(int n, const cd* LU, const int* piv, cd* B, int nrhs, int threads);
// kappa_2 of a square matrix from the extreme eigenvalues of X^H X (Lanczos) using its LU
double cond2(int n, const cd* X, const cd* LU, const int* piv);
// banded real LU with partial pivoting for the temporal B_t (dense storage, band-limited loops)
bool band_lu_real(int n, int kl, int ku, double* A, int* piv);
void band_lu_real_solve(int n, int kl, int ku, const double* LU, const int* piv, double* b);
void band_lu_real_solve_T(int n, int kl, int ku, const double* LU, const int* piv, double* b);
}  // namespace la

// result of step 1
struct TimeDecomp {
    int n = 0;
    std::vector<cd> X;   // row-major n x n, unit 2-norm columns
    std::vector<cd> s;   // eigenvalues
    std::vector<cd> Y;   // row-major, Y = X^{-1} (i B)^{-1}
    double kappa = 0;
    double min_neg_im = 0;
    // the complex Schur form behind the eigen-decomposition, (i B_t)^{-1} M_t = Z T Z^H (column-major),
    // and B_t^{-1} (column-major): the Bartels-Stewart solver's step 1
    std::vector<cd> Zs, Ts;
    std::vector<double> Binv;
};

st_status time_decompose(const TimeMats& tm, int threads, TimeDecomp& out);

}  // namespace stfdm

struct st_time {
    stfdm::TimeMats tm;
};
struct st_space {
    stfdm::SpaceMats sm;
};
