/*
 * stfdm.h -- C ABI of the GB300 space-time fast-diagonalisation solver for the
 * linear Schroedinger equation  i d_t psi - Laplace_x psi = f  on Omega x (0,T),
 * psi = 0 on the boundary of Omega, psi(., 0) = psi0  (Section 1, eq. (1)).
 *
 * Discretisation (Section 3): conforming space-time Galerkin FEM with
 * tensor-product continuous piecewise polynomials, Q^p_h = S_hx (x) S_ht,
 * giving the global system (eq. LGS)
 *
 *        K psi = f,     K = i B_t (x) M_x + M_t (x) A_x,
 *
 * with spatial mass/stiffness M_x, A_x (eq. matrix_x) and temporal mass and
 * first-derivative matrices M_t, B_t (eq. matrix_t); the temporal DOF at t_0
 * is removed (trial space = test space = Q^p_{h,0,}).  The initial condition
 * enters by the lifting psi = psi_hat + psi0 (Section 3, eq. VF_FEM), which
 * changes the right-hand side to  F~ = F - m_t (x) A_x psi0  with
 * m_t[k] = int_0^T phi_k dt.
 *
 * Solver (Section 3, fast diagonalisation choice):
 *   step 1  (i B_t)^{-1} M_t = X_t S_t X_t^{-1},  S_t = diag(s_k),  Y_t = X_t^{-1} (i B_t)^{-1}
 *   step 2  G = Y_t F~                          (dense n_t x n_t contraction)
 *   step 3  (M_x + s_k A_x) w_k = g_k, k = 1..n_t, independent (eq. LGS_x, zero sum term)
 *   step 4  Psi = X_t W  (+ psi0)
 *
 * Data layout of every space-time array: row-major (n_t, n_x), row = time DOF
 * t_1..t_{n_t} (for P2 in time: t_{1/2}, t_1, t_{3/2}, ...), column = interior
 * spatial node in lexicographic order with x1 fastest; complex numbers are
 * interleaved (re, im), i.e. the memory layout of C99 double complex /
 * torch.complex128 ("c128") or float complex / torch.complex64 ("c64").
 * Spatial vectors (psi0) have n_x entries in the same node order.
 *
 * Ownership: handles (st_time, st_space, st_fdm) are opaque and owned by the
 * library until the matching st_destroy_*.  All space-time arrays passed to
 * the solve entry points are DEVICE pointers owned by the caller; the library
 * never frees them.  Handle-internal device workspace is allocated by the
 * library (at setup, or at the first solve that needs it) and freed by
 * st_destroy_fdm.  Every device entry point is asynchronous on the given CUDA
 * stream (a cudaStream_t passed as void*, NULL = legacy default stream) except
 * where it says it synchronises; two calls on the same handle must not run
 * concurrently (they share the handle's workspace).
 *
 * Errors: no C++ exception crosses this ABI.  Every entry point returns an
 * st_status (0 = ST_OK, negative = error); st_last_error_message() gives a
 * human-readable detail of the last error of the calling thread.
 */
#ifndef STFDM_H
#define STFDM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int st_status;

#define ST_OK                    0
#define ST_ERR_ARG              -1   /* invalid argument (NULL, size, range, unsupported combination) */
#define ST_ERR_OOM              -2   /* host or device allocation failed */
#define ST_ERR_CUDA             -3   /* a CUDA runtime call or kernel launch failed */
#define ST_ERR_ILL_CONDITIONED  -4   /* kappa_2(X_t) > kappa_max, or some Im s_k clearly > 0 */
#define ST_ERR_ZERO_PIVOT       -5   /* a pivot of an LDL^T factorisation was zero or not finite */
#define ST_ERR_NOT_CONVERGED    -6   /* eigen-iteration or refinement did not reach its tolerance */
#define ST_ERR_TIMEOUT          -7   /* a bounded device-side wait expired */
#define ST_ERR_UNSUPPORTED      -8   /* not built for this device / configuration */

/* precision modes of a solve */
#define ST_FP64   0   /* c128 in/out, every step in FP64 */
#define ST_FP32   1   /* c64 in/out, every step in FP32 (complex64); error stated, not refined */
#define ST_MIXED  2   /* c128 in/out: complex-FP32 FDM sweeps refined on an FP64 Kronecker residual */

/* time transform selectors for st_time_transform (step 2 / step 4 / adjoint) */
#define ST_XFORM_Y    0   /* out = Y_t in        (forward transform, step 2) */
#define ST_XFORM_X    1   /* out = X_t in        (back transform, step 4)    */
#define ST_XFORM_XT   2   /* out = X_t^T in      (adjoint, first transform)  */
#define ST_XFORM_YT   3   /* out = Y_t^T in      (adjoint, last transform)   */

typedef struct st_time st_time;
typedef struct st_space st_space;
typedef struct st_fdm st_fdm;

/* spatial solvers of step 3 (st_setup_opts.spatial_solver) */
#define ST_SPATIAL_AUTO          0   /* banded for structured grids, multifrontal for meshes */
#define ST_SPATIAL_BANDED        1   /* pivot-free banded LDL^T (structured grids only) */
#define ST_SPATIAL_MULTIFRONTAL  2   /* pivot-free sparse-direct multifrontal LDL^T, nested dissection */

typedef struct {
    double kappa_max;   /* reject X_t with kappa_2 above this; <= 0 selects 1e10 (Section 3: X_t must be regular) */
    int device;         /* CUDA device ordinal for the handle's device data; < 0 = the current device */
    int host_threads;   /* threads for the host FP64 setup; <= 0 = hardware concurrency */
    int spatial_solver; /* ST_SPATIAL_*; 0 = automatic */
} st_setup_opts;

typedef struct {
    int precision;      /* ST_FP64, ST_FP32 or ST_MIXED */
    double tol;         /* ST_MIXED: stop when ||F~ - K psi_hat||_2 / ||F~||_2 <= tol; <= 0 selects 1e-12 */
    int max_sweeps;     /* ST_MIXED: at most this many FDM32 applications; <= 0 selects 40 */
    int keep_factors;   /* ST_MIXED: 1 = store all n_t LDL^T factors and reuse them in later sweeps
                           when they fit the memory budget, 0 = refactor every sweep, -1 = automatic */
    int fixed_sweeps;   /* ST_MIXED: > 0 runs exactly this many classical refinement sweeps with no
                           host synchronisation (no convergence test; the final residual is reported
                           when info is non-NULL) */
    int method;         /* ST_MIXED: ST_REFINE_GMRES (default) or ST_REFINE_CLASSIC */
    double err_tol;     /* ST_MIXED with GMRES: > 0 also requires the error estimate ||FDM32(R)|| / ||psi_hat||
                           (one extra FP32 application each time the residual target is met) to be
                           <= err_tol; while it is not, the residual target is lowered and the
                           iteration continues.  A small residual does not bound the error by itself:
                           the error can reach cond(K) times the residual.  <= 0: off */
} st_solve_opts;

/* refinement methods of ST_MIXED.  Both compute the residual in FP64 and correct with the
 * complex-FP32 FDM.  CLASSIC: psi += FDM32(R) each sweep.  GMRES: flexible GMRES in FP64,
 * right-preconditioned by FDM32 (restarted); a few eigen-indices whose shifted spatial matrix
 * is nearly singular in FP32 slow the classical sweeps down, GMRES removes them in a few
 * extra iterations.  max_sweeps counts FDM32 applications in both. */
#define ST_REFINE_GMRES   0
#define ST_REFINE_CLASSIC 1

typedef struct {
    int sweeps;                  /* FDM sweeps run (1 for ST_FP64 / ST_FP32) */
    int factors_kept;            /* 1 if the LDL^T factors were reused across sweeps, 2 if only
                                    those of the leading systems that fit in memory (GMRES) */
    double rel_residual;         /* final ||F~ - K psi_hat|| / ||F~|| (computed for ST_MIXED; -1 otherwise) */
    double residual_history[16]; /* rel. residual before each sweep (ST_MIXED), then the final one */
    double kappa_x;              /* kappa_2(X_t) */
    double min_neg_im_shift;     /* min_k (-Im s_k); >= 0 up to rounding */
    double setup_seconds;        /* host time of st_fdm_setup's FP64 decomposition */
    int tensor_cores;            /* 1 if the complex-FP32 time transforms ran on the tcgen05 tensor cores */
    int kernel_launches;         /* kernels this call launched (st_fdm_solve, st_adjoint_solve; 0 in batched solves) */
    int restart;                 /* ST_MIXED with GMRES: the restart length m used (0 otherwise) */
    double rel_error_estimate;   /* ST_MIXED with GMRES and err_tol > 0: the last ||FDM32(R)|| / ||psi_hat|| (-1 otherwise) */
    int kept_systems;            /* ST_MIXED: spatial systems whose factors stayed in memory across
                                    applications (n_t when all were kept, 0 when none) */
    int reorth_steps;            /* ST_MIXED with GMRES: Arnoldi steps whose Gram-Schmidt pass was
                                    repeated (the first removed more than half of the new vector's
                                    norm squared); 0 in batched solves, which always run two passes */
} st_solve_info;

/* ------------------------------------------------------------------ status */
const char* st_status_string(st_status s);
const char* st_last_error_message(void);
int st_abi_version(void);   /* returns STFDM_ABI_VERSION of the built library */
#define STFDM_ABI_VERSION 8

/* ------------------------------------------------------------------ assembly (host) */
/* Temporal matrices of eq. (matrix_t), Section 3.  p_t in {1, 2}: continuous piecewise
 * linear / quadratic Lagrange elements on 0 = t_0 < t_1 < ... < t_{N_t} = T (t_nodes has
 * N_t + 1 strictly increasing host doubles, t_nodes[0] = 0).  Builds the reduced (t_0 DOF
 * removed) banded M_t, B_t (half bandwidth p_t), n_t = p_t N_t, and m_t.  *out is owned by
 * the library.  Errors: ST_ERR_ARG (bad p_t, N_t < 1, nodes not increasing / t0 != 0). */
st_status st_assemble_time(int p_t, int N_t, const double* t_nodes, st_time** out);
/* Dense copies for inspection (host, row-major n_t x n_t; any pointer may be NULL). */
st_status st_time_get(const st_time* t, int* n_t, double* M_t, double* B_t, double* m_t, double* dof_times);

/* Spatial matrices of eq. (matrix_x): P1 on (0,Lx) x (0,Ly) split into n_squares^2 rectangles,
 * each cut along its SW-NE diagonal; interior (Dirichlet) DOFs only, n_x = (n_squares-1)^2,
 * lexicographic x1 fastest, half bandwidth b = n_squares.  The matrices are 7-point stencils:
 * M_x: centre h1 h2/2, W/E/S/N/SW/NE h1 h2/12;  A_x: centre 2(h2/h1 + h1/h2), W/E -h2/h1,
 * S/N -h1/h2, SW/NE 0.  Errors: ST_ERR_ARG (n_squares < 2, non-positive lengths). */
st_status st_assemble_space(int n_squares, double Lx, double Ly, st_space** out);
/* coeffs[8] = {Mc, Mw(=Me), Ms(=Mn), Mdiag(SW/NE), Ac, Aw, As, Adiag}; m = n_squares - 1. */
st_status st_space_get(const st_space* s, int* m, int* n_x, double* coeffs);

/* Spatial matrices of eq. (matrix_x) on a general conforming simplicial mesh (the spaces S^p_hx of
 * Section 2 for d = 2, 3): Lagrange P1 or P2 (p_x), triangles (dim = 2) or tetrahedra (dim = 3).
 * coords: host doubles (n_vertices, dim) row-major; cells: host ints (n_cells, dim + 1), vertex
 * indices (any orientation).  DOFs: the vertices in input order, then for P2 one per edge, the
 * edges ordered by their (smaller vertex, larger vertex) pair; DOFs on a boundary facet (a facet of
 * exactly one cell) are removed (Dirichlet), the interior DOFs keep this order (it is the order of
 * every spatial index of the solver's arrays).  The integrals are exact (barycentric monomials).
 * The handle works with every entry point except the structured-grid helpers (st_space_get,
 * st_error_norms, st_load_quadrature, st_residual_noalloc) and batched plans; its spatial systems
 * are solved by the multifrontal solver.  Errors: ST_ERR_ARG (dim, p_x, index out of range, a
 * degenerate cell, a facet shared by more than two cells, no interior DOF), ST_ERR_OOM. */
st_status st_assemble_mesh(int dim, int p_x, int n_vertices, const double* coords, int n_cells, const int* cells,
                           st_space** out);
/* The spatial matrices in CSR over the interior DOFs (one pattern for M_x and A_x, sorted columns;
 * for a structured grid its 7-point stencils): rowptr[n_x + 1], col[nnz], M[nnz], A[nnz], and the
 * interior DOFs' coordinates xyz[n_x * dim]; any output may be NULL (query sizes first). */
st_status st_space_get_mesh(const st_space* s, int* dim, int* p_x, int* n_x, long long* nnz, int* rowptr, int* col,
                            double* M, double* A, double* xyz);
/* The sparse-direct solver's plan for a space (host only): nested dissection by coordinate bisection
 * with leaves of at most `leaf` DOFs (<= 0: 16, the solver's own choice) and its multifrontal assembly tree.  Outputs (any may
 * be NULL): fronts, launch levels, the largest front, factor entries per system, real flops of one
 * factorisation (8 per complex multiply-add), perm[n_x] (elimination position -> DOF), per front
 * its first pivot position, pivot count and update-row count, and the update rows of all fronts
 * concatenated (elimination positions, ascending per front). */
st_status st_space_mf_plan(const st_space* s, int leaf, int* n_fronts, int* n_levels, int* max_front,
                           long long* factor_entries, double* flops, int* perm, int* front_first, int* front_np,
                           int* front_nu, int* urows);

/* Step 1 on the host, no device needed (Section 3, fast diagonalisation): X_t (unit 2-norm
 * columns), s (eigenvalues), Y_t = X_t^{-1} (i B_t)^{-1}, kappa_2(X_t).  X, Y: host
 * complex128 row-major n_t x n_t; s: host complex128 n_t; any output may be NULL.
 * Errors: ST_ERR_NOT_CONVERGED (QR iteration), ST_ERR_ARG. */
st_status st_time_decompose(const st_time* t, int host_threads, double* X, double* s, double* Y,
                            double* kappa2);

/* ------------------------------------------------------------------ setup */
/* Builds the solver handle: step 1 in FP64 on the host (timed separately), then uploads
 * X_t, Y_t, X_t^T, Y_t^T, s_k, Y_t m_t (FP64 and FP32 copies) and the band coefficients to the
 * device.  Errors: ST_ERR_ILL_CONDITIONED (kappa_2 > kappa_max, or some Im s_k > 1e-8 max|s|:
 * in exact arithmetic Im s_k < 0, which keeps every C_k = M_x + s_k A_x pivot-free; shifts with
 * |Im s_k| at rounding level are accepted and zero pivots are reported by the solves),
 * ST_ERR_CUDA, ST_ERR_OOM. */
st_status st_fdm_setup(const st_time* t, const st_space* s, const st_setup_opts* opts, st_fdm** out);
st_status st_fdm_get(const st_fdm* h, int* n_t, int* n_x, int* m, double* kappa2, double* min_neg_im_shift);

/* ------------------------------------------------------------------ solves (device) */
/* The full solve, steps 2-4 (+ lifting, + refinement for ST_MIXED).
 * F: device (n_t, n_x) load vector (c128 for ST_FP64/ST_MIXED, c64 for ST_FP32).
 * psi0: device n_x initial values at the interior nodes (same complex type) or NULL (= 0).
 * psi: device (n_t, n_x) output, the nodal values of psi_h at t_1..t_{n_t}; must not alias F.
 * info: may be NULL.  ST_MIXED (unless fixed_sweeps > 0) synchronises the stream once per
 * sweep to read the residual norm.  Errors: ST_ERR_ARG, ST_ERR_CUDA, ST_ERR_OOM,
 * ST_ERR_ZERO_PIVOT, ST_ERR_NOT_CONVERGED (info is still filled). */
st_status st_fdm_solve(st_fdm* h, const void* F, const void* psi0, void* psi,
                       const st_solve_opts* opts, st_solve_info* info, void* stream);

/* Bartels-Stewart solve in FP64 (Section 3, step 1 with the Schur choice, eq. LGS_x): with
 * (i B_t)^{-1} M_t = Z T Z^H (Z unitary, T upper triangular), Psi_hat = Z W and G = Z^H (i B_t)^{-1} F~,
 *     (M_x + T_ll A_x) w_l = g_l - A_x sum_{k>l} T_lk w_k,   l = n_t - 1, ..., 0.
 * The n_t spatial matrices are factorised together (the FDM's spatial solver, factors kept), then the
 * coupled solves run one after another.  Z is perfectly conditioned, so the result does not carry the
 * rounding of kappa_2(X_t); the solves are sequential in l.  The Schur transforms are set up on the
 * first call (host FP64, O(n_t^3)).  F, psi0 (may be NULL), psi: device c128 as in st_fdm_solve; psi
 * must not alias F.  Needs memory for all n_t FP64 factors.  Errors: ST_ERR_ARG, ST_ERR_OOM,
 * ST_ERR_CUDA, ST_ERR_ZERO_PIVOT (when info is non-NULL; the call then synchronises). */
st_status st_bs_solve(st_fdm* h, const void* F, const void* psi0, void* psi, st_solve_info* info, void* stream);

/* FP64 Kronecker residual R = F~ - K (psi - 1 (x) psi0) with F~ = F - m_t (x) A_x psi0
 * (eq. LGS; c128 arrays, psi0 may be NULL).  R may be NULL (norm only); it may alias F but not psi
 * or psi0 (ST_ERR_ARG).  rel_norm (host, may be
 * NULL) receives ||R||_2 / ||F~||_2; when it is non-NULL the call synchronises the stream. */
st_status st_residual(st_fdm* h, const void* F, const void* psi0, const void* psi, void* R,
                      double* rel_norm, void* stream);

/* Adjoint solve K^H lambda = G with the same FDM machinery:
 * K^{-H} = conj o (Y_t^T (x) I) blockdiag(C_k^{-1}) (X_t^T (x) I) o conj, C_k = M_x + s_k A_x
 * (complex symmetric, so C_k^{-T} = C_k^{-1} reuses the forward factors).
 * G, lambda: device (n_t, n_x), c128 for ST_FP64/ST_MIXED (ST_MIXED refines on the FP64 adjoint
 * residual), c64 for ST_FP32. */
st_status st_adjoint_solve(st_fdm* h, const void* G, void* lambda, const st_solve_opts* opts,
                           st_solve_info* info, void* stream);

/* Gradient of a loss J(psi) with respect to psi0 from grad_psi = dJ/dpsi-bar (PyTorch's complex
 * convention) and grad_F = K^{-H} grad_psi:  grad_psi0 = sum_l grad_psi[l,:] - A_x (m_t^T grad_F).
 * c128 device arrays; grad_psi0 has n_x entries. */
st_status st_adjoint_lift(st_fdm* h, const void* grad_psi, const void* grad_F, void* grad_psi0,
                          void* stream);

/* Many independent problems of uneven size in one call.  ST_MIXED with GMRES refinement runs as
 * one batched plan (st_batch_create + st_batch_solve below, created and destroyed inside the
 * call); ST_FP64, ST_FP32 and the classic / fixed-sweep refinements solve the problems one after
 * another with st_fdm_solve.  Arrays of `count` handles and device pointers as in st_fdm_solve
 * (psi0 may be NULL, or hold NULL entries); infos may be NULL or hold `count` entries. */
st_status st_fdm_solve_batched(st_fdm* const* hs, int count, const void* const* F,
                               const void* const* psi0, void* const* psi,
                               const st_solve_opts* opts, st_solve_info* infos, void* stream);

/* ------------------------------------------------------------------ batched plans */
/* A plan solves `count` independent problems (handles from st_fdm_setup, all on one device, of
 * any mixture of spatial meshes, n_t and temporal degree) in the mixed precision of st_fdm_solve:
 * per problem FP64 flexible GMRES on K psi_hat = F~ (eq. LGS), right-preconditioned by its
 * complex-FP32 fast-diagonalisation solve (Section 3, steps 2-4).  The problems advance together:
 *   - every phase is one grouped launch over all problems (packed vectors, block tables); the
 *     spatial solves of all (problem, k) pairs are one persistent launch over a cost-sorted work
 *     list, each CTA factorising (banded LDL^T) and solving one system at a time;
 *   - a restart cycle needs no host decision, so it is captured once in a CUDA graph and replayed;
 *   - an autotuner times the candidate transform tile shapes and CTAs per SM of the spatial solve
 *     on the plan's data at creation and keeps the fastest (cached per shape signature).
 * The plan owns its workspace: the GMRES basis ((m+1) complex128 + m complex64 vectors of the
 * packed length), one factor slot per resident CTA, the transform buffer, and -- unless
 * opts->no_keep -- kept LDL^T factors for the problems with the widest bands (b <= 256) that fit in
 * the free memory left at creation: their later applications only run the substitutions.  Solves on one plan must not overlap; the handles must outlive the plan.
 * The paper solves one problem at a time; batching is an extension. */
typedef struct st_batch st_batch;

typedef struct {
    double tol;        /* relative residual target per problem, default 1e-12 */
    int max_sweeps;    /* FP32 preconditioner applications per problem, default 40 */
    int restart;       /* GMRES restart length m, 0 = automatic (<= 20, basis within half the free memory) */
    int no_graph;      /* 1: launch each cycle directly instead of replaying a captured CUDA graph */
    int no_tune;       /* 1: skip the autotuner (square 64 x 64 transform tiles, maximum CTAs per SM) */
    int no_keep;       /* 1: refactorise every spatial system at every preconditioner application */
} st_batch_opts;

typedef struct {
    int count;                 /* problems */
    int items;                 /* spatial systems (sum of n_t) */
    int restart;               /* GMRES restart length */
    int xform_tile_m, xform_tile_n;   /* transform tile (time rows x spatial columns) */
    int solve_ctas_per_sm;     /* CTAs per SM of the persistent factor-and-solve */
    int solve_grid;            /* its grid */
    int graph_nodes;           /* nodes of the captured cycle graph (0 before the first solve) */
    int cycles;                /* restart cycles run by the last solve */
    int tuned;                 /* 0: defaults, 1: tuned at creation, 2: taken from the tuning cache */
    double tune_seconds;       /* time spent tuning */
    long long unknowns;        /* total space-time unknowns */
    unsigned long long workspace_bytes;
    int kept_problems;         /* problems whose LDL^T factors are kept across applications */
    unsigned long long kept_factor_bytes;
} st_batch_stats;

/* Builds the plan and, unless opts->no_tune, runs the autotuner on the device (synchronous).
 * opts may be NULL.  Errors: ST_ERR_ARG (no/NULL handles, different devices, negative option),
 * ST_ERR_OOM, ST_ERR_UNSUPPORTED (spatial band too wide for shared memory), ST_ERR_CUDA. */
st_status st_batch_create(st_fdm* const* hs, int count, const st_batch_opts* opts, st_batch** out);

/* Solves all problems: F[p] (n_t, n_x) c128 right-hand side, psi0[p] n_x c128 initial value (the
 * array or an entry may be NULL = 0), psi[p] (n_t, n_x) c128 output; all device pointers owned by
 * the caller, psi[p] must not alias F[p].  Work runs on the plan's own stream, ordered after the
 * caller's `stream` and before anything later enqueued on it; the call returns when done (it reads
 * one counter per restart cycle).  infos (NULL or `count` entries) is filled for every problem,
 * also on ST_ERR_NOT_CONVERGED (the first problem that missed the tolerance is named in
 * st_last_error_message).  ST_ERR_ZERO_PIVOT if a spatial factorisation met a zero pivot. */
st_status st_batch_solve(st_batch* b, const void* const* F, const void* const* psi0, void* const* psi,
                         st_solve_info* infos, void* stream);
/* Step 3 alone for the whole batch: W[k,:] = (M_x + s_k A_x)^{-1} G[k,:] for every k of every
 * problem in one persistent launch, in place on the plan's complex64 transform buffer, on `stream`
 * (asynchronous; the pivot flag is reported by the next st_batch_solve).  st_batch_spatial_get
 * copies problem p's (n_t, n_x) c64 slice of that buffer to (to_plan = 0) or from (to_plan = 1) the
 * device array G.  Used by the tests and to time the kernel; not needed for st_batch_solve. */
st_status st_batch_spatial_solve(st_batch* b, void* stream);
st_status st_batch_spatial_get(const st_batch* b, int p, void* G, int to_plan, void* stream);
st_status st_batch_stats_get(const st_batch* b, st_batch_stats* out);
void st_destroy_batch(st_batch* b);

/* ------------------------------------------------------------------ single steps (device) */
/* Step 2 / step 4 / adjoint transforms: out = T in with T selected by `which` (ST_XFORM_*),
 * in/out (n_t, n_x) device arrays, c128 (precision ST_FP64) or c64 (ST_FP32; ST_MIXED = the
 * 3xTF32 tensor-core path on c64 data).  Must not alias. */
st_status st_time_transform(st_fdm* h, int which, int precision, const void* in, void* out, void* stream);

/* Step 3: W[k,:] = (M_x + s_k A_x)^{-1} G[k,:] for all k by pivot-free banded LDL^T
 * (complex symmetric, no conjugation), factor and solve in one launch.  G, W: (n_t, n_x)
 * device arrays (c128 for ST_FP64, c64 for ST_FP32/ST_MIXED); W may alias G. */
st_status st_spatial_solve(st_fdm* h, int precision, const void* G, void* W, void* stream);

/* Step 3 split in two, for timing and for callers that reuse the factors: st_spatial_factor
 * factorises all n_t matrices C_k = M_x + s_k A_x and keeps the factors in the handle (banded or
 * multifrontal, FP64 or FP32; ST_ERR_OOM when they do not fit); st_spatial_substitute then solves
 * W[k,:] = C_k^{-1} G[k,:] for all k with them (forward and backward substitutions only).  G, W as in
 * st_spatial_solve (W may alias G).  A later solve of another precision or mode may drop the kept
 * factors; st_spatial_substitute then fails with ST_ERR_ARG.  Both synchronise the stream (status). */
st_status st_spatial_factor(st_fdm* h, int precision, void* stream);
st_status st_spatial_substitute(st_fdm* h, int precision, const void* G, void* W, void* stream);

/* Interpolated load F = (M_t,full (x) M_x) f_nodal (rows t_1.. of the full temporal mass
 * matrix applied to nodal values f at all DOF times t_0, t_1, ...): f_nodal (n_t + 1, n_x) c128,
 * F (n_t, n_x) c128 (device).  Assembly helper, not part of the solve. */
st_status st_load_nodal(st_fdm* h, const void* f_nodal, void* F, void* stream);

/* ------------------------------------------------------------------ manufactured solutions */
/* Exact solutions for error measurement (Section 4): */
#define ST_EXACT_C1 0     /* psi = sin(pi x1) sin(pi x2) (1 + t) e^{-it} */
#define ST_EXACT_PAPER 1  /* psi = e^{it} sin(pi x1) sin(pi x2) sin(t x1 x2), the paper's example */

/* Space-time errors of a discrete solution (Section 4): out[0] = ||psi - psi_h||_{L2(Q)},
 * out[1] = |psi - psi_h|_{H1(Q)} = (||d_t e||^2 + ||grad_x e||^2)^{1/2}, psi_h the trial-space
 * function with nodal values psi0 at t_0 (device n_x c128, NULL = 0) and psi at t_1.. (device
 * (n_t, n_x) c128).  Tensor quadrature per prism: q_t Gauss-Legendre points in time, q_x x q_x
 * collapsed Gauss points per triangle (0 = 4; at most 8).  out: host double[2]; synchronous on
 * `stream`.  ST_ERR_UNSUPPORTED for more than 65535 time elements. */
st_status st_error_norms(st_fdm* h, int exact, const void* psi, const void* psi0, int q_t, int q_x,
                         double* out, void* stream);

/* Load vector of the manufactured right-hand side f = i d_t psi - Laplace psi by quadrature:
 * F[k, a] = int_Q f phi_k varphi_a for the time DOFs t_1.. and interior nodes (eq. LGS right-hand
 * side before the lifting), F device (n_t, n_x) c128, rules as in st_error_norms.  Asynchronous.
 * Assembly helper (the paper integrates f with a high-order rule). */
st_status st_load_quadrature(st_fdm* h, int exact, int q_t, int q_x, void* F, void* stream);

/* ------------------------------------------------------------------ allocation-free residual */
/* The FP64 residual of st_residual, for callers that must not allocate device memory while
 * they run: frameworks that own all device memory through their own pool, and loops that cannot
 * take cudaMalloc's implicit device synchronisation.  It has no counterpart in the
 * paper; it computes the same R = F~ - K (psi - 1 (x) psi0) as st_residual.
 * F, psi: device (n_t, n_x) c128; psi0: device n_x c128 or NULL; R: device (n_t, n_x) c128 output
 * or NULL (it may alias F but not psi or psi0: ST_ERR_ARG); norms: device double[2] output receiving ||R||_2^2 and ||F~||_2^2 (the caller divides;
 * nothing is copied to the host and the call never synchronises).
 * It calls no allocating routine: its only scratch is a fixed 1 MiB array of per-block partial
 * sums inside the library, resident on every device that loads it until the process exits.  The
 * limit is ceil(n_x/256) * ceil(n_t/16) <= 65536 (e.g. n_x = 65,025 with n_t <= 4096);
 * larger problems get ST_ERR_ARG.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress, which may load the module).  All calls share the array: calls that overlap on the GPU (other streams or
 * host threads) race and must be serialised by the caller. */
st_status st_residual_noalloc(const st_fdm* h, const void* F, const void* psi0, const void* psi, void* R,
                              double* norms, void* stream);

/* ------------------------------------------------------------------ failure detection */
/* Test hook for the bounded device-side waits (no counterpart in the paper).  Every asynchronous
 * pipeline in the library waits on shared-memory mbarriers with a time limit, after which the CTA
 * records an error, lets the copies it has in flight land and returns, and the entry point reports
 * ST_ERR_TIMEOUT instead of hanging.  With seconds > 0, every later substitution launch of the
 * handle (the backward substitution of st_spatial_solve, the substitutions of the solves) makes its
 * copy-issuing thread first wait, for at most `seconds`, on an mbarrier that receives neither a
 * copy nor an arrival: the wait runs out before any copy is issued, the kernel takes its timeout
 * exit and the entry point returns ST_ERR_TIMEOUT.  seconds = 0 (the default) turns the probe off;
 * the handle stays usable.  Errors: ST_ERR_ARG (NULL handle, seconds outside [0, 1]). */
st_status st_set_wait_probe(st_fdm* h, double seconds);

/* ------------------------------------------------------------------ teardown */
void st_destroy_time(st_time* t);
void st_destroy_space(st_space* s);
void st_destroy_fdm(st_fdm* h);

#ifdef __cplusplus
}
#endif
#endif /* STFDM_H */
