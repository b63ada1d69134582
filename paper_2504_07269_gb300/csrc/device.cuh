// Device-side shared declarations: complex helpers, the solver handle, kernel launchers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "internal.h"

namespace stfdm {

// kernel launches issued by the calling host thread (counted by every launcher; a solve reports
// the difference in st_solve_info::kernel_launches)
void note_launches(int n);
long long launches_issued();

// ------------------------------------------------------------------ complex helpers
template <typename T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };
template <typename T> using C = typename cplx<T>::type;

template <typename T> __host__ __device__ __forceinline__ C<T> mk(T x, T y) { return C<T>{x, y}; }
template <typename T> __host__ __device__ __forceinline__ C<T> cadd(C<T> a, C<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __host__ __device__ __forceinline__ C<T> csub(C<T> a, C<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __host__ __device__ __forceinline__ C<T> cmul(C<T> a, C<T> b) {
    return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __host__ __device__ __forceinline__ C<T> cscale(C<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// acc -= a * b
template <typename T> __device__ __forceinline__ void cfms(C<T>& acc, C<T> a, C<T> b) {
    acc.x = fma(-a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}
// acc += a * b
template <typename T> __device__ __forceinline__ void cfma(C<T>& acc, C<T> a, C<T> b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
template <typename T> __host__ __device__ __forceinline__ C<T> cinv(C<T> a) {
    T d = a.x * a.x + a.y * a.y;
    return mk<T>(a.x / d, -a.y / d);
}
template <typename To, typename Ti> __host__ __device__ __forceinline__ C<To> ccast(C<Ti> a) {
    return mk<To>((To)a.x, (To)a.y);
}

// ------------------------------------------------------------------ handle
struct DevTime {
    double* Mb = nullptr;     // n_t x 5 band of M_t
    double* Bb = nullptr;     // n_t x 5 band of B_t
    double* BTb = nullptr;    // n_t x 5 band of B_t^T
    double* Mfull0 = nullptr; // full M_t rows 1..n_t, column t_0
    double* m = nullptr;      // m_t
    double* nodes = nullptr;  // time mesh nodes t_0 .. t_N
};

// which transform matrix
enum XformSel { XF_Y = 0, XF_X = 1, XF_XT = 2, XF_YT = 3 };


template <typename TA, typename TB, typename TC>
struct XformArgs {
    int M, N, K;
    const C<TA>* A;      // row-major M x K
    int lda;
    const C<TB>* B;      // row-major K x N
    long long ldb;
    C<TC>* Cm;           // row-major M x N
    long long ldc;
    int conj_b, conj_out, accumulate;
    const double* b_scale;    // device scalar multiplying B, or NULL
    const double* out_scale;  // device scalar for accumulate, or NULL
    const C<TC>* add_row;     // N-vector added to every output row, or NULL
    const double2* r1_u;      // rank-one term subtracted: r1_u[i] r1_v[j], or NULL
    const double2* r1_v;
};
template <typename TA, typename TB, typename TC, typename TACC>
cudaError_t xform_simt_launch(const XformArgs<TA, TB, TC>& a, cudaStream_t st);

template <typename T>
struct BandArgs {
    int n;          // n_x
    int m;          // interior nodes per grid row
    int b;          // half bandwidth m + 1
    int n_sys;      // number of systems in this launch
    int k0;         // index of the first system
    T Mc, Mw, Ms, Md, Ac, Aw, As, Ad;   // stencil coefficients of M_x and A_x
    const C<T>* shifts;   // s_k
    C<T>* rhs;            // (n_sys, n): g_k in, w_k out
    C<T>* win;            // gridDim.x windows of (b + NB) x (b + 1)
    C<T>* L;              // factor columns: L[j*b + o - 1] = L(j + o, j), o = 1..b
    C<T>* D;              // pivots
    int keep;             // 1: factors stored per system k, 0: per system of this launch (slot k - k0)
    int* status;          // status[0] set to 1 on a zero / non-finite pivot
    unsigned long long probe_ns = 0;   // > 0: substitution producers first wait this long on a barrier
                                       // that nothing completes (test of the bounded waits)
};
// panel width code: the panel width (32/16/8), negative for the unstaged complex64 kernel, 0 = too wide
template <typename T> int band_pick_nb(int b, size_t smem_optin);
template <typename T> size_t band_smem_for(int nb, int b);
template <typename T> int band_occupancy(int nb, int b);
template <typename T> cudaError_t band_factor_solve_launch(const BandArgs<T>& a, int nb, int grid, cudaStream_t st);
template <> int band_pick_nb<float>(int b, size_t smem_optin);
template <> int band_pick_nb<double>(int b, size_t smem_optin);
template <> size_t band_smem_for<float>(int nb, int b);
template <> size_t band_smem_for<double>(int nb, int b);
template <> int band_occupancy<float>(int nb, int b);
template <> int band_occupancy<double>(int nb, int b);
template <> cudaError_t band_factor_solve_launch<float>(const BandArgs<float>& a, int nb, int grid, cudaStream_t st);
template <> cudaError_t band_factor_solve_launch<double>(const BandArgs<double>& a, int nb, int grid, cudaStream_t st);
template <typename T> cudaError_t subst_launch(const BandArgs<T>& a, int k0, int nsys, bool fwd, cudaStream_t st);

// grouped factor-and-solve over the systems of a batch of problems (complex64)
struct BatchBand {
    int n, m, b, pad;
    float Mc, Mw, Ms, Md, Ac, Aw, As, Ad;
    const float2* shifts;   // s_k of the problem
    float2* rhs;            // its (n_t, n) right-hand sides in, solutions out
    float2* Lkeep;          // kept factors (n_t systems of n b entries) or NULL: refactorised per use
    float2* Dkeep;          // kept pivots (n_t x n)
};
size_t band_batch_smem(int b_max);
cudaError_t band_batch_prepare(int b_max);
int band_batch_occupancy(int b_max);
cudaError_t band_batch_launch(const BatchBand* probs, const int2* items, int n_items, const int* active,
                              const int* factored, int* counter, int b_max, float2* win, float2* Lslots, size_t L_stride,
                              float2* Dslots, size_t D_stride, int* status, int grid, cudaStream_t st);
cudaError_t subst_batch_launch(const BatchBand* probs, const int2* items, int n_items, const int* active,
                               const int* factored, int b_max, int* status, bool fwd, cudaStream_t st);

// batched solve: per-problem descriptor and per-problem GMRES state (device arrays)
struct BatchProb {
    int n_t, n_x, m, tband;   // tband: nonzero temporal band diagonals (3 for P1 time, 5 for P2)
    double Mc, Mw, Ms, Md, Ac, Aw, As, Ad;
    const double* Mb;       // n_t x 5 band of M_t
    const double* Bb;       // n_t x 5 band of B_t
    const double* m_t;
    const float2* Y32;      // Y_t (row-major n_t x n_t, complex64)
    const float2* X32;      // X_t
    const double2* F;       // right-hand side (caller's array)
    double2* x;             // iterate = the caller's output array
    const double2* apsi0;   // A_x psi0 or NULL
    long long off;          // offset of the problem in packed space-time vectors
    double psc;             // power-of-two scale of the preconditioner input
};

struct BatchGm {
    double* rr;       // [P] ||r||^2 of the last residual
    double* ff;       // [P] ||F~||^2
    double* bnorm;    // [P] ||F~|| (negative before the first cycle)
    double* rel;      // [P] last relative residual
    double* hist;     // [P][16]
    int* nh;          // [P]
    int* its;         // [P] preconditioner applications so far
    int* stopped;     // [P] 1: converged, 2: out of iterations, 3: non-finite residual
    int* active;      // [P] iterating in the current cycle
    int* jdone;       // [P] Arnoldi steps of the current cycle
    double* inv;      // [P] scale for the next basis vector
    double2* H;       // [P][(m + 1) m] rotated Hessenberg matrix, row-major
    double2* g;       // [P][m + 1]
    double2* sn;      // [P][m]
    double* cs;       // [P][m]
    double2* h;       // [P][3][KB_MAXV] Gram-Schmidt coefficients (pass 1, pass 2, norm)
    double2* y;       // [P][m]
    int* pending;     // [1] problems not stopped at the start of the cycle
};

// multifrontal spatial solver (general meshes): device copy of a plan front
struct MfFrontDev {
    int first, np, nu, parent;
    long long foff, uoff, uvoff;
    int urows_off, relpos_off, orig_off, orig_cnt, child_off, child_cnt;
};

template <typename T>
struct MfArgs {
    const MfFrontDev* fronts;
    const int* level_fronts;
    int lvl_off;
    const int* urows;
    const int* relpos;
    const int* children;
    const int* orig_r;
    const int* orig_c;
    const int* orig_k;
    const int* perm;       // new -> old node
    const double* Mv;      // CSR values of M_x and A_x
    const double* Av;
    const C<T>* shifts;    // s_k
    int k0;                // first system of the launch
    C<T>* fac;             // factor blocks; system slot = fac_keep ? k : k - k0
    long long fac_stride;
    int fac_keep;
    C<T>* upd;             // update matrices, slot k - k0
    long long upd_stride;
    C<T>* uvec;            // update vectors, slot k - k0
    long long uvec_stride;
    C<T>* rhs;             // (systems, n): right-hand sides in, solutions out
    int n;
    int* status;
};
template <typename T> cudaError_t mf_factor_launch(MfArgs<T> a, int lvl_off, int nfronts, int nsys, cudaStream_t st);
template <typename T>
cudaError_t mf_solve_launch(MfArgs<T> a, int lvl_off, int nfronts, int nsys, int max_front, bool fwd, cudaStream_t st);
template <typename T>
cudaError_t mf_level_launch(MfArgs<T> a, int lvl_off, const int* ncls, int nlarge, int nsys, int max_front, int what,
                            cudaStream_t st);

// CSR spatial operators on the device (general meshes)
struct CsrDev {
    int n;
    const int* rowptr;
    const int* col;
    const double* M;
    const double* A;
};

// tensor-core (tcgen05, 3xTF32) time transforms
int tc_round_up(int v, int m);
bool tc_make_map(CUtensorMap* map, const float* base, int rows, int cols);
void tc_split_matrix(const cd* T, int n, int M_pad, int K_pad, float* out);
cudaError_t tc_split_launch(const void* in, bool in_c128, int K, int N, int K_pad, int N2_pad, const double* scale,
                            int conj, float* bt, cudaStream_t st);
cudaError_t tc_gemm_launch(const CUtensorMap& mapA, const CUtensorMap& mapB, int M_pad, int N2_pad, int K_pad, int M,
                           int N, void* out, bool out_c128, int conj_out, int accumulate, const double* out_scale,
                           const void* add_row, const double2* r1_u, const double2* r1_v, int* err, cudaStream_t st);

}  // namespace stfdm

struct st_fdm {
    stfdm::TimeMats tm;
    stfdm::SpaceMats sm;
    stfdm::TimeDecomp td;
    double setup_seconds = 0;
    int device = 0;
    int sm_count = 0;
    size_t smem_optin = 0;
    // device constants
    double2* xf64[4] = {nullptr, nullptr, nullptr, nullptr};  // Y, X, X^T, Y^T (row-major n_t x n_t)
    float2* xf32[4] = {nullptr, nullptr, nullptr, nullptr};
    float* xf_tf32[4][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
    double2* s64 = nullptr;
    float2* s32 = nullptr;
    double2* Ym64 = nullptr;  // Y_t m_t (lifting correction after the forward transform)
    stfdm::DevTime dt;
    // workspace (allocated on demand, grown as needed)
    void* ws_big = nullptr;       // R (c128) or G (c128) : n_t n_x complex double
    size_t ws_big_bytes = 0;
    void* ws_g32 = nullptr;       // c64 n_t n_x (mixed: scaled residual / G / W)
    size_t ws_g32_bytes = 0;
    void* ws_win = nullptr;       // banded factorisation windows (per CTA slot)
    size_t ws_win_bytes = 0;
    void* ws_L = nullptr;         // LDL^T factors
    size_t ws_L_bytes = 0;
    void* ws_D = nullptr;
    size_t ws_D_bytes = 0;
    void* ws_vec = nullptr;       // small vectors: A_x psi0 (c128 n_x) etc.
    size_t ws_vec_bytes = 0;
    double* ws_red = nullptr;     // reduction partials + scalars
    size_t ws_red_bytes = 0;
    int* ws_status = nullptr;     // device status flags
    void* ws_kry = nullptr;       // GMRES basis V (m+1) and preconditioned directions Z (m), c128
    size_t ws_kry_bytes = 0;
    double2** kry_ptrs = nullptr; // device array of 2m+2 vector pointers: V_0..V_m, Z_0..Z_{m-1}, w
    void* kry_small = nullptr;    // multi-dot partials and coefficient buffers
    size_t kry_small_bytes = 0;
    int kry_m = 0;
    // tensor-core transforms: split matrices [4 parts][M_pad][K_pad] per transform, input planes
    int tc_ok = 0;
    int tc_M_pad = 0, tc_K_pad = 0, tc_N2_pad = 0;
    float* tc_A[4] = {nullptr, nullptr, nullptr, nullptr};
    CUtensorMap tc_mapA[4];
    float* tc_bt = nullptr;       // [2][N2_pad][K_pad]
    size_t tc_bt_bytes = 0;
    CUtensorMap tc_mapB;
    void* ws_norm = nullptr;      // error-norm partial sums
    size_t ws_norm_bytes = 0;
    void* ws_Lt = nullptr;        // partial keep: factors of the systems refactorised every application
    size_t ws_Lt_bytes = 0;
    void* ws_Dt = nullptr;
    size_t ws_Dt_bytes = 0;
    int kept_sys = 0;             // partial keep: ws_L holds the factors of systems 0 .. kept_sys - 1
    int factors_valid = 0;        // ws_L holds the factors of all n_t systems (keep mode) or of the kept ones
    int factors_prec = -1;
    unsigned long long wait_probe_ns = 0;   // st_set_wait_probe: copied into the substitution launches
    // general meshes / sparse-direct spatial solver
    int spatial = 0;              // 0 = banded LDL^T (structured grids), 1 = multifrontal
    int* csr_rowptr = nullptr;    // device CSR of M_x, A_x (general meshes; the residual and lifting)
    int* csr_col = nullptr;
    double* csr_M = nullptr;
    double* csr_A = nullptr;
    stfdm::MfPlan mf;             // host plan
    stfdm::MfFrontDev* mf_fronts = nullptr;
    int* mf_ints = nullptr;       // perm, urows, relpos, children, orig_r, orig_c, orig_k, level_fronts
    const int *mf_perm = nullptr, *mf_urows = nullptr, *mf_relpos = nullptr, *mf_children = nullptr;
    const int *mf_orig_r = nullptr, *mf_orig_c = nullptr, *mf_orig_k = nullptr, *mf_level = nullptr;
    double* mf_csrv = nullptr;    // M_x, A_x values on the plan's CSR (structured grids)
    long long mf_csrv_nnz = 0;
    void* mf_upd = nullptr;       // update matrices for a chunk of systems
    size_t mf_upd_bytes = 0;
    void* mf_uvec = nullptr;      // update vectors for a chunk of systems
    size_t mf_uvec_bytes = 0;
    // Bartels-Stewart (Schur choice of step 1; FP64 reference path), set up at its first use
    double2* bs_Z = nullptr;      // Z (row-major n_t x n_t): back transform
    double2* bs_Y = nullptr;      // Z^H (i B_t)^{-1}: forward transform
    double2* bs_T = nullptr;      // Schur form T (row-major, upper triangular)
    double2* bs_shift = nullptr;  // T_ll, the shifts of the spatial systems in Schur order
    double2* bs_Ym = nullptr;     // bs_Y m_t (lifting)
    void* bs_w = nullptr;         // (n_t, n_x): accumulated couplings, then the solved w_l
    size_t bs_w_bytes = 0;
    const double2* shift_override = nullptr;   // FP64 factorisations use these shifts when set
};
