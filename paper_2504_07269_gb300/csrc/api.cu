// C ABI of the solver: handle setup (step 1 on the host, upload), the full solve in
// FP64 / FP32 / mixed precision with FP64 iterative refinement, the FP64 residual, the
// adjoint solve, single-step entry points and the batched solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "device.cuh"
#include "plan_rules.h"

namespace stfdm {

thread_local long long t_launches = 0;
void note_launches(int n) { t_launches += n; }
long long launches_issued() { return t_launches; }

// launchers implemented in the kernel files
cudaError_t launch_stencil_A(const SpaceMats& sm, const void* in, bool in_c64, const double2* add, double sign,
                             double2* out, cudaStream_t st);
int residual_num_partials(int n_t, int n_x);
cudaError_t launch_residual(const SpaceMats& sm, int n_t, int time_band, const double* Mb, const double* Bb, double bsign,
                            const double2* F, const double2* apsi0, const double* m_t, const double2* U,
                            const double2* psi0, double2* R, double* partials, double* scalars, cudaStream_t st);
cudaError_t launch_add_row(int n_t, int n_x, void* psi, const void* psi0, bool c64, cudaStream_t st);
cudaError_t launch_load_nodal(const SpaceMats& sm, int n_t, const double* Mb, const double* Mfull0,
                              const double2* f, double2* F, cudaStream_t st);
cudaError_t launch_colsums(int n_t, int n_x, const double2* U1, const double2* U2, const double* w, double2* out1,
                           double2* out2, cudaStream_t st);
cudaError_t launch_multidot(const double2* const* Vdev, int nv, const double2* w, size_t n, double2* partial,
                            double2* out, cudaStream_t st);
cudaError_t launch_multiaxpy(const double2* const* Vdev, int nv, const double2* c, double sign, double2* y, size_t n,
                             cudaStream_t st);
cudaError_t launch_scale(const double2* x, double alpha, double2* y, size_t n, cudaStream_t st);
cudaError_t launch_gs_project(const double2* const* Vdev, int nv, int shift, const double2* w, size_t n,
                              double2* partial, double2* out, cudaStream_t st);
cudaError_t launch_gs_update(const double2* const* Vdev, int nv, int shift, const double2* c, double2* w, size_t n,
                             double2* partial, double2* out, cudaStream_t st);
cudaError_t launch_set_scalars(double* dst, double a, double b, cudaStream_t st);
cudaError_t launch_bs_accum(int n_t, int n_x, int l, const double2* T, double2* W, cudaStream_t st);
int krylov_partial_count();
int krylov_max_vectors();

}  // namespace stfdm

using namespace stfdm;

#define CUDA_TRY(expr)                                                                       \
    do {                                                                                     \
        cudaError_t _e = (expr);                                                             \
        if (_e != cudaSuccess)                                                               \
            return fail(ST_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e));    \
    } while (0)

namespace {

st_status dev_alloc(void** p, size_t bytes, const char* what) {
    *p = nullptr;
    if (bytes == 0) return ST_OK;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? ST_ERR_OOM : ST_ERR_CUDA,
                    std::string("cudaMalloc(") + what + ", " + std::to_string(bytes) + " B): " + cudaGetErrorString(e));
    }
    return ST_OK;
}

// grow a workspace buffer (contents not preserved)
st_status grow(void*& p, size_t& have, size_t need, const char* what) {
    if (need <= have && p) return ST_OK;
    if (p) cudaFree(p);
    p = nullptr;
    have = 0;
    st_status s = dev_alloc(&p, need, what);
    if (s == ST_OK) have = need;
    return s;
}

// exactly `need` bytes (reallocated unless the size matches)
st_status resize(void*& p, size_t& have, size_t need, const char* what) {
    if (need == have && p) return ST_OK;
    if (p) cudaFree(p);
    p = nullptr;
    have = 0;
    st_status s = dev_alloc(&p, need, what);
    if (s == ST_OK) have = need;
    return s;
}

template <typename T>
st_status upload(T** dst, const void* src, size_t bytes, const char* what) {
    st_status s = dev_alloc((void**)dst, bytes, what);
    if (s != ST_OK) return s;
    CUDA_TRY(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    return ST_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (dev >= 0 && dev != prev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

inline cudaStream_t S(void* stream) { return reinterpret_cast<cudaStream_t>(stream); }

void free_handle(st_fdm* h) {
    if (!h) return;
    DeviceGuard g(h->device);
    for (int i = 0; i < 4; ++i) {
        cudaFree(h->xf64[i]);
        cudaFree(h->xf32[i]);
        cudaFree(h->xf_tf32[i][0]);
        cudaFree(h->xf_tf32[i][1]);
    }
    cudaFree(h->s64);
    cudaFree(h->s32);
    cudaFree(h->Ym64);
    cudaFree(h->dt.Mb);
    cudaFree(h->dt.Bb);
    cudaFree(h->dt.BTb);
    cudaFree(h->dt.Mfull0);
    cudaFree(h->dt.m);
    cudaFree(h->dt.nodes);
    cudaFree(h->ws_norm);
    cudaFree(h->ws_big);
    cudaFree(h->ws_g32);
    cudaFree(h->ws_win);
    cudaFree(h->ws_L);
    cudaFree(h->ws_D);
    cudaFree(h->ws_Lt);
    cudaFree(h->ws_Dt);
    cudaFree(h->ws_vec);
    cudaFree(h->ws_red);
    cudaFree(h->ws_status);
    cudaFree(h->ws_kry);
    cudaFree(h->kry_ptrs);
    cudaFree(h->kry_small);
    for (int i = 0; i < 4; ++i) cudaFree(h->tc_A[i]);
    cudaFree(h->tc_bt);
    cudaFree(h->csr_rowptr);
    cudaFree(h->csr_col);
    cudaFree(h->csr_M);
    cudaFree(h->csr_A);
    cudaFree(h->mf_fronts);
    cudaFree(h->mf_ints);
    cudaFree(h->mf_csrv);
    cudaFree(h->mf_upd);
    cudaFree(h->mf_uvec);
    cudaFree(h->bs_Z);
    cudaFree(h->bs_Y);
    cudaFree(h->bs_T);
    cudaFree(h->bs_shift);
    cudaFree(h->bs_Ym);
    cudaFree(h->bs_w);
    delete h;
}

// ------------------------------------------------------------------ transforms
template <typename TA, typename TB, typename TC, typename TACC>
st_status xform(const TA* A2, int n_t, int n_x, const void* in, void* out, int conj_b, int conj_out,
                int accumulate, const double* b_scale, const double* out_scale, const void* add_row,
                const double2* r1_u, const double2* r1_v, cudaStream_t st) {
    XformArgs<TA, TB, TC> a;
    a.M = n_t;
    a.N = n_x;
    a.K = n_t;
    a.A = reinterpret_cast<const C<TA>*>(A2);
    a.lda = n_t;
    a.B = reinterpret_cast<const C<TB>*>(in);
    a.ldb = n_x;
    a.Cm = reinterpret_cast<C<TC>*>(out);
    a.ldc = n_x;
    a.conj_b = conj_b;
    a.conj_out = conj_out;
    a.accumulate = accumulate;
    a.b_scale = b_scale;
    a.out_scale = out_scale;
    a.add_row = reinterpret_cast<const C<TC>*>(add_row);
    a.r1_u = r1_u;
    a.r1_v = r1_v;
    CUDA_TRY((xform_simt_launch<TA, TB, TC, TACC>(a, st)));
    return ST_OK;
}

// Complex-FP32 time transform: the tensor-core path (3xTF32, tcgen05 + TMA) when available,
// else the SIMT kernel.  in: c128 (in_c128) or c64, scaled by *b_scale and conjugated if conj_b;
// out: c128 (out_c128) or c64, with the epilogue options of the SIMT kernel.
st_status ensure_tc_input(st_fdm* h) {
    const size_t need = (size_t)2 * h->tc_N2_pad * h->tc_K_pad * sizeof(float);
    if (h->tc_bt && h->tc_bt_bytes >= need) return ST_OK;
    cudaFree(h->tc_bt);
    h->tc_bt = nullptr;
    h->tc_bt_bytes = 0;
    st_status s = dev_alloc(reinterpret_cast<void**>(&h->tc_bt), need, "tensor-core input planes");
    if (s != ST_OK) return s;
    h->tc_bt_bytes = need;
    CUDA_TRY(cudaMemset(h->tc_bt, 0, need));   // padding rows stay zero
    if (!tc_make_map(&h->tc_mapB, h->tc_bt, 2 * h->tc_N2_pad, h->tc_K_pad))
        return fail(ST_ERR_CUDA, "tensor map for the transform input");
    return ST_OK;
}

st_status xform32(st_fdm* h, int which, const void* in, bool in_c128, const double* b_scale, int conj_b, void* out,
                  bool out_c128, int conj_out, int accumulate, const double* out_scale, const void* add_row,
                  const double2* r1_u, const double2* r1_v, cudaStream_t st) {
    const int n_t = h->tm.n_t, n_x = h->sm.n_x;
    if (h->tc_ok) {
        st_status s = ensure_tc_input(h);
        if (s != ST_OK) return s;
        CUDA_TRY(tc_split_launch(in, in_c128, n_t, n_x, h->tc_K_pad, h->tc_N2_pad, b_scale, conj_b, h->tc_bt, st));
        CUDA_TRY(tc_gemm_launch(h->tc_mapA[which], h->tc_mapB, h->tc_M_pad, h->tc_N2_pad, h->tc_K_pad, n_t, n_x, out,
                                out_c128, conj_out, accumulate, out_scale, add_row, r1_u, r1_v, h->ws_status + 1, st));
        return ST_OK;
    }
    const float* A = reinterpret_cast<float*>(h->xf32[which]);
    if (in_c128 && !out_c128)
        return xform<float, double, float, float>(A, n_t, n_x, in, out, conj_b, conj_out, accumulate, b_scale, out_scale,
                                                  add_row, r1_u, r1_v, st);
    if (!in_c128 && out_c128)
        return xform<float, float, double, float>(A, n_t, n_x, in, out, conj_b, conj_out, accumulate, b_scale,
                                                  out_scale, add_row, r1_u, r1_v, st);
    if (!in_c128 && !out_c128)
        return xform<float, float, float, float>(A, n_t, n_x, in, out, conj_b, conj_out, accumulate, b_scale, out_scale,
                                                 add_row, r1_u, r1_v, st);
    return fail(ST_ERR_UNSUPPORTED, "xform32: c128 -> c128");
}

// ------------------------------------------------------------------ banded solves
template <typename T>
const C<T>* shifts_of(const st_fdm* h);
template <>
const double2* shifts_of<double>(const st_fdm* h) { return h->s64; }
template <>
const float2* shifts_of<float>(const st_fdm* h) { return h->s32; }
// the shifts of the factorisations: the eigenvalues s_k, or (FP64, Bartels-Stewart) the Schur diagonal
template <typename T>
const C<T>* active_shifts(const st_fdm* h) { return shifts_of<T>(h); }
template <>
const double2* active_shifts<double>(const st_fdm* h) { return h->shift_override ? h->shift_override : h->s64; }

// Partial keep when not all complex64 factors fit: the number of leading systems whose factors
// stay in memory (partial_keep_systems), with one wave of transient factors (one system per
// resident CTA), its windows and a 2 GiB reserve set aside.
// One wave of transient factors: grid = resident CTAs of the complex64 factor kernel, per = bytes
// of one system's L and D, fixed = the wave's factors, its windows and a 2 GiB reserve.
bool partial_keep_geometry(const st_fdm* h, int& grid, size_t& per, size_t& fixed) {
    if (h->spatial == 1) return false;   // the sparse-direct factors are kept whole or refactorised
    const int n_t = h->tm.n_t, n = h->sm.n_x, b = h->sm.m + 1;
    const int nb = band_pick_nb<float>(b, h->smem_optin);
    if (nb == 0) return false;
    int occ = band_occupancy<float>(nb, b);
    if (occ < 1) occ = 1;
    grid = std::max(1, std::min(n_t, occ * h->sm_count));
    per = (size_t)n * (size_t)(b + 1) * sizeof(float2);
    fixed = (size_t)grid * per + (size_t)grid * (size_t)(b + 32) * (size_t)(b + 1) * sizeof(float2) + ((size_t)2 << 30);
    return true;
}

int partial_keep_count(st_fdm* h) {
    if (h->spatial == 1) return 0;
    int grid = 0;
    size_t per = 0, fixed = 0;
    if (!partial_keep_geometry(h, grid, per, fixed)) return 0;
    size_t freeb = 0, total = 0;
    if (cudaMemGetInfo(&freeb, &total) != cudaSuccess) return 0;
    // buffers that this solve may reallocate count as free
    const size_t avail = freeb + h->ws_L_bytes + h->ws_D_bytes + h->ws_Lt_bytes + h->ws_Dt_bytes;
    return partial_keep_systems(h->tm.n_t, grid, per, avail, fixed);
}

bool mf_factors_fit(st_fdm* h, size_t elem);

bool factors_fit(st_fdm* h, size_t elem) {
    if (h->spatial == 1) return mf_factors_fit(h, elem);
    size_t freeb = 0, total = 0;
    if (cudaMemGetInfo(&freeb, &total) != cudaSuccess) return false;
    const size_t need = (size_t)h->tm.n_t * h->sm.n_x * (size_t)(h->sm.m + 1 + 1) * elem;
    size_t have = h->ws_L_bytes + h->ws_D_bytes;
    return need <= (size_t)(0.85 * (double)(freeb + have));
}

// ------------------------------------------------------------------ sparse-direct spatial solves
// Multifrontal factor-and-solve of all n_t systems (general meshes, or structured grids set up
// with ST_SPATIAL_MULTIFRONTAL).  mode 0: factors transient, systems in chunks; 1: factor all
// systems into kept storage, then solve; 2: solve with the kept factors.  The update matrices and
// vectors live only for a chunk of systems.
bool mf_factors_fit(st_fdm* h, size_t elem) {
    size_t freeb = 0, total = 0;
    if (cudaMemGetInfo(&freeb, &total) != cudaSuccess) return false;
    const size_t need = (size_t)h->tm.n_t * (size_t)h->mf.factor_entries * elem;
    const size_t have = h->ws_L_bytes + h->mf_upd_bytes + h->mf_uvec_bytes;
    return need <= (size_t)(0.8 * (double)(freeb + have));
}

template <typename T>
MfArgs<T> mf_args(const st_fdm* h, C<T>* G);
template <typename T>
cudaError_t mf_levels(const st_fdm* h, MfArgs<T>& a, int k0, int cnt, int what, cudaStream_t st);

template <typename T>
st_status mf_run(st_fdm* h, C<T>* G, int mode, cudaStream_t st) {
    const MfPlan& P = h->mf;
    const int n_t = h->tm.n_t;
    const size_t esz = sizeof(C<T>);
    if (mode == 2 && (!h->factors_valid || h->factors_prec != (int)sizeof(T)))
        return fail(ST_ERR_ARG, "spatial solve: no stored factors");
    size_t freeb = 0, total = 0;
    CUDA_TRY(cudaMemGetInfo(&freeb, &total));
    size_t avail = freeb + h->mf_upd_bytes + h->mf_uvec_bytes + (mode == 2 ? 0 : h->ws_L_bytes);
    if (mode == 1) {
        const size_t kept = (size_t)n_t * P.factor_entries * esz;
        if (kept > avail) return fail(ST_ERR_OOM, "spatial solve: kept factors do not fit");
        avail -= kept;
    }
    // systems per chunk: transient storage within 40% of what is available
    size_t per = (size_t)(P.update_entries + P.uvec_entries) * esz;
    if (mode == 0) per += (size_t)P.factor_entries * esz;
    if (mode == 2) per = (size_t)P.uvec_entries * esz;
    long long kc = per ? (long long)((double)avail * 0.4 / (double)per) : n_t;
    kc = std::max(1LL, std::min<long long>(kc, std::min(n_t, 65535)));
    st_status s = ST_OK;
    if (mode != 2) {
        s = grow(h->mf_upd, h->mf_upd_bytes, std::max<size_t>(16, (size_t)kc * P.update_entries * esz), "update matrices");
        if (s != ST_OK) return s;
    }
    s = grow(h->mf_uvec, h->mf_uvec_bytes, std::max<size_t>(16, (size_t)kc * P.uvec_entries * esz), "update vectors");
    if (s != ST_OK) return s;
    if (mode == 1) {
        h->factors_valid = 0;
        s = resize(h->ws_L, h->ws_L_bytes, (size_t)n_t * P.factor_entries * esz, "kept factors");
    } else if (mode == 0) {
        h->factors_valid = 0;
        s = grow(h->ws_L, h->ws_L_bytes, (size_t)kc * P.factor_entries * esz, "factors");
    }
    if (s != ST_OK) return s;
    MfArgs<T> a = mf_args<T>(h, G);
    a.fac_keep = (mode == 0) ? 0 : 1;
    auto levels = [&](int k0, int cnt, int what) -> cudaError_t { return mf_levels<T>(h, a, k0, cnt, what, st); };
    for (int k0 = 0; k0 < n_t; k0 += (int)kc) {
        const int cnt = (int)std::min<long long>(kc, n_t - k0);
        if (mode != 2) CUDA_TRY(levels(k0, cnt, 0));
        CUDA_TRY(levels(k0, cnt, 1));
        CUDA_TRY(levels(k0, cnt, 2));
    }
    if (mode == 1) {
        h->factors_valid = 1;
        h->factors_prec = (int)sizeof(T);   // the real type's size, as for banded factors
    }
    return ST_OK;
}

template <typename T>
MfArgs<T> mf_args(const st_fdm* h, C<T>* G) {
    const MfPlan& P = h->mf;
    MfArgs<T> a;
    a.fronts = h->mf_fronts;
    a.level_fronts = h->mf_level;
    a.lvl_off = 0;
    a.urows = h->mf_urows;
    a.relpos = h->mf_relpos;
    a.children = h->mf_children;
    a.orig_r = h->mf_orig_r;
    a.orig_c = h->mf_orig_c;
    a.orig_k = h->mf_orig_k;
    a.perm = h->mf_perm;
    if (h->sm.kind == 1) {
        a.Mv = h->csr_M;
        a.Av = h->csr_A;
    } else {
        a.Mv = h->mf_csrv;
        a.Av = h->mf_csrv + h->mf_csrv_nnz;
    }
    a.shifts = active_shifts<T>(h);
    a.fac = reinterpret_cast<C<T>*>(h->ws_L);
    a.fac_stride = P.factor_entries;
    a.fac_keep = 1;
    a.k0 = 0;
    a.upd = reinterpret_cast<C<T>*>(h->mf_upd);
    a.upd_stride = P.update_entries;
    a.uvec = reinterpret_cast<C<T>*>(h->mf_uvec);
    a.uvec_stride = P.uvec_entries;
    a.rhs = G;
    a.n = h->sm.n_x;
    a.status = h->ws_status;
    return a;
}

// what: 0 = factorise, 1 = forward substitution, 2 = backward substitution, systems k0 .. k0 + cnt - 1
template <typename T>
cudaError_t mf_levels(const st_fdm* h, MfArgs<T>& a, int k0, int cnt, int what, cudaStream_t st) {
    const MfPlan& P = h->mf;
    const int H = (int)P.level_ptr.size() - 1;
    a.k0 = k0;
    for (int i = 0; i < H; ++i) {
        const int l = (what == 2) ? H - 1 - i : i;   // backward substitution from the root
        const int n = P.level_ptr[l + 1] - P.level_ptr[l];
        const int* ncls = P.level_ncls.data() + (size_t)l * MF_NCLS;
        int nsmall = 0;
        for (int c = 0; c < MF_NCLS; ++c) nsmall += ncls[c];
        cudaError_t e = mf_level_launch<T>(a, P.level_ptr[l], ncls, n - nsmall, cnt, P.max_front, what, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// the launch arguments common to every banded kernel of a handle (windows and factor storage unset)
template <typename T>
BandArgs<T> band_args(const st_fdm* h, C<T>* G) {
    const SpaceMats& sm = h->sm;
    BandArgs<T> a;
    a.n = sm.n_x;
    a.m = sm.m;
    a.b = sm.m + 1;
    a.n_sys = h->tm.n_t;
    a.k0 = 0;
    a.Mc = (T)sm.Mc; a.Mw = (T)sm.Mw; a.Ms = (T)sm.Ms; a.Md = (T)sm.Md;
    a.Ac = (T)sm.Ac; a.Aw = (T)sm.Aw; a.As = (T)sm.As; a.Ad = (T)sm.Ad;
    a.shifts = active_shifts<T>(h);
    a.rhs = G;
    a.win = nullptr;
    a.L = nullptr;
    a.D = nullptr;
    a.keep = 0;
    a.status = h->ws_status;
    a.probe_ns = h->wait_probe_ns;
    return a;
}

// mode: 0 = factor and solve (factors transient, in chunks of systems), 1 = factor, keep all
//       factors, and solve, 2 = forward + backward substitution with the kept factors;
//       partial keep (h->kept_sys systems kept, the rest refactorised in waves of one CTA each):
//       3 = first application (the kept systems factorised into ws_L), 4 = later applications
//       (substitutions for the kept systems)
template <typename T>
st_status band_run(st_fdm* h, C<T>* G, int mode, cudaStream_t st) {
    if (h->spatial == 1) {
        if (mode == 3 || mode == 4) return fail(ST_ERR_ARG, "spatial solve: partial keep is for banded factors");
        return mf_run<T>(h, G, mode, st);
    }
    const SpaceMats& sm = h->sm;
    const int n = sm.n_x, b = sm.m + 1, n_t = h->tm.n_t;
    const int nb = band_pick_nb<T>(b, h->smem_optin);
    if (nb == 0) return fail(ST_ERR_UNSUPPORTED, "spatial solve: band too wide for shared memory");
    int occ = band_occupancy<T>(nb, b);
    if (occ < 1) occ = 1;
    const int grid = std::max(1, std::min(n_t, occ * h->sm_count));
    BandArgs<T> a = band_args<T>(h, G);
    const int nbw = nb == 64 ? 32 : (nb < 0 ? -nb : nb);   // panel width of the selected kernel
    const size_t WR = (size_t)b + nbw;
    if (mode == 3 || mode == 4) {
        const int K = h->kept_sys;
        if (K <= 0 || K >= n_t) return fail(ST_ERR_ARG, "spatial solve: kept-system count out of range");
        if (mode == 4 && (!h->factors_valid || h->factors_prec != (int)sizeof(T)))
            return fail(ST_ERR_ARG, "spatial solve: no stored factors");
        st_status s = ST_OK;
        if (mode == 3) {
            // exactly K systems' worth: a larger buffer left by an earlier solve would hold memory
            // that the choice of K counted as free
            h->factors_valid = 0;
            s = resize(h->ws_L, h->ws_L_bytes, (size_t)K * n * b * sizeof(C<T>), "kept band factors");
            if (s != ST_OK) return s;
            s = resize(h->ws_D, h->ws_D_bytes, (size_t)K * n * sizeof(C<T>), "kept band pivots");
            if (s != ST_OK) return s;
        }
        s = grow(h->ws_win, h->ws_win_bytes, (size_t)grid * WR * (b + 1) * sizeof(C<T>), "band windows");
        if (s != ST_OK) return s;
        s = grow(h->ws_Lt, h->ws_Lt_bytes, (size_t)grid * n * b * sizeof(C<T>), "band factors");
        if (s != ST_OK) return s;
        s = grow(h->ws_Dt, h->ws_Dt_bytes, (size_t)grid * n * sizeof(C<T>), "band pivots");
        if (s != ST_OK) return s;
        a.win = reinterpret_cast<C<T>*>(h->ws_win);
        // systems 0 .. K-1: factors stored per system k
        a.L = reinterpret_cast<C<T>*>(h->ws_L);
        a.D = reinterpret_cast<C<T>*>(h->ws_D);
        a.keep = 1;
        a.k0 = 0;
        a.n_sys = K;
        if (mode == 3) {
            CUDA_TRY(band_factor_solve_launch<T>(a, nb, std::min(grid, K), st));
        } else {
            CUDA_TRY(subst_launch<T>(a, 0, K, true, st));
        }
        CUDA_TRY(subst_launch<T>(a, 0, K, false, st));
        // systems K .. n_t-1: factor and solve, one wave of CTAs per launch, factors per CTA slot
        a.L = reinterpret_cast<C<T>*>(h->ws_Lt);
        a.D = reinterpret_cast<C<T>*>(h->ws_Dt);
        a.keep = 0;
        for (int k0 = K; k0 < n_t; k0 += grid) {
            const int cnt = std::min(grid, n_t - k0);
            a.k0 = k0;
            a.n_sys = cnt;
            CUDA_TRY(band_factor_solve_launch<T>(a, nb, cnt, st));
            CUDA_TRY(subst_launch<T>(a, k0, cnt, false, st));
        }
        if (mode == 3) {
            h->factors_valid = 1;
            h->factors_prec = (int)sizeof(T);
        }
        return ST_OK;
    }
    if (mode == 2) {
        if (!h->factors_valid || h->factors_prec != (int)sizeof(T) || h->kept_sys != 0)
            return fail(ST_ERR_ARG, "spatial solve: no stored factors");
        a.win = nullptr;
        a.L = reinterpret_cast<C<T>*>(h->ws_L);
        a.D = reinterpret_cast<C<T>*>(h->ws_D);
        a.keep = 1;
        CUDA_TRY(subst_launch<T>(a, 0, n_t, true, st));
        CUDA_TRY(subst_launch<T>(a, 0, n_t, false, st));
        return ST_OK;
    }
    st_status s = grow(h->ws_win, h->ws_win_bytes, (size_t)grid * WR * (b + 1) * sizeof(C<T>), "band windows");
    if (s != ST_OK) return s;
    // transient factors: all systems in one launch when their factors fit, else chunks of `grid`
    int chunk = (mode == 1) ? n_t : grid;
    if (mode == 0 && chunk < n_t && factors_fit(h, sizeof(C<T>))) chunk = n_t;
    s = grow(h->ws_L, h->ws_L_bytes, (size_t)chunk * n * b * sizeof(C<T>), "band factors");
    if (s != ST_OK) return s;
    s = grow(h->ws_D, h->ws_D_bytes, (size_t)chunk * n * sizeof(C<T>), "band pivots");
    if (s != ST_OK) return s;
    h->factors_valid = 0;
    h->kept_sys = 0;
    a.win = reinterpret_cast<C<T>*>(h->ws_win);
    a.L = reinterpret_cast<C<T>*>(h->ws_L);
    a.D = reinterpret_cast<C<T>*>(h->ws_D);
    a.keep = (mode == 1) ? 1 : 0;
    for (int k0 = 0; k0 < n_t; k0 += chunk) {
        const int cnt = std::min(chunk, n_t - k0);
        a.k0 = k0;
        a.n_sys = cnt;
        CUDA_TRY(band_factor_solve_launch<T>(a, nb, std::min(grid, cnt), st));
        CUDA_TRY(subst_launch<T>(a, k0, cnt, false, st));
    }
    if (mode == 1) {
        h->factors_valid = 1;
        h->factors_prec = (int)sizeof(T);
    }
    return ST_OK;
}

// nonzero diagonals of the temporal band matrices: 3 for P1 time, 5 for P2
int time_band(const st_fdm* h) { return h->tm.p == 1 ? 3 : 5; }

st_status check_status_flag(st_fdm* h, cudaStream_t st) {
    int flag[2] = {0, 0};
    CUDA_TRY(cudaMemcpyAsync(flag, h->ws_status, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (flag[1]) return fail(ST_ERR_TIMEOUT, "a bounded pipeline wait expired (tensor-core transform or factor streaming)");
    if (flag[0]) return fail(ST_ERR_ZERO_PIVOT, "spatial solve: zero or non-finite pivot");
    return ST_OK;
}

st_status ensure_common(st_fdm* h) {
    const size_t nx = (size_t)h->sm.n_x;
    st_status s = grow(h->ws_vec, h->ws_vec_bytes, 4 * nx * sizeof(double2), "vectors");
    if (s != ST_OK) return s;
    return ST_OK;
}

double2* vec_slot(st_fdm* h, int i) { return reinterpret_cast<double2*>(h->ws_vec) + (size_t)i * h->sm.n_x; }

// A direct (single-application) solve needs neither the refinement's basis nor the partial keep's
// transient wave: release them, so that its own transient factors find the memory.
void release_refinement_workspace(st_fdm* h) {
    const bool busy = h->ws_kry || h->ws_Lt || h->ws_Dt;
    if (!busy) return;
    cudaFree(h->ws_kry);   // cudaFree waits for the device work in flight, like grow()'s reallocations
    h->ws_kry = nullptr;
    h->ws_kry_bytes = 0;
    h->kry_m = 0;
    cudaFree(h->ws_Lt);
    h->ws_Lt = nullptr;
    h->ws_Lt_bytes = 0;
    cudaFree(h->ws_Dt);
    h->ws_Dt = nullptr;
    h->ws_Dt_bytes = 0;
    h->kept_sys = 0;
}

// ------------------------------------------------------------------ solves
st_status solve_fp64(st_fdm* h, const void* F, const void* psi0, void* psi, cudaStream_t st) {
    const int n_t = h->tm.n_t, n_x = h->sm.n_x;
    release_refinement_workspace(h);
    st_status s = ensure_common(h);
    if (s != ST_OK) return s;
    s = grow(h->ws_big, h->ws_big_bytes, (size_t)n_t * n_x * sizeof(double2), "G");
    if (s != ST_OK) return s;
    double2* apsi0 = nullptr;
    if (psi0) {
        apsi0 = vec_slot(h, 0);
        CUDA_TRY(launch_stencil_A(h->sm, psi0, false, nullptr, 1.0, apsi0, st));
    }
    double2* G = reinterpret_cast<double2*>(h->ws_big);
    s = xform<double, double, double, double>(reinterpret_cast<double*>(h->xf64[XF_Y]), n_t, n_x, F, G, 0, 0, 0,
                                              nullptr, nullptr, nullptr, psi0 ? h->Ym64 : nullptr, apsi0, st);
    if (s != ST_OK) return s;
    s = band_run<double>(h, G, 0, st);
    if (s != ST_OK) return s;
    return xform<double, double, double, double>(reinterpret_cast<double*>(h->xf64[XF_X]), n_t, n_x, G, psi, 0, 0, 0,
                                                 nullptr, nullptr, psi0, nullptr, nullptr, st);
}

st_status solve_fp32(st_fdm* h, const void* F, const void* psi0, void* psi, cudaStream_t st) {
    const int n_t = h->tm.n_t, n_x = h->sm.n_x;
    release_refinement_workspace(h);
    st_status s = ensure_common(h);
    if (s != ST_OK) return s;
    s = grow(h->ws_g32, h->ws_g32_bytes, (size_t)n_t * n_x * sizeof(float2), "G32");
    if (s != ST_OK) return s;
    double2* apsi0 = nullptr;
    if (psi0) {
        apsi0 = vec_slot(h, 0);
        CUDA_TRY(launch_stencil_A(h->sm, psi0, true, nullptr, 1.0, apsi0, st));
    }
    float2* G = reinterpret_cast<float2*>(h->ws_g32);
    s = xform32(h, XF_Y, F, false, nullptr, 0, G, false, 0, 0, nullptr, nullptr, psi0 ? h->Ym64 : nullptr, apsi0, st);
    if (s != ST_OK) return s;
    s = band_run<float>(h, G, 0, st);
    if (s != ST_OK) return s;
    return xform32(h, XF_X, G, false, nullptr, 0, psi, false, 0, 0, nullptr, psi0, nullptr, nullptr, st);
}


// Mixed precision: complex-FP32 FDM sweeps on the FP64 residual (forward: K, adjoint: K^H).
st_status solve_mixed(st_fdm* h, bool adjoint, const void* F, const void* psi0, void* psi, const st_solve_opts& o,
                      st_solve_info* info, cudaStream_t st) {
    const int n_t = h->tm.n_t, n_x = h->sm.n_x;
    st_status s = ensure_common(h);
    if (s != ST_OK) return s;
    s = grow(h->ws_big, h->ws_big_bytes, (size_t)n_t * n_x * sizeof(double2), "R");
    if (s != ST_OK) return s;
    s = grow(h->ws_g32, h->ws_g32_bytes, (size_t)n_t * n_x * sizeof(float2), "G32");
    if (s != ST_OK) return s;
    double2* apsi0 = nullptr;
    if (psi0 && !adjoint) {
        apsi0 = vec_slot(h, 0);
        CUDA_TRY(launch_stencil_A(h->sm, psi0, false, nullptr, 1.0, apsi0, st));
    }
    double2* R = reinterpret_cast<double2*>(h->ws_big);
    float2* G = reinterpret_cast<float2*>(h->ws_g32);
    double* scal = h->ws_red;                      // [0..3] scalars
    double* parts = h->ws_red + 8;
    const double tol = o.tol > 0 ? o.tol : 1e-12;
    const int maxs = o.max_sweeps > 0 ? std::min(o.max_sweeps, 15) : 12;
    const bool fixed = o.fixed_sweeps > 0;
    const int nsweeps = fixed ? std::min(o.fixed_sweeps, 15) : maxs;
    bool keep = false;
    if (o.keep_factors == 1) keep = true;
    else if (o.keep_factors == -1) keep = factors_fit(h, sizeof(float2));
    const double* Bband = adjoint ? h->dt.BTb : h->dt.Bb;
    const double bsign = adjoint ? -1.0 : 1.0;
    CUDA_TRY(cudaMemsetAsync(psi, 0, (size_t)n_t * n_x * sizeof(double2), st));
    CUDA_TRY(cudaMemsetAsync(h->ws_status, 0, 2 * sizeof(int), st));
    int sweeps = 0;
    double hist[16];
    int nh = 0;
    double rel = -1;
    bool converged = false;
    for (int sw = 0; sw <= nsweeps; ++sw) {
        CUDA_TRY(launch_residual(h->sm, n_t, time_band(h), h->dt.Mb, Bband, bsign, reinterpret_cast<const double2*>(F), apsi0,
                                 h->dt.m, sw == 0 ? nullptr : reinterpret_cast<const double2*>(psi), nullptr, R, parts,
                                 scal, st));
        if (!fixed || sw == nsweeps) {
            if (!fixed || info) {
                double hs[2];
                CUDA_TRY(cudaMemcpyAsync(hs, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
                CUDA_TRY(cudaStreamSynchronize(st));
                rel = (hs[1] > 0) ? std::sqrt(hs[0] / hs[1]) : 0.0;
                if (nh < 16) hist[nh++] = rel;
                if (!std::isfinite(rel)) return fail(ST_ERR_NOT_CONVERGED, "refinement: non-finite residual");
                if (!fixed && rel <= tol) {
                    converged = true;
                    break;
                }
            }
        }
        if (sw == nsweeps) break;
        // delta = K^{-1} R (or K^{-H} R) in complex FP32, psi += delta (scaled)
        s = xform32(h, adjoint ? XF_XT : XF_Y, R, true, scal + 2, adjoint ? 1 : 0, G, false, 0, 0, nullptr, nullptr,
                    nullptr, nullptr, st);
        if (s != ST_OK) return s;
        int mode = 0;
        if (keep) mode = (sw == 0) ? 1 : 2;
        s = band_run<float>(h, G, mode, st);
        if (s != ST_OK) {
            if (mode == 1 && s == ST_ERR_OOM) {  // fall back to refactoring every sweep
                keep = false;
                s = band_run<float>(h, G, 0, st);
            }
            if (s != ST_OK) return s;
        }
        s = xform32(h, adjoint ? XF_YT : XF_X, G, false, nullptr, 0, psi, true, adjoint ? 1 : 0, 1, scal + 3, nullptr,
                    nullptr, nullptr, st);
        if (s != ST_OK) return s;
        ++sweeps;
    }
    if (psi0 && !adjoint) CUDA_TRY(launch_add_row(n_t, n_x, psi, psi0, false, st));
    if (info) {
        info->sweeps = sweeps;
        info->factors_kept = keep ? 1 : 0;
        info->kept_systems = keep ? n_t : 0;
        info->rel_residual = rel;
        for (int i = 0; i < 16; ++i) info->residual_history[i] = (i < nh) ? hist[i] : -1.0;
    }
    if (!fixed || info) {
        s = check_status_flag(h, st);
        if (s != ST_OK) return s;
    }
    if (!fixed && !converged) return fail(ST_ERR_NOT_CONVERGED, "refinement: tolerance not reached in max_sweeps");
    return ST_OK;
}


// ------------------------------------------------------------------ GMRES-based refinement
// FP64 flexible GMRES(m) for K x = F~ (or K^H x = G), right-preconditioned by the complex-FP32
// FDM: z = FDM32(v).  The Arnoldi basis V, the directions Z, the operator apply and the
// orthogonalisation (classical Gram-Schmidt, done twice) are FP64 on the device; the small
// Hessenberg least-squares problem (Givens rotations) is solved on the host.
st_status precond32(st_fdm* h, bool adjoint, const double2* v, double2* z, bool& keep, bool& first,
                    const double* scal, cudaStream_t st) {
    float2* G = reinterpret_cast<float2*>(h->ws_g32);
    st_status s = xform32(h, adjoint ? XF_XT : XF_Y, v, true, scal, adjoint ? 1 : 0, G, false, 0, 0, nullptr, nullptr,
                          nullptr, nullptr, st);
    if (s != ST_OK) return s;
    int mode = keep ? (first ? 1 : 2) : (h->kept_sys > 0 ? (first ? 3 : 4) : 0);
    s = band_run<float>(h, G, mode, st);
    if (s == ST_ERR_OOM && (mode == 1 || mode == 3)) {
        h->kept_sys = 0;
        s = band_run<float>(h, G, 0, st);
        keep = false;
    }
    if (s != ST_OK) return s;
    first = false;
    return xform32(h, adjoint ? XF_YT : XF_X, G, false, nullptr, 0, z, true, adjoint ? 1 : 0, 0, scal + 1, nullptr,
                   nullptr, nullptr, st);
}

// exact: reallocate unless the size matches (memory planned for kept factors must really be free)
st_status ensure_krylov(st_fdm* h, int m, bool exact = false) {
    const size_t N = (size_t)h->tm.n_t * h->sm.n_x;
    const size_t need = (size_t)(2 * m + 1) * N * sizeof(double2);
    st_status s = exact ? resize(h->ws_kry, h->ws_kry_bytes, need, "GMRES basis")
                        : grow(h->ws_kry, h->ws_kry_bytes, need, "GMRES basis");
    if (s != ST_OK) return s;
    if (!h->kry_ptrs) {
        s = dev_alloc(reinterpret_cast<void**>(&h->kry_ptrs), sizeof(double2*) * 2 * (krylov_max_vectors() + 1),
                      "GMRES pointers");
        if (s != ST_OK) return s;
    }
    s = grow(h->kry_small, h->kry_small_bytes, sizeof(double2) * (krylov_partial_count() + 4 * krylov_max_vectors()),
             "GMRES scalars");
    if (s != ST_OK) return s;
    std::vector<double2*> ptrs(2 * m + 2);
    double2* base = reinterpret_cast<double2*>(h->ws_kry);
    for (int i = 0; i < 2 * m + 1; ++i) ptrs[i] = base + (size_t)i * N;
    ptrs[2 * m + 1] = reinterpret_cast<double2*>(h->ws_big);  // w (shares the residual buffer)
    CUDA_TRY(cudaMemcpy(h->kry_ptrs, ptrs.data(), sizeof(double2*) * ptrs.size(), cudaMemcpyHostToDevice));
    h->kry_m = m;
    return ST_OK;
}

st_status solve_mixed_gmres(st_fdm* h, bool adjoint, const void* F, const void* psi0, void* psi,
                            const st_solve_opts& o, st_solve_info* info, cudaStream_t st) {
    const int n_t = h->tm.n_t, n_x = h->sm.n_x;
    const size_t N = (size_t)n_t * n_x;
    st_status s = ensure_common(h);
    if (s != ST_OK) return s;
    s = grow(h->ws_big, h->ws_big_bytes, N * sizeof(double2), "R");
    if (s != ST_OK) return s;
    s = grow(h->ws_g32, h->ws_g32_bytes, N * sizeof(float2), "G32");
    if (s != ST_OK) return s;
    const double tol = o.tol > 0 ? o.tol : 1e-12;
    const int maxit = o.max_sweeps > 0 ? o.max_sweeps : 40;
    bool keep = false;
    if (o.keep_factors == 1) keep = true;
    else if (o.keep_factors == -1) keep = factors_fit(h, sizeof(float2));
    // restart length: at most 20, and the basis within a third of the free memory; when not all
    // factors fit (partial keep), the longest basis that costs no refactorisation wave more than the
    // shortest (4 vectors) would
    int m = std::min(20, krylov_max_vectors() - 1);
    const bool partial_keep = !keep && o.keep_factors == -1;
    {
        size_t freeb = 0, total = 0;
        cudaMemGetInfo(&freeb, &total);
        size_t avail = freeb + h->ws_kry_bytes;
        if (keep) {
            // the kept factors will take `fac` bytes, reusing what ws_L holds already
            const size_t fac = h->spatial == 1 ? (size_t)n_t * (size_t)h->mf.factor_entries * sizeof(float2)
                                               : (size_t)n_t * n_x * (size_t)(h->sm.m + 2) * sizeof(float2);
            avail += h->ws_L_bytes + h->ws_D_bytes;
            avail = avail > fac ? avail - fac : 0;
        }
        int grid = 0;
        size_t per = 0, fixed = 0;
        if (partial_keep && partial_keep_geometry(h, grid, per, fixed)) {
            avail += h->ws_L_bytes + h->ws_D_bytes + h->ws_Lt_bytes + h->ws_Dt_bytes;
            m = single_restart_for_partial_keep(N, n_t, grid, per, avail, fixed, m, 4);
        } else {
            while (m > 2 && (size_t)(2 * m + 1) * N * sizeof(double2) > avail / 3) --m;
        }
    }
    s = ensure_krylov(h, m, partial_keep);
    if (s != ST_OK) return s;
    // when not all factors fit, keep those of as many systems as the memory left allows
    h->kept_sys = partial_keep ? partial_keep_count(h) : 0;
    double2* const* P = h->kry_ptrs;                 // device pointer array
    double2* V0 = reinterpret_cast<double2*>(h->ws_kry);
    auto Vp = [&](int i) { return V0 + (size_t)i * N; };
    auto Zp = [&](int i) { return V0 + (size_t)(m + 1 + i) * N; };
    double2* w = reinterpret_cast<double2*>(h->ws_big);
    double2* partial = reinterpret_cast<double2*>(h->kry_small);
    double2* hb = partial + krylov_partial_count();   // 4 coefficient buffers of KRY_MAXV
    const int MV = krylov_max_vectors();
    double* scal = h->ws_red;       // [0..3] residual scalars, [4..5] preconditioner scaling
    double* parts = h->ws_red + 8;
    double2* apsi0 = nullptr;
    if (psi0 && !adjoint) {
        apsi0 = vec_slot(h, 0);
        CUDA_TRY(launch_stencil_A(h->sm, psi0, false, nullptr, 1.0, apsi0, st));
    }
    const double* Bband = adjoint ? h->dt.BTb : h->dt.Bb;
    const double bsign = adjoint ? -1.0 : 1.0;
    // unit-norm basis vectors have entries ~ N^{-1/2}: scale by a power of two near sqrt(N) for FP32
    const double psc = std::ldexp(1.0, (int)std::lround(0.5 * std::log2((double)N)));
    CUDA_TRY(launch_set_scalars(scal + 4, psc, 1.0 / psc, st));
    CUDA_TRY(cudaMemsetAsync(psi, 0, N * sizeof(double2), st));
    CUDA_TRY(cudaMemsetAsync(h->ws_status, 0, 2 * sizeof(int), st));
    double2* x = reinterpret_cast<double2*>(psi);
    // the iterate's pointer after the basis, for its norm in the error estimate
    CUDA_TRY(cudaMemcpyAsync(const_cast<double2**>(P) + 2 * m + 2, &x, sizeof(double2*), cudaMemcpyHostToDevice, st));
    double hist[16];
    int nh = 0;
    int its = 0, reorth = 0;
    double bnorm = -1, rel = -1, err_est = -1;
    double cur_tol = tol;
    bool converged = false, first = true, x_zero = true;
    bool z0_ready = false;   // Z_0 = FDM32(V_0) of the current residual, left by a failed error estimate
    std::vector<cd> H((size_t)(m + 1) * m), g(m + 1), sn(m);
    std::vector<double> cs(m);
    std::vector<double2> hh(3 * MV);
    while (true) {
        CUDA_TRY(launch_residual(h->sm, n_t, time_band(h), h->dt.Mb, Bband, bsign, reinterpret_cast<const double2*>(F), apsi0,
                                 h->dt.m, x_zero ? nullptr : x, nullptr, w, parts, scal, st));
        double hs[2];
        CUDA_TRY(cudaMemcpyAsync(hs, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        const double beta = std::sqrt(hs[0]);
        if (bnorm < 0) bnorm = std::sqrt(hs[1]);
        rel = bnorm > 0 ? beta / bnorm : 0.0;
        if (nh < 15) hist[nh++] = rel;
        if (!std::isfinite(rel)) return fail(ST_ERR_NOT_CONVERGED, "refinement: non-finite residual");
        if (rel <= cur_tol || beta == 0.0) {
            if (!(o.err_tol > 0) || beta == 0.0) {
                converged = true;
                break;
            }
            if (its >= maxit) break;
            // error estimate: the FP32 FDM of the residual, relative to the iterate
            CUDA_TRY(launch_scale(w, 1.0 / beta, Vp(0), N, st));
            s = precond32(h, adjoint, Vp(0), Zp(0), keep, first, scal + 4, st);
            if (s != ST_OK) return s;
            ++its;
            CUDA_TRY(launch_multidot(P + m + 1, 1, Zp(0), N, partial, hb, st));
            CUDA_TRY(launch_multidot(P + 2 * m + 2, 1, x, N, partial, hb + MV, st));
            CUDA_TRY(cudaMemcpyAsync(hh.data(), hb, 2 * MV * sizeof(double2), cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            const double zz = std::max(0.0, hh[0].x), xx = std::max(0.0, hh[MV].x);
            err_est = xx > 0 ? beta * std::sqrt(zz / xx) : HUGE_VAL;
            if (err_est <= o.err_tol) {
                converged = true;
                break;
            }
            // lower the residual target by the factor the estimate is off, and keep iterating; the next
            // cycle starts from this residual, whose preconditioned direction is already in Z_0
            cur_tol = std::max(1e-16, std::min(0.5 * rel, rel * (0.5 * o.err_tol / err_est)));
            z0_ready = true;
            continue;
        }
        if (its >= maxit) break;
        CUDA_TRY(launch_scale(w, 1.0 / beta, Vp(0), N, st));
        std::fill(g.begin(), g.end(), cd(0));
        g[0] = beta;
        int jdone = 0;
        for (int j = 0; j < m; ++j) {
            if (j == 0 && z0_ready) {
                z0_ready = false;   // same iterate, same residual, same V_0: reuse its FDM32 application
            } else {
                s = precond32(h, adjoint, Vp(j), Zp(j), keep, first, scal + 4, st);
                if (s != ST_OK) return s;
                ++its;
            }
            // w = K z_j (operator apply: no right-hand side)
            CUDA_TRY(launch_residual(h->sm, n_t, time_band(h), h->dt.Mb, Bband, bsign, nullptr, nullptr, h->dt.m, Zp(j), nullptr,
                                     w, parts, scal, st));
            // Classical Gram-Schmidt on d = w - v_j, h = e_j + V^H d: with the FP32-FDM preconditioner
            // w = K z_j is close to v_j, and orthogonalising the small difference d instead of w keeps
            // the pass's rounding relative to ||d||, not ||w||.  A second pass runs only when the first
            // removed more than half of ||d||^2 (Daniel-Gragg-Kaufman-Stewart criterion).
            CUDA_TRY(launch_gs_project(P, j + 1, j, w, N, partial, hb, st));
            CUDA_TRY(launch_gs_update(P, j + 1, j, hb, w, N, partial, hb + 2 * MV, st));
            CUDA_TRY(cudaMemcpyAsync(hh.data(), hb, 3 * MV * sizeof(double2), cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            const double dd = hh[j + 1].x;
            double nn = hh[2 * MV].x;
            for (int i = 0; i <= j; ++i) hh[MV + i] = make_double2(0, 0);
            if (nn < 0.5 * dd) {
                ++reorth;
                CUDA_TRY(launch_gs_project(P, j + 1, -1, w, N, partial, hb + MV, st));
                CUDA_TRY(launch_gs_update(P, j + 1, -1, hb + MV, w, N, partial, hb + 2 * MV, st));
                CUDA_TRY(cudaMemcpyAsync(hh.data() + MV, hb + MV, 2 * MV * sizeof(double2), cudaMemcpyDeviceToHost, st));
                CUDA_TRY(cudaStreamSynchronize(st));
                nn = hh[2 * MV].x;
            }
            const double hn = std::sqrt(std::max(0.0, nn));
            for (int i = 0; i <= j; ++i)
                H[(size_t)i * m + j] = cd(hh[i].x + hh[MV + i].x + (i == j ? 1.0 : 0.0), hh[i].y + hh[MV + i].y);
            H[(size_t)(j + 1) * m + j] = hn;
            // previous rotations, then the new one (G = [[c, s], [-conj s, c]])
            for (int i = 0; i < j; ++i) {
                cd a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
                H[(size_t)(i + 1) * m + j] = -std::conj(sn[i]) * a + cs[i] * b;
            }
            {
                cd a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
                double aa = std::abs(a), ab = std::abs(b);
                if (ab == 0.0) {
                    cs[j] = 1.0;
                    sn[j] = 0.0;
                } else if (aa == 0.0) {
                    cs[j] = 0.0;
                    sn[j] = std::conj(b) / ab;
                } else {
                    double rho = std::hypot(aa, ab);
                    cs[j] = aa / rho;
                    sn[j] = (a / aa) * std::conj(b) / rho;
                }
                H[(size_t)j * m + j] = cs[j] * a + sn[j] * b;
                H[(size_t)(j + 1) * m + j] = 0.0;
                cd gj = g[j];
                g[j] = cs[j] * gj;
                g[j + 1] = -std::conj(sn[j]) * gj;
            }
            jdone = j + 1;
            const double est = std::abs(g[j + 1]) / bnorm;
            if (est <= 0.5 * cur_tol || j == m - 1 || its >= maxit || hn <= 1e-300) break;
            CUDA_TRY(launch_scale(w, 1.0 / hn, Vp(j + 1), N, st));
        }
        // y = R^{-1} g, x += Z y
        std::vector<cd> y(jdone);
        for (int i = jdone - 1; i >= 0; --i) {
            cd acc = g[i];
            for (int k = i + 1; k < jdone; ++k) acc -= H[(size_t)i * m + k] * y[k];
            y[i] = acc / H[(size_t)i * m + i];
        }
        std::vector<double2> yd(jdone);
        for (int i = 0; i < jdone; ++i) yd[i] = make_double2(y[i].real(), y[i].imag());
        CUDA_TRY(cudaMemcpyAsync(hb + 3 * MV, yd.data(), jdone * sizeof(double2), cudaMemcpyHostToDevice, st));
        CUDA_TRY(launch_multiaxpy(P + m + 1, jdone, hb + 3 * MV, 1.0, x, N, st));
        CUDA_TRY(cudaStreamSynchronize(st));  // yd lives on the host stack
        x_zero = false;
    }
    if (psi0 && !adjoint) CUDA_TRY(launch_add_row(n_t, n_x, psi, psi0, false, st));
    if (info) {
        info->sweeps = its;
        info->factors_kept = keep ? 1 : (h->kept_sys > 0 ? 2 : 0);
        info->restart = m;
        info->kept_systems = keep ? n_t : h->kept_sys;
        info->reorth_steps = reorth;
        info->rel_error_estimate = err_est;
        info->rel_residual = rel;
        for (int i = 0; i < 16; ++i) info->residual_history[i] = (i < nh) ? hist[i] : -1.0;
    }
    s = check_status_flag(h, st);
    if (s != ST_OK) return s;
    if (!converged) return fail(ST_ERR_NOT_CONVERGED, "refinement: tolerance not reached in max_sweeps");
    return ST_OK;
}

st_status adjoint_direct(st_fdm* h, bool fp32, const void* G, void* lambda, cudaStream_t st) {
    const int n_t = h->tm.n_t, n_x = h->sm.n_x;
    release_refinement_workspace(h);
    st_status s;
    if (!fp32) {
        s = grow(h->ws_big, h->ws_big_bytes, (size_t)n_t * n_x * sizeof(double2), "H");
        if (s != ST_OK) return s;
        double2* H = reinterpret_cast<double2*>(h->ws_big);
        s = xform<double, double, double, double>(reinterpret_cast<double*>(h->xf64[XF_XT]), n_t, n_x, G, H, 1, 0, 0,
                                                  nullptr, nullptr, nullptr, nullptr, nullptr, st);
        if (s != ST_OK) return s;
        s = band_run<double>(h, H, 0, st);
        if (s != ST_OK) return s;
        return xform<double, double, double, double>(reinterpret_cast<double*>(h->xf64[XF_YT]), n_t, n_x, H, lambda, 0,
                                                     1, 0, nullptr, nullptr, nullptr, nullptr, nullptr, st);
    }
    s = grow(h->ws_g32, h->ws_g32_bytes, (size_t)n_t * n_x * sizeof(float2), "H32");
    if (s != ST_OK) return s;
    float2* H = reinterpret_cast<float2*>(h->ws_g32);
    s = xform32(h, XF_XT, G, false, nullptr, 1, H, false, 0, 0, nullptr, nullptr, nullptr, nullptr, st);
    if (s != ST_OK) return s;
    s = band_run<float>(h, H, 0, st);
    if (s != ST_OK) return s;
    return xform32(h, XF_YT, H, false, nullptr, 0, lambda, false, 1, 0, nullptr, nullptr, nullptr, nullptr, st);
}

// ------------------------------------------------------------------ Bartels-Stewart (FP64)
// The Schur choice of step 1 (Section 3): (i B_t)^{-1} M_t = Z T Z^H with Z unitary and T upper
// triangular, so that with Psi_hat = Z W and G = Z^H (i B_t)^{-1} F~ the spatial problems of eq. LGS_x
// couple through T:
//     (M_x + T_ll A_x) w_l = g_l - A_x sum_{k > l} T_lk w_k,     l = n_t - 1, ..., 0.
// All n_t spatial matrices are factorised at once (the FDM's kernels, at the shifts T_ll, factors
// kept); the coupled solves then run one system at a time from the last, each followed by a rank-one
// update of the couplings of all earlier rows.  A reference path: robust where X_t is
// ill-conditioned, with no time parallelism in its solves.
st_status bs_prepare(st_fdm* h) {
    if (h->bs_Z) return ST_OK;
    const int n = h->tm.n_t;
    const TimeDecomp& td = h->td;
    if (td.Zs.size() != (size_t)n * n || td.Ts.size() != (size_t)n * n || td.Binv.size() != (size_t)n * n)
        return fail(ST_ERR_ARG, "Bartels-Stewart: no Schur form");
    std::vector<cd> Z((size_t)n * n), T((size_t)n * n, cd(0.0)), Y((size_t)n * n), sh(n), ym(n, cd(0.0));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            Z[(size_t)i * n + j] = td.Zs[i + (size_t)j * n];
            if (i <= j) T[(size_t)i * n + j] = td.Ts[i + (size_t)j * n];
        }
    for (int i = 0; i < n; ++i) sh[i] = td.Ts[i + (size_t)i * n];
    // Y = Z^H (i B_t)^{-1} = Z^H (-i B_t^{-1})
    {
        const int nth = std::max(1, std::min<int>(16, (int)std::thread::hardware_concurrency()));
        std::vector<std::thread> pool;
        for (int t = 0; t < nth; ++t)
            pool.emplace_back([&, t]() {
                for (int i = t; i < n; i += nth)
                    for (int j = 0; j < n; ++j) {
                        cd acc = 0.0;
                        for (int k = 0; k < n; ++k) acc += std::conj(td.Zs[k + (size_t)i * n]) * td.Binv[k + (size_t)j * n];
                        Y[(size_t)i * n + j] = cd(0.0, -1.0) * acc;
                    }
            });
        for (auto& th : pool) th.join();
    }
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) ym[i] += Y[(size_t)i * n + k] * h->tm.m[k];
    st_status s = upload(&h->bs_Z, Z.data(), Z.size() * sizeof(double2), "Schur Z");
    if (s == ST_OK) s = upload(&h->bs_Y, Y.data(), Y.size() * sizeof(double2), "Schur Y");
    if (s == ST_OK) s = upload(&h->bs_T, T.data(), T.size() * sizeof(double2), "Schur T");
    if (s == ST_OK) s = upload(&h->bs_shift, sh.data(), sh.size() * sizeof(double2), "Schur shifts");
    if (s == ST_OK) s = upload(&h->bs_Ym, ym.data(), ym.size() * sizeof(double2), "Schur Y m_t");
    if (s != ST_OK) {
        cudaFree(h->bs_Z);
        h->bs_Z = nullptr;
    }
    return s;
}

// w_l = C_l^{-1} w_l with the kept FP64 factors of system l (row l of W)
st_status bs_solve_one(st_fdm* h, double2* W, int l, cudaStream_t st) {
    if (h->spatial == 1) {
        MfArgs<double> a = mf_args<double>(h, W);
        a.fac_keep = 1;
        CUDA_TRY(mf_levels<double>(h, a, l, 1, 1, st));
        CUDA_TRY(mf_levels<double>(h, a, l, 1, 2, st));
        return ST_OK;
    }
    BandArgs<double> a = band_args<double>(h, W);
    a.L = reinterpret_cast<double2*>(h->ws_L);
    a.D = reinterpret_cast<double2*>(h->ws_D);
    a.keep = 1;
    CUDA_TRY(subst_launch<double>(a, l, 1, true, st));
    CUDA_TRY(subst_launch<double>(a, l, 1, false, st));
    return ST_OK;
}

st_status bs_solve(st_fdm* h, const void* F, const void* psi0, void* psi, cudaStream_t st) {
    const int n_t = h->tm.n_t, n_x = h->sm.n_x;
    const size_t N = (size_t)n_t * n_x;
    release_refinement_workspace(h);
    st_status s = bs_prepare(h);
    if (s == ST_OK) s = ensure_common(h);
    if (s == ST_OK) s = grow(h->ws_big, h->ws_big_bytes, N * sizeof(double2), "G");
    if (s == ST_OK) s = grow(h->bs_w, h->bs_w_bytes, N * sizeof(double2), "Bartels-Stewart W");
    if (s != ST_OK) return s;
    double2* G = reinterpret_cast<double2*>(h->ws_big);
    double2* W = reinterpret_cast<double2*>(h->bs_w);
    double2* tmp = vec_slot(h, 2);
    double2* apsi0 = nullptr;
    if (psi0) {
        apsi0 = vec_slot(h, 0);
        CUDA_TRY(launch_stencil_A(h->sm, psi0, false, nullptr, 1.0, apsi0, st));
    }
    s = xform<double, double, double, double>(reinterpret_cast<double*>(h->bs_Y), n_t, n_x, F, G, 0, 0, 0, nullptr,
                                              nullptr, nullptr, psi0 ? h->bs_Ym : nullptr, apsi0, st);
    if (s != ST_OK) return s;
    // factorise every C_l = M_x + T_ll A_x into kept storage (on zero right-hand sides)
    CUDA_TRY(cudaMemsetAsync(W, 0, N * sizeof(double2), st));
    h->shift_override = h->bs_shift;
    s = band_run<double>(h, W, 1, st);
    h->shift_override = nullptr;
    if (s == ST_OK) {
        CUDA_TRY(cudaMemsetAsync(W, 0, N * sizeof(double2), st));
        for (int l = n_t - 1; l >= 0 && s == ST_OK; --l) {
            double2* wl = W + (size_t)l * n_x;
            // right-hand side g_l - A_x (sum_{k>l} T_lk w_k), the sum accumulated in row l
            CUDA_TRY(launch_stencil_A(h->sm, wl, false, G + (size_t)l * n_x, -1.0, tmp, st));
            CUDA_TRY(cudaMemcpyAsync(wl, tmp, (size_t)n_x * sizeof(double2), cudaMemcpyDeviceToDevice, st));
            s = bs_solve_one(h, W, l, st);
            if (s == ST_OK) CUDA_TRY(launch_bs_accum(n_t, n_x, l, h->bs_T, W, st));
        }
    }
    // the kept factors belong to the Schur shifts, not to the eigenvalues of the FDM
    h->factors_valid = 0;
    if (s != ST_OK) return s;
    return xform<double, double, double, double>(reinterpret_cast<double*>(h->bs_Z), n_t, n_x, W, psi, 0, 0, 0, nullptr,
                                                 nullptr, psi0, nullptr, nullptr, st);
}

st_status validate_opts(const st_solve_opts* o, st_solve_opts& out) {
    st_solve_opts d;
    std::memset(&d, 0, sizeof(d));
    d.precision = ST_FP64;
    d.keep_factors = -1;
    out = o ? *o : d;
    if (out.precision != ST_FP64 && out.precision != ST_FP32 && out.precision != ST_MIXED)
        return fail(ST_ERR_ARG, "solve: unknown precision");
    if (out.method != ST_REFINE_GMRES && out.method != ST_REFINE_CLASSIC)
        return fail(ST_ERR_ARG, "solve: unknown refinement method");
    return ST_OK;
}

void fill_info_common(const st_fdm* h, st_solve_info* info, int precision) {
    if (!info) return;
    info->kappa_x = h->td.kappa;
    info->min_neg_im_shift = h->td.min_neg_im;
    info->setup_seconds = h->setup_seconds;
    info->tensor_cores = (precision != ST_FP64 && h->tc_ok) ? 1 : 0;
    info->restart = 0;
    info->kept_systems = 0;
    info->reorth_steps = 0;
    info->rel_error_estimate = -1;
}

}  // namespace

// Spatial side of a handle: the device CSR of a general mesh, and the multifrontal plan when the
// sparse-direct solver is used (general meshes always; structured grids on request).
st_status setup_spatial(st_fdm* h, int choice) {
    if (choice < 0 || choice > ST_SPATIAL_MULTIFRONTAL) return fail(ST_ERR_ARG, "st_fdm_setup: unknown spatial solver");
    if (h->sm.kind == 1 && choice == ST_SPATIAL_BANDED)
        return fail(ST_ERR_UNSUPPORTED, "st_fdm_setup: the banded spatial solver needs a structured grid");
    st_status s = ST_OK;
    if (h->sm.kind == 1) {
        const MeshSpace& ms = h->sm.mesh;
        s = upload(&h->csr_rowptr, ms.rowptr.data(), ms.rowptr.size() * sizeof(int), "CSR rows");
        if (s == ST_OK) s = upload(&h->csr_col, ms.col.data(), ms.col.size() * sizeof(int), "CSR columns");
        if (s == ST_OK) s = upload(&h->csr_M, ms.Mv.data(), ms.Mv.size() * sizeof(double), "CSR M_x");
        if (s == ST_OK) s = upload(&h->csr_A, ms.Av.data(), ms.Av.size() * sizeof(double), "CSR A_x");
        if (s != ST_OK) return s;
        h->sm.d_rowptr = h->csr_rowptr;
        h->sm.d_col = h->csr_col;
        h->sm.d_M = h->csr_M;
        h->sm.d_A = h->csr_A;
    }
    h->spatial = (h->sm.kind == 1 || choice == ST_SPATIAL_MULTIFRONTAL) ? 1 : 0;
    if (!h->spatial) return ST_OK;
    MeshSpace tmp;
    const MeshSpace* ms = &h->sm.mesh;
    if (h->sm.kind == 0) {
        structured_as_mesh(h->sm, tmp);
        ms = &tmp;
        std::vector<double> v(ms->Mv);
        v.insert(v.end(), ms->Av.begin(), ms->Av.end());
        h->mf_csrv_nnz = (long long)ms->Mv.size();
        s = upload(&h->mf_csrv, v.data(), v.size() * sizeof(double), "plan CSR values");
        if (s != ST_OK) return s;
    }
    try {
        s = build_mf_plan(*ms, MF_DEFAULT_LEAF, h->mf);
    } catch (const std::bad_alloc&) {
        return fail(ST_ERR_OOM, "st_fdm_setup: multifrontal plan (host)");
    }
    if (s != ST_OK) return s;
    const MfPlan& P = h->mf;
    if (((size_t)P.max_front + 32 * 33) * sizeof(double2) > h->smem_optin)
        return fail(ST_ERR_UNSUPPORTED, "st_fdm_setup: a front of the sparse-direct solver exceeds shared memory");
    std::vector<MfFrontDev> fd(P.fronts.size());
    for (size_t i = 0; i < P.fronts.size(); ++i) {
        const MfFront& f = P.fronts[i];
        fd[i] = MfFrontDev{f.first, f.np, f.nu, f.parent, f.foff, f.uoff, f.uvoff,
                           f.urows_off, f.relpos_off, f.orig_off, f.orig_cnt, f.child_off, f.child_cnt};
    }
    s = upload(&h->mf_fronts, fd.data(), fd.size() * sizeof(MfFrontDev), "plan fronts");
    if (s != ST_OK) return s;
    const std::vector<int>* parts[8] = {&P.perm, &P.urows, &P.relpos, &P.children, &P.orig_r, &P.orig_c, &P.orig_k,
                                        &P.level_fronts};
    std::vector<int> all;
    size_t offs[8];
    for (int i = 0; i < 8; ++i) {
        offs[i] = all.size();
        all.insert(all.end(), parts[i]->begin(), parts[i]->end());
    }
    all.push_back(0);
    s = upload(&h->mf_ints, all.data(), all.size() * sizeof(int), "plan indices");
    if (s != ST_OK) return s;
    h->mf_perm = h->mf_ints + offs[0];
    h->mf_urows = h->mf_ints + offs[1];
    h->mf_relpos = h->mf_ints + offs[2];
    h->mf_children = h->mf_ints + offs[3];
    h->mf_orig_r = h->mf_ints + offs[4];
    h->mf_orig_c = h->mf_ints + offs[5];
    h->mf_orig_k = h->mf_ints + offs[6];
    h->mf_level = h->mf_ints + offs[7];
    return ST_OK;
}

// ==================================================================== setup
extern "C" st_status st_fdm_setup(const st_time* t, const st_space* sp, const st_setup_opts* opts, st_fdm** out) {
    if (!out) return fail(ST_ERR_ARG, "st_fdm_setup: out is NULL");
    *out = nullptr;
    if (!t || !sp) return fail(ST_ERR_ARG, "st_fdm_setup: NULL time or space handle");
    st_setup_opts o;
    std::memset(&o, 0, sizeof(o));
    o.device = -1;
    if (opts) o = *opts;
    const double kappa_max = o.kappa_max > 0 ? o.kappa_max : 1e10;
    st_fdm* h = new (std::nothrow) st_fdm();
    if (!h) return fail(ST_ERR_OOM, "st_fdm_setup: host allocation");
    h->tm = t->tm;
    h->sm = sp->sm;
    auto t0 = std::chrono::steady_clock::now();
    st_status s = time_decompose(h->tm, o.host_threads, h->td);
    h->setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (s != ST_OK) {
        delete h;
        return s;
    }
    if (!(h->td.kappa <= kappa_max)) {
        double k = h->td.kappa;
        delete h;
        return fail(ST_ERR_ILL_CONDITIONED, "st_fdm_setup: kappa_2(X_t) = " + std::to_string(k) + " exceeds kappa_max");
    }
    {
        // Im s_k < 0 in exact arithmetic whenever the eigenvector has v_N != 0; eigenvectors
        // localised away from t = T (graded meshes) give |Im s_k| at rounding level, i.e.
        // numerically real shifts.  Only an imaginary part clearly of the wrong sign is rejected.
        double smax = 0;
        for (const auto& v : h->td.s) smax = std::max(smax, std::abs(v));
        if (!(h->td.min_neg_im >= -1e-8 * smax)) {
            delete h;
            return fail(ST_ERR_ILL_CONDITIONED, "st_fdm_setup: an eigenvalue has Im s_k > 0");
        }
    }
    int dev = o.device;
    if (dev < 0) {
        if (cudaGetDevice(&dev) != cudaSuccess) {
            delete h;
            cudaGetLastError();
            return fail(ST_ERR_CUDA, "st_fdm_setup: no CUDA device");
        }
    }
    h->device = dev;
    DeviceGuard g(dev);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        delete h;
        cudaGetLastError();
        return fail(ST_ERR_CUDA, "st_fdm_setup: cudaGetDeviceProperties failed");
    }
    if (prop.major < 10) {
        delete h;
        return fail(ST_ERR_UNSUPPORTED, "st_fdm_setup: the library is built for sm_103a (GB300)");
    }
    h->sm_count = prop.multiProcessorCount;
    h->smem_optin = prop.sharedMemPerBlockOptin;
    const int n = h->tm.n_t;
    const size_t nn = (size_t)n * n;
    // transform matrices: Y, X, X^T, Y^T (row-major), FP64 and FP32
    std::vector<cd> mats[4];
    mats[XF_Y] = h->td.Y;
    mats[XF_X] = h->td.X;
    mats[XF_XT].resize(nn);
    mats[XF_YT].resize(nn);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            mats[XF_XT][(size_t)i * n + j] = h->td.X[(size_t)j * n + i];
            mats[XF_YT][(size_t)i * n + j] = h->td.Y[(size_t)j * n + i];
        }
    std::vector<float2> f32(nn);
    for (int w = 0; w < 4 && s == ST_OK; ++w) {
        s = upload(&h->xf64[w], mats[w].data(), nn * sizeof(double2), "transform (FP64)");
        if (s != ST_OK) break;
        for (size_t i = 0; i < nn; ++i) f32[i] = make_float2((float)mats[w][i].real(), (float)mats[w][i].imag());
        s = upload(&h->xf32[w], f32.data(), nn * sizeof(float2), "transform (FP32)");
    }
    // tensor-core transforms (sm_100 family): hi/lo TF32 splits of the four transform matrices
    if (s == ST_OK && prop.major == 10) {
        h->tc_M_pad = tc_round_up(n, 128);
        h->tc_K_pad = tc_round_up(n, 32);
        h->tc_N2_pad = tc_round_up(2 * h->sm.n_x, 128);
        std::vector<float> sp((size_t)4 * h->tc_M_pad * h->tc_K_pad);
        bool ok = true;
        for (int w = 0; w < 4 && s == ST_OK && ok; ++w) {
            tc_split_matrix(mats[w].data(), n, h->tc_M_pad, h->tc_K_pad, sp.data());
            s = upload(&h->tc_A[w], sp.data(), sp.size() * sizeof(float), "tensor-core transform");
            if (s == ST_OK) ok = tc_make_map(&h->tc_mapA[w], h->tc_A[w], 4 * h->tc_M_pad, h->tc_K_pad);
        }
        h->tc_ok = (s == ST_OK && ok) ? 1 : 0;
    }
    std::vector<float2> s32(n);
    for (int k = 0; k < n; ++k) s32[k] = make_float2((float)h->td.s[k].real(), (float)h->td.s[k].imag());
    std::vector<cd> ym(n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) ym[i] += h->td.Y[(size_t)i * n + k] * h->tm.m[k];
    std::vector<double> BT((size_t)n * 5, 0.0);
    for (int l = 0; l < n; ++l)
        for (int d = -2; d <= 2; ++d) {
            int c = l + d;
            if (c < 0 || c >= n) continue;
            // B^T[l][c] = B[c][l] = Bb[c][l - c + 2]
            BT[(size_t)l * 5 + d + 2] = h->tm.Bb[(size_t)c * 5 + (l - c) + 2];
        }
    if (s == ST_OK) s = upload(&h->s64, h->td.s.data(), n * sizeof(double2), "shifts");
    if (s == ST_OK) s = upload(&h->s32, s32.data(), n * sizeof(float2), "shifts32");
    if (s == ST_OK) s = upload(&h->Ym64, ym.data(), n * sizeof(double2), "Y m_t");
    if (s == ST_OK) s = upload(&h->dt.Mb, h->tm.Mb.data(), (size_t)n * 5 * sizeof(double), "M_t band");
    if (s == ST_OK) s = upload(&h->dt.Bb, h->tm.Bb.data(), (size_t)n * 5 * sizeof(double), "B_t band");
    if (s == ST_OK) s = upload(&h->dt.BTb, BT.data(), (size_t)n * 5 * sizeof(double), "B_t^T band");
    if (s == ST_OK) s = upload(&h->dt.Mfull0, h->tm.Mfull0.data(), (size_t)n * sizeof(double), "M_t col 0");
    if (s == ST_OK) s = upload(&h->dt.m, h->tm.m.data(), (size_t)n * sizeof(double), "m_t");
    if (s == ST_OK)
        s = upload(&h->dt.nodes, h->tm.nodes.data(), h->tm.nodes.size() * sizeof(double), "time mesh nodes");
    if (s == ST_OK) {
        size_t parts = (size_t)residual_num_partials(n, h->sm.n_x);
        s = grow(*reinterpret_cast<void**>(&h->ws_red), h->ws_red_bytes, (8 + 2 * parts) * sizeof(double), "reduction");
    }
    if (s == ST_OK) s = setup_spatial(h, o.spatial_solver);
    if (s == ST_OK) s = dev_alloc(reinterpret_cast<void**>(&h->ws_status), sizeof(int) * 4, "status");
    if (s == ST_OK && cudaMemset(h->ws_status, 0, sizeof(int) * 4) != cudaSuccess)
        s = fail(ST_ERR_CUDA, "st_fdm_setup: cudaMemset");
    if (s != ST_OK) {
        free_handle(h);
        return s;
    }
    *out = h;
    return ST_OK;
}

extern "C" st_status st_fdm_get(const st_fdm* h, int* n_t, int* n_x, int* m, double* kappa2, double* min_neg_im) {
    if (!h) return fail(ST_ERR_ARG, "st_fdm_get: NULL handle");
    if (n_t) *n_t = h->tm.n_t;
    if (n_x) *n_x = h->sm.n_x;
    if (m) *m = h->sm.m;
    if (kappa2) *kappa2 = h->td.kappa;
    if (min_neg_im) *min_neg_im = h->td.min_neg_im;
    return ST_OK;
}

extern "C" void st_destroy_fdm(st_fdm* h) { free_handle(h); }

// ==================================================================== solves
static st_status fdm_solve_impl(st_fdm* h, const void* F, const void* psi0, void* psi, const st_solve_opts* opts,
                                st_solve_info* info, void* stream) {
    if (!h) return fail(ST_ERR_ARG, "st_fdm_solve: NULL handle");
    if (!F || !psi) return fail(ST_ERR_ARG, "st_fdm_solve: NULL F or psi");
    if (F == psi) return fail(ST_ERR_ARG, "st_fdm_solve: psi must not alias F");
    st_solve_opts o;
    st_status s = validate_opts(opts, o);
    if (s != ST_OK) return s;
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    fill_info_common(h, info, o.precision);
    if (o.precision == ST_MIXED) {
        if (o.fixed_sweeps > 0 || o.method == ST_REFINE_CLASSIC) return solve_mixed(h, false, F, psi0, psi, o, info, st);
        return solve_mixed_gmres(h, false, F, psi0, psi, o, info, st);
    }
    CUDA_TRY(cudaMemsetAsync(h->ws_status, 0, 2 * sizeof(int), st));
    s = (o.precision == ST_FP64) ? solve_fp64(h, F, psi0, psi, st) : solve_fp32(h, F, psi0, psi, st);
    if (s != ST_OK) return s;
    if (info) {
        info->sweeps = 1;
        info->factors_kept = 0;
        info->rel_residual = -1;
        for (int i = 0; i < 16; ++i) info->residual_history[i] = -1;
        return check_status_flag(h, st);
    }
    return ST_OK;
}

extern "C" st_status st_fdm_solve(st_fdm* h, const void* F, const void* psi0, void* psi, const st_solve_opts* opts,
                                  st_solve_info* info, void* stream) {
    const long long l0 = launches_issued();
    const st_status s = fdm_solve_impl(h, F, psi0, psi, opts, info, stream);
    if (info) info->kernel_launches = (int)(launches_issued() - l0);
    return s;
}

extern "C" st_status st_residual(st_fdm* h, const void* F, const void* psi0, const void* psi, void* R,
                                 double* rel_norm, void* stream) {
    if (!h || !F || !psi) return fail(ST_ERR_ARG, "st_residual: NULL argument");
    // R is written while other threads still read the stencil neighbours of psi and psi0
    if (R && (R == psi || R == psi0)) return fail(ST_ERR_ARG, "st_residual: R must not alias psi or psi0");
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    st_status s = ensure_common(h);
    if (s != ST_OK) return s;
    double2* apsi0 = nullptr;
    if (psi0) {
        apsi0 = vec_slot(h, 1);
        CUDA_TRY(launch_stencil_A(h->sm, psi0, false, nullptr, 1.0, apsi0, st));
    }
    double* scal = h->ws_red + 4;
    double* parts = h->ws_red + 8;
    CUDA_TRY(launch_residual(h->sm, h->tm.n_t, time_band(h), h->dt.Mb, h->dt.Bb, 1.0, reinterpret_cast<const double2*>(F), apsi0,
                             h->dt.m, reinterpret_cast<const double2*>(psi), reinterpret_cast<const double2*>(psi0),
                             reinterpret_cast<double2*>(R), parts, scal, st));
    if (rel_norm) {
        double hs[2];
        CUDA_TRY(cudaMemcpyAsync(hs, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        *rel_norm = hs[1] > 0 ? std::sqrt(hs[0] / hs[1]) : 0.0;
    }
    return ST_OK;
}

static st_status adjoint_solve_impl(st_fdm* h, const void* G, void* lambda, const st_solve_opts* opts,
                                    st_solve_info* info, void* stream) {
    if (!h || !G || !lambda) return fail(ST_ERR_ARG, "st_adjoint_solve: NULL argument");
    if (G == lambda) return fail(ST_ERR_ARG, "st_adjoint_solve: lambda must not alias G");
    st_solve_opts o;
    st_status s = validate_opts(opts, o);
    if (s != ST_OK) return s;
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    fill_info_common(h, info, o.precision);
    if (o.precision == ST_MIXED) {
        if (o.fixed_sweeps > 0 || o.method == ST_REFINE_CLASSIC) return solve_mixed(h, true, G, nullptr, lambda, o, info, st);
        return solve_mixed_gmres(h, true, G, nullptr, lambda, o, info, st);
    }
    CUDA_TRY(cudaMemsetAsync(h->ws_status, 0, 2 * sizeof(int), st));
    s = adjoint_direct(h, o.precision == ST_FP32, G, lambda, st);
    if (s != ST_OK) return s;
    if (info) {
        info->sweeps = 1;
        info->factors_kept = 0;
        info->rel_residual = -1;
        for (int i = 0; i < 16; ++i) info->residual_history[i] = -1;
        return check_status_flag(h, st);
    }
    return ST_OK;
}

extern "C" st_status st_adjoint_solve(st_fdm* h, const void* G, void* lambda, const st_solve_opts* opts,
                                      st_solve_info* info, void* stream) {
    const long long l0 = launches_issued();
    const st_status s = adjoint_solve_impl(h, G, lambda, opts, info, stream);
    if (info) info->kernel_launches = (int)(launches_issued() - l0);
    return s;
}

extern "C" st_status st_adjoint_lift(st_fdm* h, const void* grad_psi, const void* grad_F, void* grad_psi0,
                                     void* stream) {
    if (!h || !grad_psi || !grad_F || !grad_psi0) return fail(ST_ERR_ARG, "st_adjoint_lift: NULL argument");
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    st_status s = ensure_common(h);
    if (s != ST_OK) return s;
    double2* s1 = vec_slot(h, 2);
    double2* s2 = vec_slot(h, 3);
    CUDA_TRY(launch_colsums(h->tm.n_t, h->sm.n_x, reinterpret_cast<const double2*>(grad_psi),
                            reinterpret_cast<const double2*>(grad_F), h->dt.m, s1, s2, st));
    CUDA_TRY(launch_stencil_A(h->sm, s2, false, s1, -1.0, reinterpret_cast<double2*>(grad_psi0), st));
    return ST_OK;
}

extern "C" st_status st_bs_solve(st_fdm* h, const void* F, const void* psi0, void* psi, st_solve_info* info,
                                 void* stream) {
    if (!h || !F || !psi) return fail(ST_ERR_ARG, "st_bs_solve: NULL argument");
    if (F == psi) return fail(ST_ERR_ARG, "st_bs_solve: psi must not alias F");
    const long long l0 = launches_issued();
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    fill_info_common(h, info, ST_FP64);
    CUDA_TRY(cudaMemsetAsync(h->ws_status, 0, 2 * sizeof(int), st));
    st_status s = bs_solve(h, F, psi0, psi, st);
    if (s == ST_OK && info) {
        info->sweeps = 1;
        info->factors_kept = 1;
        info->kept_systems = h->tm.n_t;
        info->rel_residual = -1;
        for (int i = 0; i < 16; ++i) info->residual_history[i] = -1;
        s = check_status_flag(h, st);
    }
    if (info) info->kernel_launches = (int)(launches_issued() - l0);
    return s;
}

extern "C" st_status st_time_transform(st_fdm* h, int which, int precision, const void* in, void* out, void* stream) {
    if (!h || !in || !out) return fail(ST_ERR_ARG, "st_time_transform: NULL argument");
    if (in == out) return fail(ST_ERR_ARG, "st_time_transform: out must not alias in");
    if (which < 0 || which > 3) return fail(ST_ERR_ARG, "st_time_transform: bad selector");
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    const int n_t = h->tm.n_t, n_x = h->sm.n_x;
    if (precision == ST_FP64)
        return xform<double, double, double, double>(reinterpret_cast<double*>(h->xf64[which]), n_t, n_x, in, out, 0,
                                                     0, 0, nullptr, nullptr, nullptr, nullptr, nullptr, st);
    if (precision == ST_FP32)
        return xform<float, float, float, float>(reinterpret_cast<float*>(h->xf32[which]), n_t, n_x, in, out, 0, 0, 0,
                                                 nullptr, nullptr, nullptr, nullptr, nullptr, st);
    if (precision == ST_MIXED) {
        CUDA_TRY(cudaMemsetAsync(h->ws_status, 0, 2 * sizeof(int), st));
        st_status s = xform32(h, which, in, false, nullptr, 0, out, false, 0, 0, nullptr, nullptr, nullptr, nullptr, st);
        if (s != ST_OK) return s;
        return check_status_flag(h, st);
    }
    return fail(ST_ERR_ARG, "st_time_transform: unknown precision");
}

extern "C" st_status st_spatial_solve(st_fdm* h, int precision, const void* G, void* W, void* stream) {
    if (!h || !G || !W) return fail(ST_ERR_ARG, "st_spatial_solve: NULL argument");
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    const size_t elems = (size_t)h->tm.n_t * h->sm.n_x;
    const size_t esz = precision == ST_FP64 ? sizeof(double2) : sizeof(float2);
    if (precision != ST_FP64 && precision != ST_FP32 && precision != ST_MIXED)
        return fail(ST_ERR_ARG, "st_spatial_solve: unknown precision");
    release_refinement_workspace(h);
    if (W != G) CUDA_TRY(cudaMemcpyAsync(W, G, elems * esz, cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(cudaMemsetAsync(h->ws_status, 0, 2 * sizeof(int), st));
    st_status s = (precision == ST_FP64) ? band_run<double>(h, reinterpret_cast<double2*>(W), 0, st)
                                         : band_run<float>(h, reinterpret_cast<float2*>(W), 0, st);
    if (s != ST_OK) return s;
    return check_status_flag(h, st);
}

extern "C" st_status st_spatial_factor(st_fdm* h, int precision, void* stream) {
    if (!h) return fail(ST_ERR_ARG, "st_spatial_factor: NULL argument");
    if (precision != ST_FP64 && precision != ST_FP32) return fail(ST_ERR_ARG, "st_spatial_factor: FP64 or FP32");
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    release_refinement_workspace(h);
    const size_t elems = (size_t)h->tm.n_t * h->sm.n_x;
    const size_t esz = precision == ST_FP64 ? sizeof(double2) : sizeof(float2);
    // the factorisation runs with its fused (or following) substitutions on a zero right-hand side
    st_status s = grow(h->ws_big, h->ws_big_bytes, elems * esz, "scratch right-hand side");
    if (s != ST_OK) return s;
    CUDA_TRY(cudaMemsetAsync(h->ws_big, 0, elems * esz, st));
    CUDA_TRY(cudaMemsetAsync(h->ws_status, 0, 2 * sizeof(int), st));
    h->kept_sys = 0;
    s = (precision == ST_FP64) ? band_run<double>(h, reinterpret_cast<double2*>(h->ws_big), 1, st)
                               : band_run<float>(h, reinterpret_cast<float2*>(h->ws_big), 1, st);
    if (s != ST_OK) return s;
    return check_status_flag(h, st);
}

extern "C" st_status st_spatial_substitute(st_fdm* h, int precision, const void* G, void* W, void* stream) {
    if (!h || !G || !W) return fail(ST_ERR_ARG, "st_spatial_substitute: NULL argument");
    if (precision != ST_FP64 && precision != ST_FP32) return fail(ST_ERR_ARG, "st_spatial_substitute: FP64 or FP32");
    const size_t esz = precision == ST_FP64 ? sizeof(double2) : sizeof(float2);
    if (!h->factors_valid || h->factors_prec != (int)(esz / 2) || h->kept_sys != 0)
        return fail(ST_ERR_ARG, "st_spatial_substitute: no kept factors of this precision (call st_spatial_factor)");
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    const size_t elems = (size_t)h->tm.n_t * h->sm.n_x;
    if (W != G) CUDA_TRY(cudaMemcpyAsync(W, G, elems * esz, cudaMemcpyDeviceToDevice, st));
    st_status s = (precision == ST_FP64) ? band_run<double>(h, reinterpret_cast<double2*>(W), 2, st)
                                         : band_run<float>(h, reinterpret_cast<float2*>(W), 2, st);
    if (s != ST_OK) return s;
    return check_status_flag(h, st);
}

extern "C" st_status st_load_nodal(st_fdm* h, const void* f_nodal, void* F, void* stream) {
    if (!h || !f_nodal || !F) return fail(ST_ERR_ARG, "st_load_nodal: NULL argument");
    if (h->tm.n_t > 65535) return fail(ST_ERR_UNSUPPORTED, "st_load_nodal: n_t > 65535");
    DeviceGuard g(h->device);
    CUDA_TRY(launch_load_nodal(h->sm, h->tm.n_t, h->dt.Mb, h->dt.Mfull0, reinterpret_cast<const double2*>(f_nodal),
                               reinterpret_cast<double2*>(F), S(stream)));
    return ST_OK;
}


extern "C" st_status st_set_wait_probe(st_fdm* h, double seconds) {
    if (!h) return fail(ST_ERR_ARG, "st_set_wait_probe: NULL handle");
    if (!(seconds >= 0.0) || seconds > 1.0) return fail(ST_ERR_ARG, "st_set_wait_probe: seconds must be in [0, 1]");
    h->wait_probe_ns = (unsigned long long)(seconds * 1e9);
    return ST_OK;
}
