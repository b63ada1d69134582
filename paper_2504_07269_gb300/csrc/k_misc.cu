// Kernels around the three solver steps:
//   * A_x applied to a spatial vector (lifting, eq. VF_FEM: F~ = F - m_t (x) A_x psi0);
//   * the FP64 Kronecker residual R = F~ - K U, K = i B_t (x) M_x + M_t (x) A_x (eq. LGS),
//     fused with the 2-norm partial sums of R and F~ (and its adjoint K^H);
//   * deterministic two-level norm reduction and refinement scaling;
//   * psi = psi_hat + psi0;  the interpolated load (M_t,full (x) M_x) f;  weighted column sums.
// All space-time arrays are (n_t, n_x) row-major complex; spatial nodes are x1-fastest with
// m per grid row; the 7-point stencil (W, E, S, N, SW, NE) is zero outside the grid.
#include <cuda_runtime.h>

#include "device.cuh"

namespace stfdm {

struct Stencil {
    int m;
    double Mc, Mw, Ms, Md, Ac, Aw, As, Ad;
};

template <typename TI>
__device__ __forceinline__ void stencil_MA(const Stencil& s, const C<TI>* u, int x, double2& Pm, double2& Qa) {
    const int m = s.m;
    const int xi = x % m, yj = x / m;
    auto ld = [&](int idx) {
        C<TI> v = u[idx];
        return make_double2((double)v.x, (double)v.y);
    };
    // neighbours outside the grid read as zero; each pair is one addition (the FP64 pipe bounds the
    // kernels that call this on GB300)
    const double2 z = make_double2(0, 0);
    const bool w_ = xi > 0, e_ = xi < m - 1, s_ = yj > 0, n_ = yj < m - 1;
    const double2 c = ld(x);
    const double2 vw = w_ ? ld(x - 1) : z, ve = e_ ? ld(x + 1) : z;
    const double2 vs = s_ ? ld(x - m) : z, vn = n_ ? ld(x + m) : z;
    const double2 vsw = (w_ && s_) ? ld(x - m - 1) : z, vne = (e_ && n_) ? ld(x + m + 1) : z;
    const double2 we = make_double2(vw.x + ve.x, vw.y + ve.y);
    const double2 sn = make_double2(vs.x + vn.x, vs.y + vn.y);
    const double2 dg = make_double2(vsw.x + vne.x, vsw.y + vne.y);
    Pm.x = s.Mc * c.x + s.Mw * we.x + s.Ms * sn.x + s.Md * dg.x;
    Pm.y = s.Mc * c.y + s.Mw * we.y + s.Ms * sn.y + s.Md * dg.y;
    Qa.x = s.Ac * c.x + s.Aw * we.x + s.As * sn.x;
    Qa.y = s.Ac * c.y + s.Aw * we.y + s.As * sn.y;
    if (s.Ad != 0.0) {   // zero for the squares' right triangles (right angle opposite the diagonal)
        Qa.x = fma(s.Ad, dg.x, Qa.x);
        Qa.y = fma(s.Ad, dg.y, Qa.y);
    }
}

// General meshes: M_x and A_x in CSR over the interior DOFs (one pattern for both).
struct Csr {
    int m;   // unused (keeps the interface of Stencil)
    const int* rowptr;
    const int* col;
    const double* M;
    const double* A;
};

template <typename TI>
__device__ __forceinline__ void stencil_MA(const Csr& s, const C<TI>* u, int x, double2& Pm, double2& Qa) {
    double2 p = make_double2(0, 0), q = make_double2(0, 0);
    for (int e = s.rowptr[x]; e < s.rowptr[x + 1]; ++e) {
        const C<TI> v = u[s.col[e]];
        const double mv = s.M[e], av = s.A[e];
        p.x += mv * (double)v.x;
        p.y += mv * (double)v.y;
        q.x += av * (double)v.x;
        q.y += av * (double)v.y;
    }
    Pm = p;
    Qa = q;
}

// out[x] = (add ? add[x] : 0) + sign * (A_x in)[x]
template <typename TI, typename Op>
__global__ void k_stencil_A(Op s, int n_x, const C<TI>* in, const double2* add, double sign, double2* out) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n_x) return;
    double2 P, Q;
    stencil_MA<TI>(s, in, x, P, Q);
    double2 r = add ? add[x] : make_double2(0, 0);
    r.x += sign * Q.x;
    r.y += sign * Q.y;
    out[x] = r;
}

template <typename Op>
struct ResArgs {
    int n_t, n_x;
    Op s;
    const double* Mb;   // n_t x 5 band of M_t
    const double* Bb;   // n_t x 5 band of B_t (or B_t^T)
    double bsign;       // +1: K;  -1 with B_t^T: K^H
    const double2* F;      // right-hand side, or NULL: then R = K U (operator apply)
    const double2* apsi0;  // A_x psi0 or NULL
    const double* m_t;
    const double2* U;      // current iterate or NULL (= 0)
    const double2* psi0;   // if set, the iterate is U - 1 (x) psi0
    double2* R;            // output or NULL
    double* partials;      // 2 per block: ||R||^2, ||F~||^2
};

constexpr int RES_LT = 64;

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

// TB: nonzero diagonals of the temporal bands (3 for P1 time, 5 for P2).  One thread per spatial
// node x and RES_LT consecutive time rows: the spatial products (M_x u_k, A_x u_k) of rows k - 2 .. k + 2
// slide through registers, each computed once per block (plus four halo rows).  The block's band
// coefficients (bsign B_t, M_t) sit in shared memory.
template <int TB, typename Op>
__global__ void __launch_bounds__(256) k_residual(ResArgs<Op> a) {
    __shared__ double red[32];
    __shared__ double2 coef[RES_LT][5];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int l0 = blockIdx.y * RES_LT;
    const int l1 = min(l0 + RES_LT, a.n_t);
    for (int i = threadIdx.x; i < (l1 - l0) * 5; i += blockDim.x) {
        const int l = l0 + i / 5, d = i % 5;
        coef[i / 5][d] = make_double2(a.bsign * a.Bb[l * 5 + d], a.Mb[l * 5 + d]);
    }
    __syncthreads();
    double rr = 0, ff = 0;
    if (x < a.n_x) {
        double2 P[5], Q[5];
        auto load_row = [&](int k, double2& p, double2& q) {
            if (k < 0 || k >= a.n_t || !a.U) {
                p = make_double2(0, 0);
                q = make_double2(0, 0);
            } else {
                stencil_MA<double>(a.s, a.U + (size_t)k * a.n_x, x, p, q);
            }
        };
        double2 P0 = make_double2(0, 0), Q0 = make_double2(0, 0);
        if (a.psi0) stencil_MA<double>(a.s, a.psi0, x, P0, Q0);
        auto load_row_shift = [&](int k, double2& p, double2& q) {
            load_row(k, p, q);
            if (a.psi0 && a.U && k >= 0 && k < a.n_t) {
                p.x -= P0.x; p.y -= P0.y;
                q.x -= Q0.x; q.y -= Q0.y;
            }
        };
        for (int d = 1; d < 5; ++d) load_row_shift(l0 - 3 + d, P[d], Q[d]);
        const double2 ap = a.apsi0 ? a.apsi0[x] : make_double2(0, 0);
        for (int l = l0; l < l1; ++l) {
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                P[d] = P[d + 1];
                Q[d] = Q[d + 1];
            }
            load_row_shift(l + 2, P[4], Q[4]);
            double2 kv = make_double2(0, 0);
#pragma unroll
            for (int d = 2 - TB / 2; d <= 2 + TB / 2; ++d) {
                const double2 cm = coef[l - l0][d];   // (bsign B_t, M_t) at (l, l + d - 2)
                // P2 in time: the interior node of an element couples only with its own element, so
                // its outer diagonals are zero (the branch is the same for the whole block)
                if (TB == 5 && cm.x == 0.0 && cm.y == 0.0) continue;
                // += i * bc * P + mc * Q
                kv.x = fma(-cm.x, P[d].y, kv.x);
                kv.x = fma(cm.y, Q[d].x, kv.x);
                kv.y = fma(cm.x, P[d].x, kv.y);
                kv.y = fma(cm.y, Q[d].y, kv.y);
            }
            // residual F~ - K U, or the plain product K U when no right-hand side is given
            double2 r = kv;
            if (a.F) {
                const double2 f = a.F[(size_t)l * a.n_x + x];
                const double ml = a.m_t[l];
                const double2 ft = make_double2(f.x - ml * ap.x, f.y - ml * ap.y);
                r = make_double2(ft.x - kv.x, ft.y - kv.y);
                ff = fma(ft.x, ft.x, ff);
                ff = fma(ft.y, ft.y, ff);
            }
            if (a.R) a.R[(size_t)l * a.n_x + x] = r;
            rr = fma(r.x, r.x, rr);
            rr = fma(r.y, r.y, rr);
        }
    }
    double s1 = block_sum(rr, red);
    double s2 = block_sum(ff, red);
    if (threadIdx.x == 0) {
        const size_t bid = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        a.partials[2 * bid] = s1;
        a.partials[2 * bid + 1] = s2;
    }
}

// scalars[0] = ||R||^2, [1] = ||F~||^2, [2] = scale = 2^e with 2^e * rms(R) in [1, 2), [3] = 1/scale
__global__ void k_reduce_finalize(const double* partials, int nparts, double* scalars, double count) {
    __shared__ double red[32];
    double s1 = 0, s2 = 0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        s1 += partials[2 * i];
        s2 += partials[2 * i + 1];
    }
    double t1 = block_sum(s1, red);
    double t2 = block_sum(s2, red);
    if (threadIdx.x == 0) {
        scalars[0] = t1;
        scalars[1] = t2;
        double rms = sqrt(t1 / count);
        double sc = 1.0;
        if (rms > 0 && isfinite(rms)) {
            int e;
            frexp(rms, &e);          // rms = f 2^e, f in [0.5, 1)
            sc = ldexp(1.0, 1 - e);  // sc * rms in [1, 2)
        }
        scalars[2] = sc;
        scalars[3] = 1.0 / sc;
    }
}

// psi[l, x] += psi0[x]
template <typename T>
__global__ void k_add_row(int n_t, int n_x, C<T>* psi, const C<T>* psi0) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = (size_t)n_t * n_x;
    for (; i < total; i += (size_t)gridDim.x * blockDim.x) {
        int x = (int)(i % n_x);
        C<T> v = psi[i], p = psi0[x];
        psi[i] = mk<T>(v.x + p.x, v.y + p.y);
    }
}

// F[l, x] = sum_k Mfull[l+1, k] (M_x f_k)[x] over full time indices k (t_0 included)
template <typename Op>
__global__ void k_load_nodal(int n_t, int n_x, Op s, const double* Mb, const double* Mfull0,
                             const double2* f, double2* F) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int l = blockIdx.y;
    if (x >= n_x || l >= n_t) return;
    double2 acc = make_double2(0, 0);
    // column t_0
    {
        double2 P, Q;
        stencil_MA<double>(s, f, x, P, Q);
        double c = Mfull0[l];
        acc.x += c * P.x;
        acc.y += c * P.y;
    }
    for (int d = -2; d <= 2; ++d) {
        int k = l + d;  // reduced column index -> full row k + 1 of f
        if (k < 0 || k >= n_t) continue;
        double c = Mb[l * 5 + d + 2];
        if (c == 0.0) continue;
        double2 P, Q;
        stencil_MA<double>(s, f + (size_t)(k + 1) * n_x, x, P, Q);
        acc.x += c * P.x;
        acc.y += c * P.y;
    }
    F[(size_t)l * n_x + x] = acc;
}

// out1[x] = sum_l U1[l, x];  out2[x] = sum_l w[l] U2[l, x]
__global__ void k_colsums(int n_t, int n_x, const double2* U1, const double2* U2, const double* w, double2* out1,
                          double2* out2) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n_x) return;
    double2 a = make_double2(0, 0), b = make_double2(0, 0);
    for (int l = 0; l < n_t; ++l) {
        double2 u = U1[(size_t)l * n_x + x], v = U2[(size_t)l * n_x + x];
        a.x += u.x;
        a.y += u.y;
        b.x += w[l] * v.x;
        b.y += w[l] * v.y;
    }
    out1[x] = a;
    out2[x] = b;
}

// Bartels-Stewart coupling (eq. LGS_x, Schur choice): once w_l is solved, every earlier row
// r < l of the accumulator gains T[r, l] w_l (T row-major n_t x n_t, upper triangular).
__global__ void k_bs_accum(int n_t, int n_x, int l, const double2* T, double2* W) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (x >= n_x || r >= l) return;
    const double2 t = T[(size_t)r * n_t + l];
    const double2 w = W[(size_t)l * n_x + x];
    double2& a = W[(size_t)r * n_x + x];
    a.x += t.x * w.x - t.y * w.y;
    a.y += t.x * w.y + t.y * w.x;
}

cudaError_t launch_bs_accum(int n_t, int n_x, int l, const double2* T, double2* W, cudaStream_t st) {
    if (l <= 0) return cudaSuccess;
    k_bs_accum<<<dim3((n_x + 255) / 256, l), 256, 0, st>>>(n_t, n_x, l, T, W);
    note_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ launchers
static Stencil make_stencil(const SpaceMats& sm) {
    return Stencil{sm.m, sm.Mc, sm.Mw, sm.Ms, sm.Md, sm.Ac, sm.Aw, sm.As, sm.Ad};
}
static Csr make_csr(const SpaceMats& sm) { return Csr{0, sm.d_rowptr, sm.d_col, sm.d_M, sm.d_A}; }

template <typename Op>
static cudaError_t stencil_A_op(const Op& s, int n_x, const void* in, bool in_c64, const double2* add, double sign,
                                double2* out, cudaStream_t st) {
    int grid = (n_x + 255) / 256;
    if (in_c64) k_stencil_A<float, Op><<<grid, 256, 0, st>>>(s, n_x, (const float2*)in, add, sign, out);
    else k_stencil_A<double, Op><<<grid, 256, 0, st>>>(s, n_x, (const double2*)in, add, sign, out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_stencil_A(const SpaceMats& sm, const void* in, bool in_c64, const double2* add, double sign,
                             double2* out, cudaStream_t st) {
    if (sm.kind == 1) return stencil_A_op(make_csr(sm), sm.n_x, in, in_c64, add, sign, out, st);
    return stencil_A_op(make_stencil(sm), sm.n_x, in, in_c64, add, sign, out, st);
}

int residual_num_partials(int n_t, int n_x) {
    return ((n_x + 255) / 256) * ((n_t + RES_LT - 1) / RES_LT);
}

template <typename Op>
static cudaError_t residual_op(const Op& op, const SpaceMats& sm, int n_t, int time_band, const double* Mb,
                               const double* Bb, double bsign, const double2* F, const double2* apsi0, const double* m_t,
                               const double2* U, const double2* psi0, double2* R, double* partials, double* scalars,
                               cudaStream_t st) {
    ResArgs<Op> a;
    a.n_t = n_t;
    a.n_x = sm.n_x;
    a.s = op;
    a.Mb = Mb;
    a.Bb = Bb;
    a.bsign = bsign;
    a.F = F;
    a.apsi0 = apsi0;
    a.m_t = m_t;
    a.U = U;
    a.psi0 = psi0;
    a.R = R;
    a.partials = partials;
    dim3 grid((sm.n_x + 255) / 256, (n_t + RES_LT - 1) / RES_LT);
    if (time_band == 3) k_residual<3, Op><<<grid, 256, 0, st>>>(a);
    else k_residual<5, Op><<<grid, 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_finalize<<<1, 256, 0, st>>>(partials, (int)(grid.x * grid.y), scalars, (double)n_t * sm.n_x);
    note_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_residual(const SpaceMats& sm, int n_t, int time_band, const double* Mb, const double* Bb, double bsign,
                            const double2* F, const double2* apsi0, const double* m_t, const double2* U,
                            const double2* psi0, double2* R, double* partials, double* scalars, cudaStream_t st) {
    if (sm.kind == 1)
        return residual_op(make_csr(sm), sm, n_t, time_band, Mb, Bb, bsign, F, apsi0, m_t, U, psi0, R, partials, scalars, st);
    return residual_op(make_stencil(sm), sm, n_t, time_band, Mb, Bb, bsign, F, apsi0, m_t, U, psi0, R, partials, scalars,
                       st);
}

cudaError_t launch_add_row(int n_t, int n_x, void* psi, const void* psi0, bool c64, cudaStream_t st) {
    size_t total = (size_t)n_t * n_x;
    int grid = (int)std::min<size_t>((total + 255) / 256, 152 * 32);
    if (c64) k_add_row<float><<<grid, 256, 0, st>>>(n_t, n_x, (float2*)psi, (const float2*)psi0);
    else k_add_row<double><<<grid, 256, 0, st>>>(n_t, n_x, (double2*)psi, (const double2*)psi0);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_load_nodal(const SpaceMats& sm, int n_t, const double* Mb, const double* Mfull0,
                              const double2* f, double2* F, cudaStream_t st) {
    dim3 grid((sm.n_x + 255) / 256, n_t);
    if (sm.kind == 1) k_load_nodal<Csr><<<grid, 256, 0, st>>>(n_t, sm.n_x, make_csr(sm), Mb, Mfull0, f, F);
    else k_load_nodal<Stencil><<<grid, 256, 0, st>>>(n_t, sm.n_x, make_stencil(sm), Mb, Mfull0, f, F);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_colsums(int n_t, int n_x, const double2* U1, const double2* U2, const double* w, double2* out1,
                           double2* out2, cudaStream_t st) {
    k_colsums<<<(n_x + 255) / 256, 256, 0, st>>>(n_t, n_x, U1, U2, w, out1, out2);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace stfdm
