// Grouped kernels of the batched solve: many independent problems of uneven size (n_x, n_t,
// temporal degree) advance together, one launch per phase for all of them.
//
// Every space-time vector of the batch is packed: problem p occupies elements
// [off_p, off_p + n_t^p n_x^p) in the (n_t, n_x) row-major layout of the single solve.  A launch
// covers all problems through a block table (first block of each problem, prefix sums); a block
// finds its problem by binary search and returns at once when that problem is masked out.
//
// Phases (per problem they compute exactly what the single-problem path computes):
//   * kb_residual      FP64 Kronecker residual F~ - K x (eq. LGS with the lifting of eq. VF_FEM)
//                      or the operator apply K z (z complex64), with per-block norm partials;
//   * kb_xform         the time transforms G = psc Y_t V and Z = psc^{-1} X_t W (steps 2 and 4 of
//                      the Kronecker solver, Section 3) as tiled complex-FP32 contractions;
//   * kb_multidot / kb_multiaxpy / kb_scale / kb_update_x   the FP64 vector work of flexible GMRES;
//   * kb_cycle_start / kb_arnoldi / kb_solve_y   per-problem GMRES control (one thread per problem:
//                      restart test, Hessenberg column, Givens rotations, least-squares solve),
//                      so that a whole restart cycle runs without the host and can be captured
//                      in a CUDA graph.
#include <cuda_runtime.h>

#include "device.cuh"

namespace stfdm {

constexpr int KB_MAXV = 32;
constexpr int KB_SEG = 8192;     // elements per vector-kernel block
constexpr int KB_THREADS = 256;
constexpr int KB_RES_LT = 16;    // time rows per residual block

__device__ __forceinline__ int kb_find(const int* blk0, int P, int b) {
    int lo = 0, hi = P - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (blk0[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ bool kb_run(const int* on, const int* off, int p) {
    return (!on || on[p]) && (!off || !off[p]);
}

__device__ __forceinline__ double kb_block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

// P = M_x u, Q = A_x u at node x (7-point stencils, zero outside the grid)
template <typename TI>
__device__ __forceinline__ void kb_stencil(const BatchProb& pr, const TI* u, int x, double2& Pm, double2& Qa) {
    const int m = pr.m;
    const int xi = x % m, yj = x / m;
    auto ld = [&](int i) { return make_double2((double)u[i].x, (double)u[i].y); };
    const double2 c = ld(x);
    double2 we = make_double2(0, 0), sn = make_double2(0, 0), dg = make_double2(0, 0);
    if (xi > 0) { const double2 v = ld(x - 1); we.x += v.x; we.y += v.y; }
    if (xi < m - 1) { const double2 v = ld(x + 1); we.x += v.x; we.y += v.y; }
    if (yj > 0) { const double2 v = ld(x - m); sn.x += v.x; sn.y += v.y; }
    if (yj < m - 1) { const double2 v = ld(x + m); sn.x += v.x; sn.y += v.y; }
    if (xi > 0 && yj > 0) { const double2 v = ld(x - m - 1); dg.x += v.x; dg.y += v.y; }
    if (xi < m - 1 && yj < m - 1) { const double2 v = ld(x + m + 1); dg.x += v.x; dg.y += v.y; }
    Pm = make_double2(pr.Mc * c.x + pr.Mw * we.x + pr.Ms * sn.x + pr.Md * dg.x,
                      pr.Mc * c.y + pr.Mw * we.y + pr.Ms * sn.y + pr.Md * dg.y);
    Qa = make_double2(pr.Ac * c.x + pr.Aw * we.x + pr.As * sn.x + pr.Ad * dg.x,
                      pr.Ac * c.y + pr.Aw * we.y + pr.As * sn.y + pr.Ad * dg.y);
}

// RES: w = F - m_t (x) A_x psi0 - K x with partial sums of |w|^2 and |F~|^2;  else w = K z
// (z = Zp + off, complex64).  K = i B_t (x) M_x + M_t (x) A_x.
template <typename TI, bool RES>
__global__ void __launch_bounds__(KB_THREADS) kb_residual(const BatchProb* probs, const int* blk0, int P, const int* on,
                                                          const int* off, const TI* Zp, double2* w, double* partials) {
    __shared__ double red[32];
    const int p = kb_find(blk0, P, blockIdx.x);
    if (!kb_run(on, off, p)) return;
    const BatchProb& pr = probs[p];
    const int n_t = pr.n_t, n_x = pr.n_x;
    const int local = blockIdx.x - blk0[p];
    const int nbx = (n_x + KB_THREADS - 1) / KB_THREADS;
    const int bx = local % nbx, by = local / nbx;
    const int x = bx * KB_THREADS + threadIdx.x;
    const int l0 = by * KB_RES_LT, l1 = min(l0 + KB_RES_LT, n_t);
    const TI* U = RES ? reinterpret_cast<const TI*>(pr.x) : Zp + pr.off;
    double rr = 0, ff = 0;
    if (x < n_x) {
        double2 Pv[5], Qv[5];
        auto row = [&](int k, double2& a, double2& q) {
            if (k < 0 || k >= n_t) {
                a = make_double2(0, 0);
                q = make_double2(0, 0);
            } else {
                kb_stencil<TI>(pr, U + (size_t)k * n_x, x, a, q);
            }
        };
        for (int d = 1; d < 5; ++d) row(l0 - 3 + d, Pv[d], Qv[d]);
        const double2 ap = (RES && pr.apsi0) ? pr.apsi0[x] : make_double2(0, 0);
        for (int l = l0; l < l1; ++l) {
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                Pv[d] = Pv[d + 1];
                Qv[d] = Qv[d + 1];
            }
            row(l + 2, Pv[4], Qv[4]);
            double2 kv = make_double2(0, 0);
            const int dlo = 2 - pr.tband / 2, dhi = 2 + pr.tband / 2;
#pragma unroll
            for (int d = 0; d < 5; ++d) {
                if (d < dlo || d > dhi) continue;
                const double bc = pr.Bb[l * 5 + d], mc = pr.Mb[l * 5 + d];
                kv.x += -bc * Pv[d].y + mc * Qv[d].x;
                kv.y += bc * Pv[d].x + mc * Qv[d].y;
            }
            double2 r = kv;
            if (RES) {
                const double2 f = pr.F[(size_t)l * n_x + x];
                const double ml = pr.m_t[l];
                const double2 ft = make_double2(f.x - ml * ap.x, f.y - ml * ap.y);
                r = make_double2(ft.x - kv.x, ft.y - kv.y);
                rr += r.x * r.x + r.y * r.y;
                ff += ft.x * ft.x + ft.y * ft.y;
            }
            w[pr.off + (size_t)l * n_x + x] = r;
        }
    }
    if (RES) {
        const double s1 = kb_block_sum(rr, red);
        const double s2 = kb_block_sum(ff, red);
        if (threadIdx.x == 0) {
            partials[2 * (size_t)blockIdx.x] = s1;
            partials[2 * (size_t)blockIdx.x + 1] = s2;
        }
    }
}

// rr[p], ff[p] from the residual partials of problem p's blocks (fixed order: deterministic)
__global__ void kb_norm_finalize(const double* partials, const int* blk0, int P, const int* off, double* rr,
                                 double* ff) {
    __shared__ double red[32];
    const int p = blockIdx.x;
    if (off && off[p]) return;
    double s1 = 0, s2 = 0;
    for (int b = blk0[p] + threadIdx.x; b < blk0[p + 1]; b += blockDim.x) {
        s1 += partials[2 * (size_t)b];
        s2 += partials[2 * (size_t)b + 1];
    }
    const double t1 = kb_block_sum(s1, red);
    const double t2 = kb_block_sum(s2, red);
    if (threadIdx.x == 0) {
        rr[p] = t1;
        ff[p] = t2;
    }
}

__global__ void kb_init(BatchGm gm, int P, int m) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    gm.bnorm[p] = -1.0;
    gm.rel[p] = -1.0;
    gm.nh[p] = 0;
    gm.its[p] = 0;
    gm.stopped[p] = 0;
    gm.active[p] = 0;
    gm.jdone[p] = 0;
    for (int i = 0; i < 16; ++i) gm.hist[p * 16 + i] = -1.0;
}

// restart test of every problem; starts a new cycle (g = beta e_1, V_0 = r / beta) for the rest
__global__ void kb_cycle_start(BatchGm gm, int P, int m, double tol, int maxit) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    gm.jdone[p] = 0;
    gm.active[p] = 0;
    if (gm.stopped[p]) return;
    const double beta = sqrt(gm.rr[p]);
    if (gm.bnorm[p] < 0) gm.bnorm[p] = sqrt(gm.ff[p]);
    const double bn = gm.bnorm[p];
    const double rel = bn > 0 ? beta / bn : 0.0;
    gm.rel[p] = rel;
    if (gm.nh[p] < 15) gm.hist[p * 16 + gm.nh[p]++] = rel;
    if (!isfinite(rel)) {
        gm.stopped[p] = 3;
        return;
    }
    if (rel <= tol || beta == 0.0) {
        gm.stopped[p] = 1;
        return;
    }
    if (gm.its[p] >= maxit) {
        gm.stopped[p] = 2;
        return;
    }
    gm.active[p] = 1;
    double2* g = gm.g + (size_t)p * (m + 1);
    g[0] = make_double2(beta, 0);
    for (int i = 1; i <= m; ++i) g[i] = make_double2(0, 0);
    gm.inv[p] = 1.0 / beta;
    atomicAdd(gm.pending, 1);
}

// partial[blk * KB_MAXV + i] = sum over the block's elements of conj(V_i) w, V_i = Vb + i * vs
__global__ void __launch_bounds__(KB_THREADS) kb_multidot(const BatchProb* probs, const int* seg0, int P, const int* on,
                                                          const double2* Vb, size_t vs, int nv, const double2* w,
                                                          double2* partial) {
    constexpr int CH = 4;
    __shared__ double2 red[KB_THREADS / 32][CH];
    const int p = kb_find(seg0, P, blockIdx.x);
    if (!kb_run(on, nullptr, p)) return;
    const BatchProb& pr = probs[p];
    const size_t np = (size_t)pr.n_t * pr.n_x;
    const size_t s0 = (size_t)(blockIdx.x - seg0[p]) * KB_SEG, s1 = min(s0 + KB_SEG, np);
    const int i0 = blockIdx.y * CH;
    double2 acc[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = make_double2(0, 0);
    for (size_t e = s0 + threadIdx.x; e < s1; e += KB_THREADS) {
        const size_t gi = pr.off + e;
        const double2 wx = w[gi];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            if (i0 + c < nv) {
                const double2 v = Vb[(size_t)(i0 + c) * vs + gi];
                acc[c].x += v.x * wx.x + v.y * wx.y;
                acc[c].y += v.x * wx.y - v.y * wx.x;
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        double ax = acc[c].x, ay = acc[c].y;
        for (int o = 16; o > 0; o >>= 1) {
            ax += __shfl_down_sync(0xffffffffu, ax, o);
            ay += __shfl_down_sync(0xffffffffu, ay, o);
        }
        if (lane == 0) red[warp][c] = make_double2(ax, ay);
    }
    __syncthreads();
    if (threadIdx.x < CH && i0 + (int)threadIdx.x < nv) {
        double2 s = make_double2(0, 0);
        for (int wi = 0; wi < KB_THREADS / 32; ++wi) {
            s.x += red[wi][threadIdx.x].x;
            s.y += red[wi][threadIdx.x].y;
        }
        partial[(size_t)blockIdx.x * KB_MAXV + i0 + threadIdx.x] = s;
    }
}

// out[p][i] = sum over problem p's blocks of partial[.][i], i < nv
__global__ void kb_dot_finalize(const double2* partial, const int* seg0, int P, const int* on, int nv, double2* out,
                                int out_stride) {
    const int p = blockIdx.x, i = threadIdx.x;
    if (i >= nv || (on && !on[p])) return;
    double2 s = make_double2(0, 0);
    for (int b = seg0[p]; b < seg0[p + 1]; ++b) {
        const double2 v = partial[(size_t)b * KB_MAXV + i];
        s.x += v.x;
        s.y += v.y;
    }
    out[(size_t)p * out_stride + i] = s;
}

// w -= sum_i c[p][i] V_i  over problem p's elements
__global__ void __launch_bounds__(KB_THREADS) kb_multiaxpy(const BatchProb* probs, const int* seg0, int P, const int* on,
                                                           const double2* Vb, size_t vs, int nv, const double2* c,
                                                           int c_stride, double2* w) {
    __shared__ double2 cs[KB_MAXV];
    const int p = kb_find(seg0, P, blockIdx.x);
    if (!kb_run(on, nullptr, p)) return;
    if (threadIdx.x < nv) cs[threadIdx.x] = c[(size_t)p * c_stride + threadIdx.x];
    __syncthreads();
    const BatchProb& pr = probs[p];
    const size_t np = (size_t)pr.n_t * pr.n_x;
    const size_t s0 = (size_t)(blockIdx.x - seg0[p]) * KB_SEG, s1 = min(s0 + KB_SEG, np);
    for (size_t e = s0 + threadIdx.x; e < s1; e += KB_THREADS) {
        const size_t gi = pr.off + e;
        double2 acc = w[gi];
        for (int i = 0; i < nv; ++i) {
            const double2 v = Vb[(size_t)i * vs + gi];
            const double2 ci = cs[i];
            acc.x -= ci.x * v.x - ci.y * v.y;
            acc.y -= ci.x * v.y + ci.y * v.x;
        }
        w[gi] = acc;
    }
}

// out = inv[p] * w over problem p's elements
__global__ void __launch_bounds__(KB_THREADS) kb_scale(const BatchProb* probs, const int* seg0, int P, const int* on,
                                                       const double* inv, const double2* w, double2* out) {
    const int p = kb_find(seg0, P, blockIdx.x);
    if (!kb_run(on, nullptr, p)) return;
    const BatchProb& pr = probs[p];
    const double a = inv[p];
    const size_t np = (size_t)pr.n_t * pr.n_x;
    const size_t s0 = (size_t)(blockIdx.x - seg0[p]) * KB_SEG, s1 = min(s0 + KB_SEG, np);
    for (size_t e = s0 + threadIdx.x; e < s1; e += KB_THREADS) {
        const double2 v = w[pr.off + e];
        out[pr.off + e] = make_double2(a * v.x, a * v.y);
    }
}

// x_p += sum_{i < jdone[p]} y[p][i] Z_i  (Z complex64, packed)
__global__ void __launch_bounds__(KB_THREADS) kb_update_x(const BatchProb* probs, const int* seg0, int P,
                                                          const int* jdone, const float2* Zb, size_t zs,
                                                          const double2* y, int m) {
    __shared__ double2 ys[KB_MAXV];
    const int p = kb_find(seg0, P, blockIdx.x);
    const int nv = jdone[p];
    if (nv <= 0) return;
    if (threadIdx.x < nv) ys[threadIdx.x] = y[(size_t)p * m + threadIdx.x];
    __syncthreads();
    const BatchProb& pr = probs[p];
    const size_t np = (size_t)pr.n_t * pr.n_x;
    const size_t s0 = (size_t)(blockIdx.x - seg0[p]) * KB_SEG, s1 = min(s0 + KB_SEG, np);
    for (size_t e = s0 + threadIdx.x; e < s1; e += KB_THREADS) {
        double2 acc = pr.x[e];
        for (int i = 0; i < nv; ++i) {
            const float2 z = Zb[(size_t)i * zs + pr.off + e];
            const double2 c = ys[i];
            acc.x += c.x * (double)z.x - c.y * (double)z.y;
            acc.y += c.x * (double)z.y + c.y * (double)z.x;
        }
        pr.x[e] = acc;
    }
}

// Arnoldi step j of every active problem: column j of H from the two Gram-Schmidt passes and
// ||w||, the earlier rotations, a new rotation, the residual estimate |g_{j+1}|; ends the cycle
// of a problem that reached the tolerance, the restart length or the iteration limit.
__global__ void kb_arnoldi(BatchGm gm, int P, int m, int j, double tol, int maxit) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P || !gm.active[p]) return;
    const double2* h1 = gm.h + (size_t)p * 3 * KB_MAXV;
    const double2* h2 = h1 + KB_MAXV;
    const double hn = sqrt(fmax(0.0, h1[2 * KB_MAXV].x));
    double2* H = gm.H + (size_t)p * (m + 1) * m;
    double2* g = gm.g + (size_t)p * (m + 1);
    double2* sn = gm.sn + (size_t)p * m;
    double* cs = gm.cs + (size_t)p * m;
    for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = make_double2(h1[i].x + h2[i].x, h1[i].y + h2[i].y);
    H[(size_t)(j + 1) * m + j] = make_double2(hn, 0);
    // previous rotations G_i = [[c, s], [-conj s, c]]
    for (int i = 0; i < j; ++i) {
        const double2 a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
        const double c = cs[i];
        const double2 s = sn[i];
        // c a + s b ;  -conj(s) a + c b
        H[(size_t)i * m + j] = make_double2(c * a.x + s.x * b.x - s.y * b.y, c * a.y + s.x * b.y + s.y * b.x);
        H[(size_t)(i + 1) * m + j] = make_double2(-(s.x * a.x + s.y * a.y) + c * b.x, -(s.x * a.y - s.y * a.x) + c * b.y);
    }
    {
        const double2 a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
        const double aa = hypot(a.x, a.y), ab = hypot(b.x, b.y);
        double c;
        double2 s;
        if (ab == 0.0) {
            c = 1.0;
            s = make_double2(0, 0);
        } else if (aa == 0.0) {
            c = 0.0;
            s = make_double2(b.x / ab, -b.y / ab);   // conj(b) / |b|
        } else {
            const double rho = hypot(aa, ab);
            c = aa / rho;
            // (a / |a|) conj(b) / rho
            const double2 ua = make_double2(a.x / aa, a.y / aa);
            s = make_double2((ua.x * b.x + ua.y * b.y) / rho, (ua.y * b.x - ua.x * b.y) / rho);
        }
        cs[j] = c;
        sn[j] = s;
        H[(size_t)j * m + j] = make_double2(c * a.x + s.x * b.x - s.y * b.y, c * a.y + s.x * b.y + s.y * b.x);
        H[(size_t)(j + 1) * m + j] = make_double2(0, 0);
        const double2 gj = g[j];
        g[j] = make_double2(c * gj.x, c * gj.y);
        g[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
    }
    gm.its[p] += 1;
    gm.jdone[p] = j + 1;
    const double est = hypot(g[j + 1].x, g[j + 1].y) / gm.bnorm[p];
    if (est <= 0.5 * tol || j == m - 1 || gm.its[p] >= maxit || hn <= 1e-300) {
        gm.active[p] = 0;
    } else {
        gm.inv[p] = 1.0 / hn;
    }
}

// y = R^{-1} g of the cycle's Arnoldi steps (R: the rotated, upper triangular H)
__global__ void kb_solve_y(BatchGm gm, int P, int m) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int nd = gm.jdone[p];
    const double2* H = gm.H + (size_t)p * (m + 1) * m;
    const double2* g = gm.g + (size_t)p * (m + 1);
    double2* y = gm.y + (size_t)p * m;
    for (int i = nd - 1; i >= 0; --i) {
        double2 acc = g[i];
        for (int k = i + 1; k < nd; ++k) {
            const double2 h = H[(size_t)i * m + k], v = y[k];
            acc.x -= h.x * v.x - h.y * v.y;
            acc.y -= h.x * v.y + h.y * v.x;
        }
        const double2 d = H[(size_t)i * m + i];
        const double dd = d.x * d.x + d.y * d.y;
        y[i] = make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd);
    }
}

// a problem that iterated in this application and keeps its factors has them stored now
__global__ void kb_mark_factored(const BatchBand* probs, const int* active, int* factored, int P) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P && probs[p].Lkeep && active[p]) factored[p] = 1;
}

// out_p = scale_p * T_p in_p for every masked-in problem, T_p = Y_t (which 0, scale psc) or X_t
// (which 1, scale 1/psc); complex64 arithmetic and output, TB input (complex128 or complex64).
// Tiles of BM time rows x BN spatial columns, 256 threads, (BM/16) x (BN/16) outputs per thread.
template <typename TB, int BM, int BN>
__global__ void __launch_bounds__(256) kb_xform(const BatchProb* probs, const int* tile0, int P, const int* on,
                                                int which, const TB* in, float2* out) {
    constexpr int BK = 8, TM = BM / 16, TN = BN / 16;
    __shared__ float2 As[BK][BM + 1];
    __shared__ float2 Bs[BK][BN + 1];
    const int p = kb_find(tile0, P, blockIdx.x);
    if (!kb_run(on, nullptr, p)) return;
    const BatchProb& pr = probs[p];
    const int M = pr.n_t, N = pr.n_x, K = pr.n_t;
    const float2* A = which == 0 ? pr.Y32 : pr.X32;
    const TB* B = in + pr.off;
    float2* Cm = out + pr.off;
    const float sc = (float)(which == 0 ? pr.psc : 1.0 / pr.psc);
    const int local = blockIdx.x - tile0[p];
    const int ntn = (N + BN - 1) / BN;
    const int m0 = (local / ntn) * BM, n0 = (local % ntn) * BN;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    float2 acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) acc[i][jj] = make_float2(0, 0);
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int e = tid; e < BM * BK; e += 256) {
            const int r = e / BK, kk = e - r * BK;
            const int gm = m0 + r, gk = k0 + kk;
            As[kk][r] = (gm < M && gk < K) ? A[(size_t)gm * K + gk] : make_float2(0, 0);
        }
        for (int e = tid; e < BK * BN; e += 256) {
            const int kk = e / BN, c = e - kk * BN;
            const int gk = k0 + kk, gn = n0 + c;
            float2 v = make_float2(0, 0);
            if (gk < K && gn < N) {
                const TB t = B[(size_t)gk * N + gn];
                v = make_float2((float)t.x * sc, (float)t.y * sc);
            }
            Bs[kk][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float2 av[TM], bv[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int jj = 0; jj < TN; ++jj) bv[jj] = Bs[kk][tx + 16 * jj];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int jj = 0; jj < TN; ++jj) cfma<float>(acc[i][jj], av[i], bv[jj]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) {
            const int gn = n0 + tx + 16 * jj;
            if (gn < N) Cm[(size_t)gm * N + gn] = acc[i][jj];
        }
    }
}

// ------------------------------------------------------------------ launchers
int kb_seg_blocks(long long n) { return (int)((n + KB_SEG - 1) / KB_SEG); }
int kb_res_blocks(int n_t, int n_x) {
    return ((n_x + KB_THREADS - 1) / KB_THREADS) * ((n_t + KB_RES_LT - 1) / KB_RES_LT);
}
int kb_max_vectors() { return KB_MAXV; }

// transform tile shapes the autotuner chooses from
constexpr int KB_XF_SHAPES = 3;
static const int kb_xf_bm[KB_XF_SHAPES] = {64, 32, 128};
static const int kb_xf_bn[KB_XF_SHAPES] = {64, 128, 32};
int kb_xform_shapes() { return KB_XF_SHAPES; }
void kb_xform_shape(int s, int* bm, int* bn) {
    *bm = kb_xf_bm[s];
    *bn = kb_xf_bn[s];
}

template <typename TB>
static cudaError_t xform_shape_launch(int shape, int ntiles, const BatchProb* probs, const int* tile0, int P,
                                      const int* on, int which, const TB* in, float2* out, cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
    switch (shape) {
        case 0: kb_xform<TB, 64, 64><<<ntiles, 256, 0, st>>>(probs, tile0, P, on, which, in, out); break;
        case 1: kb_xform<TB, 32, 128><<<ntiles, 256, 0, st>>>(probs, tile0, P, on, which, in, out); break;
        default: kb_xform<TB, 128, 32><<<ntiles, 256, 0, st>>>(probs, tile0, P, on, which, in, out); break;
    }
    return cudaGetLastError();
}

cudaError_t kb_launch_xform(int shape, int ntiles, const BatchProb* probs, const int* tile0, int P, const int* on,
                            int which, const void* in, bool in_c128, float2* out, cudaStream_t st) {
    if (in_c128)
        return xform_shape_launch<double2>(shape, ntiles, probs, tile0, P, on, which, (const double2*)in, out, st);
    return xform_shape_launch<float2>(shape, ntiles, probs, tile0, P, on, which, (const float2*)in, out, st);
}

cudaError_t kb_launch_residual(int nblocks, const BatchProb* probs, const int* blk0, int P, const int* off,
                               double* partials, double2* w, double* rr, double* ff, cudaStream_t st) {
    if (nblocks <= 0) return cudaSuccess;
    kb_residual<double2, true><<<nblocks, KB_THREADS, 0, st>>>(probs, blk0, P, nullptr, off, nullptr, w, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    kb_norm_finalize<<<P, 256, 0, st>>>(partials, blk0, P, off, rr, ff);
    return cudaGetLastError();
}

cudaError_t kb_launch_apply(int nblocks, const BatchProb* probs, const int* blk0, int P, const int* on, const float2* Z,
                            double2* w, cudaStream_t st) {
    if (nblocks <= 0) return cudaSuccess;
    kb_residual<float2, false><<<nblocks, KB_THREADS, 0, st>>>(probs, blk0, P, on, nullptr, Z, w, nullptr);
    return cudaGetLastError();
}

cudaError_t kb_launch_multidot(int nseg, const BatchProb* probs, const int* seg0, int P, const int* on,
                               const double2* Vb, size_t vs, int nv, const double2* w, double2* partial, double2* out,
                               int out_stride, cudaStream_t st) {
    if (nv < 1 || nv > KB_MAXV) return cudaErrorInvalidValue;
    dim3 grid(nseg, (nv + 3) / 4);
    kb_multidot<<<grid, KB_THREADS, 0, st>>>(probs, seg0, P, on, Vb, vs, nv, w, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    kb_dot_finalize<<<P, KB_MAXV, 0, st>>>(partial, seg0, P, on, nv, out, out_stride);
    return cudaGetLastError();
}

cudaError_t kb_launch_multiaxpy(int nseg, const BatchProb* probs, const int* seg0, int P, const int* on,
                                const double2* Vb, size_t vs, int nv, const double2* c, int c_stride, double2* w,
                                cudaStream_t st) {
    if (nv < 1 || nv > KB_MAXV) return cudaErrorInvalidValue;
    kb_multiaxpy<<<nseg, KB_THREADS, 0, st>>>(probs, seg0, P, on, Vb, vs, nv, c, c_stride, w);
    return cudaGetLastError();
}

cudaError_t kb_launch_scale(int nseg, const BatchProb* probs, const int* seg0, int P, const int* on, const double* inv,
                            const double2* w, double2* out, cudaStream_t st) {
    kb_scale<<<nseg, KB_THREADS, 0, st>>>(probs, seg0, P, on, inv, w, out);
    return cudaGetLastError();
}

cudaError_t kb_launch_update_x(int nseg, const BatchProb* probs, const int* seg0, int P, const int* jdone,
                               const float2* Z, size_t zs, const double2* y, int m, cudaStream_t st) {
    kb_update_x<<<nseg, KB_THREADS, 0, st>>>(probs, seg0, P, jdone, Z, zs, y, m);
    return cudaGetLastError();
}

cudaError_t kb_launch_init(const BatchGm& gm, int P, int m, cudaStream_t st) {
    kb_init<<<(P + 127) / 128, 128, 0, st>>>(gm, P, m);
    return cudaGetLastError();
}

cudaError_t kb_launch_cycle_start(const BatchGm& gm, int P, int m, double tol, int maxit, cudaStream_t st) {
    kb_cycle_start<<<(P + 127) / 128, 128, 0, st>>>(gm, P, m, tol, maxit);
    return cudaGetLastError();
}

cudaError_t kb_launch_arnoldi(const BatchGm& gm, int P, int m, int j, double tol, int maxit, cudaStream_t st) {
    kb_arnoldi<<<(P + 127) / 128, 128, 0, st>>>(gm, P, m, j, tol, maxit);
    return cudaGetLastError();
}

cudaError_t kb_launch_mark_factored(const BatchBand* probs, const int* active, int* factored, int P, cudaStream_t st) {
    kb_mark_factored<<<(P + 127) / 128, 128, 0, st>>>(probs, active, factored, P);
    return cudaGetLastError();
}

cudaError_t kb_launch_solve_y(const BatchGm& gm, int P, int m, cudaStream_t st) {
    kb_solve_y<<<(P + 127) / 128, 128, 0, st>>>(gm, P, m);
    return cudaGetLastError();
}

}  // namespace stfdm
