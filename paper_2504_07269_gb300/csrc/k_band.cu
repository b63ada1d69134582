// Step 3 of the Kronecker solver (Section 3, eq. LGS_x with the fast-diagonalisation
// choice, where the coupling sum vanishes): the n_t independent spatial problems
//
//        C_k w_k = g_k,     C_k = M_x + s_k A_x,   k = 1..n_t,
//
// each factorised as C_k = L_k D_k L_k^T (complex symmetric, no conjugation, no pivoting:
// Im s_k < 0 makes Im C_k definite, so every leading minor is non-zero) in band form and
// solved in the same launch.
//
// Band structure: interior nodes lexicographic, x1 fastest, m per row; C_k is a 7-point
// stencil with half bandwidth b = m + 1 and the factor fills the whole band.
//
// Generic kernel (complex128, and complex64 when the blocked one does not fit); one CTA per
// system at a time, persistent over systems:
//   * right-looking blocked band LDL^T with panels of NB columns;
//   * the active window -- rows c0 .. c0+NB+b-1 of the band, stored by row as offsets
//     o = i - j in [0, b] -- lives in a per-CTA global scratch buffer (row-circular);
//   * a panel (NB columns x (NB+b) rows) is copied to shared memory and factorised
//     there with one barrier per column; its L columns and pivots then drive a rank-NB
//     update of the b x b trailing triangle of the window, register-tiled 8 rows x 2
//     columns per lane (L D formed on the fly);
//   * forward substitution L z = g and y = D^{-1} z are fused into the panel sweep, and
//     the columns of L (b entries each) and D are written out for the backward
//     substitution L^T w = y (k_subst.cu), which streams them back in reverse order.
#include <cuda_runtime.h>

#include <cstdio>

#include "device.cuh"

namespace stfdm {



template <typename T>
__device__ __forceinline__ C<T> stencil_entry(const BandArgs<T>& a, C<T> s, int i, int o) {
    // entry (i, i - o) of M_x + s A_x, o in [0, b]
    const int xi = i % a.m, yj = i / a.m;
    T re = 0, im = 0;
    if (o == 0) {
        re = a.Mc + s.x * a.Ac;
        im = s.y * a.Ac;
    } else if (o == a.m && yj >= 1) {
        re = a.Ms + s.x * a.As;
        im = s.y * a.As;
    } else if (o == 1 && xi >= 1) {
        re = a.Mw + s.x * a.Aw;
        im = s.y * a.Aw;
    } else if (o == a.m + 1 && xi >= 1 && yj >= 1) {
        re = a.Md + s.x * a.Ad;
        im = s.y * a.Ad;
    }
    return mk<T>(re, im);
}

template <typename T>
__device__ __forceinline__ bool bad_pivot(C<T> d) {
    T a = fabs(d.x) + fabs(d.y);
    return !(a > (T)0) || !isfinite(a);
}

// Shared memory layout (dynamic), WR = b + NB:
//   P   [NB][WR]  panel, by panel column; after the panel factorisation column q holds
//                 L(c0 + r, c0 + q) for r > q and the pivot d_q at r = q
//   zb  [WR]      circular forward-substitution vector (rows c0 .. c0+WR-1)
template <typename T, int NB>
__device__ void band_factor_one(const BandArgs<T>& a, int k, int ks, char* smem) {
    const int n = a.n, b = a.b, WR = b + NB, WB = b + 1;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
    C<T>* P = reinterpret_cast<C<T>*>(smem);
    C<T>* zb = P + NB * WR;
    const C<T> s = a.shifts[k];
    C<T>* z = a.rhs + (size_t)k * n;
    const size_t slot = a.keep ? (size_t)k : (size_t)ks;
    C<T>* Lk = a.L + slot * (size_t)n * b;
    C<T>* Dk = a.D + slot * (size_t)n;
    C<T>* W = a.win + (size_t)blockIdx.x * WR * WB;

    // window rows 0 .. min(WR, n) - 1 from the stencil, forward-substitution vector
    const int r0n = min(WR, n);
    for (int idx = tid; idx < r0n * WB; idx += nth) {
        int i = idx / WB, o = idx - i * WB;
        W[(size_t)(i % WR) * WB + o] = (o <= i) ? stencil_entry(a, s, i, o) : mk<T>(0, 0);
    }
    for (int i = tid; i < r0n; i += nth) zb[i % WR] = z[i];
    __syncthreads();

    for (int c0 = 0; c0 < n; c0 += NB) {
        const int nbk = min(NB, n - c0);
        const int rows_p = min(WR, n - c0);
        // 1. panel to shared memory
        for (int idx = tid; idx < NB * WR; idx += nth) {
            int q = idx / WR, r = idx - q * WR;
            C<T> v = mk<T>(0, 0);
            if (q < nbk && r >= q && r < rows_p && r - q <= b)
                v = W[(size_t)((c0 + r) % WR) * WB + (r - q)];
            P[idx] = v;
        }
        __syncthreads();
        // 2. unblocked LDL^T of the panel on unscaled columns (one barrier per column):
        //    column q2 > q loses P(r, q) P(q2, q) / d_q; the columns are scaled by 1/d_q afterwards
        for (int q = 0; q < nbk; ++q) {
            C<T> d = P[q * WR + q];
            if (bad_pivot<T>(d)) {
                if (tid == 0) atomicExch(a.status, 1);
                d = mk<T>((T)1e-30, 0);
                if (tid == 0) P[q * WR + q] = d;
            }
            const C<T> dinv = cinv<T>(d);
            for (int r = q + 1 + tid; r < rows_p; r += nth) {
                const C<T> x = P[q * WR + r];
                const int q2max = min(nbk - 1, r);
                for (int q2 = q + 1; q2 <= q2max; ++q2) {
                    const C<T> f = cmul<T>(P[q * WR + q2], dinv);
                    cfms<T>(P[q2 * WR + r], x, f);
                }
            }
            __syncthreads();
        }
        // 3. scale to L, write L columns and pivots out
        for (int idx = tid; idx < nbk * WR; idx += nth) {
            int q = idx / WR, r = idx - q * WR;
            if (r > q && r < rows_p) P[idx] = cmul<T>(P[idx], cinv<T>(P[q * WR + q]));
        }
        __syncthreads();
        for (int idx = tid; idx < nbk * b; idx += nth) {
            int q = idx / b, o = idx - q * b + 1;
            int r = q + o;
            Lk[(size_t)(c0 + q) * b + (o - 1)] = (r < rows_p) ? P[q * WR + r] : mk<T>(0, 0);
        }
        if (tid < nbk) Dk[c0 + tid] = P[tid * WR + tid];
        // 4. forward substitution inside the panel, one warp: lane q holds z(c0 + q)
        if (warp == 0) {
            for (int base = 0; base < nbk; base += 32) {
                const int q = base + lane;
                C<T> zq = (q < nbk) ? zb[(c0 + q) % WR] : mk<T>(0, 0);
                // contributions of the earlier 32-blocks of the panel
                for (int q1 = 0; q1 < base; ++q1)
                    if (q < nbk) cfms<T>(zq, P[q1 * WR + q], zb[(c0 + q1) % WR]);
                for (int q1 = base; q1 < min(base + 32, nbk); ++q1) {
                    const C<T> z1 = mk<T>(__shfl_sync(0xffffffffu, zq.x, q1 - base),
                                          __shfl_sync(0xffffffffu, zq.y, q1 - base));
                    if (q > q1 && q < nbk) cfms<T>(zq, P[q1 * WR + q], z1);
                }
                if (q < nbk) zb[(c0 + q) % WR] = zq;
                __syncwarp();
            }
        }
        __syncthreads();
        // 5. forward substitution below the panel; y = z / d of the panel rows out
        for (int r = nbk + tid; r < rows_p; r += nth) {
            C<T> acc = zb[(c0 + r) % WR];
            for (int q = 0; q < nbk; ++q) cfms<T>(acc, P[q * WR + r], zb[(c0 + q) % WR]);
            zb[(c0 + r) % WR] = acc;
        }
        if (tid < nbk) z[c0 + tid] = cmul<T>(zb[(c0 + tid) % WR], cinv<T>(P[tid * WR + tid]));
        // 6. trailing update of the b x b triangle: W(r, r2) -= sum_q L(r, q) d_q L(r2, q);
        {
            const int R6 = rows_p - nbk;
            const int ngroups = (R6 + 7) >> 3;
            for (int rg = warp; rg < ngroups; rg += nwarps) {
                const int rr0 = rg * 8;
                const int nseg = (rr0 + 7) / 64 + 1;
                for (int cs = 0; cs < nseg; ++cs) {
                    const int cc0 = cs * 64 + lane, cc1 = cc0 + 32;
                    C<T> acc[8][2];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int rr = rr0 + j;
                        const size_t rowbase = (size_t)((c0 + nbk + rr) % WR) * WB;
                        acc[j][0] = (rr < R6 && cc0 <= rr) ? W[rowbase + (rr - cc0)] : mk<T>(0, 0);
                        acc[j][1] = (rr < R6 && cc1 <= rr) ? W[rowbase + (rr - cc1)] : mk<T>(0, 0);
                    }
                    const int ci0 = min(nbk + cc0, WR - 1), ci1 = min(nbk + cc1, WR - 1);
                    const int jmax = min(7, WR - 1 - nbk - rr0);
                    for (int q = 0; q < nbk; ++q) {
                        const C<T> dq = P[q * WR + q];
                        const C<T> a0 = cmul<T>(P[q * WR + ci0], dq);
                        const C<T> a1 = cmul<T>(P[q * WR + ci1], dq);
                        const C<T>* prow = P + q * WR + nbk + rr0;
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const C<T> p = prow[min(j, jmax)];
                            cfms<T>(acc[j][0], p, a0);
                            cfms<T>(acc[j][1], p, a1);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int rr = rr0 + j;
                        const size_t rowbase = (size_t)((c0 + nbk + rr) % WR) * WB;
                        if (rr < R6 && cc0 <= rr) W[rowbase + (rr - cc0)] = acc[j][0];
                        if (rr < R6 && cc1 <= rr) W[rowbase + (rr - cc1)] = acc[j][1];
                    }
                }
            }
        }
        __syncthreads();
        // 7. rows entering the window take the freed slots of the panel rows
        {
            const int i0 = c0 + WR;
            const int cnt = min(nbk, n - i0);
            for (int idx = tid; idx < cnt * WB; idx += nth) {
                int x = idx / WB, o = idx - x * WB;
                int i = i0 + x;
                W[(size_t)(i % WR) * WB + o] = stencil_entry(a, s, i, o);
            }
            for (int x = tid; x < cnt; x += nth) zb[(i0 + x) % WR] = z[i0 + x];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ complex64, blocked panel
// Panel of 32 columns, two CTAs of 256 threads per SM (one CTA's serial panel work overlaps
// the other's trailing update).  Warp 0 factors the 32 x 32 top block in registers (lane =
// row; the pivot and L entries travel by shuffles) and publishes U = D L11^T; every row r
// below then solves l_r U = p_r by a register-resident forward substitution (no barriers).
// The trailing update uses an 8 x 2 register tile per lane with L D formed on the fly and
// skips 32-column sub-blocks that lie entirely above the diagonal.
constexpr int V4_THREADS = 256;
constexpr int V4_NB = 32;

__device__ __forceinline__ float2 shfl2(float2 v, int src) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// One system: shift s, right-hand side z (y = D^{-1} L^{-1} g out), factor columns Lk and pivots
// Dk, the CTA's window W of (b + 32) x (b + 1) entries; n, m, b, the stencil and status from a.
__device__ __forceinline__ void band_factor_v4(const BandArgs<float>& a, const float2 s, float2* z, float2* Lk,
                                               float2* Dk, float2* W, char* smem) {
    using T = float;
    constexpr int NB = V4_NB;
    const int n = a.n, b = a.b, m = a.m, WR = b + NB, WB = b + 1;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
    float2* P = reinterpret_cast<float2*>(smem);     // [NB][WR]  panel -> L (pivots on the diagonal)
    float2* Us = P + NB * WR;                          // [NB][NB]  U[q'][q] = d_q' L(q, q') for q' < q
    float2* dinv = Us + NB * NB;                       // [NB]
    float2* zb = dinv + NB;                            // [WR]
    // a new band row i (one warp): zero except the stencil offsets 0, 1, m, m + 1
    auto fill_row = [&](int i) {
        float2* row = W + (size_t)(i % WR) * WB;
        const int xi = i % m, yj = i / m;
        const float2 e0 = mk<T>(a.Mc + s.x * a.Ac, s.y * a.Ac);
        const float2 e1 = (xi >= 1) ? mk<T>(a.Mw + s.x * a.Aw, s.y * a.Aw) : mk<T>(0, 0);
        const float2 em = (yj >= 1) ? mk<T>(a.Ms + s.x * a.As, s.y * a.As) : mk<T>(0, 0);
        const float2 ed = (xi >= 1 && yj >= 1) ? mk<T>(a.Md + s.x * a.Ad, s.y * a.Ad) : mk<T>(0, 0);
        for (int o = lane; o < WB; o += 32) {
            float2 v = mk<T>(0, 0);
            if (o <= i) {
                if (o == 0) v = e0;
                else if (o == m) v = em;
                else if (o == 1) v = e1;
                else if (o == m + 1) v = ed;
            }
            row[o] = v;
        }
    };

    const int r0n = min(WR, n);
    for (int i = warp; i < r0n; i += nwarps) fill_row(i);
    for (int i = tid; i < r0n; i += nth) zb[i % WR] = z[i];
    __syncthreads();

    for (int c0 = 0; c0 < n; c0 += NB) {
        const int nbk = min(NB, n - c0);
        const int rows_p = min(WR, n - c0);
        const int rbase = c0 % WR;
        // 1. panel to shared memory: each thread reads whole rows (contiguous offsets), loads batched
        for (int r = tid; r < WR; r += nth) {
            int sl = rbase + r;
            if (sl >= WR) sl -= WR;
            const float2* wrow = W + (size_t)sl * WB;
#pragma unroll
            for (int h = 0; h < NB; h += 16) {
                float2 v[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int q = h + u;
                    v[u] = (q < nbk && r >= q && r < rows_p && r - q <= b) ? wrow[r - q] : mk<T>(0, 0);
                }
#pragma unroll
                for (int u = 0; u < 16; ++u) P[(h + u) * WR + r] = v[u];
            }
        }
        __syncthreads();
        // 2a. LDL^T of the 32 x 32 top block by the whole CTA, two columns per step (one barrier per
        //     step): thread t owns row r = t / 8 at columns q2 = q + 2 + t % 8 (+ 8, ...) <= r and applies
        //     the eliminations of columns q and q + 1 together from the values before the step,
        //       A''(r, q2) = A(r, q2) - A(r, q) A(q2, q) / d_q - A'(r, q+1) A'(q2, q+1) / d'_{q+1},
        //       A'(i, q+1) = A(i, q+1) - A(i, q) A(q+1, q) / d_q,  d'_{q+1} = A'(q+1, q+1)
        //     (unscaled form); column q + 1's new entries are stored after the step's barrier.  A last
        //     odd column has no rows below it inside the block.
        {
            const int r = tid >> 3, g = tid & 7;
            float2 pend = mk<T>(0, 0);
            int pend_col = -1;
            for (int q = 0; q + 1 < nbk; q += 2) {
                if (pend_col >= 0) {
                    P[pend_col * WR + r] = pend;
                    pend_col = -1;
                }
                float2 d0 = P[q * WR + q];
                if (bad_pivot<T>(d0)) d0 = mk<T>(1e-30f, 0);
                const float2 di0 = cinv<T>(d0);
                const float2 f = cmul<T>(P[q * WR + (q + 1)], di0);      // A(q+1, q) / d_q
                float2 d1 = P[(q + 1) * WR + (q + 1)];
                cfms<T>(d1, P[q * WR + (q + 1)], f);
                const float2 d1s = bad_pivot<T>(d1) ? mk<T>(1e-30f, 0) : d1;
                const float2 di1 = cinv<T>(d1s);
                if (r > q + 1 && r < nbk) {
                    const float2 x0 = P[q * WR + r];
                    float2 x1 = P[(q + 1) * WR + r];
                    cfms<T>(x1, x0, f);
                    for (int q2 = q + 2 + g; q2 <= r; q2 += 8) {
                        const float2 c0 = P[q * WR + q2];
                        float2 c1 = P[(q + 1) * WR + q2];
                        cfms<T>(c1, c0, f);
                        float2 v = P[q2 * WR + r];
                        cfms<T>(v, x0, cmul<T>(c0, di0));
                        cfms<T>(v, x1, cmul<T>(c1, di1));
                        P[q2 * WR + r] = v;
                    }
                    if (g == 0) {
                        pend = x1;
                        pend_col = q + 1;
                    }
                } else if (r == q + 1 && g == 0) {
                    pend = d1;
                    pend_col = q + 1;
                }
                __syncthreads();
            }
            if (pend_col >= 0) P[pend_col * WR + r] = pend;
            __syncthreads();
        }
        // pivots, 1/d, scaled L11 and U[q'][q] = d_q' L(q, q')
        if (tid < nbk) {
            float2 d = P[tid * WR + tid];
            if (bad_pivot<T>(d)) {
                atomicExch(a.status, 1);
                d = mk<T>(1e-30f, 0);
                P[tid * WR + tid] = d;
            }
            dinv[tid] = cinv<T>(d);
        }
        __syncthreads();
        for (int idx = tid; idx < NB * NB; idx += nth) {
            const int q = idx / NB, r = idx % NB;   // entry (r, q) of the top block
            float2 u = mk<T>(0, 0);
            if (q < r && r < nbk) {
                const float2 lrq = cmul<T>(P[q * WR + r], dinv[q]);
                u = cmul<T>(P[q * WR + q], lrq);       // d_q L(r, q) = unscaled entry
                P[q * WR + r] = lrq;
            }
            Us[q * NB + r] = u;                        // U[q][r] = d_q L(r, q)
        }
        __syncthreads();
        // 2b. rows below the top block: l_r[q] = (p_r[q] - sum_{q'<q} l_r[q'] U[q'][q]) / d_q
        for (int r = nbk + tid; r < rows_p; r += nth) {
            float2 l[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                float2 acc = P[q * WR + r];
#pragma unroll
                for (int q1 = 0; q1 < q; ++q1) cfms<T>(acc, l[q1], Us[q1 * NB + q]);
                l[q] = (q < nbk) ? cmul<T>(acc, dinv[q]) : mk<T>(0, 0);
            }
#pragma unroll
            for (int q = 0; q < NB; ++q)
                if (q < nbk) P[q * WR + r] = l[q];
        }
        __syncthreads();
        // 3. warp 0: forward substitution inside the panel; the others write L and D out
        if (warp == 0) {
            const int q = lane;
            int sq = rbase + q;
            if (sq >= WR) sq -= WR;
            float2 zq = (q < nbk) ? zb[sq] : mk<T>(0, 0);
            for (int q1 = 0; q1 < nbk; ++q1) {
                const float2 z1 = shfl2(zq, q1);
                if (q > q1 && q < nbk) cfms<T>(zq, P[q1 * WR + q], z1);
            }
            if (q < nbk) zb[sq] = zq;
        } else {
            for (int q = 0; q < nbk; ++q)
                for (int o = tid - 31; o <= b; o += nth - 32) {
                    const int r = q + o;
                    Lk[(size_t)(c0 + q) * b + (o - 1)] = (r < rows_p) ? P[q * WR + r] : mk<T>(0, 0);
                }
            if (tid - 32 < nbk) Dk[c0 + tid - 32] = P[(tid - 32) * WR + (tid - 32)];
        }
        __syncthreads();
        // 4. forward substitution below the panel; y = z / d of the panel rows out
        for (int r = nbk + tid; r < rows_p; r += nth) {
            int sl = rbase + r;
            if (sl >= WR) sl -= WR;
            float2 acc = zb[sl];
            int sq = rbase;
            for (int q = 0; q < nbk; ++q) {
                cfms<T>(acc, P[q * WR + r], zb[sq]);
                if (++sq == WR) sq = 0;
            }
            zb[sl] = acc;
        }
        if (tid < nbk) {
            int sq = rbase + tid;
            if (sq >= WR) sq -= WR;
            z[c0 + tid] = cmul<T>(zb[sq], dinv[tid]);
        }
        // 5. trailing update, items of 8 rows x 64 columns, 2 columns per lane: the panel's products
        //    sum_q L(r, q) d_q L(c, q) are accumulated on their own and subtracted from the window
        //    entry once (the entries are loaded before the sum, hiding their latency), which rounds
        //    less than updating the entry term by term.
        {
            const int R6 = rows_p - nbk;
            const int ngroups = (R6 + 7) >> 3;
            for (int rg = warp; rg < ngroups; rg += nwarps) {
                const int rr0 = rg * 8;
                const int nseg = (rr0 + 7) / 64 + 1;
                const int jmax = min(7, WR - 1 - nbk - rr0);
                int rowb[8];   // window offsets of the 8 rows (< WR WB)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    int sl = rbase + nbk + rr0 + j;
                    while (sl >= WR) sl -= WR;
                    rowb[j] = sl * WB;
                }
                for (int cs = 0; cs < nseg; ++cs) {
                    const int cc0 = cs * 64 + lane, cc1 = cc0 + 32;
                    const bool act1 = (cs * 64 + 32) <= (rr0 + 7);   // second sub-block touches the triangle
                    float2 acc[8][2], wv[8][2];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int rr = rr0 + j;
                        wv[j][0] = (rr < R6 && cc0 <= rr) ? W[rowb[j] + (rr - cc0)] : mk<T>(0, 0);
                        wv[j][1] = (act1 && rr < R6 && cc1 <= rr) ? W[rowb[j] + (rr - cc1)] : mk<T>(0, 0);
                        acc[j][0] = mk<T>(0, 0);
                        acc[j][1] = mk<T>(0, 0);
                    }
                    const int ci0 = min(nbk + cc0, WR - 1), ci1 = min(nbk + cc1, WR - 1);
                    if (act1) {
#pragma unroll 2
                        for (int q = 0; q < nbk; ++q) {
                            const float2 dq = P[q * WR + q];
                            const float2 a0 = cmul<T>(P[q * WR + ci0], dq);
                            const float2 a1 = cmul<T>(P[q * WR + ci1], dq);
                            const float2* prow = P + q * WR + nbk + rr0;
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                const float2 pv = prow[min(j, jmax)];
                                cfma<T>(acc[j][0], pv, a0);
                                cfma<T>(acc[j][1], pv, a1);
                            }
                        }
                    } else {
#pragma unroll 2
                        for (int q = 0; q < nbk; ++q) {
                            const float2 a0 = cmul<T>(P[q * WR + ci0], P[q * WR + q]);
                            const float2* prow = P + q * WR + nbk + rr0;
#pragma unroll
                            for (int j = 0; j < 8; ++j) cfma<T>(acc[j][0], prow[min(j, jmax)], a0);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int rr = rr0 + j;
                        if (rr < R6 && cc0 <= rr) W[rowb[j] + (rr - cc0)] = csub<T>(wv[j][0], acc[j][0]);
                        if (act1 && rr < R6 && cc1 <= rr) W[rowb[j] + (rr - cc1)] = csub<T>(wv[j][1], acc[j][1]);
                    }
                }
            }
        }
        __syncthreads();
        // 6. rows entering the window take the freed slots of the panel rows
        {
            const int i0 = c0 + WR;
            const int cnt = min(nbk, n - i0);
            for (int x = warp; x < cnt; x += nwarps) fill_row(i0 + x);
            for (int x = tid; x < cnt; x += nth) zb[(i0 + x) % WR] = z[i0 + x];
        }
        __syncthreads();
    }
}

size_t band_factor_v4_smem(int b) {
    const int WR = b + V4_NB;
    return sizeof(float2) * ((size_t)V4_NB * WR + V4_NB * V4_NB + V4_NB + WR);
}

size_t band_batch_smem(int b_max) {
    const size_t bwd = sizeof(float2) * ((size_t)b_max + 32 + 32 + 32 * 33);
    const size_t f = band_factor_v4_smem(b_max);
    return f > bwd ? f : bwd;
}

__global__ void __launch_bounds__(V4_THREADS, 2) k_band_factor_v4(BandArgs<float> a) {
    extern __shared__ __align__(16) char smem[];
    const int WR = a.b + V4_NB, WB = a.b + 1;
    for (int ks = blockIdx.x; ks < a.n_sys; ks += gridDim.x) {
        const int k = a.k0 + ks;
        const size_t slot = a.keep ? (size_t)k : (size_t)ks;
        band_factor_v4(a, a.shifts[k], a.rhs + (size_t)k * a.n, a.L + slot * (size_t)a.n * a.b, a.D + slot * (size_t)a.n,
                       a.win + (size_t)blockIdx.x * WR * WB, smem);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ backward substitution by one CTA
// The same for bands wider than 256 (entries loaded when they are used).
__device__ __forceinline__ void band_bwd_cta_wide(int n, int b, const float2* __restrict__ L, float2* z, char* smem) {
    using T = float;
    const int RB = b + 32;
    float2* ring = reinterpret_cast<float2*>(smem);   // [RB]: w of row r at r % RB
    float2* tcon = ring + RB;                          // [32]: contributions from below the block
    float2* Ls = tcon + 32;                            // [32][33]: Ls[r][q] = L(j0 + r, j0 + q), q < r
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int j0 = ((n - 1) / 32) * 32; j0 >= 0; j0 -= 32) {
        const int j1 = min(j0 + 32, n);
        // the block's strictly lower triangle of L, 4 entries per thread
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = tid + 256 * e, r = idx >> 5, q = idx & 31, o = r - q;
            Ls[r * 33 + q] = (o >= 1 && o <= b && j0 + r < j1) ? L[(size_t)(j0 + q) * b + (o - 1)] : mk<T>(0, 0);
        }
        for (int cc = 0; cc < 4; ++cc) {
            const int c = warp * 4 + cc, j = j0 + c;
            float2 acc = mk<T>(0, 0);
            if (j < j1) {
                const int ohi = min(b, n - 1 - j);
                const float2* Lj = L + (size_t)j * b - 1;
#pragma unroll 4
                for (int o = j1 - j + lane; o <= ohi; o += 32) {
                    int r = j + o;
                    r -= (r / RB) * RB;
                    cfma<T>(acc, Lj[o], ring[r]);
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
            }
            if (lane == 0) tcon[c] = acc;
        }
        __syncthreads();
        if (warp == 0) {
            const int j = j0 + lane;
            float2 acc = (j < j1) ? csub<T>(z[j], tcon[lane]) : mk<T>(0, 0);
#pragma unroll
            for (int r = 31; r > 0; --r) {
                const float2 wr = mk<T>(__shfl_sync(0xffffffffu, acc.x, r), __shfl_sync(0xffffffffu, acc.y, r));
                if (lane < r) cfms<T>(acc, Ls[r * 33 + lane], wr);
            }
            if (j < j1) {
                ring[j % RB] = acc;
                z[j] = acc;
            }
        }
        __syncthreads();
    }
}

// L^T w = y for one system whose factor columns L (L[j*b + o - 1] = L(j + o, j)) this CTA has just
// written; z holds y on entry and w on exit.  Rows are solved in blocks of 32 from the bottom:
//   A. every warp forms, for 4 of the block's columns j, the contribution of the already solved
//      rows below the block, sum_{j + o >= j1} L(j + o, j) w_{j+o} (lanes across the band);
//   B. warp 0 solves the 32 x 32 unit upper triangle of the block by shuffles, lane = row, with
//      the block's in-triangle entries of L staged in shared memory.
// The solved w of the last b + 32 rows stay in a shared-memory ring.  For b <= 256 the entries of
// L that block j0 - 32 needs (they do not depend on w) are loaded into registers while warp 0
// solves block j0, so the loads' latency is off the block-to-block chain.
__device__ __forceinline__ void band_bwd_cta(int n, int b, const float2* __restrict__ L, float2* z, char* smem) {
    using T = float;
    if (b > 256) {
        band_bwd_cta_wide(n, b, L, z, smem);
        return;
    }
    constexpr int NO = 8;   // band offsets per lane and column (b <= 8 x 32)
    const int RB = b + 32;
    float2* ring = reinterpret_cast<float2*>(smem);   // [RB]: w of row r at r % RB
    float2* tcon = ring + RB;                          // [32]: contributions from below the block
    float2* Ls = tcon + 32;                            // [32][33]: Ls[r][q] = L(j0 + r, j0 + q), q < r
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float2 lv[4][NO];   // lv[cc][t] = L(j1 + lane + 32 t, j) for the warp's column j = j0 + 4 warp + cc
    float2 lt[4];       // the thread's 4 entries of the block's strictly lower triangle
    auto load = [&](int j0) {
        const int j1 = min(j0 + 32, n);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = tid + 256 * e, r = idx >> 5, q = idx & 31, o = r - q;
            lt[e] = (o >= 1 && o <= b && j0 + r < j1) ? L[(size_t)(j0 + q) * b + (o - 1)] : mk<T>(0, 0);
        }
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            const int j = j0 + warp * 4 + cc;
            // columns past the end of the block (j >= j1) read nothing: ohi = 0 < o
            const int ohi = (j < j1) ? min(b, n - 1 - j) : 0;
            const float2* Lj = L + (size_t)j * b - 1;
#pragma unroll
            for (int t = 0; t < NO; ++t) {
                const int o = j1 - j + lane + 32 * t;
                lv[cc][t] = (o >= 1 && o <= ohi) ? Lj[o] : mk<T>(0, 0);
            }
        }
    };
    int j0 = ((n - 1) / 32) * 32;
    load(j0);
    for (; j0 >= 0; j0 -= 32) {
        const int j1 = min(j0 + 32, n);
        const int j1m = j1 % RB;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = tid + 256 * e;
            Ls[(idx >> 5) * 33 + (idx & 31)] = lt[e];
        }
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            const int c = warp * 4 + cc, j = j0 + c;
            const int ohi = (j < j1) ? min(b, n - 1 - j) : 0;
            float2 acc = mk<T>(0, 0);
#pragma unroll
            for (int t = 0; t < NO; ++t) {
                const int o = j1 - j + lane + 32 * t;
                if (o >= 1 && o <= ohi) {
                    int r = j1m + lane + 32 * t;   // (j + o) % RB: j + o - j1 < b < RB
                    if (r >= RB) r -= RB;
                    cfma<T>(acc, lv[cc][t], ring[r]);
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
            }
            if (lane == 0) tcon[c] = acc;
        }
        __syncthreads();
        if (j0 >= 32) load(j0 - 32);
        if (warp == 0) {
            const int j = j0 + lane;
            float2 acc = (j < j1) ? csub<T>(z[j], tcon[lane]) : mk<T>(0, 0);
#pragma unroll
            for (int r = 31; r > 0; --r) {
                const float2 wr = mk<T>(__shfl_sync(0xffffffffu, acc.x, r), __shfl_sync(0xffffffffu, acc.y, r));
                if (lane < r) cfms<T>(acc, Ls[r * 33 + lane], wr);
            }
            if (j < j1) {
                ring[j % RB] = acc;
                z[j] = acc;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ grouped factor-and-solve
// All systems (problem p, shift k) of a batch of problems of uneven size in one persistent launch:
// each CTA takes the next item of a cost-sorted work list (atomic counter), factorises it with the
// blocked-panel kernel (forward substitution fused) into its private factor slot and solves the
// backward substitution itself.  Items of problems whose `active` flag is 0 are skipped.
__global__ void __launch_bounds__(V4_THREADS, 2)
k_band_batch_v4(const BatchBand* probs, const int2* items, int n_items, const int* active, const int* factored,
                int* counter, float2* win, size_t win_stride, float2* Lslots, size_t L_stride, float2* Dslots,
                size_t D_stride, int* status) {
    extern __shared__ __align__(16) char smem[];
    __shared__ int s_item;
    __shared__ BandArgs<float> s_args;   // the current item's geometry and stencil (keeps registers free)
    __shared__ float2 s_shift;
    __shared__ float2* s_z;
    __shared__ float2* s_L;   // factor columns: the problem's kept storage or this CTA's slot
    __shared__ float2* s_D;
    for (;;) {
        if (threadIdx.x == 0) {
            const int it = atomicAdd(counter, 1);
            int run = 0;
            if (it < n_items) {
                const int2 pk = items[it];
                const BatchBand& pb = probs[pk.x];
                // skip problems that are not iterating, and kept factors that are already stored
                // (their systems are solved by the grouped substitutions)
                const bool skip = (active && !active[pk.x]) || (pb.Lkeep && factored && factored[pk.x]);
                run = skip ? 2 : 1;
                if (run == 1) {
                    s_args.n = pb.n;
                    s_args.m = pb.m;
                    s_args.b = pb.b;
                    s_args.Mc = pb.Mc; s_args.Mw = pb.Mw; s_args.Ms = pb.Ms; s_args.Md = pb.Md;
                    s_args.Ac = pb.Ac; s_args.Aw = pb.Aw; s_args.As = pb.As; s_args.Ad = pb.Ad;
                    s_args.status = status;
                    s_shift = pb.shifts[pk.y];
                    s_z = pb.rhs + (size_t)pk.y * pb.n;
                    if (pb.Lkeep) {
                        s_L = pb.Lkeep + (size_t)pk.y * pb.n * pb.b;
                        s_D = pb.Dkeep + (size_t)pk.y * pb.n;
                    } else {
                        s_L = Lslots + (size_t)blockIdx.x * L_stride;
                        s_D = Dslots + (size_t)blockIdx.x * D_stride;
                    }
                }
            }
            s_item = run;
        }
        __syncthreads();
        const int run = s_item;
        if (run == 0) break;
        if (run == 1) {
            band_factor_v4(s_args, s_shift, s_z, s_L, s_D, win + (size_t)blockIdx.x * win_stride, smem);
            __syncthreads();
            band_bwd_cta(s_args.n, s_args.b, s_L, s_z, smem);
        }
        __syncthreads();
    }
}

cudaError_t band_batch_launch(const BatchBand* probs, const int2* items, int n_items, const int* active,
                              const int* factored, int* counter, int b_max, float2* win, float2* Lslots, size_t L_stride,
                              float2* Dslots, size_t D_stride, int* status, int grid, cudaStream_t st) {
    const size_t smem = band_batch_smem(b_max);
    const size_t win_stride = (size_t)(b_max + V4_NB) * (b_max + 1);
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_band_batch_v4<<<grid, V4_THREADS, smem, st>>>(probs, items, n_items, active, factored, counter, win, win_stride,
                                                    Lslots, L_stride, Dslots, D_stride, status);
    return cudaGetLastError();
}

cudaError_t band_batch_prepare(int b_max) {
    return cudaFuncSetAttribute(k_band_batch_v4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)band_batch_smem(b_max));
}

int band_batch_occupancy(int b_max) {
    int occ = 0;
    if (band_batch_prepare(b_max) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_band_batch_v4, V4_THREADS, band_batch_smem(b_max));
    cudaGetLastError();
    return occ;
}


template <typename T, int NB>
__global__ void __launch_bounds__(256, 2) k_band_factor_solve(BandArgs<T> a) {
    extern __shared__ __align__(16) char smem[];
    for (int ks = blockIdx.x; ks < a.n_sys; ks += gridDim.x) {
        band_factor_one<T, NB>(a, a.k0 + ks, ks, smem);
        __syncthreads();
    }
}

template <typename T, int NB>
size_t band_factor_smem(int b) {
    const int WR = b + NB;
    return sizeof(C<T>) * ((size_t)NB * WR + WR);
}
// ------------------------------------------------------------------ host launchers

template <typename T, int NB>
static cudaError_t launch_factor_nb(const BandArgs<T>& a, int grid, cudaStream_t st) {
    size_t smem = band_factor_smem<T, NB>(a.b);
    cudaError_t e = cudaFuncSetAttribute(k_band_factor_solve<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_band_factor_solve<T, NB><<<grid, 256, smem, st>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

// Panel width code: complex64 uses the blocked-panel kernel (code 64) when it fits, else the
// generic kernel (negative codes); complex128 uses the generic kernel with the widest panel.
template <typename T>
int band_pick_nb(int b, size_t smem_optin);
template <>
int band_pick_nb<double>(int b, size_t smem_optin) {
    if (band_factor_smem<double, 32>(b) <= smem_optin) return 32;
    if (band_factor_smem<double, 16>(b) <= smem_optin) return 16;
    if (band_factor_smem<double, 8>(b) <= smem_optin) return 8;
    return 0;
}
template <>
int band_pick_nb<float>(int b, size_t smem_optin) {
    if (band_factor_v4_smem(b) <= smem_optin) return 64;   // blocked panel of 32 (code 64)
    if (band_factor_smem<float, 16>(b) <= smem_optin) return -16;  // generic kernel
    if (band_factor_smem<float, 8>(b) <= smem_optin) return -8;
    return 0;
}

template <typename T>
size_t band_smem_for(int nb, int b);
template <>
size_t band_smem_for<double>(int nb, int b) {
    return nb == 32 ? band_factor_smem<double, 32>(b) : nb == 16 ? band_factor_smem<double, 16>(b)
                                                                : band_factor_smem<double, 8>(b);
}
template <>
size_t band_smem_for<float>(int nb, int b) {
    if (nb == 64) return band_factor_v4_smem(b);
    return nb == -16 ? band_factor_smem<float, 16>(b) : band_factor_smem<float, 8>(b);
}

template <typename T>
cudaError_t band_factor_solve_launch(const BandArgs<T>& a, int nb, int grid, cudaStream_t st);
template <>
cudaError_t band_factor_solve_launch<double>(const BandArgs<double>& a, int nb, int grid, cudaStream_t st) {
    if (nb == 32) return launch_factor_nb<double, 32>(a, grid, st);
    if (nb == 16) return launch_factor_nb<double, 16>(a, grid, st);
    return launch_factor_nb<double, 8>(a, grid, st);
}
template <>
cudaError_t band_factor_solve_launch<float>(const BandArgs<float>& a, int nb, int grid, cudaStream_t st) {
    if (nb == 64) {
        size_t smem = band_factor_v4_smem(a.b);
        cudaError_t e = cudaFuncSetAttribute(k_band_factor_v4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_band_factor_v4<<<grid, V4_THREADS, smem, st>>>(a);
        note_launches(1);
        return cudaGetLastError();
    }
    if (nb == -16) return launch_factor_nb<float, 16>(a, grid, st);
    return launch_factor_nb<float, 8>(a, grid, st);
}

template <typename T, int NB>
static int occupancy_nb(int b) {
    int occ = 0;
    size_t smem = band_factor_smem<T, NB>(b);
    cudaFuncSetAttribute(k_band_factor_solve<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_band_factor_solve<T, NB>, 256, smem);
    cudaGetLastError();
    return occ;
}

template <typename T>
int band_occupancy(int nb, int b);
template <>
int band_occupancy<double>(int nb, int b) {
    return nb == 32 ? occupancy_nb<double, 32>(b) : nb == 16 ? occupancy_nb<double, 16>(b) : occupancy_nb<double, 8>(b);
}
template <>
int band_occupancy<float>(int nb, int b) {
    if (nb == 64) {
        int occ = 0;
        size_t smem = band_factor_v4_smem(b);
        cudaFuncSetAttribute(k_band_factor_v4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_band_factor_v4, V4_THREADS, smem);
        cudaGetLastError();
        return occ;
    }
    return nb == -16 ? occupancy_nb<float, 16>(b) : occupancy_nb<float, 8>(b);
}


}  // namespace stfdm
