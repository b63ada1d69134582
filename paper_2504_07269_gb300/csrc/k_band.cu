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
// Kernel design (one CTA per system at a time, persistent over systems):
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
        // 6. trailing update of the b x b triangle: W(r, r2) -= sum_q L(r, q) d_q L(r2, q)
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
template <typename T>
struct BandPlan {
    int nb = 16;
    int grid = 0;
    size_t smem = 0;
};

template <typename T, int NB>
static cudaError_t launch_factor_nb(const BandArgs<T>& a, int grid, cudaStream_t st) {
    size_t smem = band_factor_smem<T, NB>(a.b);
    cudaError_t e = cudaFuncSetAttribute(k_band_factor_solve<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_band_factor_solve<T, NB><<<grid, 256, smem, st>>>(a);
    return cudaGetLastError();
}
// Chooses the panel width that fits the shared-memory budget.
template <typename T>
int band_pick_nb(int b, size_t smem_optin) {
    if (band_factor_smem<T, 32>(b) <= smem_optin) return 32;
    if (band_factor_smem<T, 16>(b) <= smem_optin) return 16;
    if (band_factor_smem<T, 8>(b) <= smem_optin) return 8;
    return 0;
}

template <typename T>
size_t band_smem_for(int nb, int b) {
    return nb == 32 ? band_factor_smem<T, 32>(b) : nb == 16 ? band_factor_smem<T, 16>(b) : band_factor_smem<T, 8>(b);
}

template <typename T>
cudaError_t band_factor_solve_launch(const BandArgs<T>& a, int nb, int grid, cudaStream_t st) {
    if (nb == 32) return launch_factor_nb<T, 32>(a, grid, st);
    if (nb == 16) return launch_factor_nb<T, 16>(a, grid, st);
    return launch_factor_nb<T, 8>(a, grid, st);
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
int band_occupancy(int nb, int b) {
    return nb == 32 ? occupancy_nb<T, 32>(b) : nb == 16 ? occupancy_nb<T, 16>(b) : occupancy_nb<T, 8>(b);
}

template int band_occupancy<float>(int, int);
template int band_occupancy<double>(int, int);
template int band_pick_nb<float>(int, size_t);
template int band_pick_nb<double>(int, size_t);
template size_t band_smem_for<float>(int, int);
template size_t band_smem_for<double>(int, int);
template cudaError_t band_factor_solve_launch<float>(const BandArgs<float>&, int, int, cudaStream_t);
template cudaError_t band_factor_solve_launch<double>(const BandArgs<double>&, int, int, cudaStream_t);

}  // namespace stfdm
