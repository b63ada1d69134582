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
//     there; its L and L*D columns then drive a rank-NB update of the b x b trailing
//     triangle of the window, register-tiled 8 rows x 2 columns per lane;
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
//   P  [NB][WR]  panel, column-major by panel column (L after factorisation)
//   LD [NB][WR]  L * D of the panel
//   zb [WR]      circular forward-substitution vector (rows c0 .. c0+WR-1)
template <typename T, int NB>
__device__ void band_factor_one(const BandArgs<T>& a, int k, int ks, char* smem) {
    const int n = a.n, b = a.b, WR = b + NB, WB = b + 1;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
    (void)lane;
    C<T>* P = reinterpret_cast<C<T>*>(smem);
    C<T>* LD = P + NB * WR;
    C<T>* zb = LD + NB * WR;
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
        // 2. unblocked LDL^T of the panel
        for (int q = 0; q < nbk; ++q) {
            C<T> d = P[q * WR + q];
            if (bad_pivot<T>(d)) {
                if (tid == 0) atomicExch(a.status, 1);
                d = mk<T>((T)1e-30, 0);
            }
            const C<T> dinv = cinv<T>(d);
            for (int r = q + 1 + tid; r < rows_p; r += nth) P[q * WR + r] = cmul<T>(P[q * WR + r], dinv);
            __syncthreads();
            const int rem = nbk - q - 1;
            for (int idx = tid; idx < rem * rows_p; idx += nth) {
                int q2 = q + 1 + idx / rows_p, r = idx % rows_p;
                if (r >= q2) {
                    C<T> ldq2 = cmul<T>(d, P[q * WR + q2]);
                    cfms<T>(P[q2 * WR + r], P[q * WR + r], ldq2);
                }
            }
            __syncthreads();
        }
        // 3. L*D for the trailing rows, 4. factor columns out, 5a. panel forward substitution
        for (int idx = tid; idx < NB * WR; idx += nth) {
            int q = idx / WR, r = idx - q * WR;
            if (q < nbk && r >= nbk && r < rows_p) LD[idx] = cmul<T>(P[idx], P[q * WR + q]);
        }
        for (int idx = tid; idx < nbk * b; idx += nth) {
            int q = idx / b, o = idx - q * b + 1;
            int r = q + o;
            Lk[(size_t)(c0 + q) * b + (o - 1)] = (r < rows_p) ? P[q * WR + r] : mk<T>(0, 0);
        }
        if (tid < nbk) Dk[c0 + tid] = P[tid * WR + tid];
        if (tid == 0) {
            for (int q = 0; q < nbk; ++q) {
                C<T> acc = zb[(c0 + q) % WR];
                for (int q1 = 0; q1 < q; ++q1) cfms<T>(acc, P[q1 * WR + q], zb[(c0 + q1) % WR]);
                zb[(c0 + q) % WR] = acc;
            }
        }
        __syncthreads();
        // 5b. forward substitution below the panel; y = z / d of the panel rows out
        for (int r = nbk + tid; r < rows_p; r += nth) {
            C<T> acc = zb[(c0 + r) % WR];
            for (int q = 0; q < nbk; ++q) cfms<T>(acc, P[q * WR + r], zb[(c0 + q) % WR]);
            zb[(c0 + r) % WR] = acc;
        }
        if (tid < nbk) z[c0 + tid] = cmul<T>(zb[(c0 + tid) % WR], cinv<T>(P[tid * WR + tid]));
        __syncthreads();
        // 6. trailing update of the b x b triangle: W(r, r2) -= sum_q L(r, q) (L D)(r2, q)
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
                    for (int q = 0; q < nbk; ++q) {
                        const C<T> a0 = LD[q * WR + ci0];
                        const C<T> a1 = LD[q * WR + ci1];
                        const C<T>* prow = P + q * WR + nbk + rr0;
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const C<T> p = prow[min(j, WR - 1 - nbk - rr0)];
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
__global__ void __launch_bounds__(256) k_band_factor_solve(BandArgs<T> a) {
    extern __shared__ __align__(16) char smem[];
    for (int ks = blockIdx.x; ks < a.n_sys; ks += gridDim.x) {
        band_factor_one<T, NB>(a, a.k0 + ks, ks, smem);
        __syncthreads();
    }
}

template <typename T, int NB>
size_t band_factor_smem(int b) {
    const int WR = b + NB;
    return sizeof(C<T>) * ((size_t)2 * NB * WR + WR);
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
    if (band_factor_smem<T, 16>(b) <= smem_optin) return 16;
    if (band_factor_smem<T, 8>(b) <= smem_optin) return 8;
    return 0;
}

template <typename T>
size_t band_smem_for(int nb, int b) {
    return nb == 16 ? band_factor_smem<T, 16>(b) : band_factor_smem<T, 8>(b);
}

template <typename T>
cudaError_t band_factor_solve_launch(const BandArgs<T>& a, int nb, int grid, cudaStream_t st) {
    if (nb == 16) return launch_factor_nb<T, 16>(a, grid, st);
    return launch_factor_nb<T, 8>(a, grid, st);
}
template <typename T>
int band_occupancy(int nb, int b) {
    int occ = 0;
    size_t smem = band_smem_for<T>(nb, b);
    if (nb == 16) {
        cudaFuncSetAttribute(k_band_factor_solve<T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_band_factor_solve<T, 16>, 256, smem);
    } else {
        cudaFuncSetAttribute(k_band_factor_solve<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_band_factor_solve<T, 8>, 256, smem);
    }
    cudaGetLastError();
    return occ;
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
