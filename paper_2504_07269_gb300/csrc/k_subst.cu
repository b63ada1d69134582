// Forward and backward substitution with stored banded LDL^T factors (step 3 of the
// Kronecker solver, Section 3, applied with factors computed once and reused across the
// refinement iterations):  L z = g,  y = D^{-1} z,  L^T w = y,  per system k.
//
// One warp per system.  Row i of the active band is owned by lane i mod 32; each lane keeps
// its R = ceil(b/32) active rows in registers, ordered so that slot 0 is always its nearest
// row past the current column (a lane shifts its slots when it owns the pivot), which keeps
// every register index static.  A column j of L (b entries, contiguous) is read by the 32
// lanes as R coalesced 32-entry segments.  Forward: the pivot z_j is broadcast with a shuffle
// and every lane updates its rows.  Backward: every lane forms its part of the dot product
// L(j+1.., j) . w(j+1..), a butterfly reduction gives w_j.  Columns are read G at a time so
// that G * b entries per warp are in flight: the kernels stream the factors at HBM speed.
#include <cuda_runtime.h>

#include "device.cuh"

namespace stfdm {

template <typename T>
__device__ __forceinline__ C<T> shfl(C<T> v, int src) {
    return mk<T>(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

template <typename T, int R, int G>
__global__ void __launch_bounds__(128) k_subst_fwd(BandArgs<T> a, int k0, int nsys) {
    const int lane = threadIdx.x & 31;
    const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    const int n = a.n, b = a.b;
    for (int ks = wid; ks < nsys; ks += nw) {
        const int k = k0 + ks;
        C<T>* z = a.rhs + (size_t)k * n;
        const size_t slot = a.keep ? (size_t)k : (size_t)ks;
        const C<T>* L = a.L + slot * (size_t)n * b;
        const C<T>* D = a.D + slot * (size_t)n;
        C<T> zr[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int i = lane + 32 * t;
            zr[t] = (i < n) ? z[i] : mk<T>(0, 0);
        }
        C<T> outv = mk<T>(0, 0);
        for (int j0 = 0; j0 < n; j0 += G) {
            C<T> Lg[G][R];
            C<T> dg = mk<T>(1, 0);
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int j = j0 + g;
                const int o0 = ((lane - j - 1) & 31) + 1;
#pragma unroll
                for (int t = 0; t < R; ++t) {
                    const int o = o0 + 32 * t;
                    Lg[g][t] = (j < n && o <= b && j + o < n) ? L[(size_t)j * b + (o - 1)] : mk<T>(0, 0);
                }
            }
            if (lane < G && j0 + lane < n) dg = D[j0 + lane];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int j = j0 + g;
                if (j >= n) break;
                const int pl = j & 31;
                const C<T> zj = shfl<T>(zr[0], pl);
                const C<T> dj = shfl<T>(dg, g);
                if (lane == pl) {
                    outv = cmul<T>(zj, cinv<T>(dj));
#pragma unroll
                    for (int t = 0; t < R - 1; ++t) zr[t] = zr[t + 1];
                    const int inew = j + 32 * R;
                    zr[R - 1] = (inew < n) ? z[inew] : mk<T>(0, 0);
                }
#pragma unroll
                for (int t = 0; t < R; ++t) cfms<T>(zr[t], Lg[g][t], zj);
                if (pl == 31 || j == n - 1) {
                    if (lane <= pl) z[j - pl + lane] = outv;
                }
            }
        }
    }
}

template <typename T, int R, int G>
__global__ void __launch_bounds__(128) k_subst_bwd(BandArgs<T> a, int k0, int nsys) {
    const int lane = threadIdx.x & 31;
    const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    const int n = a.n, b = a.b;
    for (int ks = wid; ks < nsys; ks += nw) {
        const int k = k0 + ks;
        C<T>* z = a.rhs + (size_t)k * n;  // y in, w out
        const size_t slot = a.keep ? (size_t)k : (size_t)ks;
        const C<T>* L = a.L + slot * (size_t)n * b;
        // wr[t] = w of the lane's t-th nearest solved row past the current column (0 beyond n)
        C<T> wr[R];
#pragma unroll
        for (int t = 0; t < R; ++t) wr[t] = mk<T>(0, 0);
        C<T> outv = mk<T>(0, 0);
        for (int j0 = n - 1; j0 >= 0; j0 -= G) {
            C<T> Lg[G][R];
            C<T> yg = mk<T>(0, 0);
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int j = j0 - g;
                const int o0 = ((lane - j - 1) & 31) + 1;
#pragma unroll
                for (int t = 0; t < R; ++t) {
                    const int o = o0 + 32 * t;
                    Lg[g][t] = (j >= 0 && o <= b && j + o < n) ? L[(size_t)j * b + (o - 1)] : mk<T>(0, 0);
                }
            }
            if (lane < G && j0 - lane >= 0) yg = z[j0 - lane];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int j = j0 - g;
                if (j < 0) break;
                C<T> part = mk<T>(0, 0);
#pragma unroll
                for (int t = 0; t < R; ++t) cfma<T>(part, Lg[g][t], wr[t]);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    part.x += __shfl_xor_sync(0xffffffffu, part.x, off);
                    part.y += __shfl_xor_sync(0xffffffffu, part.y, off);
                }
                const C<T> yj = shfl<T>(yg, g);
                const C<T> wj = csub<T>(yj, part);
                const int pl = j & 31;
                if (lane == pl) {
                    outv = wj;
#pragma unroll
                    for (int t = R - 1; t > 0; --t) wr[t] = wr[t - 1];
                    wr[0] = wj;
                }
                if (pl == 0 || j == 0) {
                    const int top = min(31, n - 1 - (j - pl));
                    if (lane >= pl && lane <= top) z[j - pl + lane] = outv;
                }
            }
        }
    }
}

template <typename T, int R, int G>
static cudaError_t launch_rg(const BandArgs<T>& a, int k0, int nsys, bool fwd, cudaStream_t st) {
    const int warps_per_block = 4;
    const int blocks = (nsys + warps_per_block - 1) / warps_per_block;
    if (fwd) k_subst_fwd<T, R, G><<<blocks, 32 * warps_per_block, 0, st>>>(a, k0, nsys);
    else k_subst_bwd<T, R, G><<<blocks, 32 * warps_per_block, 0, st>>>(a, k0, nsys);
    return cudaGetLastError();
}

template <typename T>
cudaError_t subst_launch(const BandArgs<T>& a, int k0, int nsys, bool fwd, cudaStream_t st);

// complex128: fewer columns per group so that the register ring fits without spilling
template <>
cudaError_t subst_launch<double>(const BandArgs<double>& a, int k0, int nsys, bool fwd, cudaStream_t st) {
    const int R = (a.b + 31) / 32;
    if (nsys <= 0) return cudaSuccess;
    if (R <= 1) return launch_rg<double, 1, 8>(a, k0, nsys, fwd, st);
    if (R <= 2) return launch_rg<double, 2, 8>(a, k0, nsys, fwd, st);
    if (R <= 4) return launch_rg<double, 4, 6>(a, k0, nsys, fwd, st);
    if (R <= 8) return launch_rg<double, 8, 4>(a, k0, nsys, fwd, st);
    if (R <= 13) return launch_rg<double, 13, 2>(a, k0, nsys, fwd, st);
    if (R <= 16) return launch_rg<double, 16, 2>(a, k0, nsys, fwd, st);
    return cudaErrorInvalidValue;
}

template <>
cudaError_t subst_launch<float>(const BandArgs<float>& a, int k0, int nsys, bool fwd, cudaStream_t st) {
    const int R = (a.b + 31) / 32;
    if (nsys <= 0) return cudaSuccess;
    if (R <= 1) return launch_rg<float, 1, 8>(a, k0, nsys, fwd, st);
    if (R <= 2) return launch_rg<float, 2, 8>(a, k0, nsys, fwd, st);
    if (R <= 4) return launch_rg<float, 4, 8>(a, k0, nsys, fwd, st);
    if (R <= 8) return launch_rg<float, 8, 6>(a, k0, nsys, fwd, st);
    if (R <= 13) return launch_rg<float, 13, 4>(a, k0, nsys, fwd, st);
    if (R <= 16) return launch_rg<float, 16, 3>(a, k0, nsys, fwd, st);
    return cudaErrorInvalidValue;
}

}  // namespace stfdm
