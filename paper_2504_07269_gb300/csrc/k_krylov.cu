// Vector kernels of the FP64 flexible GMRES that drives the mixed-precision refinement:
// multi-dot products V^H w (deterministic two-level reduction), w -= V h / x += Z y
// (multi-axpy), and scaling.  Vectors are complex128 of length n (a whole space-time array).
#include <cuda_runtime.h>

#include "device.cuh"

namespace stfdm {

constexpr int KRY_MAXV = 32;  // at most this many basis vectors in one call
constexpr int KRY_BLOCKS = 608;

// partial[b * nv + i] = sum over this block's x of conj(V_i[x]) w[x]; blockIdx.y selects a
// chunk of KRY_CHUNK vectors (w is read once per chunk)
constexpr int KRY_CHUNK = 4;
__global__ void __launch_bounds__(256) k_multidot(const double2* const* V, int nv, const double2* w, size_t n,
                                                  double2* partial) {
    __shared__ double2 red[8][KRY_CHUNK];
    const int i0 = blockIdx.y * KRY_CHUNK;
    const double2* Vc[KRY_CHUNK];
#pragma unroll
    for (int c = 0; c < KRY_CHUNK; ++c) Vc[c] = (i0 + c < nv) ? V[i0 + c] : nullptr;
    double2 acc[KRY_CHUNK];
#pragma unroll
    for (int c = 0; c < KRY_CHUNK; ++c) acc[c] = make_double2(0, 0);
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x) {
        const double2 wx = w[x];
#pragma unroll
        for (int c = 0; c < KRY_CHUNK; ++c) {
            if (Vc[c]) {
                const double2 v = Vc[c][x];
                acc[c].x += v.x * wx.x + v.y * wx.y;
                acc[c].y += v.x * wx.y - v.y * wx.x;
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < KRY_CHUNK; ++c) {
        double ax = acc[c].x, ay = acc[c].y;
        for (int off = 16; off > 0; off >>= 1) {
            ax += __shfl_down_sync(0xffffffffu, ax, off);
            ay += __shfl_down_sync(0xffffffffu, ay, off);
        }
        if (lane == 0) red[warp][c] = make_double2(ax, ay);
    }
    __syncthreads();
    if (threadIdx.x < KRY_CHUNK && i0 + (int)threadIdx.x < nv) {
        double2 s = make_double2(0, 0);
        for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) {
            s.x += red[wi][threadIdx.x].x;
            s.y += red[wi][threadIdx.x].y;
        }
        partial[(size_t)blockIdx.x * nv + i0 + threadIdx.x] = s;
    }
}

__global__ void k_multidot_finalize(const double2* partial, int nblocks, int nv, double2* out) {
    const int i = threadIdx.x;
    if (i >= nv) return;
    double2 s = make_double2(0, 0);
    for (int b = 0; b < nblocks; ++b) {
        s.x += partial[(size_t)b * nv + i].x;
        s.y += partial[(size_t)b * nv + i].y;
    }
    out[i] = s;
}

// y[x] += sign * sum_i c[i] V_i[x]
__global__ void __launch_bounds__(256) k_multiaxpy(const double2* const* V, int nv, const double2* c, double sign,
                                                   double2* y, size_t n) {
    __shared__ double2 cs[KRY_MAXV];
    if (threadIdx.x < nv) cs[threadIdx.x] = c[threadIdx.x];
    __syncthreads();
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x) {
        double2 acc = y[x];
        for (int i = 0; i < nv; ++i) {
            const double2 v = V[i][x];
            const double2 ci = cs[i];
            acc.x += sign * (ci.x * v.x - ci.y * v.y);
            acc.y += sign * (ci.x * v.y + ci.y * v.x);
        }
        y[x] = acc;
    }
}

// y = alpha * x (real alpha)
__global__ void k_scale(const double2* x, double alpha, double2* y, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double2 v = x[i];
        y[i] = make_double2(alpha * v.x, alpha * v.y);
    }
}

__global__ void k_set_scalars(double* dst, double a, double b) {
    dst[0] = a;
    dst[1] = b;
}

cudaError_t launch_multidot(const double2* const* Vdev, int nv, const double2* w, size_t n, double2* partial,
                            double2* out, cudaStream_t st) {
    if (nv < 1 || nv > KRY_MAXV) return cudaErrorInvalidValue;
    dim3 grid(KRY_BLOCKS, (nv + KRY_CHUNK - 1) / KRY_CHUNK);
    k_multidot<<<grid, 256, 0, st>>>(Vdev, nv, w, n, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_multidot_finalize<<<1, KRY_MAXV, 0, st>>>(partial, KRY_BLOCKS, nv, out);
    note_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_multiaxpy(const double2* const* Vdev, int nv, const double2* c, double sign, double2* y, size_t n,
                             cudaStream_t st) {
    if (nv < 1 || nv > KRY_MAXV) return cudaErrorInvalidValue;
    k_multiaxpy<<<KRY_BLOCKS, 256, 0, st>>>(Vdev, nv, c, sign, y, n);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_scale(const double2* x, double alpha, double2* y, size_t n, cudaStream_t st) {
    k_scale<<<KRY_BLOCKS, 256, 0, st>>>(x, alpha, y, n);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_set_scalars(double* dst, double a, double b, cudaStream_t st) {
    k_set_scalars<<<1, 1, 0, st>>>(dst, a, b);
    note_launches(1);
    return cudaGetLastError();
}

int krylov_partial_count() { return KRY_BLOCKS * KRY_MAXV; }
int krylov_max_vectors() { return KRY_MAXV; }

}  // namespace stfdm
