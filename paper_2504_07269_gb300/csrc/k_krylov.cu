// Vector kernels of the FP64 flexible GMRES that drives the mixed-precision refinement:
// multi-dot products V^H w (deterministic two-level reduction), w -= V h / x += Z y
// (multi-axpy), and scaling.  Vectors are complex128 of length n (a whole space-time array).
#include <cuda_runtime.h>

#include "device.cuh"

namespace stfdm {

constexpr int KRY_MAXV = 32;  // at most this many basis vectors in one call
constexpr int KRY_BLOCKS = 608;

// The FP64 pipe, not the bytes, bounds these kernels on GB300 (a complex multiply-add is four FP64
// FMAs per 16 bytes read): every complex product is written as exactly four fused multiply-adds.

// acc += conj(v) d
__device__ __forceinline__ void cdot_acc(double2& acc, double2 v, double2 d) {
    acc.x = fma(v.x, d.x, acc.x);
    acc.x = fma(v.y, d.y, acc.x);
    acc.y = fma(v.x, d.y, acc.y);
    acc.y = fma(-v.y, d.x, acc.y);
}
// d -= c v
__device__ __forceinline__ void caxpy_sub(double2& d, double2 c, double2 v) {
    d.x = fma(-c.x, v.x, d.x);
    d.x = fma(c.y, v.y, d.x);
    d.y = fma(-c.x, v.y, d.y);
    d.y = fma(-c.y, v.x, d.y);
}

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
                cdot_acc(acc[c], v, wx);
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
    if (threadIdx.x < nv) cs[threadIdx.x] = make_double2(-sign * c[threadIdx.x].x, -sign * c[threadIdx.x].y);
    __syncthreads();
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x) {
        double2 acc = y[x];
        for (int i = 0; i < nv; ++i) caxpy_sub(acc, cs[i], V[i][x]);
        y[x] = acc;
    }
}

// One Gram-Schmidt pass of the Arnoldi step on d = w - V_s (s = shift >= 0; d = w when shift < 0).
// Project: partial[b * (nv + 1) + i] = this block's part of conj(V_i)^T d for i < nv, and of ||d||^2 in
// slot nv; blockIdx.y selects a chunk of GS_CHUNK vectors (w and V_s are read once per chunk, the
// norm is summed by chunk 0 only).  Chunks of 4 with five blocks per SM ran faster than chunks of 8
// (three blocks per SM) or 16 (two): 79 / 107 / 206 ms per 384^2/P2-1024 solve.
constexpr int GS_CHUNK = 4;
constexpr int GS_BLOCKS = 760;   // 5 x 152 SMs: k_gs_project (48 registers) keeps five 256-thread blocks per SM
__global__ void __launch_bounds__(256) k_gs_project(const double2* const* V, int nv, int shift, const double2* w,
                                                    size_t n, double2* partial) {
    __shared__ double2 red[8][GS_CHUNK + 1];
    const int i0 = blockIdx.y * GS_CHUNK;
    const int cnt = min(GS_CHUNK, nv - i0);
    const double2* Vc[GS_CHUNK];
#pragma unroll
    for (int c = 0; c < GS_CHUNK; ++c) Vc[c] = (c < cnt) ? V[i0 + c] : nullptr;
    const double2* Vs = shift >= 0 ? V[shift] : nullptr;
    double2 acc[GS_CHUNK + 1];
#pragma unroll
    for (int c = 0; c <= GS_CHUNK; ++c) acc[c] = make_double2(0, 0);
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x) {
        double2 d = w[x];
        if (Vs) {
            const double2 vs = Vs[x];
            d.x -= vs.x;
            d.y -= vs.y;
        }
#pragma unroll
        for (int c = 0; c < GS_CHUNK; ++c)
            if (Vc[c]) cdot_acc(acc[c], Vc[c][x], d);
        if (blockIdx.y == 0) {
            acc[GS_CHUNK].x = fma(d.x, d.x, acc[GS_CHUNK].x);
            acc[GS_CHUNK].x = fma(d.y, d.y, acc[GS_CHUNK].x);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c <= GS_CHUNK; ++c) {
        double ax = acc[c].x, ay = acc[c].y;
        for (int off = 16; off > 0; off >>= 1) {
            ax += __shfl_down_sync(0xffffffffu, ax, off);
            ay += __shfl_down_sync(0xffffffffu, ay, off);
        }
        if (lane == 0) red[warp][c] = make_double2(ax, ay);
    }
    __syncthreads();
    const int t = threadIdx.x;
    if (t <= GS_CHUNK) {
        const int slot = (t == GS_CHUNK) ? nv : i0 + t;
        if ((t < cnt) || (t == GS_CHUNK && blockIdx.y == 0)) {
            double2 s = make_double2(0, 0);
            for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) {
                s.x += red[wi][t].x;
                s.y += red[wi][t].y;
            }
            partial[(size_t)blockIdx.x * (nv + 1) + slot] = s;
        }
    }
}

// Update: w = d - sum_i c_i V_i (d as above), and partial[b] = this block's part of ||w||^2.
__global__ void __launch_bounds__(256) k_gs_update(const double2* const* V, int nv, int shift, const double2* c,
                                                   double2* w, size_t n, double2* partial) {
    __shared__ double2 cs[KRY_MAXV];
    __shared__ double red[8];
    if (threadIdx.x < nv) cs[threadIdx.x] = c[threadIdx.x];
    __syncthreads();
    const double2* Vs = shift >= 0 ? V[shift] : nullptr;
    double nn = 0;
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x) {
        double2 d = w[x];
        if (Vs) {
            const double2 vs = Vs[x];
            d.x -= vs.x;
            d.y -= vs.y;
        }
        for (int i = 0; i < nv; ++i) caxpy_sub(d, cs[i], V[i][x]);
        w[x] = d;
        nn = fma(d.x, d.x, nn);
        nn = fma(d.y, d.y, nn);
    }
    for (int off = 16; off > 0; off >>= 1) nn += __shfl_down_sync(0xffffffffu, nn, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = nn;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) s += red[wi];
        partial[blockIdx.x] = make_double2(s, 0);
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

cudaError_t launch_gs_project(const double2* const* Vdev, int nv, int shift, const double2* w, size_t n,
                              double2* partial, double2* out, cudaStream_t st) {
    if (nv < 1 || nv + 1 > KRY_MAXV || shift >= nv) return cudaErrorInvalidValue;
    if ((size_t)GS_BLOCKS * (nv + 1) > (size_t)KRY_BLOCKS * KRY_MAXV) return cudaErrorInvalidValue;   // partials
    dim3 grid(GS_BLOCKS, (nv + GS_CHUNK - 1) / GS_CHUNK);
    k_gs_project<<<grid, 256, 0, st>>>(Vdev, nv, shift, w, n, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_multidot_finalize<<<1, KRY_MAXV, 0, st>>>(partial, GS_BLOCKS, nv + 1, out);
    note_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_gs_update(const double2* const* Vdev, int nv, int shift, const double2* c, double2* w, size_t n,
                             double2* partial, double2* out, cudaStream_t st) {
    if (nv < 1 || nv > KRY_MAXV || shift >= nv) return cudaErrorInvalidValue;
    k_gs_update<<<KRY_BLOCKS, 256, 0, st>>>(Vdev, nv, shift, c, w, n, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_multidot_finalize<<<1, KRY_MAXV, 0, st>>>(partial, KRY_BLOCKS, 1, out);
    note_launches(2);
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
