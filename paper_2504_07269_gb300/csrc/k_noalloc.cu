// st_residual_noalloc: the FP64 Kronecker residual with its norms, for callers that must
// not allocate device memory while they run.
//
// Who needs it: code that owns all device memory through its own pool and forbids driver
// allocations after start-up, and loops that cannot afford cudaMalloc's implicit device-wide
// synchronisation.  The handle
// (st_fdm_setup) is still created beforehand, at a point where allocating is fine.
//
// The only scratch the computation needs -- one pair of partial sums per thread block -- lives
// in a fixed, file-scope device array below instead of handle workspace.  A_x psi0 is formed
// inside the kernel from psi0, so no vector buffer is needed either.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "device.cuh"

namespace stfdm {
namespace {

constexpr int NOALLOC_THREADS = 256;     // spatial nodes per block
constexpr int NOALLOC_ROWS = 16;         // time rows per block
constexpr int NOALLOC_MAX_BLOCKS = 65536;

// Partial sums (||R||^2, ||F~||^2) of every block: 65536 blocks x 2 doubles = 1 MiB.  It is
// loaded with the library's code on every device that uses it and stays there until the
// process exits.  All calls share it and it keeps the previous call's contents; each call
// writes every slot it reads, so nothing has to be cleared.  Calls that overlap on the GPU
// (on different streams, or from different host threads) race on it.
static __device__ __align__(256) double g_noalloc_partials[2 * NOALLOC_MAX_BLOCKS];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

struct NaStencil {
    int m;
    double Mc, Mw, Ms, Md, Ac, Aw, As, Ad;
};

__device__ __forceinline__ void na_stencil(const NaStencil& s, const double2* u, int x, double2& Pm, double2& Qa) {
    const int m = s.m;
    const int xi = x % m, yj = x / m;
    double2 c = u[x];
    double2 we = make_double2(0, 0), sn = make_double2(0, 0), dg = make_double2(0, 0);
    if (xi > 0) { we.x += u[x - 1].x; we.y += u[x - 1].y; }
    if (xi < m - 1) { we.x += u[x + 1].x; we.y += u[x + 1].y; }
    if (yj > 0) { sn.x += u[x - m].x; sn.y += u[x - m].y; }
    if (yj < m - 1) { sn.x += u[x + m].x; sn.y += u[x + m].y; }
    if (xi > 0 && yj > 0) { dg.x += u[x - m - 1].x; dg.y += u[x - m - 1].y; }
    if (xi < m - 1 && yj < m - 1) { dg.x += u[x + m + 1].x; dg.y += u[x + m + 1].y; }
    Pm = make_double2(s.Mc * c.x + s.Mw * we.x + s.Ms * sn.x + s.Md * dg.x,
                      s.Mc * c.y + s.Mw * we.y + s.Ms * sn.y + s.Md * dg.y);
    Qa = make_double2(s.Ac * c.x + s.Aw * we.x + s.As * sn.x + s.Ad * dg.x,
                      s.Ac * c.y + s.Aw * we.y + s.As * sn.y + s.Ad * dg.y);
}

__device__ __forceinline__ double na_block_sum(double v, double* red) {
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

// R = F - m_t (x) A_x psi0 - K (psi - 1 (x) psi0), K = i B_t (x) M_x + M_t (x) A_x, and the
// block's partial sums of |R|^2 and |F~|^2 into partials[2 * block].
__global__ void __launch_bounds__(NOALLOC_THREADS)
k_residual_noalloc(int n_t, int n_x, NaStencil s, const double* Mb, const double* Bb, const double* m_t,
                   const double2* F, const double2* psi0, const double2* psi, double2* R, double* partials) {
    __shared__ double red[32];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int l0 = blockIdx.y * NOALLOC_ROWS;
    const int l1 = min(l0 + NOALLOC_ROWS, n_t);
    double rr = 0, ff = 0;
    if (x < n_x) {
        double2 P0 = make_double2(0, 0), Q0 = make_double2(0, 0);
        if (psi0) na_stencil(s, psi0, x, P0, Q0);       // Q0 = (A_x psi0)[x]
        double2 P[5], Q[5];
        auto row = [&](int k, double2& p, double2& q) {
            if (k < 0 || k >= n_t) {
                p = make_double2(0, 0);
                q = make_double2(0, 0);
                return;
            }
            na_stencil(s, psi + (size_t)k * n_x, x, p, q);
            p.x -= P0.x; p.y -= P0.y;
            q.x -= Q0.x; q.y -= Q0.y;
        };
        for (int d = 1; d < 5; ++d) row(l0 - 3 + d, P[d], Q[d]);
        for (int l = l0; l < l1; ++l) {
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                P[d] = P[d + 1];
                Q[d] = Q[d + 1];
            }
            row(l + 2, P[4], Q[4]);
            const double2 f = F[(size_t)l * n_x + x];
            const double ml = m_t[l];
            const double2 ft = make_double2(f.x - ml * Q0.x, f.y - ml * Q0.y);
            double2 kv = make_double2(0, 0);
#pragma unroll
            for (int d = 0; d < 5; ++d) {
                const double bc = Bb[l * 5 + d], mc = Mb[l * 5 + d];
                kv.x += -bc * P[d].y + mc * Q[d].x;
                kv.y += bc * P[d].x + mc * Q[d].y;
            }
            const double2 r = make_double2(ft.x - kv.x, ft.y - kv.y);
            if (R) R[(size_t)l * n_x + x] = r;
            rr += r.x * r.x + r.y * r.y;
            ff += ft.x * ft.x + ft.y * ft.y;
        }
    }
    const double s1 = na_block_sum(rr, red);
    const double s2 = na_block_sum(ff, red);
    if (threadIdx.x == 0) {
        const size_t bid = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        partials[2 * bid] = s1;
        partials[2 * bid + 1] = s2;
    }
}

// norms[0] = ||R||^2, norms[1] = ||F~||^2 (fixed summation order: deterministic)
__global__ void k_noalloc_finalize(const double* partials, int nparts, double* norms) {
    __shared__ double red[32];
    double s1 = 0, s2 = 0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        s1 += partials[2 * i];
        s2 += partials[2 * i + 1];
    }
    const double t1 = na_block_sum(s1, red);
    const double t2 = na_block_sum(s2, red);
    if (threadIdx.x == 0) {
        norms[0] = t1;
        norms[1] = t2;
    }
}

// Device address of the partial-sum array on `dev`, looked up once per device (with that
// device current) and cached.
st_status noalloc_scratch(int dev, double** out) {
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(ST_ERR_UNSUPPORTED, "st_residual_noalloc: device ordinal");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p)
            return fail(ST_ERR_CUDA, std::string("st_residual_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_noalloc_addr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_addr[dev];
    return ST_OK;
}

}  // namespace
}  // namespace stfdm

using namespace stfdm;

extern "C" st_status st_residual_noalloc(const st_fdm* h, const void* F, const void* psi0, const void* psi, void* R,
                                         double* norms, void* stream) {
    if (!h || !F || !psi || !norms) return fail(ST_ERR_ARG, "st_residual_noalloc: NULL argument");
    if (h->sm.kind != 0) return fail(ST_ERR_UNSUPPORTED, "st_residual_noalloc: structured grids only");
    // R is written while other threads still read the stencil neighbours of psi and psi0
    if (R && (R == psi || R == psi0)) return fail(ST_ERR_ARG, "st_residual_noalloc: R must not alias psi or psi0");
    const int n_t = h->tm.n_t, n_x = h->sm.n_x;
    const dim3 grid((n_x + NOALLOC_THREADS - 1) / NOALLOC_THREADS, (n_t + NOALLOC_ROWS - 1) / NOALLOC_ROWS);
    const size_t nblocks = (size_t)grid.x * grid.y;
    if (nblocks > (size_t)NOALLOC_MAX_BLOCKS)
        return fail(ST_ERR_ARG, "st_residual_noalloc: problem too large for the fixed scratch (at most " +
                                    std::to_string(NOALLOC_MAX_BLOCKS) + " blocks of 256 nodes x 16 time rows, got " +
                                    std::to_string(nblocks) + ")");
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return fail(ST_ERR_CUDA, "st_residual_noalloc: cudaGetDevice");
    if (prev != h->device && cudaSetDevice(h->device) != cudaSuccess)
        return fail(ST_ERR_CUDA, "st_residual_noalloc: cudaSetDevice");
    double* partials = nullptr;
    st_status s = noalloc_scratch(h->device, &partials);
    if (s == ST_OK) {
        const SpaceMats& sm = h->sm;
        const NaStencil st{sm.m, sm.Mc, sm.Mw, sm.Ms, sm.Md, sm.Ac, sm.Aw, sm.As, sm.Ad};
        cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
        k_residual_noalloc<<<grid, NOALLOC_THREADS, 0, cs>>>(
            n_t, n_x, st, h->dt.Mb, h->dt.Bb, h->dt.m, static_cast<const double2*>(F),
            static_cast<const double2*>(psi0), static_cast<const double2*>(psi), static_cast<double2*>(R), partials);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) {
            k_noalloc_finalize<<<1, 256, 0, cs>>>(partials, (int)nblocks, norms);
            e = cudaGetLastError();
            if (e == cudaSuccess) note_launches(2);
        }
        if (e != cudaSuccess) s = fail(ST_ERR_CUDA, std::string("st_residual_noalloc: launch: ") + cudaGetErrorString(e));
    }
    if (prev != h->device) cudaSetDevice(prev);
    return s;
}
