// Step 3 of the Kronecker solver (Section 3, eq. LGS_x, fast-diagonalisation choice) on general
// meshes: the n_t independent spatial systems C_k w_k = g_k, C_k = M_x + s_k A_x (complex
// symmetric), by a sparse direct multifrontal LDL^T factorisation without pivoting (Im s_k < 0
// makes Im C_k definite, so every principal submatrix is nonsingular in any ordering).  The
// ordering and assembly tree come from the host plan (nested dissection, host_mf.cpp); every C_k
// has the same sparsity, so the device work is batched over k.
//
// Launch levels are fronts of equal height in the assembly tree.  Fronts of up to 64 rows are
// factorised by one warp each (the whole lower triangle in shared memory), fronts of up to 128 rows
// are solved by one warp each (the front vector in registers); the larger ones take one CTA per
// (front, system k):
//   factor  the front (np pivots, nu update rows, f = np + nu) is assembled from the entries of
//           M_x + s_k A_x in its pivot columns and the children's update matrices (extend-add),
//           then its pivot columns are factorised by 32-column panels: the panel's top block by an
//           unscaled right-looking elimination in shared memory, the rows below by a per-row
//           substitution against it, the remaining pivot columns by a rank-32 update in 64 x 64
//           register tiles.  The update matrix for the parent then takes one symmetric rank-np
//           update over all pivot columns (each 64 x 64 tile read and written once).  The front
//           lives in global memory: the pivot columns (f x np, column-major) are the stored factor
//           (L below the diagonal, D on it); the trailing nu x nu block is the update matrix.
//   forward front vector = right-hand side at the pivots + the children's update vectors; the
//           unit lower pivot block is solved by 32-row blocks (warp 0 by shuffles, the rows below
//           by all threads); y = z / d goes to the solution, the rest to the update vector.
//   backward from the root down: the update rows' solutions (ancestors' pivots) are gathered,
//           the pivot block's transposed system is solved by 32-row blocks from the bottom.
// Solutions stay in the caller's node order: the kernels index through the permutation.
#include <cuda_runtime.h>

#include <algorithm>

#include "device.cuh"

namespace stfdm {

template <typename T> struct MfNB;
template <> struct MfNB<float> { static constexpr int v = 32; };
template <> struct MfNB<double> { static constexpr int v = 16; };

constexpr int MF_THREADS = 256;
constexpr int MF_TILE = 64;

template <typename T>
__device__ __forceinline__ C<T> shfl_c(C<T> v, int src) {
    return mk<T>(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

template <typename T>
__device__ __forceinline__ bool mf_bad(C<T> d) {
    const T a = fabs(d.x) + fabs(d.y);
    return !(a > (T)0) || !isfinite(a);
}

// ------------------------------------------------------------------ factorisation
// 4 consecutive complex entries from shared memory (16-byte aligned): two 16-byte loads for
// complex64, four for complex128
template <typename T>
__device__ __forceinline__ void ld4(const C<T>* p, C<T> (&v)[4]);
template <>
__device__ __forceinline__ void ld4<float>(const float2* p, float2 (&v)[4]) {
    const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
    v[0] = make_float2(a.x, a.y);
    v[1] = make_float2(a.z, a.w);
    v[2] = make_float2(b.x, b.y);
    v[3] = make_float2(b.z, b.w);
}
template <>
__device__ __forceinline__ void ld4<double>(const double2* p, double2 (&v)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = p[i];
}

// Symmetric rank-k update of the front's lower triangle, dst(r, c) -= sum_q L(r, q) d_q L(c, q) over
// the pivot columns q in [qa, qb), for rows r in [base, rend) and columns c in [base, cend), c <= r.
// 64 x 64 tiles; per tile the sum runs over all of [qa, qb) in register accumulators (4 x 4 complex
// per thread) and the destination is read and written once.  Operands are staged q-major in shared
// memory (As[q][row], Bs[q][col] = L d) by chunks of NB columns.  The (tile, chunk) steps form one
// sequence, and the next step's operands (the next chunk, or the next tile's first chunk) are loaded
// into registers while the current one is multiplied, so a tile's loads overlap the previous tile's
// products and write-back.  d_q is read from the factor's diagonal (written before the call).
template <typename T, typename At>
__device__ __forceinline__ void mf_syrk_tiles(const C<T>* Fp, int f, int base, int rend, int cend, int qa, int qb,
                                              C<T>* As, C<T>* Bs, At at) {
    constexpr int NB = MfNB<T>::v;
    constexpr int PER = NB * MF_TILE / MF_THREADS;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int ntr = (rend - base + MF_TILE - 1) / MF_TILE, ntc = (cend - base + MF_TILE - 1) / MF_TILE;
    const int nch = (qb - qa + NB - 1) / NB;
    if (ntc <= 0 || ntr <= 0 || nch <= 0) return;
    C<T> ra[PER], rbv[PER];
    auto fetch = [&](int I, int J, int c) {
        const int rb = base + I * MF_TILE, cb = base + J * MF_TILE, q0 = qa + c * NB;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = tid + k * MF_THREADS, q = q0 + e / MF_TILE, rr = e % MF_TILE;
            const bool okq = q < qb;
            ra[k] = (okq && rb + rr < rend) ? Fp[(size_t)q * f + rb + rr] : mk<T>(0, 0);
            rbv[k] = (okq && cb + rr < cend) ? Fp[(size_t)q * f + cb + rr] : mk<T>(0, 0);
        }
    };
    C<T> acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = mk<T>(0, 0);
    int I = 0, J = 0, c = 0;   // the current step: tile (I, J), I >= J, column chunk c
    fetch(0, 0, 0);
    while (true) {
        const int q0 = qa + c * NB;
        __syncthreads();   // the previous step's products are done with As / Bs
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = tid + k * MF_THREADS, q = q0 + e / MF_TILE;
            As[e] = ra[k];
            Bs[e] = q < qb ? cmul<T>(rbv[k], Fp[(size_t)q * f + q]) : mk<T>(0, 0);   // d_q, an L1 hit
        }
        __syncthreads();
        int nI = I, nJ = J, nc = c + 1;
        if (nc == nch) {
            nc = 0;
            if (++nI == ntr) nI = ++nJ;
        }
        const bool more = nJ < ntc;
        if (more) fetch(nI, nJ, nc);
        const int wq = min(NB, qb - q0);
        if (wq == NB) {
#pragma unroll 4
            for (int q = 0; q < NB; ++q) {
                C<T> av[4], bv[4];
                ld4<T>(As + q * MF_TILE + tx * 4, av);
                ld4<T>(Bs + q * MF_TILE + ty * 4, bv);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) cfma<T>(acc[i][j], av[i], bv[j]);
            }
        } else {
            for (int q = 0; q < wq; ++q) {
                C<T> av[4], bv[4];
                ld4<T>(As + q * MF_TILE + tx * 4, av);
                ld4<T>(Bs + q * MF_TILE + ty * 4, bv);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) cfma<T>(acc[i][j], av[i], bv[j]);
            }
        }
        if (c == nch - 1) {   // the tile's sum is complete: subtract it from the destination
            const int rb = base + I * MF_TILE, cb = base + J * MF_TILE;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int cc = cb + ty * 4 + j;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int r = rb + tx * 4 + i;
                    if (r < rend && cc < cend && r >= cc) {
                        C<T>& dst = at(r, cc);
                        dst = csub<T>(dst, acc[i][j]);
                    }
                    acc[i][j] = mk<T>(0, 0);
                }
            }
        }
        if (!more) break;
        I = nI;
        J = nJ;
        c = nc;
    }
}

template <typename T>
__global__ void __launch_bounds__(MF_THREADS, 2) k_mf_factor(MfArgs<T> a) {
    constexpr int NB = MfNB<T>::v;
    extern __shared__ __align__(16) unsigned char mf_smem[];
    C<T>* As = reinterpret_cast<C<T>*>(mf_smem);             // [NB][MF_TILE]  rows of the tile, q-major
    C<T>* Bs = As + NB * MF_TILE;                            // [NB][MF_TILE]  columns times d, q-major
    C<T>* Tt = Bs + NB * MF_TILE;                            // [NB][NB + 1] top block, row-major
    C<T>* dinv = Tt + NB * (NB + 1);                         // [NB]
    const MfFrontDev fr = a.fronts[a.level_fronts[a.lvl_off + blockIdx.x]];
    const int k = a.k0 + blockIdx.y;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int np = fr.np, nu = fr.nu, f = np + nu;
    const C<T> s = a.shifts[k];
    C<T>* Fp = a.fac + (size_t)(a.fac_keep ? k : blockIdx.y) * a.fac_stride + fr.foff;
    C<T>* S = a.upd + (size_t)blockIdx.y * a.upd_stride + fr.uoff;
    // entry (r, c), r >= c, of the front
    auto at = [&](int r, int c) -> C<T>& { return c < np ? Fp[(size_t)c * f + r] : S[(size_t)(c - np) * nu + (r - np)]; };

    // A. assembly
    for (size_t i = tid; i < (size_t)f * np; i += nth) Fp[i] = mk<T>(0, 0);
    for (size_t i = tid; i < (size_t)nu * nu; i += nth) S[i] = mk<T>(0, 0);
    __syncthreads();
    for (int e = tid; e < fr.orig_cnt; e += nth) {
        const int q = a.orig_k[fr.orig_off + e];
        const double m = a.Mv[q], av = a.Av[q];
        Fp[(size_t)a.orig_c[fr.orig_off + e] * f + a.orig_r[fr.orig_off + e]] =
            mk<T>((T)(m + (double)s.x * av), (T)((double)s.y * av));
    }
    __syncthreads();
    // extend-add of the children's update matrices.  The child's relative positions are staged in
    // shared memory (in the operand tiles, unused until the panels), and each thread handles eight
    // entries at a time: a child's entries land on distinct positions of the front, so the eight
    // destinations are loaded together and stored together.
    constexpr int EA = 8;
    int* rps = reinterpret_cast<int*>(As);
    constexpr int RPS_CAP = (int)(2 * NB * MF_TILE * sizeof(C<T>) / sizeof(int));
    for (int ci = 0; ci < fr.child_cnt; ++ci) {
        const MfFrontDev ch = a.fronts[a.children[fr.child_off + ci]];
        const C<T>* Sc = a.upd + (size_t)blockIdx.y * a.upd_stride + ch.uoff;
        const int cn = ch.nu, tot = cn * cn;
        const int* rp = a.relpos + ch.relpos_off;
        if (cn <= RPS_CAP) {
            for (int t = tid; t < cn; t += nth) rps[t] = rp[t];
            __syncthreads();
            rp = rps;
        }
        for (int i0 = tid; i0 < tot; i0 += EA * nth) {
            C<T>* dp[EA];
            C<T> v[EA];
#pragma unroll
            for (int u = 0; u < EA; ++u) {
                const int i = i0 + u * nth;
                const int t2 = i / cn, t1 = i - t2 * cn;
                const bool ok = i < tot && t1 >= t2;
                dp[u] = ok ? &at(rp[t1], rp[t2]) : nullptr;
                v[u] = ok ? Sc[i] : mk<T>(0, 0);
            }
            C<T> d[EA];
#pragma unroll
            for (int u = 0; u < EA; ++u) d[u] = dp[u] ? *dp[u] : mk<T>(0, 0);
#pragma unroll
            for (int u = 0; u < EA; ++u)
                if (dp[u]) *dp[u] = cadd<T>(d[u], v[u]);
        }
        __syncthreads();
    }

    // B. LDL^T of the pivot columns, panels of NB columns; the trailing update of each panel reaches
    //    only the remaining pivot columns (all their rows)
    for (int c0 = 0; c0 < np; c0 += NB) {
        const int w = min(NB, np - c0);
        for (int i = tid; i < NB * NB; i += nth) {
            const int r = i / NB, q = i - r * NB;
            Tt[r * (NB + 1) + q] = (r < w && q <= r) ? Fp[(size_t)(c0 + q) * f + c0 + r] : mk<T>(0, 0);
        }
        __syncthreads();
        // unscaled right-looking elimination of the top block: column q below the diagonal ends as
        // d_q L(r, q), the diagonal as d_q
        for (int q = 0; q < w; ++q) {
            C<T> d = Tt[q * (NB + 1) + q];
            if (mf_bad<T>(d)) d = mk<T>((T)1e-30, 0);
            const C<T> di = cinv<T>(d);
            const int rem = w - q - 1;
            for (int i = tid; i < rem * rem; i += nth) {
                const int r = q + 1 + i / rem, c = q + 1 + i % rem;
                if (c > r) continue;
                const C<T> lrq = cmul<T>(Tt[r * (NB + 1) + q], di);
                cfms<T>(Tt[r * (NB + 1) + c], lrq, Tt[c * (NB + 1) + q]);
            }
            __syncthreads();
        }
        if (tid < w) {
            C<T> d = Tt[tid * (NB + 1) + tid];
            if (mf_bad<T>(d)) {
                atomicExch(a.status, 1);
                d = mk<T>((T)1e-30, 0);
                Tt[tid * (NB + 1) + tid] = d;
            }
            dinv[tid] = cinv<T>(d);
        }
        __syncthreads();
        for (int i = tid; i < w * w; i += nth) {
            const int q = i / w, r = i - q * w;
            if (r < q) continue;
            Fp[(size_t)(c0 + q) * f + c0 + r] = (r == q) ? Tt[r * (NB + 1) + q] : cmul<T>(Tt[r * (NB + 1) + q], dinv[q]);
        }
        // rows below the top block: L(r, q) = (A(r, q) - sum_{q' < q} L(r, q') d_q' L(q, q')) / d_q
        for (int r = c0 + w + tid; r < f; r += nth) {
            C<T> l[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                if (q < w) {
                    C<T> acc = Fp[(size_t)(c0 + q) * f + r];
#pragma unroll
                    for (int q1 = 0; q1 < q; ++q1) cfms<T>(acc, l[q1], Tt[q * (NB + 1) + q1]);
                    l[q] = cmul<T>(acc, dinv[q]);
                } else {
                    l[q] = mk<T>(0, 0);
                }
            }
#pragma unroll
            for (int q = 0; q < NB; ++q)
                if (q < w) Fp[(size_t)(c0 + q) * f + r] = l[q];
        }
        __syncthreads();
        if (c0 + w < np) mf_syrk_tiles<T>(Fp, f, c0 + w, f, np, c0, c0 + w, As, Bs, at);
        __syncthreads();
    }
    // C. the update matrix for the parent: S -= L_u D L_u^T over all np pivot columns at once
    if (nu > 0) mf_syrk_tiles<T>(Fp, f, np, f, f, 0, np, As, Bs, at);
}

// ------------------------------------------------------------------ substitutions
// forward: y = D^{-1} L^{-1} (g + children's update vectors) at the pivots, update vector out
template <typename T>
__global__ void __launch_bounds__(MF_THREADS) k_mf_fwd(MfArgs<T> a) {
    extern __shared__ __align__(16) unsigned char mf_smem[];
    C<T>* tri = reinterpret_cast<C<T>*>(mf_smem);  // [32][33] the block's triangle of L, staged
    C<T>* x = tri + 32 * 33;                        // [f]
    const MfFrontDev fr = a.fronts[a.level_fronts[a.lvl_off + blockIdx.x]];
    const int k = a.k0 + blockIdx.y;
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int np = fr.np, nu = fr.nu, f = np + nu;
    const C<T>* Fp = a.fac + (size_t)(a.fac_keep ? k : blockIdx.y) * a.fac_stride + fr.foff;
    C<T>* g = a.rhs + (size_t)k * a.n;
    C<T>* uv = a.uvec + (size_t)blockIdx.y * a.uvec_stride;
    for (int t = tid; t < f; t += nth) x[t] = t < np ? g[a.perm[fr.first + t]] : mk<T>(0, 0);
    __syncthreads();
    for (int ci = 0; ci < fr.child_cnt; ++ci) {
        const MfFrontDev ch = a.fronts[a.children[fr.child_off + ci]];
        const int* rp = a.relpos + ch.relpos_off;
        for (int t = tid; t < ch.nu; t += nth) {
            const C<T> v = uv[ch.uvoff + t];
            C<T>& d = x[rp[t]];
            d.x += v.x;
            d.y += v.y;
        }
        __syncthreads();
    }
    for (int q0 = 0; q0 < np; q0 += 32) {
        const int wq = min(32, np - q0);
        // stage the block's triangle (coalesced: consecutive threads, consecutive rows of a column)
        for (int i = tid; i < wq * 32; i += nth) {
            const int c = i >> 5, r = i & 31;
            if (r < wq) tri[r * 33 + c] = Fp[(size_t)(q0 + c) * f + q0 + r];
        }
        __syncthreads();
        if (warp == 0) {
            C<T> v = lane < wq ? x[q0 + lane] : mk<T>(0, 0);
            for (int q = 0; q < wq; ++q) {
                const C<T> z = shfl_c<T>(v, q);
                if (lane > q && lane < wq) cfms<T>(v, tri[lane * 33 + q], z);
            }
            if (lane < wq) x[q0 + lane] = v;
        }
        __syncthreads();
        for (int r = q0 + wq + tid; r < f; r += nth) {
            C<T> acc = x[r];
            for (int q = 0; q < wq; ++q) cfms<T>(acc, Fp[(size_t)(q0 + q) * f + r], x[q0 + q]);
            x[r] = acc;
        }
        __syncthreads();
    }
    for (int t = tid; t < np; t += nth) g[a.perm[fr.first + t]] = cmul<T>(x[t], cinv<T>(Fp[(size_t)t * f + t]));
    for (int t = tid; t < nu; t += nth) uv[fr.uvoff + t] = x[np + t];
}

// backward: L^T w = y over the pivot block, with the update rows' solutions known
template <typename T>
__global__ void __launch_bounds__(MF_THREADS) k_mf_bwd(MfArgs<T> a) {
    extern __shared__ __align__(16) unsigned char mf_smem[];
    C<T>* tri = reinterpret_cast<C<T>*>(mf_smem);  // [32][33] the block's triangle of L, staged
    C<T>* x = tri + 32 * 33;                        // [f]
    const MfFrontDev fr = a.fronts[a.level_fronts[a.lvl_off + blockIdx.x]];
    const int k = a.k0 + blockIdx.y;
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
    const int np = fr.np, nu = fr.nu, f = np + nu;
    const C<T>* Fp = a.fac + (size_t)(a.fac_keep ? k : blockIdx.y) * a.fac_stride + fr.foff;
    C<T>* g = a.rhs + (size_t)k * a.n;
    for (int t = tid; t < f; t += nth)
        x[t] = g[a.perm[t < np ? fr.first + t : a.urows[fr.urows_off + t - np]]];
    __syncthreads();
    for (int q0 = ((np - 1) / 32) * 32; q0 >= 0; q0 -= 32) {
        const int wq = min(32, np - q0);
        // contributions of the solved rows below the block: one warp per column
        for (int q = warp; q < wq; q += nwarps) {
            const C<T>* col = Fp + (size_t)(q0 + q) * f;
            // four independent partial sums keep four loads per lane in flight
            C<T> acc4[4] = {mk<T>(0, 0), mk<T>(0, 0), mk<T>(0, 0), mk<T>(0, 0)};
            int r = q0 + wq + lane;
            for (; r + 96 < f; r += 128) {
#pragma unroll
                for (int u = 0; u < 4; ++u) cfma<T>(acc4[u], col[r + 32 * u], x[r + 32 * u]);
            }
            for (; r < f; r += 32) cfma<T>(acc4[0], col[r], x[r]);
            C<T> acc = cadd<T>(cadd<T>(acc4[0], acc4[1]), cadd<T>(acc4[2], acc4[3]));
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
            }
            if (lane == 0) x[q0 + q] = csub<T>(x[q0 + q], acc);
        }
        for (int i = tid; i < wq * 32; i += nth) {
            const int c = i >> 5, r = i & 31;
            if (r < wq) tri[r * 33 + c] = Fp[(size_t)(q0 + c) * f + q0 + r];
        }
        __syncthreads();
        if (warp == 0) {
            C<T> v = lane < wq ? x[q0 + lane] : mk<T>(0, 0);
            for (int i = wq - 1; i >= 0; --i) {
                const C<T> wi = shfl_c<T>(v, i);
                if (lane < i) cfms<T>(v, tri[i * 33 + lane], wi);
            }
            if (lane < wq) x[q0 + lane] = v;
        }
        __syncthreads();
    }
    for (int t = tid; t < np; t += nth) g[a.perm[fr.first + t]] = x[t];
}

// ------------------------------------------------------------------ small fronts
// Fronts with f <= FM (32 or 64): one warp per (front, system), W warps per CTA, the whole front's
// lower triangle packed by rows in the warp's shared-memory tile (entry (r, c), c <= r, at
// r (r + 1) / 2 + c); lane l owns rows l, l + 32, ...  Items are (front, system) pairs, system
// fastest, so the warps of a CTA share a front's metadata.
template <typename T, int FM>
struct SmallCfg {
    static constexpr int R = FM / 32;                                                      // rows per lane
    static constexpr int W = (FM == 32) ? 8 : (sizeof(T) == 4 ? 6 : 3);                    // warps per CTA
    static constexpr int TILE = FM * (FM + 1) / 2 + FM;                                    // entries per warp
    static constexpr size_t SMEM = sizeof(C<T>) * (size_t)W * TILE;
};
__device__ __forceinline__ int tri_row(int r) { return (r * (r + 1)) >> 1; }

// resident CTAs per SM that the shared-memory tiles allow (complex64 fronts of <= 32 rows: six);
// the register budget is held to it
template <typename T, int FM>
__global__ void __launch_bounds__(SmallCfg<T, FM>::W * 32, (sizeof(T) == 4 && FM == 32) ? 6 : 2)
k_mf_factor_small(MfArgs<T> a, int nfronts, int nsys) {
    using Cfg = SmallCfg<T, FM>;
    constexpr int R = Cfg::R;
    extern __shared__ __align__(16) unsigned char mf_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long item = (long long)blockIdx.x * Cfg::W + warp;
    if (item >= (long long)nfronts * nsys) return;
    const int fi = (int)(item / nsys), ks = (int)(item - (long long)fi * nsys);
    C<T>* F = reinterpret_cast<C<T>*>(mf_smem) + (size_t)warp * Cfg::TILE;
    const MfFrontDev fr = a.fronts[a.level_fronts[a.lvl_off + fi]];
    const int k = a.k0 + ks;
    const int np = fr.np, nu = fr.nu, f = np + nu;
    const C<T> s = a.shifts[k];
    C<T>* Fp = a.fac + (size_t)(a.fac_keep ? k : ks) * a.fac_stride + fr.foff;
    C<T>* S = a.upd + (size_t)ks * a.upd_stride + fr.uoff;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int r = lane + 32 * i;
        if (r < f)
            for (int c = 0; c <= r; ++c) F[tri_row(r) + c] = mk<T>(0, 0);
    }
    __syncwarp();
    for (int e = lane; e < fr.orig_cnt; e += 32) {
        const int q = a.orig_k[fr.orig_off + e];
        const double m = a.Mv[q], av = a.Av[q];
        F[tri_row(a.orig_r[fr.orig_off + e]) + a.orig_c[fr.orig_off + e]] =
            mk<T>((T)(m + (double)s.x * av), (T)((double)s.y * av));
    }
    __syncwarp();
    // extend-add: each lane loads EB of the child's entries (and their positions) before adding them
    // into the shared-memory front (EB = 4 for fronts of <= 32 rows keeps their registers within the
    // six resident CTAs the tiles allow)
    constexpr int EB = (R == 1) ? 4 : 8;
    for (int ci = 0; ci < fr.child_cnt; ++ci) {
        const MfFrontDev ch = a.fronts[a.children[fr.child_off + ci]];
        const C<T>* Sc = a.upd + (size_t)ks * a.upd_stride + ch.uoff;
        const int* rp = a.relpos + ch.relpos_off;
        const int cn = ch.nu, tot = cn * cn;
        for (int i0 = lane; i0 < tot; i0 += EB * 32) {
            int pos[EB];
            C<T> v[EB];
#pragma unroll
            for (int u = 0; u < EB; ++u) {
                const int i = i0 + 32 * u;
                const int t2 = i / cn, t1 = i - t2 * cn;
                const bool ok = i < tot && t1 >= t2;
                pos[u] = ok ? tri_row(rp[t1]) + rp[t2] : -1;
                v[u] = ok ? Sc[i] : mk<T>(0, 0);
            }
#pragma unroll
            for (int u = 0; u < EB; ++u)
                if (pos[u] >= 0) {
                    C<T>& dst = F[pos[u]];
                    dst.x += v[u].x;
                    dst.y += v[u].y;
                }
        }
        __syncwarp();
    }
    // right-looking unscaled elimination of the np pivots; the trailing block is the update matrix
    bool bad = false;
    for (int q = 0; q < np; ++q) {
        C<T> d = F[tri_row(q) + q];
        if (mf_bad<T>(d)) {
            bad = true;
            d = mk<T>((T)1e-30, 0);
        }
        const C<T> di = cinv<T>(d);
        C<T> u[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int r = lane + 32 * i;
            u[i] = (r > q && r < f) ? cmul<T>(F[tri_row(r) + q], di) : mk<T>(0, 0);   // L(r, q)
        }
        for (int c = q + 1; c < f; ++c) {
            const C<T> uc = F[tri_row(c) + q];              // d_q L(c, q), still unscaled
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const int r = lane + 32 * i;
                if (r >= c && r < f) cfms<T>(F[tri_row(r) + c], u[i], uc);
            }
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int r = lane + 32 * i;
            if (r > q && r < f) F[tri_row(r) + q] = u[i];
        }
        if (lane == 0) F[tri_row(q) + q] = d;
        __syncwarp();
    }
    if (bad && lane == 0) atomicExch(a.status, 1);
    // factor block (f x np, column-major) and update matrix (nu x nu, column-major) out
    for (int c = 0; c < np; ++c)
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int r = lane + 32 * i;
            if (r >= c && r < f) Fp[(size_t)c * f + r] = F[tri_row(r) + c];
        }
    for (int c = np; c < f; ++c)
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int r = lane + 32 * i;
            if (r >= c && r < f) S[(size_t)(c - np) * nu + (r - np)] = F[tri_row(r) + c];
        }
}

// Substitutions for fronts with f <= FM (32, 64, 96 or 128): one warp per (front, system), the front
// vector in registers
// (lane l holds rows l, l + 32, ...), the pivot value of each step broadcast by a shuffle from its
// owner, the factor entries read straight from global memory (column q of the block is contiguous,
// so a step's loads are coalesced; they do not depend on the chain and are issued ahead of it).
// Shared memory only gathers the children's update vectors (forward).
template <typename T, int FM>
struct SolveSmallCfg {
    static constexpr int R = FM / 32;
    static constexpr int W = 8;
    static constexpr size_t SMEM = sizeof(C<T>) * (size_t)W * FM;
};

template <typename T, int R>
__device__ __forceinline__ C<T> row_value(const C<T> (&v)[R], int q) {
    C<T> src = v[0];
#pragma unroll
    for (int i = 1; i < R; ++i)
        if ((q >> 5) == i) src = v[i];
    return shfl_c<T>(src, q & 31);
}

// factor entries of steps q0 .. q0 + PF - 1 (forward: column q below the diagonal) or q1 - 1 down to
// q1 - PF (backward), zero outside the front's pivot block; lane l takes rows l, l + 32, ...
template <typename T, int R, int PF>
__device__ __forceinline__ void small_load_fwd(C<T> (&Lq)[PF][R], const C<T>* Fp, int f, int np, int q0, int lane) {
#pragma unroll
    for (int u = 0; u < PF; ++u)
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int q = q0 + u, r = lane + 32 * i;
            Lq[u][i] = (q < np && r > q && r < f) ? Fp[(size_t)q * f + r] : mk<T>(0, 0);
        }
}
template <typename T, int R, int PF>
__device__ __forceinline__ void small_load_bwd(C<T> (&Lq)[PF][R], const C<T>* Fp, int f, int q1, int lane) {
#pragma unroll
    for (int u = 0; u < PF; ++u)
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int q = q1 - 1 - u, r = lane + 32 * i;
            Lq[u][i] = (q >= 0 && r > q && r < f) ? Fp[(size_t)q * f + r] : mk<T>(0, 0);
        }
}

template <typename T, int FM>
__global__ void __launch_bounds__(SolveSmallCfg<T, FM>::W * 32, sizeof(T) == 4 ? (FM == 32 ? 5 : (FM == 64 ? 4 : 2)) : 1)
k_mf_solve_small(MfArgs<T> a, int nfronts, int nsys, int fwd) {
    using Cfg = SolveSmallCfg<T, FM>;
    // PF steps' factor entries are loaded ahead of the chain.  For two rows per lane the first batch
    // is issued before the right-hand side and the children's update vectors are gathered, so both
    // latencies overlap; for one row per lane the registers this takes cost more resident warps
    // than the overlap gains, and every batch is loaded where it is used.
    constexpr int R = Cfg::R, PF = 8;
    constexpr bool HOIST = (R > 1);
    extern __shared__ __align__(16) unsigned char mf_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long item = (long long)blockIdx.x * Cfg::W + warp;
    if (item >= (long long)nfronts * nsys) return;
    const int fi = (int)(item / nsys), ks = (int)(item - (long long)fi * nsys);
    const MfFrontDev fr = a.fronts[a.level_fronts[a.lvl_off + fi]];
    const int k = a.k0 + ks;
    const int np = fr.np, nu = fr.nu, f = np + nu;
    const C<T>* Fp = a.fac + (size_t)(a.fac_keep ? k : ks) * a.fac_stride + fr.foff;
    C<T>* g = a.rhs + (size_t)k * a.n;
    C<T> v[R];
    C<T> Lq[PF][R];
    if (fwd) {
        if (HOIST) small_load_fwd<T, R, PF>(Lq, Fp, f, np, 0, lane);
        C<T>* uv = a.uvec + (size_t)ks * a.uvec_stride;
        C<T>* x = reinterpret_cast<C<T>*>(mf_smem) + (size_t)warp * FM;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int r = lane + 32 * i;
            if (r < f) x[r] = r < np ? g[a.perm[fr.first + r]] : mk<T>(0, 0);
        }
        __syncwarp();
        for (int ci = 0; ci < fr.child_cnt; ++ci) {
            const MfFrontDev ch = a.fronts[a.children[fr.child_off + ci]];
            const int* rp = a.relpos + ch.relpos_off;
            for (int t = lane; t < ch.nu; t += 32) {
                const C<T> u = uv[ch.uvoff + t];
                C<T>& d = x[rp[t]];
                d.x += u.x;
                d.y += u.y;
            }
            __syncwarp();
        }
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int r = lane + 32 * i;
            v[i] = r < f ? x[r] : mk<T>(0, 0);
        }
        for (int q0 = 0; q0 < np; q0 += PF) {
            if (q0 > 0 || !HOIST) small_load_fwd<T, R, PF>(Lq, Fp, f, np, q0, lane);
#pragma unroll
            for (int u = 0; u < PF; ++u) {
                const int q = q0 + u;
                if (q >= np) break;
                const C<T> z = row_value<T, R>(v, q);
#pragma unroll
                for (int i = 0; i < R; ++i) cfms<T>(v[i], Lq[u][i], z);   // zero entries above the step
            }
        }
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int r = lane + 32 * i;
            if (r < np) g[a.perm[fr.first + r]] = cmul<T>(v[i], cinv<T>(Fp[(size_t)r * f + r]));
            else if (r < f) uv[fr.uvoff + r - np] = v[i];
        }
    } else {
        if (HOIST) small_load_bwd<T, R, PF>(Lq, Fp, f, np, lane);
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int r = lane + 32 * i;
            v[i] = r < f ? g[a.perm[r < np ? fr.first + r : a.urows[fr.urows_off + r - np]]] : mk<T>(0, 0);
        }
        for (int q1 = np; q1 > 0; q1 -= PF) {
            if (q1 < np || !HOIST) small_load_bwd<T, R, PF>(Lq, Fp, f, q1, lane);
#pragma unroll
            for (int u = 0; u < PF; ++u) {
                const int q = q1 - 1 - u;
                if (q < 0) break;
                C<T> acc = mk<T>(0, 0);
#pragma unroll
                for (int i = 0; i < R; ++i) cfma<T>(acc, Lq[u][i], v[i]);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
                    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
                }
                if (lane == (q & 31)) {
#pragma unroll
                    for (int i = 0; i < R; ++i)
                        if ((q >> 5) == i) v[i] = csub<T>(v[i], acc);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int r = lane + 32 * i;
            if (r < np) g[a.perm[fr.first + r]] = v[i];
        }
    }
}

template <typename T, int FM>
cudaError_t mf_small_launch(MfArgs<T> a, int lvl_off, int nfronts, int nsys, int what, cudaStream_t st) {
    using Cfg = SmallCfg<T, FM>;
    if (nfronts <= 0 || nsys <= 0) return cudaSuccess;
    a.lvl_off = lvl_off;
    const long long items = (long long)nfronts * nsys;
    const long long blocks = (items + Cfg::W - 1) / Cfg::W;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    cudaError_t e;
    if (what == 0) {
        if constexpr (FM <= 64) {   // larger fronts are factorised by the CTA kernel
            e = cudaFuncSetAttribute(k_mf_factor_small<T, FM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)Cfg::SMEM);
            if (e != cudaSuccess) return e;
            k_mf_factor_small<T, FM><<<(unsigned)blocks, Cfg::W * 32, Cfg::SMEM, st>>>(a, nfronts, nsys);
        } else {
            return cudaErrorInvalidValue;
        }
    } else {
        using SCfg = SolveSmallCfg<T, FM>;
        const long long sblocks = (items + SCfg::W - 1) / SCfg::W;
        if (sblocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
        k_mf_solve_small<T, FM><<<(unsigned)sblocks, SCfg::W * 32, SCfg::SMEM, st>>>(a, nfronts, nsys, what == 1 ? 1 : 0);
    }
    note_launches(1);
    return cudaGetLastError();
}

// one launch level: the first ncls[0] fronts from lvl_off have f <= 32, the next ncls[1] f <= 64,
// ncls[2] f <= 96, ncls[3] f <= 128, the remaining nlarge are large; what: 0 factorise, 1 forward,
// 2 backward.  Substitutions run one warp per front up to f = 128.  Factorisations run one warp per
// front only up to f = 64: from f = 65 on, the CTA kernel's tiled updates beat one warp's
// sequential pivot loop over the larger shared-memory tile (measured on the 384^2 grid: 216 ms by
// warps for the fronts of 65 to 128 rows against about 90 ms by CTAs).
template <typename T>
cudaError_t mf_level_launch(MfArgs<T> a, int lvl_off, const int* ncls, int nlarge, int nsys, int max_front, int what,
                            cudaStream_t st) {
    int off = lvl_off;
    cudaError_t e = mf_small_launch<T, 32>(a, off, ncls[0], nsys, what, st);
    off += ncls[0];
    if (e == cudaSuccess) e = mf_small_launch<T, 64>(a, off, ncls[1], nsys, what, st);
    off += ncls[1];
    if (e != cudaSuccess) return e;
    if (what == 0) {
        const int n = ncls[2] + ncls[3] + nlarge;
        return n > 0 ? mf_factor_launch<T>(a, off, n, nsys, st) : cudaSuccess;
    }
    e = mf_small_launch<T, 96>(a, off, ncls[2], nsys, what, st);
    off += ncls[2];
    if (e == cudaSuccess) e = mf_small_launch<T, 128>(a, off, ncls[3], nsys, what, st);
    off += ncls[3];
    if (e != cudaSuccess || nlarge <= 0) return e;
    return mf_solve_launch<T>(a, off, nlarge, nsys, max_front, what == 1, st);
}

// ------------------------------------------------------------------ launchers
template <typename T>
size_t mf_factor_smem() {
    constexpr int NB = MfNB<T>::v;
    return sizeof(C<T>) * (2 * (size_t)NB * MF_TILE + (size_t)NB * (NB + 1) + NB);
}

template <typename T>
cudaError_t mf_factor_launch(MfArgs<T> a, int lvl_off, int nfronts, int nsys, cudaStream_t st) {
    if (nfronts <= 0 || nsys <= 0) return cudaSuccess;
    a.lvl_off = lvl_off;
    const size_t smem = mf_factor_smem<T>();
    cudaError_t e = cudaFuncSetAttribute(k_mf_factor<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mf_factor<T>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    k_mf_factor<T><<<dim3(nfronts, nsys), MF_THREADS, smem, st>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t mf_solve_launch(MfArgs<T> a, int lvl_off, int nfronts, int nsys, int max_front, bool fwd, cudaStream_t st) {
    if (nfronts <= 0 || nsys <= 0) return cudaSuccess;
    a.lvl_off = lvl_off;
    const size_t smem = sizeof(C<T>) * ((size_t)max_front + 32 * 33);
    cudaError_t e;
    if (fwd) {
        e = cudaFuncSetAttribute(k_mf_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_mf_fwd<T><<<dim3(nfronts, nsys), MF_THREADS, smem, st>>>(a);
    } else {
        e = cudaFuncSetAttribute(k_mf_bwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_mf_bwd<T><<<dim3(nfronts, nsys), MF_THREADS, smem, st>>>(a);
    }
    note_launches(1);
    return cudaGetLastError();
}

template cudaError_t mf_level_launch<float>(MfArgs<float>, int, const int*, int, int, int, int, cudaStream_t);
template cudaError_t mf_level_launch<double>(MfArgs<double>, int, const int*, int, int, int, int, cudaStream_t);
template cudaError_t mf_factor_launch<float>(MfArgs<float>, int, int, int, cudaStream_t);
template cudaError_t mf_factor_launch<double>(MfArgs<double>, int, int, int, cudaStream_t);
template cudaError_t mf_solve_launch<float>(MfArgs<float>, int, int, int, int, bool, cudaStream_t);
template cudaError_t mf_solve_launch<double>(MfArgs<double>, int, int, int, int, bool, cudaStream_t);

}  // namespace stfdm
