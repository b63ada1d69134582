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
// L(j+1.., j) . w(j+1..), a butterfly reduction gives w_j.
//
// The factor columns stream through shared memory: per CTA one producer lane issues 1-D bulk
// copies (TMA) of G consecutive columns (G b contiguous entries) into a ring of SUB_STAGES
// buffers, completed on mbarriers, while the consumer warp works on earlier groups; each CTA
// thus keeps SUB_STAGES x G x b entries in flight, enough to run the HBM at full rate with one
// system per CTA.  All waits are bounded in time; a timeout sets status[1] and ends the kernel
// after the copies in flight have landed.
#include <cuda_runtime.h>

#include <algorithm>

#include "async.cuh"
#include "device.cuh"

namespace stfdm {

template <typename T>
__device__ __forceinline__ C<T> shfl(C<T> v, int src) {
    return mk<T>(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

constexpr int SUB_STAGES = 3;
constexpr unsigned long long SUB_WAIT_NS = 2000000000ull;   // 2 s per wait

struct SubShared {
    uint64_t full[SUB_STAGES];
    uint64_t empty[SUB_STAGES];
    uint64_t never;  // initialised, never arrived on: the target of the wait probe
    int err;
    int issued;      // bulk copies issued by the producer
    int consumed;    // stages released by the consumer
};

// One system for the substitution kernels: n rows, half bandwidth b, its factor columns L, pivots
// D and right-hand side z (solution on exit); n = 0 marks an item to skip.
template <typename T>
struct SubSys {
    int n, b;
    const C<T>* L;
    const C<T>* D;
    C<T>* z;
};

// the systems k0 .. k0 + nsys - 1 of one problem
template <typename T>
struct SingleSrc {
    BandArgs<T> a;
    int k0, nsys;
    __device__ int count() const { return nsys; }
    __device__ unsigned long long probe_ns() const { return a.probe_ns; }
    __device__ SubSys<T> get(int ks) const {
        const int k = k0 + ks;
        const size_t slot = a.keep ? (size_t)k : (size_t)ks;
        return SubSys<T>{a.n, a.b, a.L + slot * (size_t)a.n * a.b, a.D + slot * (size_t)a.n, a.rhs + (size_t)k * a.n};
    }
};

// the kept-factor systems of a batch (work list of (problem, k)); items of problems that are not
// iterating, or whose factors are not stored yet, are skipped
struct GroupSrc {
    const BatchBand* probs;
    const int2* items;
    int n_items;
    const int* active;
    const int* factored;
    __device__ int count() const { return n_items; }
    __device__ unsigned long long probe_ns() const { return 0; }
    __device__ SubSys<float> get(int ks) const {
        const int2 pk = items[ks];
        const BatchBand& pb = probs[pk.x];
        if ((active && !active[pk.x]) || !factored[pk.x] || !pb.Lkeep) return SubSys<float>{0, 0, nullptr, nullptr, nullptr};
        return SubSys<float>{pb.n, pb.b, pb.Lkeep + (size_t)pk.y * pb.n * pb.b, pb.Dkeep + (size_t)pk.y * pb.n,
                             pb.rhs + (size_t)pk.y * pb.n};
    }
};

// Producer lane: the column groups of every system of this CTA, in the consumer's order.
// Forward: groups [gG, gG + G) from the top; backward: the same G-aligned groups from the last.
// Stage s of the ring starts at s G sb entries (sb >= every system's b).
template <typename T, int G, bool FWD, typename Src>
__device__ void subst_produce(const Src& src, int sb, C<T>* ring, SubShared* sh) {
    int it = 0;
    // wait probe: a wait on a barrier that receives no copy and no arrival runs out, and the CTA
    // takes the same exit as on a real timeout (nothing has been issued yet)
    if (src.probe_ns() > 0 && !async::bar_wait(&sh->never, 0, src.probe_ns())) {
        atomicExch(&sh->err, 1);
        sh->issued = 0;
        return;
    }
    for (int ks = blockIdx.x; ks < src.count(); ks += gridDim.x) {
        const SubSys<T> sys = src.get(ks);
        if (sys.n == 0) continue;
        const int n = sys.n, b = sys.b, ngroups = (n + G - 1) / G;
        for (int g = 0; g < ngroups; ++g, ++it) {
            const int s = it % SUB_STAGES;
            if (it >= SUB_STAGES &&
                !async::bar_wait(&sh->empty[s], ((it / SUB_STAGES) & 1) ^ 1, SUB_WAIT_NS)) {
                atomicExch(&sh->err, 1);
                sh->issued = it;
                return;
            }
            if (*(volatile int*)&sh->err) {
                sh->issued = it;
                return;
            }
            const int start = FWD ? g * G : ((n - 1) / G) * G - g * G;
            const int cols = min(G, n - start);
            const uint32_t bytes = (uint32_t)((size_t)cols * b * sizeof(C<T>));   // n b is even: 16-byte multiple
            async::bar_expect_tx(&sh->full[s], bytes);
            async::bulk_g2s(ring + (size_t)s * G * sb, sys.L + (size_t)start * b, bytes, &sh->full[s]);
        }
    }
    sh->issued = it;
}

// after both roles finished: wait (bounded) for copies that were issued but never consumed
__device__ void subst_drain(SubShared* sh) {
    for (int it = sh->consumed; it < sh->issued; ++it)
        async::bar_wait(&sh->full[it % SUB_STAGES], (it / SUB_STAGES) & 1, SUB_WAIT_NS);
}

template <typename T, int G>
__device__ void subst_setup(SubShared* sh) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < SUB_STAGES; ++s) {
            async::bar_init(&sh->full[s], 1);
            async::bar_init(&sh->empty[s], 1);
        }
        async::bar_init(&sh->never, 1);
        sh->err = 0;
        sh->issued = 0;
        sh->consumed = 0;
        async::fence_barrier_init();
    }
    __syncthreads();
}

// Forward substitution L z = g, y = D^{-1} z, by blocks of G columns (G divides 32).  Lane l
// keeps in zr[t] the running z of row jb + 32 t + l, t = 0..R (jb: the 32-row group of the block;
// R = ceil(b / 32)).  Per block [j0, j0 + G):
//   1. the block's own rows by a G-step chain: z_c broadcast from its lane, the later block rows
//      subtract L(r, c) z_c;
//   2. every other row below the block subtracts sum_c L(r, c) z_c (independent accumulations);
//   3. the block's y = z / d is stored; after the last block of a group the slots shift by one.
template <typename T, int R, int G, typename Src>
__global__ void __launch_bounds__(64) k_subst_fwd(Src src, int sb, int* status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    C<T>* ring = reinterpret_cast<C<T>*>(smem_raw);
    SubShared* sh = reinterpret_cast<SubShared*>(smem_raw + (size_t)SUB_STAGES * G * sb * sizeof(C<T>));
    subst_setup<T, G>(sh);
    const int lane = threadIdx.x & 31;
    if (threadIdx.x >= 32) {
        if (lane == 0) subst_produce<T, G, true>(src, sb, ring, sh);
    } else {
        int it = 0;
        bool ok = true;
        for (int ks = blockIdx.x; ks < src.count() && ok; ks += gridDim.x) {
            const SubSys<T> sys = src.get(ks);
            if (sys.n == 0) continue;
            const int n = sys.n, b = sys.b, ngroups = (n + G - 1) / G;
            C<T>* z = sys.z;
            const C<T>* D = sys.D;
            C<T> zr[R + 1];
#pragma unroll
            for (int t = 0; t <= R; ++t) {
                const int i = lane + 32 * t;
                zr[t] = (i < n) ? z[i] : mk<T>(0, 0);
            }
            C<T> znext = (lane + 32 * (R + 1) < n) ? z[lane + 32 * (R + 1)] : mk<T>(0, 0);
            C<T> dnext = (lane < G && lane < n) ? D[lane] : mk<T>(1, 0);
            for (int g = 0; g < ngroups; ++g, ++it) {
                const int j0 = g * G, jb = j0 & ~31, l0 = j0 & 31;
                const int s = it % SUB_STAGES;
                if (!async::bar_wait_or_abort(&sh->full[s], (it / SUB_STAGES) & 1, SUB_WAIT_NS, &sh->err)) {
                    atomicExch(&sh->err, 1);
                    ok = false;
                    break;
                }
                const C<T>* Ls = ring + (size_t)s * G * sb;
                const C<T> dg = dnext;
                if (lane < G && j0 + G + lane < n) dnext = D[j0 + G + lane];   // the next block's pivots
                const bool inblk = lane >= l0 && lane < l0 + G;
                // 1. the block's rows
                C<T> zb[G];
#pragma unroll
                for (int gg = 0; gg < G; ++gg) {
                    zb[gg] = shfl<T>(zr[0], l0 + gg);
                    const int o = lane - (l0 + gg);
                    if (inblk && o >= 1 && o <= b && jb + lane < n) cfms<T>(zr[0], Ls[(size_t)gg * b + (o - 1)], zb[gg]);
                }
                // 2. the rows below the block
#pragma unroll
                for (int gg = 0; gg < G; ++gg) {
                    const int c = j0 + gg;
                    if (c >= n) break;
#pragma unroll
                    for (int t = 0; t <= R; ++t) {
                        const int r = jb + 32 * t + lane, o = r - c;
                        if ((t > 0 || lane >= l0 + G) && o >= 1 && o <= b && r < n)
                            cfms<T>(zr[t], Ls[(size_t)gg * b + (o - 1)], zb[gg]);
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    async::bar_arrive(&sh->empty[s]);
                    sh->consumed = it + 1;
                }
                // 3. y of the block's rows
                {
                    const C<T> d = shfl<T>(dg, (lane - l0) & 31);
                    if (inblk && jb + lane < n) z[jb + lane] = cmul<T>(zr[0], cinv<T>(d));
                }
                if (((j0 + G) & 31) == 0) {
#pragma unroll
                    for (int t = 0; t < R; ++t) zr[t] = zr[t + 1];
                    zr[R] = znext;
                    const int i = jb + 32 * (R + 2) + lane;
                    znext = (i < n) ? z[i] : mk<T>(0, 0);
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        subst_drain(sh);
        if (sh->err) atomicExch(status + 1, 1);
    }
}

// Backward substitution L^T w = y by blocks of G columns from the bottom.  Lane l keeps in wr[t]
// the solved w of row jb + 32 t + l (0 for rows not solved yet).  Per block [j0, j0 + G):
//   1. for every column c of the block, the part of sum_o L(c + o, c) w_{c+o} over the solved rows
//      below the block: per-lane partial sums over the slots, butterfly sums across the lanes;
//   2. the block's rows by a G-step chain from the top: w_c = y_c - partial_c - sum L(i, c) w_i
//      over the block rows i > c;
//   3. the block's w are stored; below the first block of a group the slots shift by one.
template <typename T, int R, int G, typename Src>
__global__ void __launch_bounds__(64) k_subst_bwd(Src src, int sb, int* status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    C<T>* ring = reinterpret_cast<C<T>*>(smem_raw);
    SubShared* sh = reinterpret_cast<SubShared*>(smem_raw + (size_t)SUB_STAGES * G * sb * sizeof(C<T>));
    subst_setup<T, G>(sh);
    const int lane = threadIdx.x & 31;
    if (threadIdx.x >= 32) {
        if (lane == 0) subst_produce<T, G, false>(src, sb, ring, sh);
    } else {
        int it = 0;
        bool ok = true;
        for (int ks = blockIdx.x; ks < src.count() && ok; ks += gridDim.x) {
            const SubSys<T> sys = src.get(ks);
            if (sys.n == 0) continue;
            const int n = sys.n, b = sys.b, ngroups = (n + G - 1) / G;
            C<T>* z = sys.z;  // y in, w out
            C<T> wr[R + 1];
#pragma unroll
            for (int t = 0; t <= R; ++t) wr[t] = mk<T>(0, 0);
            // blocks are aligned to multiples of G; the first (highest) may be partial
            const int jtop = ((n - 1) / G) * G;
            C<T> ynext = (lane < G && jtop + lane < n) ? z[jtop + lane] : mk<T>(0, 0);
            for (int g = 0; g < ngroups; ++g, ++it) {
                const int j0 = jtop - g * G, jb = j0 & ~31, l0 = j0 & 31;
                const int s = it % SUB_STAGES;
                if (!async::bar_wait_or_abort(&sh->full[s], (it / SUB_STAGES) & 1, SUB_WAIT_NS, &sh->err)) {
                    atomicExch(&sh->err, 1);
                    ok = false;
                    break;
                }
                // the copy for this block starts at column j0 (see subst_produce)
                const C<T>* Ls = ring + (size_t)s * G * sb;
                const C<T> yg = ynext;
                if (lane < G && j0 - G + lane >= 0) ynext = z[j0 - G + lane];   // the next block's y
                const bool inblk = lane >= l0 && lane < l0 + G && jb + lane < n;
                // 1. contributions of the solved rows below the block
                C<T> part[G];
#pragma unroll
                for (int gg = 0; gg < G; ++gg) {
                    const int c = j0 + gg;
                    part[gg] = mk<T>(0, 0);
#pragma unroll
                    for (int t = 0; t <= R; ++t) {
                        const int r = jb + 32 * t + lane, o = r - c;
                        if ((t > 0 || lane >= l0 + G) && o >= 1 && o <= b && r < n && c < n)
                            cfma<T>(part[gg], Ls[(size_t)gg * b + (o - 1)], wr[t]);
                    }
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
                    for (int gg = 0; gg < G; ++gg) {
                        part[gg].x += __shfl_xor_sync(0xffffffffu, part[gg].x, off);
                        part[gg].y += __shfl_xor_sync(0xffffffffu, part[gg].y, off);
                    }
                }
                // 2. the block's rows, from the top
                C<T> acc = mk<T>(0, 0);
#pragma unroll
                for (int gg = 0; gg < G; ++gg) {
                    const C<T> y = shfl<T>(yg, gg);
                    if (lane == l0 + gg) acc = csub<T>(y, part[gg]);
                }
#pragma unroll
                for (int gg = G - 1; gg >= 0; --gg) {
                    const C<T> wi = shfl<T>(acc, l0 + gg);
                    const int o = (l0 + gg) - lane;           // row i = j0 + gg, column = this lane's row
                    if (inblk && o >= 1 && o <= b) cfms<T>(acc, Ls[(size_t)(lane - l0) * b + (o - 1)], wi);
                }
                __syncwarp();
                if (lane == 0) {
                    async::bar_arrive(&sh->empty[s]);
                    sh->consumed = it + 1;
                }
                // 3. store the block's w; keep them in slot 0
                if (inblk) {
                    z[jb + lane] = acc;
                    wr[0] = acc;
                }
                if (l0 == 0) {
#pragma unroll
                    for (int t = R; t > 0; --t) wr[t] = wr[t - 1];
                    wr[0] = mk<T>(0, 0);
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        subst_drain(sh);
        if (sh->err) atomicExch(status + 1, 1);
    }
}

template <typename T, int R, int G, typename Src>
static cudaError_t launch_src(const Src& src, int count, int sb, int* status, bool fwd, cudaStream_t st) {
    const size_t smem = (size_t)SUB_STAGES * G * sb * sizeof(C<T>) + sizeof(SubShared);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int occ = 0;
    if (fwd) {
        e = cudaFuncSetAttribute(k_subst_fwd<T, R, G, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_subst_fwd<T, R, G, Src>, 64, smem);
    } else {
        e = cudaFuncSetAttribute(k_subst_bwd<T, R, G, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_subst_bwd<T, R, G, Src>, 64, smem);
    }
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int blocks = std::max(1, std::min(count, occ * sms));
    if (fwd) k_subst_fwd<T, R, G, Src><<<blocks, 64, smem, st>>>(src, sb, status);
    else k_subst_bwd<T, R, G, Src><<<blocks, 64, smem, st>>>(src, sb, status);
    note_launches(1);
    return cudaGetLastError();
}

template <typename T, int R, int G>
static cudaError_t launch_rg(const BandArgs<T>& a, int k0, int nsys, bool fwd, cudaStream_t st) {
    const SingleSrc<T> src{a, k0, nsys};
    return launch_src<T, R, G, SingleSrc<T>>(src, nsys, a.b, a.status, fwd, st);
}

template <typename T>
cudaError_t subst_launch(const BandArgs<T>& a, int k0, int nsys, bool fwd, cudaStream_t st);

// complex128: 8 columns per stage (16 B entries)
template <>
cudaError_t subst_launch<double>(const BandArgs<double>& a, int k0, int nsys, bool fwd, cudaStream_t st) {
    const int R = (a.b + 31) / 32;
    if (nsys <= 0) return cudaSuccess;
    if (R <= 1) return launch_rg<double, 1, 8>(a, k0, nsys, fwd, st);
    if (R <= 2) return launch_rg<double, 2, 8>(a, k0, nsys, fwd, st);
    if (R <= 4) return launch_rg<double, 4, 8>(a, k0, nsys, fwd, st);
    if (R <= 8) return launch_rg<double, 8, 4>(a, k0, nsys, fwd, st);
    if (R <= 13) return launch_rg<double, 13, 2>(a, k0, nsys, fwd, st);
    if (R <= 16) return launch_rg<double, 16, 2>(a, k0, nsys, fwd, st);
    return cudaErrorInvalidValue;
}

template <>
cudaError_t subst_launch<float>(const BandArgs<float>& a, int k0, int nsys, bool fwd, cudaStream_t st) {
    const int R = (a.b + 31) / 32;
    if (nsys <= 0) return cudaSuccess;
    if (R <= 1) return launch_rg<float, 1, 16>(a, k0, nsys, fwd, st);
    if (R <= 2) return launch_rg<float, 2, 16>(a, k0, nsys, fwd, st);
    if (R <= 4) return launch_rg<float, 4, 16>(a, k0, nsys, fwd, st);
    if (R <= 8) return launch_rg<float, 8, 8>(a, k0, nsys, fwd, st);
    if (R <= 13) return launch_rg<float, 13, 4>(a, k0, nsys, fwd, st);
    if (R <= 16) return launch_rg<float, 16, 4>(a, k0, nsys, fwd, st);
    return cudaErrorInvalidValue;
}

// grouped substitutions over the kept-factor systems of a batch (complex64; b <= 256)
cudaError_t subst_batch_launch(const BatchBand* probs, const int2* items, int n_items, const int* active,
                               const int* factored, int b_max, int* status, bool fwd, cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    const GroupSrc src{probs, items, n_items, active, factored};
    const int R = (b_max + 31) / 32;
    if (R <= 4) return launch_src<float, 4, 16, GroupSrc>(src, n_items, b_max, status, fwd, st);
    if (R <= 8) return launch_src<float, 8, 8, GroupSrc>(src, n_items, b_max, status, fwd, st);
    return cudaErrorInvalidValue;
}

}  // namespace stfdm
