// Time transforms (steps 2 and 4 of the Kronecker solver, Section 3) on the tcgen05 tensor
// cores:  out[l, x] = sum_k T[l, k] in[k, x]  with T = Y_t, X_t, X_t^T or Y_t^T (n_t x n_t).
//
// Complex product as real GEMMs on the interleaved layout: with the input viewed as a real
// K x 2N matrix B (columns 2x, 2x+1 = re, im of spatial node x),
//     P = Re(T) B,  Q = Im(T) B,   out_re = P[:, 2x] - Q[:, 2x+1],  out_im = P[:, 2x+1] + Q[:, 2x].
// Each real GEMM runs as 3xTF32 (a = a_hi + a_lo with a_hi = tf32(a)): a_hi b_hi + a_hi b_lo +
// a_lo b_hi, which keeps FP32-level accuracy (plain TF32 would not let the refinement contract).
//
// Layout: both operands K-major (TN GEMM).  The transform matrices are split once at setup into
// [4 parts: re_hi, re_lo, im_hi, im_lo][M_pad][K_pad] FP32; the input is split per call by
// k_tc_split into [2: hi, lo][N2_pad][K_pad] (transposed, K contiguous).  A CTA computes one
// 128 x 128 output tile (rows of T x interleaved columns): TMA (128B swizzle) stages 4 A tiles and
// 2 B tiles of 128 x 32 per K step into shared memory (2-stage mbarrier pipeline), one thread
// issues 24 tcgen05.mma (M=128, N=128, K=8) per K step into two TMEM accumulators (P: columns
// 0..127, Q: 128..255), and four warps read them back with tcgen05.ld for the epilogue.
// Every mbarrier wait is bounded; on expiry the kernel records an error and winds down.
#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "device.cuh"

namespace stfdm {
namespace tc {

constexpr int BM = 128, BN = 128, BK = 32, STAGES = 2;
constexpr int TILE_BYTES = BM * BK * 4;            // 16 KiB per 128 x 32 FP32 tile
constexpr int STAGE_BYTES = 6 * TILE_BYTES;        // 4 A tiles + 2 B tiles
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int THREADS = 128;
constexpr uint32_t TMEM_COLS = 256;
constexpr long long SPIN_LIMIT = 1LL << 27;

struct Epi {
    int M, N;                 // rows of T (n_t), complex columns (n_x)
    void* out;
    int out_c128;
    long long ldc;            // complex elements per output row
    int conj_out, accumulate;
    const double* out_scale;
    const void* add_row;
    const double2* r1_u;
    const double2* r1_v;
    int* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: false (and the error flag set) if the phase did not complete in time
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
    for (long long i = 0; i < SPIN_LIMIT; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    atomicExch(err, 1);
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(16 >> 4) << 16;      // leading byte offset (not used by K-major swizzled layouts)
    d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
    d |= (uint64_t)1 << 46;              // descriptor version
    d |= (uint64_t)2 << 61;              // swizzle mode: 128B
    return d;
}

// instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = 128
__host__ __device__ constexpr uint32_t make_idesc() {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(THREADS, 1)
    k_xform_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M_pad,
               int N2_pad, int K_pad, Epi e) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* done = empty + STAGES;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM;      // row tile of T
    const int n0 = blockIdx.y * BN;      // interleaved real column tile
    const int nk = K_pad / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer: TMA of 4 A tiles (re_hi, re_lo, im_hi, im_lo) and 2 B tiles (hi, lo) per K step
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % STAGES;
            if (kc >= STAGES && !mbar_wait(&empty[s], ((kc / STAGES) - 1) & 1, e.err)) break;
            uint8_t* st = smem + s * STAGE_BYTES;
            mbar_expect_tx(&full[s], STAGE_BYTES);
            const int k0 = kc * BK;
#pragma unroll
            for (int p = 0; p < 4; ++p) tma_load_2d(st + p * TILE_BYTES, &mapA, k0, p * M_pad + m0, &full[s]);
#pragma unroll
            for (int p = 0; p < 2; ++p) tma_load_2d(st + (4 + p) * TILE_BYTES, &mapB, k0, p * N2_pad + n0, &full[s]);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = make_idesc();
        bool ok = true;
        for (int kc = 0; kc < nk && ok; ++kc) {
            const int s = kc % STAGES;
            if (!mbar_wait(&full[s], (kc / STAGES) & 1, e.err)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sb = smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
            for (int kk = 0; kk < BK / 8; ++kk) {
                const uint32_t off = kk * 32;   // 8 TF32 = 32 bytes along K inside the swizzled row
                const uint64_t arh = make_desc(sb + 0 * TILE_BYTES + off), arl = make_desc(sb + 1 * TILE_BYTES + off);
                const uint64_t aih = make_desc(sb + 2 * TILE_BYTES + off), ail = make_desc(sb + 3 * TILE_BYTES + off);
                const uint64_t bh = make_desc(sb + 4 * TILE_BYTES + off), bl = make_desc(sb + 5 * TILE_BYTES + off);
                const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
                mma_tf32(tmem, arh, bh, idesc, acc);
                mma_tf32(tmem, arh, bl, idesc, 1u);
                mma_tf32(tmem, arl, bh, idesc, 1u);
                mma_tf32(tmem + BN, aih, bh, idesc, acc);
                mma_tf32(tmem + BN, aih, bl, idesc, 1u);
                mma_tf32(tmem + BN, ail, bh, idesc, 1u);
            }
            mma_commit(&empty[s]);
        }
        mma_commit(done);   // arrives when every MMA issued above has completed
    }
    __syncwarp();

    // epilogue: warp w owns TMEM lanes 32w .. 32w + 31 (rows of the tile)
    const bool have = mbar_wait(done, 0, e.err);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (have && *(volatile int*)e.err == 0) {
        const int row = warp * 32 + lane;
        const int m = m0 + row;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        double osc = 1.0;
        if (e.out_scale) osc = *e.out_scale;
        for (int c = 0; c < BN; c += 16) {
            float P[16], Q[16];
            tmem_ld16(trow + c, P);
            tmem_ld16(trow + BN + c, Q);
            if (m >= e.M) continue;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int x = (n0 + c) / 2 + t;
                if (x >= e.N) break;
                double vx = (double)P[2 * t] - (double)Q[2 * t + 1];
                double vy = (double)P[2 * t + 1] + (double)Q[2 * t];
                if (e.conj_out) vy = -vy;
                if (e.r1_u) {
                    const double2 u = e.r1_u[m], w = e.r1_v[x];
                    vx -= u.x * w.x - u.y * w.y;
                    vy -= u.x * w.y + u.y * w.x;
                }
                const size_t idx = (size_t)m * e.ldc + x;
                if (e.out_c128) {
                    double2* o = reinterpret_cast<double2*>(e.out) + idx;
                    if (e.add_row) {
                        const double2 ad = reinterpret_cast<const double2*>(e.add_row)[x];
                        vx += ad.x;
                        vy += ad.y;
                    }
                    if (e.accumulate) {
                        const double2 old = *o;
                        *o = make_double2(old.x + osc * vx, old.y + osc * vy);
                    } else {
                        *o = make_double2(osc * vx, osc * vy);
                    }
                } else {
                    float2* o = reinterpret_cast<float2*>(e.out) + idx;
                    if (e.add_row) {
                        const float2 ad = reinterpret_cast<const float2*>(e.add_row)[x];
                        vx += ad.x;
                        vy += ad.y;
                    }
                    if (e.accumulate) {
                        const float2 old = *o;
                        *o = make_float2((float)(old.x + osc * vx), (float)(old.y + osc * vy));
                    } else {
                        *o = make_float2((float)(osc * vx), (float)(osc * vy));
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// hi/lo TF32 split of one FP32 value (hi rounded to nearest TF32, lo the exact remainder)
__device__ __forceinline__ void split_tf32(float v, float& hi, float& lo) {
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
    hi = __uint_as_float(h);
    lo = v - hi;
}

// B^T planes: bt[p][2x + c][k] for p = hi/lo, c = re/im, from in[k][x] (scaled, optionally conjugated)
template <typename TI>
__global__ void __launch_bounds__(256) k_tc_split(const C<TI>* in, int K, int N, int K_pad, int N2_pad,
                                                  const double* scale, int conj, float* bt) {
    __shared__ float2 tile[32][33];
    const int x0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const float sc = scale ? (float)(*scale) : 1.0f;
    for (int kk = ty; kk < 32; kk += 8) {
        const int k = k0 + kk, x = x0 + tx;
        float2 v = make_float2(0.f, 0.f);
        if (k < K && x < N) {
            const C<TI> w = in[(size_t)k * N + x];
            v = make_float2((float)w.x * sc, (float)(conj ? -w.y : w.y) * sc);
        }
        tile[kk][tx] = v;
    }
    __syncthreads();
    const size_t plane = (size_t)N2_pad * K_pad;
    for (int xx = ty; xx < 32; xx += 8) {
        const int x = x0 + xx;
        if (2 * x + 1 >= N2_pad) continue;
        const float2 v = tile[tx][xx];
        float hr, lr, hi_, li;
        split_tf32(v.x, hr, lr);
        split_tf32(v.y, hi_, li);
        const size_t r0 = (size_t)(2 * x) * K_pad + k0 + tx;
        bt[r0] = hr;
        bt[r0 + K_pad] = hi_;
        bt[plane + r0] = lr;
        bt[plane + r0 + K_pad] = li;
    }
}

}  // namespace tc

// ------------------------------------------------------------------ host side
namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
    // looked up once (thread-safe static initialisation)
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<EncodeTiledFn>(p);
        return nullptr;
    }();
    return fn;
}

// the GEMM kernel's shared-memory opt-in, once per device
constexpr int TC_MAX_DEVICES = 64;
std::atomic<int> g_tc_attr[TC_MAX_DEVICES];
}  // namespace

int tc_round_up(int v, int m) { return (v + m - 1) / m * m; }

// 2-D FP32 tensor map over a [rows][cols] row-major array, box 128 rows x 32 columns, 128B swizzle
bool tc_make_map(CUtensorMap* map, const float* base, int rows, int cols) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)tc::BM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// hi/lo split of a row-major n x n complex matrix into [4][M_pad][K_pad] FP32 (host)
void tc_split_matrix(const cd* T, int n, int M_pad, int K_pad, float* out) {
    auto tf32 = [](float v) {
        uint32_t u;
        std::memcpy(&u, &v, 4);
        if ((u & 0x7f800000u) != 0x7f800000u) {
            u += 0x0fffu + ((u >> 13) & 1u);
            u &= 0xffffe000u;
        }
        float r;
        std::memcpy(&r, &u, 4);
        return r;
    };
    const size_t plane = (size_t)M_pad * K_pad;
    std::fill(out, out + 4 * plane, 0.0f);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            const cd v = T[(size_t)i * n + k];
            const float rh = tf32((float)v.real()), ih = tf32((float)v.imag());
            const float rl = (float)(v.real() - (double)rh), il = (float)(v.imag() - (double)ih);
            const size_t o = (size_t)i * K_pad + k;
            out[o] = rh;
            out[plane + o] = rl;
            out[2 * plane + o] = ih;
            out[3 * plane + o] = il;
        }
}

cudaError_t tc_split_launch(const void* in, bool in_c128, int K, int N, int K_pad, int N2_pad, const double* scale,
                            int conj, float* bt, cudaStream_t st) {
    dim3 grid((N + 31) / 32, K_pad / 32);
    if (in_c128)
        tc::k_tc_split<double><<<grid, 256, 0, st>>>(reinterpret_cast<const double2*>(in), K, N, K_pad, N2_pad, scale,
                                                     conj, bt);
    else
        tc::k_tc_split<float><<<grid, 256, 0, st>>>(reinterpret_cast<const float2*>(in), K, N, K_pad, N2_pad, scale,
                                                    conj, bt);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t tc_gemm_launch(const CUtensorMap& mapA, const CUtensorMap& mapB, int M_pad, int N2_pad, int K_pad, int M,
                           int N, void* out, bool out_c128, int conj_out, int accumulate, const double* out_scale,
                           const void* add_row, const double2* r1_u, const double2* r1_v, int* err, cudaStream_t st) {
    int dev = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 != cudaSuccess) return e0;
    if (dev < 0 || dev >= TC_MAX_DEVICES || !g_tc_attr[dev].load()) {
        e0 = cudaFuncSetAttribute(tc::k_xform_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES);
        if (e0 != cudaSuccess) return e0;
        if (dev >= 0 && dev < TC_MAX_DEVICES) g_tc_attr[dev].store(1);
    }
    tc::Epi e;
    e.M = M;
    e.N = N;
    e.out = out;
    e.out_c128 = out_c128 ? 1 : 0;
    e.ldc = N;
    e.conj_out = conj_out;
    e.accumulate = accumulate;
    e.out_scale = out_scale;
    e.add_row = add_row;
    e.r1_u = r1_u;
    e.r1_v = r1_v;
    e.err = err;
    dim3 grid(M_pad / tc::BM, N2_pad / tc::BN);
    tc::k_xform_tc<<<grid, tc::THREADS, tc::SMEM_BYTES, st>>>(mapA, mapB, M_pad, N2_pad, K_pad, e);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace stfdm
