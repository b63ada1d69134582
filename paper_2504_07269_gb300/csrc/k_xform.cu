// Steps 2 and 4 of the Kronecker solver (Section 3): the time transforms
//   G = Y_t F~   and   Psi = X_t W   (and X_t^T, Y_t^T for the adjoint),
// dense complex contractions over the n_t time DOFs of an (n_t, n_x) array:
//   out[l, x] = sum_k T[l, k] in[k, x].
// This file holds the tiled SIMT version (FP64 and FP32 arithmetic) with fused
// prologue/epilogue options:
//   * b_scale: multiply the input by a device scalar while loading (refinement cast);
//   * conj_b / conj_out: complex conjugation of the input / the product (adjoint);
//   * r1_u, r1_v: subtract the rank-one lifting term u[l] v[x] with u = Y_t m_t,
//     v = A_x psi0 (Y_t (F - m_t (x) A_x psi0) = Y_t F - (Y_t m_t) (x) A_x psi0);
//   * add_row: add psi0 to every row (psi = psi_hat + psi0);
//   * out_scale: device scalar multiplying the product (undoes the input scaling);
//   * accumulate: out += out_scale * product (refinement update psi_hat += delta).
#include <cuda_runtime.h>

#include "device.cuh"

namespace stfdm {



constexpr int XBM = 64, XBN = 64, XBK = 8;

template <typename TA, typename TB, typename TC, typename TACC>
__global__ void __launch_bounds__(256) k_xform_simt(XformArgs<TA, TB, TC> a) {
    __shared__ C<TACC> As[XBK][XBM + 1];
    __shared__ C<TACC> Bs[XBK][XBN + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * XBM, n0 = blockIdx.x * XBN;
    TACC bsc = (TACC)1;
    if (a.b_scale) bsc = (TACC)(*a.b_scale);
    C<TACC> acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = mk<TACC>(0, 0);
    for (int k0 = 0; k0 < a.K; k0 += XBK) {
        for (int e = tid; e < XBM * XBK; e += 256) {
            int r = e / XBK, kk = e - r * XBK;
            int gm = m0 + r, gk = k0 + kk;
            C<TACC> v = mk<TACC>(0, 0);
            if (gm < a.M && gk < a.K) v = ccast<TACC, TA>(a.A[(size_t)gm * a.lda + gk]);
            As[kk][r] = v;
        }
        for (int e = tid; e < XBK * XBN; e += 256) {
            int kk = e / XBN, c = e - kk * XBN;
            int gk = k0 + kk, gn = n0 + c;
            C<TACC> v = mk<TACC>(0, 0);
            if (gk < a.K && gn < a.N) {
                v = ccast<TACC, TB>(a.B[(size_t)gk * a.ldb + gn]);
                if (a.conj_b) v.y = -v.y;
                v.x *= bsc;
                v.y *= bsc;
            }
            Bs[kk][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < XBK; ++kk) {
            C<TACC> av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cfma<TACC>(acc[i][j], av[i], bv[j]);
        }
        __syncthreads();
    }
    double osc = 1.0;
    if (a.out_scale) osc = *a.out_scale;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + ty + 16 * i;
        if (gm >= a.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + tx + 16 * j;
            if (gn >= a.N) continue;
            double vx = (double)acc[i][j].x, vy = (double)acc[i][j].y;
            if (a.conj_out) vy = -vy;
            if (a.r1_u) {
                double2 u = a.r1_u[gm], w = a.r1_v[gn];
                vx -= u.x * w.x - u.y * w.y;
                vy -= u.x * w.y + u.y * w.x;
            }
            if (a.add_row) {
                C<TC> ad = a.add_row[gn];
                vx += (double)ad.x;
                vy += (double)ad.y;
            }
            C<TC>* out = a.Cm + (size_t)gm * a.ldc + gn;
            if (a.accumulate) {
                C<TC> o = *out;
                *out = mk<TC>((TC)((double)o.x + osc * vx), (TC)((double)o.y + osc * vy));
            } else {
                *out = mk<TC>((TC)(osc * vx), (TC)(osc * vy));
            }
        }
    }
}

template <typename TA, typename TB, typename TC, typename TACC>
cudaError_t xform_simt_launch(const XformArgs<TA, TB, TC>& a, cudaStream_t st) {
    dim3 grid((a.N + XBN - 1) / XBN, (a.M + XBM - 1) / XBM);
    k_xform_simt<TA, TB, TC, TACC><<<grid, 256, 0, st>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

template cudaError_t xform_simt_launch<double, double, double, double>(const XformArgs<double, double, double>&, cudaStream_t);
template cudaError_t xform_simt_launch<float, float, float, float>(const XformArgs<float, float, float>&, cudaStream_t);
template cudaError_t xform_simt_launch<float, double, float, float>(const XformArgs<float, double, float>&, cudaStream_t);
template cudaError_t xform_simt_launch<float, float, double, float>(const XformArgs<float, float, double>&, cudaStream_t);

}  // namespace stfdm
