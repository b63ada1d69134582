// Space-time error norms and quadrature loads for the manufactured solutions of Section 4.
//
//   ||psi - psi_h||_{L2(Q)}  and  |psi - psi_h|_{H1(Q)} = (||d_t e||^2 + ||grad_x e||^2)^{1/2}
//
// for psi_h in the trial space (P1 on the SW-NE split grid in space, P1/P2 Lagrange in time, zero
// on the spatial boundary) given by its nodal values, by tensor quadrature on every prism
// (triangle x time element): Gauss-Legendre in time, collapsed Gauss-Legendre on the triangle.
// The load F[k, a] = int_Q f phi_k varphi_a of the right-hand side f = i d_t psi - Laplace psi uses
// the same rules, gathered per degree of freedom over its support (deterministic).
//
// Manufactured solutions (ST_EXACT_*):
//   C1    psi = sin(pi x1) sin(pi x2) (1 + t) e^{-it};
//   PAPER psi = e^{it} sin(pi x1) sin(pi x2) sin(t x1 x2)  (Section 4, the paper's example).
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "device.cuh"

namespace stfdm {

constexpr int NQ_MAX = 8;

struct QuadRules {
    int nt, nx;
    double tq[NQ_MAX], tw[NQ_MAX];   // Gauss-Legendre on [0, 1]
    double xq[NQ_MAX], xw[NQ_MAX];
};

// Gauss-Legendre nodes and weights on [0, 1]: Newton's method on the Legendre polynomial P_n
// (three-term recurrence), w = 2 / ((1 - z^2) P_n'(z)^2) on [-1, 1], halved for [0, 1]
static void legendre(int n, double z, double* pn, double* dpn) {
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;
    *dpn = (n == 1) ? 1.0 : n * (z * p1 - p0) / (z * z - 1.0);
}

void gauss_legendre01(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), pn, dpn;
        for (int itn = 0; itn < 100; ++itn) {
            legendre(n, z, &pn, &dpn);
            const double dz = pn / dpn;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        legendre(n, z, &pn, &dpn);
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dpn * dpn);
    }
}

struct ExactVals {
    double2 psi, dt, dx1, dx2;
};

__device__ __forceinline__ double2 cm(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cs(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

__device__ ExactVals exact_eval(int which, double x1, double x2, double t) {
    ExactVals v;
    double s1, c1, s2, c2;
    sincospi(x1, &s1, &c1);
    sincospi(x2, &s2, &c2);
    if (which == ST_EXACT_C1) {
        double st, ct;
        sincos(t, &st, &ct);
        const double2 e = make_double2(ct, -st);          // e^{-it}
        const double S = s1 * s2;
        const double2 g = cs(e, 1.0 + t);                  // (1 + t) e^{-it}
        v.psi = cs(g, S);
        v.dt = cs(cm(e, make_double2(1.0, -(1.0 + t))), S);   // e^{-it} (1 - i (1 + t))
        v.dx1 = cs(g, M_PI * c1 * s2);
        v.dx2 = cs(g, M_PI * s1 * c2);
    } else {
        double st, ct, sa, ca;
        sincos(t, &st, &ct);
        sincos(t * x1 * x2, &sa, &ca);
        const double2 e = make_double2(ct, st);           // e^{it}
        const double ab = s1 * s2;
        v.psi = cs(e, ab * sa);
        // d_t: i e^{it} a b c + e^{it} a b x1 x2 cos(t x1 x2)
        v.dt = cm(e, make_double2(ab * x1 * x2 * ca, ab * sa));
        v.dx1 = cs(e, s2 * (M_PI * c1 * sa + s1 * t * x2 * ca));
        v.dx2 = cs(e, s1 * (M_PI * c2 * sa + s2 * t * x1 * ca));
    }
    return v;
}

// f = i d_t psi - Laplace psi
__device__ double2 exact_f(int which, double x1, double x2, double t) {
    double s1, c1, s2, c2;
    sincospi(x1, &s1, &c1);
    sincospi(x2, &s2, &c2);
    if (which == ST_EXACT_C1) {
        double st, ct;
        sincos(t, &st, &ct);
        const double2 e = make_double2(ct, -st);
        // S e^{-it} [(1 + 2 pi^2)(1 + t) + i]
        return cs(cm(e, make_double2((1.0 + 2.0 * M_PI * M_PI) * (1.0 + t), 1.0)), s1 * s2);
    }
    double st, ct, sa, ca;
    sincos(t, &st, &ct);
    sincos(t * x1 * x2, &sa, &ca);
    const double2 e = make_double2(ct, st);
    const double abc = s1 * s2 * sa;
    // Laplace(abc) = -(2 pi^2 + t^2 (x1^2 + x2^2)) abc + 2 pi t cos(t x1 x2) [x2 cos(pi x1) b + x1 a cos(pi x2)]
    const double lap = -(2.0 * M_PI * M_PI + t * t * (x1 * x1 + x2 * x2)) * abc +
                       2.0 * M_PI * t * ca * (x2 * c1 * s2 + x1 * s1 * c2);
    // e^{it} [-abc + i x1 x2 a b cos(t x1 x2) - Laplace(abc)]
    return cm(e, make_double2(-abc - lap, x1 * x2 * s1 * s2 * ca));
}

// Lagrange basis of degree p (1 or 2) on [0, 1] with equispaced nodes, and derivative
__device__ __forceinline__ void tbasis(int p, double s, double* phi, double* dphi) {
    if (p == 1) {
        phi[0] = 1.0 - s;
        phi[1] = s;
        dphi[0] = -1.0;
        dphi[1] = 1.0;
    } else {
        phi[0] = (2.0 * s - 1.0) * (s - 1.0);
        phi[1] = 4.0 * s * (1.0 - s);
        phi[2] = s * (2.0 * s - 1.0);
        dphi[0] = 4.0 * s - 3.0;
        dphi[1] = 4.0 - 8.0 * s;
        dphi[2] = 4.0 * s - 1.0;
    }
}

struct NormArgs {
    int n, m, n_x, n_t, p, N_t;
    double hx, hy;
    int exact;
    const double* nodes;
    const double2* psi;    // (n_t, n_x): t_1 ..
    const double2* psi0;   // (n_x): t_0 (NULL = 0)
    double* partials;      // 2 per block
    QuadRules q;
};

__device__ __forceinline__ double2 nodal(const NormArgs& a, int row, int ii, int jj) {
    if (ii < 1 || ii > a.n - 1 || jj < 1 || jj > a.n - 1) return make_double2(0, 0);
    const int idx = (ii - 1) + a.m * (jj - 1);
    if (row == 0) return a.psi0 ? a.psi0[idx] : make_double2(0, 0);
    return a.psi[(size_t)(row - 1) * a.n_x + idx];
}

__device__ __forceinline__ double nb_block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

// one thread per (square, time element): both triangles of the square
__global__ void __launch_bounds__(256) k_error_norms(NormArgs a) {
    __shared__ double red[32];
    const int sq = blockIdx.x * blockDim.x + threadIdx.x;
    const int e = blockIdx.y;
    double e2 = 0, h2 = 0;
    if (sq < a.n * a.n) {
        const int i = sq % a.n, j = sq / a.n;
        const double t0 = a.nodes[e], tau = a.nodes[e + 1] - t0;
        // nodal values: corners SW, SE, NE, NW at the element's time rows
        double2 U[3][4];
        const int ci[4] = {i, i + 1, i + 1, i}, cj[4] = {j, j, j + 1, j + 1};
        for (int r = 0; r <= a.p; ++r)
            for (int c = 0; c < 4; ++c) U[r][c] = nodal(a, a.p * e + r, ci[c], cj[c]);
        // the two triangles: (SW, SE, NE) and (SW, NE, NW) as corner indices
        const int tv[2][3] = {{0, 1, 2}, {0, 2, 3}};
        for (int tri = 0; tri < 2; ++tri) {
            double px[3], py[3];
            for (int v = 0; v < 3; ++v) {
                px[v] = ci[tv[tri][v]] * a.hx;
                py[v] = cj[tv[tri][v]] * a.hy;
            }
            const double J00 = px[1] - px[0], J01 = px[2] - px[0], J10 = py[1] - py[0], J11 = py[2] - py[0];
            const double det = J00 * J11 - J01 * J10, adet = fabs(det);
            // gradients of the barycentric coordinates
            double gx[3], gy[3];
            gx[1] = J11 / det;
            gy[1] = -J01 / det;
            gx[2] = -J10 / det;
            gy[2] = J00 / det;
            gx[0] = -gx[1] - gx[2];
            gy[0] = -gy[1] - gy[2];
            // spatial gradient of each time row's P1 function (constant on the triangle)
            double2 G1[3], G2[3];
            for (int r = 0; r <= a.p; ++r) {
                G1[r] = make_double2(0, 0);
                G2[r] = make_double2(0, 0);
                for (int v = 0; v < 3; ++v) {
                    const double2 u = U[r][tv[tri][v]];
                    G1[r].x += gx[v] * u.x;
                    G1[r].y += gx[v] * u.y;
                    G2[r].x += gy[v] * u.x;
                    G2[r].y += gy[v] * u.y;
                }
            }
            for (int qu = 0; qu < a.q.nx; ++qu) {
                for (int qv = 0; qv < a.q.nx; ++qv) {
                    const double xi = a.q.xq[qu], eta = a.q.xq[qv] * (1.0 - xi);
                    const double wx = a.q.xw[qu] * a.q.xw[qv] * (1.0 - xi) * adet;
                    const double lam[3] = {1.0 - xi - eta, xi, eta};
                    const double x1 = px[0] + J00 * xi + J01 * eta, x2 = py[0] + J10 * xi + J11 * eta;
                    double2 Ux[3];
                    for (int r = 0; r <= a.p; ++r) {
                        Ux[r] = make_double2(0, 0);
                        for (int v = 0; v < 3; ++v) {
                            const double2 u = U[r][tv[tri][v]];
                            Ux[r].x += lam[v] * u.x;
                            Ux[r].y += lam[v] * u.y;
                        }
                    }
                    for (int qt = 0; qt < a.q.nt; ++qt) {
                        const double s = a.q.tq[qt], w = wx * a.q.tw[qt] * tau;
                        double phi[3], dphi[3];
                        tbasis(a.p, s, phi, dphi);
                        double2 uh = make_double2(0, 0), ut = make_double2(0, 0), g1 = make_double2(0, 0),
                                g2 = make_double2(0, 0);
                        for (int r = 0; r <= a.p; ++r) {
                            uh.x += phi[r] * Ux[r].x;
                            uh.y += phi[r] * Ux[r].y;
                            ut.x += dphi[r] / tau * Ux[r].x;
                            ut.y += dphi[r] / tau * Ux[r].y;
                            g1.x += phi[r] * G1[r].x;
                            g1.y += phi[r] * G1[r].y;
                            g2.x += phi[r] * G2[r].x;
                            g2.y += phi[r] * G2[r].y;
                        }
                        const ExactVals ex = exact_eval(a.exact, x1, x2, t0 + tau * s);
                        const double d0x = ex.psi.x - uh.x, d0y = ex.psi.y - uh.y;
                        const double dtx = ex.dt.x - ut.x, dty = ex.dt.y - ut.y;
                        const double d1x = ex.dx1.x - g1.x, d1y = ex.dx1.y - g1.y;
                        const double d2x = ex.dx2.x - g2.x, d2y = ex.dx2.y - g2.y;
                        e2 += w * (d0x * d0x + d0y * d0y);
                        h2 += w * (dtx * dtx + dty * dty + d1x * d1x + d1y * d1y + d2x * d2x + d2y * d2y);
                    }
                }
            }
        }
    }
    const double s1 = nb_block_sum(e2, red);
    const double s2 = nb_block_sum(h2, red);
    if (threadIdx.x == 0) {
        const size_t bid = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        a.partials[2 * bid] = s1;
        a.partials[2 * bid + 1] = s2;
    }
}

__global__ void k_norm_sum(const double* partials, size_t nparts, double* out) {
    __shared__ double red[32];
    double s1 = 0, s2 = 0;
    for (size_t i = threadIdx.x; i < nparts; i += blockDim.x) {
        s1 += partials[2 * i];
        s2 += partials[2 * i + 1];
    }
    const double t1 = nb_block_sum(s1, red);
    const double t2 = nb_block_sum(s2, red);
    if (threadIdx.x == 0) {
        out[0] = t1;
        out[1] = t2;
    }
}

// F[k - 1, a] = int_Q f phi_k varphi_a, k = 1..n_t: one thread per degree of freedom, gathered over
// the (at most two) time elements of phi_k and the six triangles around node a
struct LoadArgs {
    int n, m, n_x, n_t, p, N_t;
    double hx, hy;
    int exact;
    const double* nodes;
    double2* F;
    QuadRules q;
};

__global__ void __launch_bounds__(256) k_load_quadrature(LoadArgs a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y + 1;   // full time DOF index (t_0 excluded)
    if (x >= a.n_x) return;
    const int ii = x % a.m + 1, jj = x / a.m + 1;   // grid node
    double2 acc = make_double2(0, 0);
    // time elements containing DOF k: p e <= k <= p e + p
    const int e_lo = max(0, (k - a.p + a.p - 1) / a.p), e_hi = min(a.N_t - 1, k / a.p);
    // the six triangles around the node: (square offset, triangle, local vertex of the node)
    //   square (ii-1, jj-1): lower (SW,SE,NE) and upper (SW,NE,NW), node = NE
    //   square (ii, jj-1): upper, node = NW;  square (ii-1, jj): lower, node = SE
    //   square (ii, jj): lower and upper, node = SW
    const int sqi[6] = {ii - 1, ii - 1, ii, ii - 1, ii, ii};
    const int sqj[6] = {jj - 1, jj - 1, jj - 1, jj, jj, jj};
    const int trl[6] = {0, 1, 1, 0, 0, 1};
    const int nodev[6] = {2, 1, 2, 1, 0, 0};   // position of the node in the triangle's vertex list
    for (int e = e_lo; e <= e_hi; ++e) {
        const double t0 = a.nodes[e], tau = a.nodes[e + 1] - t0;
        const int r = k - a.p * e;   // local time basis index
        for (int tr = 0; tr < 6; ++tr) {
            const int si = sqi[tr], sj = sqj[tr];
            // corners SW, SE, NE, NW of the square; triangle vertex lists as corner indices
            const int ci[4] = {si, si + 1, si + 1, si}, cj[4] = {sj, sj, sj + 1, sj + 1};
            const int tv[2][3] = {{0, 1, 2}, {0, 2, 3}};
            double px[3], py[3];
            for (int v = 0; v < 3; ++v) {
                px[v] = ci[tv[trl[tr]][v]] * a.hx;
                py[v] = cj[tv[trl[tr]][v]] * a.hy;
            }
            const double J00 = px[1] - px[0], J01 = px[2] - px[0], J10 = py[1] - py[0], J11 = py[2] - py[0];
            const double adet = fabs(J00 * J11 - J01 * J10);
            for (int qu = 0; qu < a.q.nx; ++qu) {
                for (int qv = 0; qv < a.q.nx; ++qv) {
                    const double xi = a.q.xq[qu], eta = a.q.xq[qv] * (1.0 - xi);
                    const double wx = a.q.xw[qu] * a.q.xw[qv] * (1.0 - xi) * adet;
                    const double lam[3] = {1.0 - xi - eta, xi, eta};
                    const double x1 = px[0] + J00 * xi + J01 * eta, x2 = py[0] + J10 * xi + J11 * eta;
                    const double bx = lam[nodev[tr]];
                    for (int qt = 0; qt < a.q.nt; ++qt) {
                        const double s = a.q.tq[qt];
                        double phi[3], dphi[3];
                        tbasis(a.p, s, phi, dphi);
                        const double w = wx * a.q.tw[qt] * tau * phi[r] * bx;
                        const double2 f = exact_f(a.exact, x1, x2, t0 + tau * s);
                        acc.x += w * f.x;
                        acc.y += w * f.y;
                    }
                }
            }
        }
    }
    a.F[(size_t)(k - 1) * a.n_x + x] = acc;
}

st_status make_rules(int q_t, int q_x, QuadRules& q) {
    q.nt = q_t > 0 ? q_t : 4;
    q.nx = q_x > 0 ? q_x : 4;
    if (q.nt > NQ_MAX || q.nx > NQ_MAX) return fail(ST_ERR_ARG, "quadrature: at most 8 points per direction");
    gauss_legendre01(q.nt, q.tq, q.tw);
    gauss_legendre01(q.nx, q.xq, q.xw);
    return ST_OK;
}

}  // namespace stfdm

using namespace stfdm;

extern "C" st_status st_error_norms(st_fdm* h, int exact, const void* psi, const void* psi0, int q_t, int q_x,
                                    double* out, void* stream) {
    if (!h || !psi || !out) return fail(ST_ERR_ARG, "st_error_norms: NULL argument");
    if (h->sm.kind != 0) return fail(ST_ERR_UNSUPPORTED, "st_error_norms: structured grids only");
    if (exact != ST_EXACT_C1 && exact != ST_EXACT_PAPER) return fail(ST_ERR_ARG, "st_error_norms: unknown solution");
    if (h->tm.p != 1 && h->tm.p != 2) return fail(ST_ERR_UNSUPPORTED, "st_error_norms: temporal degree 1 or 2");
    if (h->tm.N > 65535) return fail(ST_ERR_UNSUPPORTED, "st_error_norms: more than 65535 time elements");
    NormArgs a;
    st_status s = make_rules(q_t, q_x, a.q);
    if (s != ST_OK) return s;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != h->device) cudaSetDevice(h->device);
    const SpaceMats& sm = h->sm;
    a.n = sm.n;
    a.m = sm.m;
    a.n_x = sm.n_x;
    a.n_t = h->tm.n_t;
    a.p = h->tm.p;
    a.N_t = h->tm.N;
    a.hx = sm.Lx / sm.n;
    a.hy = sm.Ly / sm.n;
    a.exact = exact;
    a.nodes = h->dt.nodes;
    a.psi = static_cast<const double2*>(psi);
    a.psi0 = static_cast<const double2*>(psi0);
    const dim3 grid((sm.n * sm.n + 255) / 256, a.N_t);
    const size_t nparts = (size_t)grid.x * grid.y;
    const size_t need = (2 * nparts + 2) * sizeof(double);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (h->ws_norm_bytes < need) {
        cudaFree(h->ws_norm);
        h->ws_norm = nullptr;
        h->ws_norm_bytes = 0;
        e = cudaMalloc(&h->ws_norm, need);
        if (e == cudaSuccess) h->ws_norm_bytes = need;
    }
    double res[2] = {0, 0};
    if (e == cudaSuccess) {
        a.partials = static_cast<double*>(h->ws_norm);
        k_error_norms<<<grid, 256, 0, st>>>(a);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_norm_sum<<<1, 1024, 0, st>>>(a.partials, nparts, a.partials + 2 * nparts);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(res, a.partials + 2 * nparts, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (prev != h->device) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ST_ERR_CUDA, std::string("st_error_norms: ") + cudaGetErrorString(e));
    }
    out[0] = std::sqrt(res[0]);
    out[1] = std::sqrt(res[1]);
    return ST_OK;
}

extern "C" st_status st_load_quadrature(st_fdm* h, int exact, int q_t, int q_x, void* F, void* stream) {
    if (!h || !F) return fail(ST_ERR_ARG, "st_load_quadrature: NULL argument");
    if (h->sm.kind != 0) return fail(ST_ERR_UNSUPPORTED, "st_load_quadrature: structured grids only");
    if (exact != ST_EXACT_C1 && exact != ST_EXACT_PAPER) return fail(ST_ERR_ARG, "st_load_quadrature: unknown solution");
    if (h->tm.p != 1 && h->tm.p != 2) return fail(ST_ERR_UNSUPPORTED, "st_load_quadrature: temporal degree 1 or 2");
    if (h->tm.n_t > 65535) return fail(ST_ERR_UNSUPPORTED, "st_load_quadrature: n_t > 65535");
    LoadArgs a;
    st_status s = make_rules(q_t, q_x, a.q);
    if (s != ST_OK) return s;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != h->device) cudaSetDevice(h->device);
    const SpaceMats& sm = h->sm;
    a.n = sm.n;
    a.m = sm.m;
    a.n_x = sm.n_x;
    a.n_t = h->tm.n_t;
    a.p = h->tm.p;
    a.N_t = h->tm.N;
    a.hx = sm.Lx / sm.n;
    a.hy = sm.Ly / sm.n;
    a.exact = exact;
    a.nodes = h->dt.nodes;
    a.F = static_cast<double2*>(F);
    const dim3 grid((sm.n_x + 255) / 256, a.n_t);
    k_load_quadrature<<<grid, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(a);
    cudaError_t e = cudaGetLastError();
    if (prev != h->device) cudaSetDevice(prev);
    if (e != cudaSuccess) return fail(ST_ERR_CUDA, std::string("st_load_quadrature: ") + cudaGetErrorString(e));
    return ST_OK;
}
