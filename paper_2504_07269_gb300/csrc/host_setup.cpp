// Step 1 of the Kronecker solver on the host in FP64 (Section 3, fast diagonalisation):
//   (i B_t)^{-1} M_t = X_t S_t X_t^{-1},  S_t = diag(s_k),  Y_t = X_t^{-1} (i B_t)^{-1}.
// X_t has unit 2-norm columns (the normalisation under which kappa_2(X_t) of Tables 2-3
// is reported); the eigenvalues are ordered by decreasing modulus.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <thread>
#include <vector>

#include "internal.h"

namespace stfdm {

st_status time_decompose(const TimeMats& tm, int threads, TimeDecomp& out) {
    const int n = tm.n_t;
    const int bw = tm.p;  // half bandwidth of M_t and B_t
    if (threads <= 0) threads = std::max(1u, std::thread::hardware_concurrency());
    threads = std::min(threads, 64);
    // dense column-major copies
    std::vector<double> B((size_t)n * n, 0.0);
    std::vector<double> M((size_t)n * n, 0.0);
    for (int l = 0; l < n; ++l)
        for (int d = -2; d <= 2; ++d) {
            int c = l + d;
            if (c < 0 || c >= n) continue;
            B[l + (size_t)c * n] = tm.Bb[(size_t)l * 5 + d + 2];
            M[l + (size_t)c * n] = tm.Mb[(size_t)l * 5 + d + 2];
        }
    std::vector<int> bpiv(n);
    std::vector<double> Blu = B;
    if (!la::band_lu_real(n, bw, bw, Blu.data(), bpiv.data()))
        return fail(ST_ERR_ILL_CONDITIONED, "time decomposition: B_t is singular");
    // A = (i B)^{-1} M = -i B^{-1} M  and  Binv = B^{-1}
    std::vector<cd> A((size_t)n * n);
    std::vector<double> Binv((size_t)n * n, 0.0);
    {
        std::vector<double> col(n);
        for (int j = 0; j < n; ++j) {
            for (int i = 0; i < n; ++i) col[i] = M[i + (size_t)j * n];
            la::band_lu_real_solve(n, bw, bw, Blu.data(), bpiv.data(), col.data());
            for (int i = 0; i < n; ++i) A[i + (size_t)j * n] = cd(0.0, -col[i]);
            std::fill(col.begin(), col.end(), 0.0);
            col[j] = 1.0;
            la::band_lu_real_solve(n, bw, bw, Blu.data(), bpiv.data(), col.data());
            for (int i = 0; i < n; ++i) Binv[i + (size_t)j * n] = col[i];
        }
    }
    std::vector<cd> Z((size_t)n * n);
    if (!la::complex_schur(n, A.data(), Z.data(), threads))
        return fail(ST_ERR_NOT_CONVERGED, "time decomposition: QR iteration did not converge");
    out.Zs = Z;
    out.Ts = A;
    std::vector<cd> Xc((size_t)n * n);
    la::schur_eigenvectors(n, A.data(), Z.data(), Xc.data(), threads);
    std::vector<cd> s(n);
    for (int k = 0; k < n; ++k) s[k] = A[k + (size_t)k * n];
    // order by decreasing |s_k|
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return std::abs(s[a]) > std::abs(s[b]); });
    std::vector<cd> X((size_t)n * n);
    out.s.resize(n);
    for (int k = 0; k < n; ++k) {
        out.s[k] = s[order[k]];
        std::copy(Xc.begin() + (size_t)order[k] * n, Xc.begin() + (size_t)(order[k] + 1) * n, X.begin() + (size_t)k * n);
    }
    // Y = X^{-1} (i B)^{-1} = X^{-1} (-i B^{-1})
    std::vector<cd> LU = X;
    std::vector<int> piv(n);
    if (!la::lu_factor(n, LU.data(), piv.data()))
        return fail(ST_ERR_ILL_CONDITIONED, "time decomposition: X_t is singular");
    std::vector<cd> Yc((size_t)n * n);
    for (size_t i = 0; i < Yc.size(); ++i) Yc[i] = cd(0.0, -Binv[i]);
    la::lu_solve(n, LU.data(), piv.data(), Yc.data(), n, threads);
    out.kappa = la::cond2(n, X.data(), LU.data(), piv.data());
    out.n = n;
    out.X.resize((size_t)n * n);
    out.Y.resize((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            out.X[(size_t)i * n + j] = X[i + (size_t)j * n];
            out.Y[(size_t)i * n + j] = Yc[i + (size_t)j * n];
        }
    out.Binv = std::move(Binv);
    double mn = 1e300;
    for (int k = 0; k < n; ++k) mn = std::min(mn, -out.s[k].imag());
    out.min_neg_im = mn;
    for (int k = 0; k < n; ++k)
        if (!std::isfinite(out.s[k].real()) || !std::isfinite(out.s[k].imag()))
            return fail(ST_ERR_NOT_CONVERGED, "time decomposition: non-finite eigenvalue");
    return ST_OK;
}

}  // namespace stfdm

using namespace stfdm;

extern "C" st_status st_time_decompose(const st_time* t, int host_threads, double* X, double* s, double* Y,
                                       double* kappa2) {
    if (!t) return fail(ST_ERR_ARG, "st_time_decompose: NULL handle");
    TimeDecomp d;
    st_status st = time_decompose(t->tm, host_threads, d);
    if (st != ST_OK) return st;
    const size_t nn = (size_t)d.n * d.n;
    if (X) std::copy(d.X.begin(), d.X.end(), reinterpret_cast<cd*>(X));
    if (Y) std::copy(d.Y.begin(), d.Y.end(), reinterpret_cast<cd*>(Y));
    if (s) std::copy(d.s.begin(), d.s.end(), reinterpret_cast<cd*>(s));
    if (kappa2) *kappa2 = d.kappa;
    (void)nn;
    return ST_OK;
}
