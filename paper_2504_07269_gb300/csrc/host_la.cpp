// Host FP64 dense linear algebra for step 1 of the Kronecker solver (Section 3):
// the eigen-decomposition (i B_t)^{-1} M_t = X_t S_t X_t^{-1} of a dense complex
// n_t x n_t matrix, Y_t = X_t^{-1} (i B_t)^{-1} and kappa_2(X_t).
//
// Methods (textbook, written from their definitions):
//   * Householder reduction to upper Hessenberg form, accumulating the unitary Z;
//   * complex single-shift implicit QR iteration with Wilkinson shifts and
//     deflation on negligible subdiagonals (Francis), giving the Schur form T;
//   * eigenvectors of T by back substitution, back-transformed by Z;
//   * LU with partial pivoting for X_t^{-1};
//   * kappa_2 from the extreme eigenvalues of X^H X and (X^H X)^{-1}, each by
//     Lanczos with full reorthogonalisation and Sturm bisection on the tridiagonal.
// Matrices are column-major here: A[i + j n].
#include <algorithm>
#include <cmath>
#include <functional>
#include <limits>
#include <thread>
#include <vector>

#include "internal.h"

namespace stfdm {
namespace la {

static inline double abs1(cd z) { return std::fabs(z.real()) + std::fabs(z.imag()); }

static void parallel_for(int threads, int begin, int end, const std::function<void(int, int)>& body) {
    int n = end - begin;
    if (n <= 0) return;
    if (threads <= 1 || n < 2 * threads) {
        body(begin, end);
        return;
    }
    std::vector<std::thread> pool;
    int chunk = (n + threads - 1) / threads;
    for (int t = 0; t < threads; ++t) {
        int b = begin + t * chunk, e = std::min(end, b + chunk);
        if (b >= e) break;
        pool.emplace_back(body, b, e);
    }
    for (auto& th : pool) th.join();
}

// Householder reduction A -> Z^H A Z upper Hessenberg; Z accumulates the reflectors.
static void hessenberg(int n, cd* A, cd* Z, int threads) {
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) Z[i + (size_t)j * n] = (i == j) ? 1.0 : 0.0;
    std::vector<cd> v(n), w(n);
    for (int k = 0; k + 2 < n; ++k) {
        const int len = n - k - 1;
        double alpha2 = 0;
        for (int i = 0; i < len; ++i) alpha2 += std::norm(A[(k + 1 + i) + (size_t)k * n]);
        double alpha = std::sqrt(alpha2);
        if (alpha == 0.0) continue;
        cd x0 = A[(k + 1) + (size_t)k * n];
        cd phase = (std::abs(x0) > 0) ? x0 / std::abs(x0) : cd(1.0, 0.0);
        for (int i = 0; i < len; ++i) v[i] = A[(k + 1 + i) + (size_t)k * n];
        v[0] += phase * alpha;
        double vn2 = 0;
        for (int i = 0; i < len; ++i) vn2 += std::norm(v[i]);
        const double tau = 2.0 / vn2;
        // left: A[k+1:, k:] -= tau v (v^H A[k+1:, c])
        parallel_for(threads, k, n, [&](int c0, int c1) {
            for (int c = c0; c < c1; ++c) {
                cd* col = A + (size_t)c * n + k + 1;
                cd t = 0;
                for (int i = 0; i < len; ++i) t += std::conj(v[i]) * col[i];
                t *= tau;
                for (int i = 0; i < len; ++i) col[i] -= v[i] * t;
            }
        });
        // right: A[:, k+1:] -= tau (A[:, k+1:] v) v^H ; same for Z
        auto right = [&](cd* M) {
            parallel_for(threads, 0, n, [&](int r0, int r1) {
                std::vector<cd> acc(r1 - r0, 0.0);
                for (int i = 0; i < len; ++i) {
                    const cd* col = M + (size_t)(k + 1 + i) * n;
                    cd vi = v[i];
                    for (int r = r0; r < r1; ++r) acc[r - r0] += col[r] * vi;
                }
                for (int i = 0; i < len; ++i) {
                    cd* col = M + (size_t)(k + 1 + i) * n;
                    cd f = tau * std::conj(v[i]);
                    for (int r = r0; r < r1; ++r) col[r] -= acc[r - r0] * f;
                }
            });
        };
        right(A);
        right(Z);
        A[(k + 1) + (size_t)k * n] = -phase * alpha;
        for (int i = k + 2; i < n; ++i) A[i + (size_t)k * n] = 0.0;
    }
}

struct Rot {
    double c;
    cd s;
};

// Givens G = [[c, s], [-conj(s), c]] with G [x; y] = [r; 0]
static inline Rot make_rot(cd x, cd y) {
    double ax = std::abs(x), ay = std::abs(y);
    if (ay == 0.0) return {1.0, 0.0};
    if (ax == 0.0) return {0.0, std::conj(y) / ay};
    double rho = std::hypot(ax, ay);
    return {ax / rho, (x / ax) * std::conj(y) / rho};
}
// rows: [a; b] <- G [a; b]
static inline void rot_rows(const Rot& g, cd& a, cd& b) {
    cd na = g.c * a + g.s * b;
    cd nb = -std::conj(g.s) * a + g.c * b;
    a = na;
    b = nb;
}
// columns: [a, b] <- [a, b] G^H
static inline void rot_cols(const Rot& g, cd& a, cd& b) {
    cd na = g.c * a + std::conj(g.s) * b;
    cd nb = -g.s * a + g.c * b;
    a = na;
    b = nb;
}

bool complex_schur(int n, cd* A, cd* Z, int threads) {
    hessenberg(n, A, Z, threads);
    auto H = [&](int i, int j) -> cd& { return A[i + (size_t)j * n]; };
    const double ulp = std::numeric_limits<double>::epsilon();
    const double smlnum = std::numeric_limits<double>::min() * (n / ulp);
    int ihi = n - 1;
    int its = 0;
    const int itmax = 60 * std::max(10, n);
    int total = 0;
    std::vector<Rot> rots(n);
    while (ihi >= 0) {
        // find the top l of the active unreduced block
        int l = ihi;
        for (; l > 0; --l) {
            double hs = abs1(H(l, l - 1));
            double tst = abs1(H(l - 1, l - 1)) + abs1(H(l, l));
            if (hs <= smlnum || hs <= ulp * tst) {
                H(l, l - 1) = 0.0;
                break;
            }
        }
        if (l == ihi) {  // 1x1 block converged
            --ihi;
            its = 0;
            continue;
        }
        if (++total > itmax) return false;
        ++its;
        // shift
        cd mu;
        if (its % 11 == 10) {
            // exceptional shift
            mu = H(ihi, ihi) + 0.75 * std::fabs(H(ihi, ihi - 1).real());
        } else {
            cd a = H(ihi - 1, ihi - 1), b = H(ihi - 1, ihi), c = H(ihi, ihi - 1), d = H(ihi, ihi);
            cd half = 0.5 * (a - d);
            cd disc = std::sqrt(half * half + b * c);
            cd e1 = 0.5 * (a + d) + disc, e2 = 0.5 * (a + d) - disc;
            mu = (std::abs(e1 - d) < std::abs(e2 - d)) ? e1 : e2;
        }
        // implicit single-shift sweep on rows/cols l..ihi
        cd x = H(l, l) - mu, y = H(l + 1, l);
        for (int k = l; k < ihi; ++k) {
            if (k > l) {
                x = H(k, k - 1);
                y = H(k + 1, k - 1);
            }
            Rot g = make_rot(x, y);
            rots[k] = g;
            int c0 = (k > l) ? k - 1 : l;
            for (int c = c0; c <= ihi; ++c) rot_rows(g, H(k, c), H(k + 1, c));
            if (k > l) H(k + 1, k - 1) = 0.0;
            int rmax = std::min(k + 2, ihi);
            for (int r = l; r <= rmax; ++r) rot_cols(g, H(r, k), H(r, k + 1));
        }
        // deferred updates outside the window: rows l..ihi for columns > ihi,
        // columns l..ihi for rows < l, and the Schur vectors
        parallel_for(threads, ihi + 1, n, [&](int c0, int c1) {
            for (int c = c0; c < c1; ++c)
                for (int k = l; k < ihi; ++k) rot_rows(rots[k], H(k, c), H(k + 1, c));
        });
        for (int k = l; k < ihi; ++k) {
            cd* ck = A + (size_t)k * n;
            cd* ck1 = A + (size_t)(k + 1) * n;
            for (int r = 0; r < l; ++r) rot_cols(rots[k], ck[r], ck1[r]);
        }
        parallel_for(threads, 0, n, [&](int r0, int r1) {
            for (int k = l; k < ihi; ++k) {
                cd* zk = Z + (size_t)k * n;
                cd* zk1 = Z + (size_t)(k + 1) * n;
                for (int r = r0; r < r1; ++r) rot_cols(rots[k], zk[r], zk1[r]);
            }
        });
    }
    // clean the strictly lower part
    for (int j = 0; j < n; ++j)
        for (int i = j + 1; i < n; ++i) H(i, j) = 0.0;
    return true;
}

void schur_eigenvectors(int n, const cd* T, const cd* Z, cd* X, int threads) {
    const double ulp = std::numeric_limits<double>::epsilon();
    double tnorm = 0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i <= j; ++i) tnorm = std::max(tnorm, abs1(T[i + (size_t)j * n]));
    const double smin_floor = std::max(ulp * tnorm, std::numeric_limits<double>::min() * 1e3);
    parallel_for(threads, 0, n, [&](int k0, int k1) {
        std::vector<cd> x(n), r(n);
        for (int k = k0; k < k1; ++k) {
            cd lam = T[k + (size_t)k * n];
            double smin = std::max(ulp * abs1(lam), smin_floor);
            for (int i = 0; i < k; ++i) r[i] = -T[i + (size_t)k * n];
            x[k] = 1.0;
            for (int j = k - 1; j >= 0; --j) {
                cd d = T[j + (size_t)j * n] - lam;
                if (abs1(d) < smin) d = smin;
                x[j] = r[j] / d;
                const cd* col = T + (size_t)j * n;
                cd xj = x[j];
                for (int i = 0; i < j; ++i) r[i] -= col[i] * xj;
            }
            cd* out = X + (size_t)k * n;
            for (int i = 0; i < n; ++i) out[i] = 0.0;
            for (int j = 0; j <= k; ++j) {
                const cd* zc = Z + (size_t)j * n;
                cd xj = x[j];
                for (int i = 0; i < n; ++i) out[i] += zc[i] * xj;
            }
            double nrm = 0;
            for (int i = 0; i < n; ++i) nrm += std::norm(out[i]);
            nrm = std::sqrt(nrm);
            // phase convention: the entry of largest modulus is real positive
            int imax = 0;
            double amax = -1;
            for (int i = 0; i < n; ++i)
                if (std::abs(out[i]) > amax) {
                    amax = std::abs(out[i]);
                    imax = i;
                }
            cd ph = std::conj(out[imax]) / std::abs(out[imax]);
            for (int i = 0; i < n; ++i) out[i] *= ph / nrm;
        }
    });
}

bool lu_factor(int n, cd* A, int* piv) {
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = std::abs(A[k + (size_t)k * n]);
        for (int i = k + 1; i < n; ++i) {
            double v = std::abs(A[i + (size_t)k * n]);
            if (v > best) {
                best = v;
                p = i;
            }
        }
        piv[k] = p;
        if (best == 0.0) return false;
        if (p != k)
            for (int j = 0; j < n; ++j) std::swap(A[k + (size_t)j * n], A[p + (size_t)j * n]);
        cd inv = 1.0 / A[k + (size_t)k * n];
        for (int i = k + 1; i < n; ++i) A[i + (size_t)k * n] *= inv;
        for (int j = k + 1; j < n; ++j) {
            cd f = A[k + (size_t)j * n];
            if (f == 0.0) continue;
            cd* cj = A + (size_t)j * n;
            const cd* ck = A + (size_t)k * n;
            for (int i = k + 1; i < n; ++i) cj[i] -= ck[i] * f;
        }
    }
    return true;
}

static void lu_solve_one(int n, const cd* LU, const int* piv, cd* b) {
    for (int k = 0; k < n; ++k)
        if (piv[k] != k) std::swap(b[k], b[piv[k]]);
    for (int j = 0; j < n; ++j) {  // L unit lower, column oriented
        cd bj = b[j];
        const cd* col = LU + (size_t)j * n;
        for (int i = j + 1; i < n; ++i) b[i] -= col[i] * bj;
    }
    for (int j = n - 1; j >= 0; --j) {
        const cd* col = LU + (size_t)j * n;
        b[j] /= col[j];
        cd bj = b[j];
        for (int i = 0; i < j; ++i) b[i] -= col[i] * bj;
    }
}

// solve X^H z = b with X = P L U:  X^H = U^H L^H P^T
static void lu_solve_H_one(int n, const cd* LU, const int* piv, cd* b) {
    for (int j = 0; j < n; ++j) {  // U^H y = b (lower triangular, row j of U^H = column j of U conj)
        const cd* col = LU + (size_t)j * n;
        cd s = b[j];
        for (int i = 0; i < j; ++i) s -= std::conj(col[i]) * b[i];
        b[j] = s / std::conj(col[j]);
    }
    for (int j = n - 1; j >= 0; --j) {  // L^H z = y (unit upper)
        const cd* col = LU + (size_t)j * n;
        cd s = b[j];
        for (int i = j + 1; i < n; ++i) s -= std::conj(col[i]) * b[i];
        b[j] = s;
    }
    for (int k = n - 1; k >= 0; --k)
        if (piv[k] != k) std::swap(b[k], b[piv[k]]);
}

void lu_solve(int n, const cd* LU, const int* piv, cd* B, int nrhs, int threads) {
    parallel_for(threads, 0, nrhs, [&](int c0, int c1) {
        for (int c = c0; c < c1; ++c) lu_solve_one(n, LU, piv, B + (size_t)c * n);
    });
}

// largest eigenvalue of the symmetric tridiagonal (a, b) by Sturm bisection
static double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b, int k) {
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < k; ++i) {
        double r = (i > 0 ? std::fabs(b[i - 1]) : 0) + (i + 1 < k ? std::fabs(b[i]) : 0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    auto count_below = [&](double x) {  // number of eigenvalues < x
        int cnt = 0;
        double d = 1.0;
        for (int i = 0; i < k; ++i) {
            double bb = (i > 0) ? b[i - 1] * b[i - 1] : 0.0;
            d = a[i] - x - (i > 0 ? bb / d : 0.0);
            if (d == 0.0) d = -1e-300;
            if (d < 0) ++cnt;
        }
        return cnt;
    };
    for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
        double mid = 0.5 * (lo + hi);
        if (count_below(mid) >= k) hi = mid;
        else lo = mid;
    }
    return hi;
}

// largest eigenvalue of a Hermitian positive definite operator by Lanczos with full
// reorthogonalisation
static double lanczos_max(int n, const std::function<void(const cd*, cd*)>& op) {
    const int kmax = std::min(n, 160);
    std::vector<std::vector<cd>> Q;
    std::vector<double> a, b;
    std::vector<cd> q(n), w(n);
    // deterministic start vector
    double nrm = 0;
    for (int i = 0; i < n; ++i) {
        q[i] = cd(1.0 + 0.37 * std::sin(1.3 * i), 0.2 * std::cos(0.7 * i));
        nrm += std::norm(q[i]);
    }
    nrm = std::sqrt(nrm);
    for (auto& z : q) z /= nrm;
    double last = 0;
    int stable = 0;
    for (int j = 0; j < kmax; ++j) {
        Q.push_back(q);
        op(q.data(), w.data());
        double alpha = 0;
        for (int i = 0; i < n; ++i) alpha += (std::conj(q[i]) * w[i]).real();
        a.push_back(alpha);
        for (int pass = 0; pass < 2; ++pass)
            for (auto& qq : Q) {
                cd h = 0;
                for (int i = 0; i < n; ++i) h += std::conj(qq[i]) * w[i];
                for (int i = 0; i < n; ++i) w[i] -= h * qq[i];
            }
        double beta = 0;
        for (int i = 0; i < n; ++i) beta += std::norm(w[i]);
        beta = std::sqrt(beta);
        double cur = tridiag_max_eig(a, b, (int)a.size());
        if (j > 4 && std::fabs(cur - last) <= 1e-14 * cur) {
            if (++stable >= 3) return cur;
        } else {
            stable = 0;
        }
        last = cur;
        if (beta <= 1e-14 * std::max(1.0, cur)) return cur;
        b.push_back(beta);
        for (int i = 0; i < n; ++i) q[i] = w[i] / beta;
    }
    return last;
}

double cond2(int n, const cd* X, const cd* LU, const int* piv) {
    auto apply_XhX = [&](const cd* v, cd* out) {
        std::vector<cd> t(n, 0.0);
        for (int j = 0; j < n; ++j) {
            const cd* col = X + (size_t)j * n;
            cd vj = v[j];
            for (int i = 0; i < n; ++i) t[i] += col[i] * vj;
        }
        for (int j = 0; j < n; ++j) {
            const cd* col = X + (size_t)j * n;
            cd s = 0;
            for (int i = 0; i < n; ++i) s += std::conj(col[i]) * t[i];
            out[j] = s;
        }
    };
    auto apply_inv = [&](const cd* v, cd* out) {  // (X^H X)^{-1} v = X^{-1} X^{-H} v
        for (int i = 0; i < n; ++i) out[i] = v[i];
        lu_solve_H_one(n, LU, piv, out);
        lu_solve_one(n, LU, piv, out);
    };
    double smax2 = lanczos_max(n, apply_XhX);
    double sinv2 = lanczos_max(n, apply_inv);
    return std::sqrt(smax2 * sinv2);
}

// Banded LU with partial pivoting on dense column-major storage; after pivoting the upper
// bandwidth grows to kl + ku, so every loop is limited to that band.
bool band_lu_real(int n, int kl, int ku, double* A, int* piv) {
    const int kuu = kl + ku;
    for (int k = 0; k < n; ++k) {
        int imax = std::min(n - 1, k + kl);
        int p = k;
        double best = std::fabs(A[k + (size_t)k * n]);
        for (int i = k + 1; i <= imax; ++i)
            if (std::fabs(A[i + (size_t)k * n]) > best) {
                best = std::fabs(A[i + (size_t)k * n]);
                p = i;
            }
        piv[k] = p;
        if (best == 0.0) return false;
        int jmax = std::min(n - 1, k + kuu);
        if (p != k)
            for (int j = k; j <= jmax; ++j) std::swap(A[k + (size_t)j * n], A[p + (size_t)j * n]);
        double inv = 1.0 / A[k + (size_t)k * n];
        for (int i = k + 1; i <= imax; ++i) A[i + (size_t)k * n] *= inv;
        for (int j = k + 1; j <= jmax; ++j) {
            double f = A[k + (size_t)j * n];
            if (f == 0.0) continue;
            for (int i = k + 1; i <= imax; ++i) A[i + (size_t)j * n] -= A[i + (size_t)k * n] * f;
        }
    }
    return true;
}

void band_lu_real_solve(int n, int kl, int ku, const double* LU, const int* piv, double* b) {
    const int kuu = kl + ku;
    for (int k = 0; k < n; ++k) {
        if (piv[k] != k) std::swap(b[k], b[piv[k]]);
        int imax = std::min(n - 1, k + kl);
        for (int i = k + 1; i <= imax; ++i) b[i] -= LU[i + (size_t)k * n] * b[k];
    }
    for (int j = n - 1; j >= 0; --j) {
        b[j] /= LU[j + (size_t)j * n];
        int imin = std::max(0, j - kuu);
        for (int i = imin; i < j; ++i) b[i] -= LU[i + (size_t)j * n] * b[j];
    }
}

// solve A^T x = b with the factorisation of A (P A = L U  ->  A^T = U^T L^T P)
void band_lu_real_solve_T(int n, int kl, int ku, const double* LU, const int* piv, double* b) {
    const int kuu = kl + ku;
    for (int j = 0; j < n; ++j) {  // U^T y = b
        int imin = std::max(0, j - kuu);
        double s = b[j];
        for (int i = imin; i < j; ++i) s -= LU[i + (size_t)j * n] * b[i];
        b[j] = s / LU[j + (size_t)j * n];
    }
    for (int k = n - 1; k >= 0; --k) {  // L^T z = y, then undo the row swaps
        int imax = std::min(n - 1, k + kl);
        double s = b[k];
        for (int i = k + 1; i <= imax; ++i) s -= LU[i + (size_t)k * n] * b[i];
        b[k] = s;
        if (piv[k] != k) std::swap(b[k], b[piv[k]]);
    }
}

}  // namespace la
}  // namespace stfdm
