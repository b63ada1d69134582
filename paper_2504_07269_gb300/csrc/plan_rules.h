// Memory-planning rules of the solver: host arithmetic only (no CUDA), so that the rules can be
// checked on their own.  Sizes are in bytes.
#pragma once

#include <cstddef>

namespace stfdm {

// GMRES basis of a batched plan with restart length m over N unknowns: m + 1 complex128 basis
// vectors and m complex64 preconditioned directions.
inline size_t batch_basis_bytes(size_t N, int m) { return N * ((size_t)(m + 1) * 16 + (size_t)m * 8); }

// Restart length a batched plan chooses by itself, starting from m (the longest allowed).  A kept
// factor saves a whole factorisation at every later application of its problem, while a longer
// basis saves only restarts, so the basis yields memory to the factors: never more than half of
// `avail`, then shortened (down to m_min) while the basis and all keepable factors (`factors`)
// together exceed 90% of `avail` less a 2 GiB reserve.
inline int batch_restart_for_factors(size_t N, size_t avail, size_t factors, int m, int m_min) {
    while (m > 2 && batch_basis_bytes(N, m) > avail / 2) --m;
    const size_t reserve = (size_t)2 << 30;
    const size_t room = avail > reserve ? (size_t)((double)(avail - reserve) * 0.9) : 0;
    while (m > m_min && batch_basis_bytes(N, m) + factors > room) --m;
    return m;
}

// Partial keep when the factors of all n_t systems (`per` bytes each) do not fit: the number K of
// leading systems whose factors stay in memory.  As many as fit in 90% of `avail` less `fixed`
// (one wave of transient factors, the windows and a reserve), rounded down so that the n_t - K
// systems refactorised at every application fill whole waves of `grid` CTAs (a part-filled wave
// costs as much as a full one).  0 if none fit, or if all would (then everything is kept).
inline int partial_keep_systems(int n_t, int grid, size_t per, size_t avail, size_t fixed) {
    if (n_t <= 0 || grid <= 0 || per == 0 || avail <= fixed) return 0;
    const long long kmax = (long long)((double)(avail - fixed) * 0.9 / (double)per);
    if (kmax <= 0 || kmax >= n_t) return 0;
    const long long waves = ((long long)n_t - kmax + grid - 1) / grid;
    const long long K = (long long)n_t - waves * grid;
    return K > 0 ? (int)K : 0;
}

// GMRES basis of the single-problem refinement with restart length m over N unknowns: m + 1
// complex128 basis vectors and m complex128 preconditioned directions.
inline size_t single_basis_bytes(size_t N, int m) { return N * (size_t)(2 * m + 1) * 16; }

// Waves of `grid` CTAs that refactorise the systems whose factors are not kept.
inline int refactor_waves(int n_t, int grid, int kept) {
    return grid > 0 ? (n_t - kept + grid - 1) / grid : 0;
}

// Restart length of the single-problem refinement when the factors of all n_t systems do not fit
// (partial keep), starting from m (the longest allowed): first at most a third of `avail`, then
// shortened (down to m_min) while a shorter basis would let so many more factors stay that a whole
// wave of refactorisation drops from every preconditioner application.  The refinement converges
// in about the same number of applications whatever the restart length, so a refactorisation wave
// costs more than the restarts a longer basis saves.
inline int single_restart_for_partial_keep(size_t N, int n_t, int grid, size_t per, size_t avail, size_t fixed,
                                           int m, int m_min) {
    while (m > 2 && single_basis_bytes(N, m) > avail / 3) --m;
    if (m_min > m) m_min = m;
    auto waves = [&](int mm) {
        const size_t b = single_basis_bytes(N, mm);
        const int K = b < avail ? partial_keep_systems(n_t, grid, per, avail - b, fixed) : 0;
        return refactor_waves(n_t, grid, K);
    };
    const int best = waves(m_min);
    while (m > m_min && waves(m) > best) --m;
    return m;
}

}  // namespace stfdm
