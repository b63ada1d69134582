// Symbolic phase of the sparse-direct spatial solver: a nested-dissection ordering of the
// interior DOFs by recursive coordinate bisection, and the multifrontal assembly tree of that
// ordering.  The paper solves the n_t spatial problems (M_x + s_k A_x) w_k = g_k of eq. LGS_x with
// a sparse direct solver; every C_k has the same sparsity, so one plan serves all k.
//
// Ordering: a node set larger than `leaf` is cut at the median of its widest coordinate; the
// nodes on the lower side that have a neighbour on the upper side form the separator.  Both
// halves are ordered first (recursively), the separator last, so that every subtree's DOFs are
// numbered contiguously, before the separator that splits it from its sibling (postorder).  Each
// leaf set and each separator is one front: its DOFs are the front's pivots, eliminated together
// (a front may hold pivots whose columns of L differ in structure; the front is dense).
//
// Assembly tree: front p's update rows U_p are the rows below its last pivot of the lower
// triangle of (C restricted to p's pivot columns) together with the update rows of its children;
// its parent is the front that holds the smallest row of U_p (every other row of U_p lies in that
// parent's front, because the fill of an eliminated column is contained in the column of its
// first off-diagonal row).  Children therefore precede their parents, and grouping the fronts by
// height (leaves 0, parent = 1 + max over children) gives launch levels whose fronts are
// independent.
#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>
#include <vector>

#include "internal.h"

namespace stfdm {
namespace {

struct Builder {
    const MeshSpace& ms;
    int leaf;
    std::vector<int> order;              // new -> old, filled in postorder
    std::vector<std::pair<int, int>> groups;   // (first new index, count) per front, creation order
    std::vector<int> mark;               // scratch: side of a node in the current split (-1 = elsewhere)

    Builder(const MeshSpace& m, int l) : ms(m), leaf(l), mark(m.n_x, -1) {}

    void emit(std::vector<int>& nodes) {
        if (nodes.empty()) return;
        const int first = (int)order.size();
        for (int v : nodes) order.push_back(v);
        groups.push_back({first, (int)nodes.size()});
    }

    void dissect(std::vector<int> nodes) {
        if ((int)nodes.size() <= leaf) {
            emit(nodes);
            return;
        }
        const int d = ms.dim;
        int axis = 0;
        double wbest = -1;
        for (int a = 0; a < d; ++a) {
            double lo = 1e300, hi = -1e300;
            for (int v : nodes) {
                const double x = ms.xyz[(size_t)v * d + a];
                lo = std::min(lo, x);
                hi = std::max(hi, x);
            }
            if (hi - lo > wbest) {
                wbest = hi - lo;
                axis = a;
            }
        }
        const size_t half = nodes.size() / 2;
        auto key = [&](int v) { return ms.xyz[(size_t)v * d + axis]; };
        std::nth_element(nodes.begin(), nodes.begin() + half, nodes.end(), [&](int a, int b) {
            const double ka = key(a), kb = key(b);
            return ka != kb ? ka < kb : a < b;
        });
        // lower side: strictly below the median value (ties go up), so that a grid line is not cut
        const double med = key(nodes[half]);
        std::vector<int> lower, upper;
        for (int v : nodes) (key(v) < med ? lower : upper).push_back(v);
        if (lower.empty() || upper.empty()) {   // degenerate coordinates: split by position instead
            lower.assign(nodes.begin(), nodes.begin() + half);
            upper.assign(nodes.begin() + half, nodes.end());
        }
        for (int v : lower) mark[v] = 0;
        for (int v : upper) mark[v] = 1;
        std::vector<int> sep, low2;
        for (int v : lower) {
            bool cut = false;
            for (int q = ms.rowptr[v]; q < ms.rowptr[v + 1] && !cut; ++q) cut = mark[ms.col[q]] == 1;
            (cut ? sep : low2).push_back(v);
        }
        for (int v : nodes) mark[v] = -1;
        std::sort(sep.begin(), sep.end(), [&](int a, int b) { return key(a) != key(b) ? key(a) < key(b) : a < b; });
        dissect(std::move(low2));
        dissect(std::move(upper));
        emit(sep);
    }
};

}  // namespace

st_status build_mf_plan(const MeshSpace& ms, int leaf, MfPlan& P) {
    const int n = ms.n_x;
    if (n <= 0) return fail(ST_ERR_ARG, "multifrontal plan: empty space");
    P = MfPlan{};
    P.n = n;
    Builder b(ms, std::max(8, leaf));
    {
        std::vector<int> all(n);
        std::iota(all.begin(), all.end(), 0);
        b.dissect(std::move(all));
    }
    P.perm = b.order;
    P.iperm.assign(n, -1);
    for (int i = 0; i < n; ++i) P.iperm[P.perm[i]] = i;
    const int F = (int)b.groups.size();
    P.fronts.resize(F);
    std::vector<int> front_of(n);
    for (int f = 0; f < F; ++f) {
        P.fronts[f].first = b.groups[f].first;
        P.fronts[f].np = b.groups[f].second;
        for (int i = 0; i < b.groups[f].second; ++i) front_of[b.groups[f].first + i] = f;
    }
    // update rows in creation (post)order; children are registered with their parent as found
    std::vector<std::vector<int>> U(F), kids(F);
    std::vector<int> stamp(n, -1);
    for (int f = 0; f < F; ++f) {
        MfFront& fr = P.fronts[f];
        const int last = fr.first + fr.np - 1;
        std::vector<int>& u = U[f];
        for (int j = fr.first; j <= last; ++j) {
            const int jo = P.perm[j];
            for (int q = ms.rowptr[jo]; q < ms.rowptr[jo + 1]; ++q) {
                const int i = P.iperm[ms.col[q]];
                if (i > last && stamp[i] != f) {
                    stamp[i] = f;
                    u.push_back(i);
                }
            }
        }
        for (int c : kids[f])
            for (int i : U[c])
                if (i > last && stamp[i] != f) {
                    stamp[i] = f;
                    u.push_back(i);
                }
        std::sort(u.begin(), u.end());
        fr.nu = (int)u.size();
        fr.parent = u.empty() ? -1 : front_of[u[0]];
        if (fr.parent >= 0) {
            if (fr.parent <= f) return fail(ST_ERR_ARG, "multifrontal plan: parent precedes child");
            kids[fr.parent].push_back(f);
        }
        int h = 0;
        for (int c : kids[f]) h = std::max(h, P.fronts[c].height + 1);
        fr.height = h;
    }
    // offsets, positions of each front's update rows in its parent's front, original entries
    long long fo = 0, uo = 0, vo = 0;
    int maxh = 0;
    for (int f = 0; f < F; ++f) {
        MfFront& fr = P.fronts[f];
        const int fs = fr.np + fr.nu;
        fr.foff = fo;
        fo += (long long)fs * fr.np;
        fr.uoff = uo;
        uo += (long long)fr.nu * fr.nu;
        fr.uvoff = vo;
        vo += fr.nu;
        fr.urows_off = (int)P.urows.size();
        P.urows.insert(P.urows.end(), U[f].begin(), U[f].end());
        fr.child_off = (int)P.children.size();
        fr.child_cnt = (int)kids[f].size();
        P.children.insert(P.children.end(), kids[f].begin(), kids[f].end());
        P.max_front = std::max(P.max_front, fs);
        P.max_np = std::max(P.max_np, fr.np);
        maxh = std::max(maxh, fr.height);
        for (int c = 0; c < fr.np; ++c) P.flops_cmac += 0.5 * (double)(fs - c - 1) * (double)(fs - c) + (fs - c - 1);
    }
    P.factor_entries = fo;
    P.update_entries = uo;
    P.uvec_entries = vo;
    for (int f = 0; f < F; ++f) {
        MfFront& fr = P.fronts[f];
        fr.relpos_off = (int)P.relpos.size();
        if (fr.parent >= 0) {
            const MfFront& pa = P.fronts[fr.parent];
            const int* pu = P.urows.data() + pa.urows_off;
            for (int i : U[f]) {
                int pos;
                if (i < pa.first + pa.np) pos = i - pa.first;
                else {
                    const int* it = std::lower_bound(pu, pu + pa.nu, i);
                    if (it == pu + pa.nu || *it != i) return fail(ST_ERR_ARG, "multifrontal plan: update row outside the parent front");
                    pos = pa.np + (int)(it - pu);
                }
                P.relpos.push_back(pos);
            }
        } else {
            P.relpos.insert(P.relpos.end(), fr.nu, -1);
        }
        // lower-triangle entries (i >= j, new numbering) of the pivot columns
        fr.orig_off = (int)P.orig_k.size();
        const int* fu = P.urows.data() + fr.urows_off;
        for (int j = fr.first; j < fr.first + fr.np; ++j) {
            const int jo = P.perm[j];
            for (int q = ms.rowptr[jo]; q < ms.rowptr[jo + 1]; ++q) {
                const int i = P.iperm[ms.col[q]];
                if (i < j) continue;
                int r;
                if (i < fr.first + fr.np) r = i - fr.first;
                else r = fr.np + (int)(std::lower_bound(fu, fu + fr.nu, i) - fu);
                P.orig_r.push_back(r);
                P.orig_c.push_back(j - fr.first);
                P.orig_k.push_back(q);
            }
        }
        fr.orig_cnt = (int)P.orig_k.size() - fr.orig_off;
    }
    P.level_ptr.assign(maxh + 2, 0);
    for (const MfFront& fr : P.fronts) P.level_ptr[fr.height + 1] += 1;
    for (int h = 0; h <= maxh; ++h) P.level_ptr[h + 1] += P.level_ptr[h];
    P.level_fronts.assign(F, 0);
    std::vector<int> fill(P.level_ptr.begin(), P.level_ptr.end() - 1);
    for (int f = 0; f < F; ++f) P.level_fronts[fill[P.fronts[f].height]++] = f;
    // within a level: the fronts that one warp handles (f <= 32, 64, 96, 128) before the large ones
    P.level_ncls.assign((size_t)(maxh + 1) * MF_NCLS, 0);
    for (int h = 0; h <= maxh; ++h) {
        auto cls = [&](int fi) {
            const int fs = P.fronts[fi].np + P.fronts[fi].nu;
            return fs <= 32 * MF_NCLS ? (fs - 1) / 32 : MF_NCLS;
        };
        std::stable_sort(P.level_fronts.begin() + P.level_ptr[h], P.level_fronts.begin() + P.level_ptr[h + 1],
                         [&](int x, int y) { return cls(x) < cls(y); });
        for (int i = P.level_ptr[h]; i < P.level_ptr[h + 1]; ++i) {
            const int c = cls(P.level_fronts[i]);
            if (c < MF_NCLS) P.level_ncls[(size_t)h * MF_NCLS + c] += 1;
        }
    }
    // Update matrices live from their front's level until their parent's level has assembled them.
    // Their offsets come from a first-fit allocation replayed level by level (a level's new matrices
    // are placed before its children's are released), so the storage is the peak of the live set,
    // not the sum over all fronts.
    {
        std::map<long long, long long> free_blocks;   // offset -> size
        long long top = 0;
        auto alloc = [&](long long sz) -> long long {
            for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it)
                if (it->second >= sz) {
                    const long long off = it->first, rest = it->second - sz;
                    free_blocks.erase(it);
                    if (rest > 0) free_blocks[off + sz] = rest;
                    return off;
                }
            const long long off = top;
            top += sz;
            return off;
        };
        auto release = [&](long long off, long long sz) {
            auto it = free_blocks.emplace(off, sz).first;
            auto nx = std::next(it);
            if (nx != free_blocks.end() && it->first + it->second == nx->first) {
                it->second += nx->second;
                free_blocks.erase(nx);
            }
            if (it != free_blocks.begin()) {
                auto pv = std::prev(it);
                if (pv->first + pv->second == it->first) {
                    pv->second += it->second;
                    free_blocks.erase(it);
                }
            }
        };
        for (int h = 0; h <= maxh; ++h) {
            for (int i = P.level_ptr[h]; i < P.level_ptr[h + 1]; ++i) {
                MfFront& fr = P.fronts[P.level_fronts[i]];
                const long long sz = (long long)fr.nu * fr.nu;
                fr.uoff = sz > 0 ? alloc(sz) : 0;
            }
            for (int i = P.level_ptr[h]; i < P.level_ptr[h + 1]; ++i) {
                const MfFront& fr = P.fronts[P.level_fronts[i]];
                for (int c = 0; c < fr.child_cnt; ++c) {
                    const MfFront& ch = P.fronts[P.children[fr.child_off + c]];
                    if (ch.nu > 0) release(ch.uoff, (long long)ch.nu * ch.nu);
                }
            }
        }
        P.update_entries = top;
        // check: at every level, the update matrices alive then (produced at or below it, consumed at
        // or above it) occupy disjoint ranges
        for (int h = 0; h <= maxh; ++h) {
            std::vector<std::pair<long long, long long>> live;
            for (const MfFront& fr : P.fronts) {
                if (fr.nu == 0 || fr.height > h) continue;
                const int consumed = fr.parent >= 0 ? P.fronts[fr.parent].height : maxh + 1;
                if (consumed < h) continue;
                live.push_back({fr.uoff, fr.uoff + (long long)fr.nu * fr.nu});
            }
            std::sort(live.begin(), live.end());
            for (size_t i = 1; i < live.size(); ++i)
                if (live[i].first < live[i - 1].second)
                    return fail(ST_ERR_ARG, "multifrontal plan: overlapping update matrices");
            for (const auto& iv : live)
                if (iv.second > top) return fail(ST_ERR_ARG, "multifrontal plan: update matrix beyond the storage");
        }
    }
    return ST_OK;
}

}  // namespace stfdm

using namespace stfdm;

extern "C" st_status st_space_mf_plan(const st_space* s, int leaf, int* n_fronts, int* n_levels, int* max_front,
                                      long long* factor_entries, double* flops, int* perm, int* front_first,
                                      int* front_np, int* front_nu, int* urows) {
    if (!s) return fail(ST_ERR_ARG, "st_space_mf_plan: NULL handle");
    MeshSpace tmp;
    const MeshSpace* ms = &s->sm.mesh;
    if (s->sm.kind == 0) {
        structured_as_mesh(s->sm, tmp);
        ms = &tmp;
    }
    MfPlan P;
    st_status st = build_mf_plan(*ms, leaf > 0 ? leaf : MF_DEFAULT_LEAF, P);
    if (st != ST_OK) return st;
    const int F = (int)P.fronts.size();
    if (n_fronts) *n_fronts = F;
    if (n_levels) *n_levels = (int)P.level_ptr.size() - 1;
    if (max_front) *max_front = P.max_front;
    if (factor_entries) *factor_entries = P.factor_entries;
    if (flops) *flops = 8.0 * P.flops_cmac;
    if (perm) std::copy(P.perm.begin(), P.perm.end(), perm);
    for (int f = 0; f < F; ++f) {
        if (front_first) front_first[f] = P.fronts[f].first;
        if (front_np) front_np[f] = P.fronts[f].np;
        if (front_nu) front_nu[f] = P.fronts[f].nu;
    }
    if (urows) std::copy(P.urows.begin(), P.urows.end(), urows);
    return ST_OK;
}
