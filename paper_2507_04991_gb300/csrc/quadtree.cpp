// Host-side quadtree of the adaptive runs (Sec. 3.2.2, Sec. 5.3): a
// 2:1-balanced periodic quadtree of square cells on [-L, L]^2 over an n x n
// base grid, its adaptation (coarsen marked families, refine marked leaves,
// restore the balance) with the map of new leaves to old ones, and the mesh
// arrays of the C ABI (node coordinates, conforming faces, 2:1 mortars).
// No GPU work; the state computations of an adaptation run in the library's
// kernels (perrk_amr_indicator, perrk_amr_transfer).
//
// A leaf is (level, ix, iy), 0 <= ix, iy < n 2^level; leaves are kept in the
// canonical order of (level, ix, iy).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "perrk_internal.h"

struct perrk_quadtree {
    int n = 0;
    double L = 1.0;
    std::vector<uint64_t> leaves;                 // packed keys in canonical order
    std::unordered_map<uint64_t, int> pos;        // key -> leaf index
};

namespace perrk {
namespace {

// cell indices are packed in 29 bits each: n 2^level < 2^29
constexpr long long kMaxCells = 1ll << 29;

inline uint64_t key(int lev, long long ix, long long iy) {
    return ((uint64_t)lev << 58) | ((uint64_t)ix << 29) | (uint64_t)iy;
}
inline int klev(uint64_t k) { return (int)(k >> 58); }
inline long long kix(uint64_t k) { return (long long)((k >> 29) & ((1ull << 29) - 1)); }
inline long long kiy(uint64_t k) { return (long long)(k & ((1ull << 29) - 1)); }

inline long long wrapi(long long i, long long m) { return ((i % m) + m) % m; }

struct Tree {
    int n;
    std::unordered_set<uint64_t> set;

    long long cells(int lev) const { return (long long)n << lev; }

    // the leaf containing cell (lev, ix, iy) (periodic), or 0 with found = false
    bool owner(int lev, long long ix, long long iy, uint64_t &out) const {
        const long long m = cells(lev);
        ix = wrapi(ix, m);
        iy = wrapi(iy, m);
        for (int l = lev; l >= 0; --l) {
            const uint64_t k = key(l, ix >> (lev - l), iy >> (lev - l));
            if (set.count(k)) {
                out = k;
                return true;
            }
        }
        return false;
    }

    static void children(uint64_t k, uint64_t *c) {
        const int l = klev(k);
        const long long i = kix(k), j = kiy(k);
        for (int q = 0; q < 4; ++q) c[q] = key(l + 1, 2 * i + (q & 1), 2 * j + (q >> 1));   // child index a + 2 b
    }

    // split leaves until no face neighbour of a leaf is two levels coarser than it
    void balance() {
        std::vector<uint64_t> queue(set.begin(), set.end());
        std::sort(queue.begin(), queue.end());
        static const int d[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
        while (!queue.empty()) {
            const uint64_t c = queue.back();
            queue.pop_back();
            if (!set.count(c)) continue;
            const int l = klev(c);
            for (auto &dd : d) {
                uint64_t o;
                if (owner(l, kix(c) + dd[0], kiy(c) + dd[1], o) && klev(o) < l - 1) {
                    set.erase(o);
                    uint64_t ch[4];
                    children(o, ch);
                    for (uint64_t x : ch) {
                        set.insert(x);
                        queue.push_back(x);
                    }
                    queue.push_back(c);
                }
            }
        }
    }

    // would merging the four children of p into p leave a face neighbour of p
    // two levels finer than p?
    bool merge_keeps_balance(uint64_t p) const {
        const int l = klev(p);
        const long long i = kix(p), j = kiy(p);
        // for each face of p, the two cells at level l + 1 across it
        const long long cand[4][2][2] = {
            {{2 * i - 1, 2 * j}, {2 * i - 1, 2 * j + 1}},      // -x
            {{2 * i + 2, 2 * j}, {2 * i + 2, 2 * j + 1}},      // +x
            {{2 * i, 2 * j - 1}, {2 * i + 1, 2 * j - 1}},      // -y
            {{2 * i, 2 * j + 2}, {2 * i + 1, 2 * j + 2}}};     // +y
        for (auto &face : cand)
            for (auto &cc : face) {
                uint64_t o;
                // the cell at level l + 1 is covered by a leaf (at level <= l + 1), or split further
                if (!owner(l + 1, cc[0], cc[1], o)) return false;
            }
        return true;
    }
};

}  // namespace
}  // namespace perrk

using namespace perrk;

static void refill(perrk_quadtree *t, const std::unordered_set<uint64_t> &set) {
    t->leaves.assign(set.begin(), set.end());
    std::sort(t->leaves.begin(), t->leaves.end(), [](uint64_t a, uint64_t b) {
        if (klev(a) != klev(b)) return klev(a) < klev(b);
        if (kix(a) != kix(b)) return kix(a) < kix(b);
        return kiy(a) < kiy(b);
    });
    t->pos.clear();
    t->pos.reserve(t->leaves.size() * 2);
    for (size_t k = 0; k < t->leaves.size(); ++k) t->pos[t->leaves[k]] = (int)k;
}

extern "C" {

perrk_status perrk_quadtree_create(int n, double L, perrk_quadtree **out) {
    if (!out || n < 1 || n > (1 << 20) || !(L > 0.0)) {
        set_error("quadtree_create: n in [1, 2^20], L > 0, out not null");
        return PERRK_INVALID_ARG;
    }
    perrk_quadtree *t = new (std::nothrow) perrk_quadtree();
    if (!t) return PERRK_OUT_OF_MEMORY;
    t->n = n;
    t->L = L;
    std::unordered_set<uint64_t> set;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) set.insert(key(0, i, j));
    refill(t, set);
    *out = t;
    return PERRK_OK;
}

void perrk_quadtree_destroy(perrk_quadtree *t) { delete t; }

int perrk_quadtree_size(const perrk_quadtree *t) { return t ? (int)t->leaves.size() : 0; }

perrk_status perrk_quadtree_leaves(const perrk_quadtree *t, int32_t *out) {
    if (!t || !out) return PERRK_INVALID_ARG;
    for (size_t k = 0; k < t->leaves.size(); ++k) {
        out[3 * k] = klev(t->leaves[k]);
        out[3 * k + 1] = (int32_t)kix(t->leaves[k]);
        out[3 * k + 2] = (int32_t)kiy(t->leaves[k]);
    }
    return PERRK_OK;
}

perrk_status perrk_quadtree_adapt(perrk_quadtree *t, const int8_t *marks, int32_t *map, int map_cap, int *n_new) {
    if (!t || !marks || !map || !n_new) return PERRK_INVALID_ARG;
    const size_t n0 = t->leaves.size();
    Tree tr{t->n, {}};
    tr.set.reserve(4 * n0 + 16);
    tr.set.insert(t->leaves.begin(), t->leaves.end());
    std::unordered_set<uint64_t> refine, coarsen;
    for (size_t k = 0; k < n0; ++k) {
        if (marks[k] > 0) {
            if (((long long)t->n << (klev(t->leaves[k]) + 1)) >= kMaxCells) {
                set_error("quadtree_adapt: refinement beyond n 2^level = 2^29 cells per direction");
                return PERRK_INVALID_ARG;
            }
            refine.insert(t->leaves[k]);
        } else if (marks[k] < 0) {
            coarsen.insert(t->leaves[k]);
        }
    }
    // families whose four leaves are all marked for coarsening merge, in
    // descending (level, ix, iy) order of the parent, where the balance allows
    std::vector<uint64_t> parents;
    for (uint64_t c : coarsen)
        if (klev(c) > 0) parents.push_back(key(klev(c) - 1, kix(c) >> 1, kiy(c) >> 1));
    std::sort(parents.begin(), parents.end(), [](uint64_t a, uint64_t b) {
        if (klev(a) != klev(b)) return klev(a) > klev(b);
        if (kix(a) != kix(b)) return kix(a) > kix(b);
        return kiy(a) > kiy(b);
    });
    parents.erase(std::unique(parents.begin(), parents.end()), parents.end());
    for (uint64_t p : parents) {
        uint64_t ch[4];
        Tree::children(p, ch);
        bool all = true;
        for (uint64_t c : ch) all = all && tr.set.count(c) && coarsen.count(c);
        if (!all) continue;
        for (uint64_t c : ch) tr.set.erase(c);
        tr.set.insert(p);
        if (!tr.merge_keeps_balance(p)) {
            tr.set.erase(p);
            for (uint64_t c : ch) tr.set.insert(c);
        }
    }
    for (uint64_t c : refine)
        if (tr.set.count(c)) {
            tr.set.erase(c);
            uint64_t ch[4];
            Tree::children(c, ch);
            for (uint64_t x : ch) tr.set.insert(x);
        }
    tr.balance();
    if ((int)tr.set.size() > map_cap) {
        set_error("quadtree_adapt: map capacity below the new leaf count (4 x the old count always suffices)");
        return PERRK_INVALID_ARG;
    }
    const std::unordered_map<uint64_t, int> &old_pos = t->pos;   // unchanged until the swap below
    perrk_quadtree fresh;
    refill(&fresh, tr.set);
    for (size_t k = 0; k < fresh.leaves.size(); ++k) {
        const uint64_t c = fresh.leaves[k];
        int32_t *r = map + 5 * k;
        auto it = old_pos.find(c);
        if (it != old_pos.end()) {
            r[0] = 0;
            r[1] = it->second;
            r[2] = r[3] = r[4] = 0;
            continue;
        }
        const int l = klev(c);
        if (l > 0) {
            auto ip = old_pos.find(key(l - 1, kix(c) >> 1, kiy(c) >> 1));
            if (ip != old_pos.end()) {
                r[0] = 1;
                r[1] = ip->second;
                r[2] = (int32_t)((kix(c) & 1) + 2 * (kiy(c) & 1));
                r[3] = r[4] = 0;
                continue;
            }
        }
        uint64_t ch[4];
        Tree::children(c, ch);
        r[0] = 2;
        for (int q = 0; q < 4; ++q) {
            auto ic = old_pos.find(ch[q]);
            if (ic == old_pos.end()) {
                set_error("quadtree_adapt: a leaf changed by more than one level");
                return PERRK_INVALID_ARG;
            }
            r[1 + q] = ic->second;
        }
    }
    t->leaves.swap(fresh.leaves);
    t->pos.swap(fresh.pos);
    *n_new = (int)t->leaves.size();
    return PERRK_OK;
}

perrk_status perrk_quadtree_mesh(const perrk_quadtree *t, double *coords, int32_t *faces, int *n_faces,
                                 int32_t *mortars, int *n_mortars, int32_t *levels) {
    if (!t || !n_faces || !n_mortars) return PERRK_INVALID_ARG;
    static const double lgl[4] = {-1.0, -0.44721359549995793928, 0.44721359549995793928, 1.0};
    // a leaf covering cell (l, i, j) at its own level or coarser
    auto covered = [&](int l, long long i, long long j) {
        for (int k = l; k >= 0; --k)
            if (t->pos.count(key(k, i >> (l - k), j >> (l - k)))) return true;
        return false;
    };
    int nf = 0, nm = 0;
    static const int d[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};   // faces 0: -x, 1: +x, 2: -y, 3: +y
    for (size_t e = 0; e < t->leaves.size(); ++e) {
        const uint64_t c = t->leaves[e];
        const int l = klev(c);
        const long long i = kix(c), j = kiy(c), m = (long long)t->n << l;
        const double h = 2.0 * t->L / (double)m;
        if (coords)
            for (int q = 0; q < 16; ++q) {
                coords[(e * 16 + q) * 2] = -t->L + ((double)i + 0.5 * (lgl[q & 3] + 1.0)) * h;
                coords[(e * 16 + q) * 2 + 1] = -t->L + ((double)j + 0.5 * (lgl[q >> 2] + 1.0)) * h;
            }
        if (levels) levels[e] = l;
        for (int f = 0; f < 4; ++f) {
            const long long ni = wrapi(i + d[f][0], m), nj = wrapi(j + d[f][1], m);
            auto it = t->pos.find(key(l, ni, nj));
            if (it != t->pos.end()) {
                if (f & 1) {
                    if (faces) {
                        int32_t *r = faces + 4 * nf;
                        r[0] = (int32_t)e;
                        r[1] = f;
                        r[2] = it->second;
                        r[3] = f - 1;
                    }
                    ++nf;
                }
                continue;
            }
            if (covered(l, ni, nj)) continue;   // a coarser neighbour lists this face in its mortar row
            uint64_t lo, hi;
            if (f < 2) {   // the finer column touching this face, lower y first
                const long long ci = 2 * ni + (f == 0 ? 1 : 0);
                lo = key(l + 1, ci, 2 * nj);
                hi = key(l + 1, ci, 2 * nj + 1);
            } else {       // the finer row touching this face, lower x first
                const long long cj = 2 * nj + (f == 2 ? 1 : 0);
                lo = key(l + 1, 2 * ni, cj);
                hi = key(l + 1, 2 * ni + 1, cj);
            }
            auto a = t->pos.find(lo), b = t->pos.find(hi);
            if (a == t->pos.end() || b == t->pos.end()) {
                set_error("quadtree_mesh: the tree is not 2:1 balanced");
                return PERRK_INVALID_ARG;
            }
            if (mortars) {
                int32_t *r = mortars + 4 * nm;
                r[0] = (int32_t)e;
                r[1] = f;
                r[2] = a->second;
                r[3] = b->second;
            }
            ++nm;
        }
    }
    *n_faces = nf;
    *n_mortars = nm;
    return PERRK_OK;
}

}  // extern "C"
