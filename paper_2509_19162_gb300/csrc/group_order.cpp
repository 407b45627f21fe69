// Order of a permutation group given by generators, by the deterministic Schreier-Sims
// algorithm (C. C. Sims, 1970; see also Seress, "Permutation Group Algorithms", ch. 4).
//
// The growth of a Cayley graph sums to the order of the generated group (Section 2.1: the
// layers partition the group).  The library uses the order only to size device buffers:
// the visited-state array of a job never needs more than |<S>| entries.
#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <vector>

#include "group_order.h"

namespace cg {

namespace {

using Perm = std::vector<uint8_t>;

Perm compose(const Perm& p, const Perm& q) {  // x -> p[q[x]]
    Perm r(p.size());
    for (size_t x = 0; x < p.size(); ++x) r[x] = p[q[x]];
    return r;
}

Perm inverse(const Perm& p) {
    Perm r(p.size());
    for (size_t x = 0; x < p.size(); ++x) r[p[x]] = (uint8_t)x;
    return r;
}

bool is_identity(const Perm& p) {
    for (size_t x = 0; x < p.size(); ++x)
        if (p[x] != x) return false;
    return true;
}

struct Level {
    int base;
    std::vector<Perm> gens;            // strong generators fixing the earlier base points
    std::vector<Perm> trans;           // trans[x]: maps base to x (empty if x not in orbit)
    std::vector<int> orbit;
};

struct Chain {
    int n;
    std::vector<Level> lv;

    void rebuild_orbit(Level& L) {
        L.trans.assign(n, Perm());
        L.orbit.clear();
        Perm id(n);
        for (int x = 0; x < n; ++x) id[x] = (uint8_t)x;
        L.trans[L.base] = id;
        L.orbit.push_back(L.base);
        for (size_t q = 0; q < L.orbit.size(); ++q) {
            const int x = L.orbit[q];
            for (const Perm& g : L.gens) {
                const int y = g[x];
                if (L.trans[y].empty()) {
                    L.trans[y] = compose(g, L.trans[x]);
                    L.orbit.push_back(y);
                }
            }
        }
    }

    // Sift g through levels from `from`; returns the residue and the level where it stopped
    // (lv.size() if it passed every level).
    Perm sift(Perm g, size_t from, size_t& stop) {
        for (size_t i = from; i < lv.size(); ++i) {
            const int x = g[lv[i].base];
            if (lv[i].trans[x].empty()) { stop = i; return g; }
            g = compose(inverse(lv[i].trans[x]), g);
        }
        stop = lv.size();
        return g;
    }

    void add_level_for(const Perm& g) {
        for (int x = 0; x < n; ++x) {
            if (g[x] != x) {
                bool used = false;
                for (auto& L : lv) used |= (L.base == x);
                if (!used) {
                    Level L;
                    L.base = x;
                    lv.push_back(L);
                    rebuild_orbit(lv.back());
                    return;
                }
            }
        }
    }
};

}  // namespace

namespace {
uint64_t group_order_uncached(int n, int k, const uint8_t* gens);

// Orders of recently seen generating sets (the key is n plus the rows as given): serving and
// batch workloads submit the same named families again and again.
std::mutex g_cache_mu;
std::map<std::vector<uint8_t>, uint64_t> g_cache;
constexpr size_t kCacheMax = 4096;
}  // namespace

uint64_t group_order(int n, int k, const uint8_t* gens) {
    std::vector<uint8_t> key;
    key.reserve(1 + (size_t)n * k);
    key.push_back((uint8_t)n);
    key.insert(key.end(), gens, gens + (size_t)n * k);
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) return it->second;
    }
    const uint64_t order = group_order_uncached(n, k, gens);
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (g_cache.size() >= kCacheMax) g_cache.clear();
    g_cache.emplace(std::move(key), order);
    return order;
}

namespace {

uint64_t group_order_uncached(int n, int k, const uint8_t* gens) {
    Chain C;
    C.n = n;
    std::vector<Perm> S;
    for (int j = 0; j < k; ++j) {
        Perm p(gens + j * n, gens + (j + 1) * n);
        if (!is_identity(p)) S.push_back(p);
    }
    if (S.empty()) return 1;
    C.add_level_for(S[0]);
    for (const Perm& g : S) {
        // Make sure every generator moves some base point.
        bool moves = false;
        for (auto& L : C.lv) moves |= (g[L.base] != L.base);
        if (!moves) C.add_level_for(g);
    }
    C.lv[0].gens = S;
    // Level i's generators are the strong generators that fix base points 0..i-1.
    for (size_t i = 1; i < C.lv.size(); ++i) {
        for (const Perm& g : S) {
            bool fixes = true;
            for (size_t b = 0; b < i; ++b) fixes &= (g[C.lv[b].base] == C.lv[b].base);
            if (fixes) C.lv[i].gens.push_back(g);
        }
    }
    for (auto& L : C.lv) C.rebuild_orbit(L);

    // Deterministic Schreier-Sims: check every Schreier generator of level i against the
    // chain below it, deepest level first; a non-trivial residue is added to the levels it
    // passed and the check restarts at the deepest level that changed.
    long i = (long)C.lv.size() - 1;
    while (i >= 0) {
        bool restarted = false;
        for (size_t oi = 0; !restarted && oi < C.lv[i].orbit.size(); ++oi) {
            const int x = C.lv[i].orbit[oi];
            for (size_t gi = 0; !restarted && gi < C.lv[i].gens.size(); ++gi) {
                const Perm s = C.lv[i].gens[gi];
                const Perm ux = C.lv[i].trans[x];
                const int y = s[x];
                Perm h = compose(inverse(C.lv[i].trans[y]), compose(s, ux));
                size_t stop = 0;
                Perm res = C.sift(h, (size_t)i + 1, stop);
                if (!is_identity(res)) {
                    if (stop == C.lv.size()) C.add_level_for(res);
                    for (size_t l = (size_t)i + 1; l <= stop && l < C.lv.size(); ++l) {
                        C.lv[l].gens.push_back(res);
                        C.rebuild_orbit(C.lv[l]);
                    }
                    i = (long)std::min(stop, C.lv.size() - 1);
                    restarted = true;
                }
            }
        }
        if (!restarted) --i;
    }
    // saturating at 2^64 - 1 (S_21 and larger groups exceed 64 bits)
    uint64_t order = 1;
    for (auto& L : C.lv) {
        const unsigned __int128 x = (unsigned __int128)order * L.orbit.size();
        order = x > (unsigned __int128)~0ull ? ~0ull : (uint64_t)x;
    }
    return order;
}

}  // namespace

}  // namespace cg
