/*
 * ORACLE (test infrastructure only).
 *
 * A plain, slow, sequential CPU computation of the growth of a permutation Cayley graph,
 * written from the paper's definition and nothing else:
 *
 *   gamma(m) = |{ v : d(v, v0) = m }|,  v0 = identity                (Section 2.1, Def. "Growth")
 *
 * where d is the word metric of the generating set (the fewest generator applications that
 * reach v), computed by the textbook breadth-first search the paper says all of its growth
 * algorithms are built on (Sections 3.1.2 and 3.1.3).  States are permutations held as byte
 * arrays; a generator g acts by gather, t[i] = s[g[i]].  The visited set is a
 * std::unordered_set of an injective packing of the permutation, used only as a hash key:
 * 4 bits per element for n <= 16, its bytes for n <= 32, 4 bits per value in 256 bits for
 * vectors of up to 64 values below 16.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline / reference arm may load
 * this file's library.  It shares no code, header or table with the CUDA library.
 *
 * Pins (in tests/test_oracle_pins.py): Mahonian numbers for adjacent transpositions,
 * unsigned Stirling numbers of the first kind for all transpositions, layer sums equal to
 * the group order (sympy's Schreier-Sims and brute-force closure), palindromic Coxeter
 * growth, published diameters (Section 3.3 table, Section 3.4 maximal-diameter tables,
 * Section 4 LX conjecture, Section 5.2 reversal sphere |S_2|), and all-pairs shortest paths
 * of the explicit graph for n <= 5.  The coset mode (growth from a vector with repeated
 * entries) is pinned in tests/test_oracle_coset_pins.py: all-pairs shortest paths of the
 * explicit coset graph, orbit sizes, and the God's numbers the paper prints for the binary
 * coset (Section 3.2 and the Schreier-graph table).
 */
#include <cstdint>
#include <cstring>
#include <unordered_set>
#include <vector>
#include <algorithm>

namespace {

// Injective key of a permutation of {0..n-1}, n <= 16: element i in bits [4i, 4i+4).
uint64_t key_of(const uint8_t* p, int n) {
    uint64_t key = 0;
    for (int i = 0; i < n; ++i) key |= (uint64_t)p[i] << (4 * i);
    return key;
}

// Injective key of a vector of up to 64 values below 16 (element i in bits [4i, 4i+4) of a
// 256-bit number), for the orbits of long vectors (Schreier coset graphs with n > 16).
struct WideKey {
    uint64_t w[4];
    bool operator==(const WideKey& o) const {
        return w[0] == o.w[0] && w[1] == o.w[1] && w[2] == o.w[2] && w[3] == o.w[3];
    }
};
struct WideHash {
    size_t operator()(const WideKey& k) const {
        return std::hash<uint64_t>()(k.w[0] ^ (k.w[1] * 0x9E3779B97F4A7C15ull) ^
                                     (k.w[2] * 0xC2B2AE3D27D4EB4Full) ^ (k.w[3] * 0x165667B19E3779F9ull));
    }
};

// Injective key of a permutation of up to 32 elements: its bytes, element i in byte i of a
// 256-bit number (growth from the identity with 16 < n <= 32).
struct ByteKeys {
    using Key = WideKey;
    using Set = std::unordered_set<WideKey, WideHash>;
    static Key of(const uint8_t* p, int n) {
        WideKey k{{0, 0, 0, 0}};
        std::memcpy(k.w, p, (size_t)n);
        return k;
    }
};

struct NarrowKeys {
    using Key = uint64_t;
    using Set = std::unordered_set<uint64_t>;
    static Key of(const uint8_t* p, int n) { return key_of(p, n); }
};
struct WideKeys {
    using Key = WideKey;
    using Set = std::unordered_set<WideKey, WideHash>;
    static Key of(const uint8_t* p, int n) {
        WideKey k{{0, 0, 0, 0}};
        for (int i = 0; i < n; ++i) k.w[i / 16] |= (uint64_t)p[i] << (4 * (i % 16));
        return k;
    }
};

bool valid_gens(int n, int k, const uint8_t* gens, int max_n = 16) {
    if (n < 1 || n > max_n || k < 1 || gens == nullptr) return false;
    for (int j = 0; j < k; ++j) {
        std::vector<int> hit(n, 0);
        for (int i = 0; i < n; ++i) {
            int v = gens[j * n + i];
            if (v >= n || hit[v]) return false;
            hit[v] = 1;
        }
    }
    return true;
}

// Apply generator g to state s by gather: t[i] = s[g[i]].
void apply(const uint8_t* s, const uint8_t* g, uint8_t* t, int n) {
    for (int i = 0; i < n; ++i) t[i] = s[g[i]];
}

template <class Keys>
struct BfsT {
    using Key = typename Keys::Key;
    int n, k;
    const uint8_t* gens;
    bool two_layer;
    typename Keys::Set seen;                           // full-visited mode
    typename Keys::Set prev, cur;                      // two-layer mode
    std::vector<uint8_t> frontier;                     // n bytes per state
    uint64_t frontier_count = 0;
    int radius = 0;

    // Breadth-first search from `start` (n values, repeats allowed: the orbit of a vector under
    // the group, i.e. a Schreier coset graph, Sections 3.1.2 and 5.2), or from the identity.
    BfsT(int n_, int k_, const uint8_t* g_, bool two, const uint8_t* start = nullptr)
        : n(n_), k(k_), gens(g_), two_layer(two) {
        frontier.resize(n);
        for (int i = 0; i < n; ++i) frontier[i] = start ? start[i] : (uint8_t)i;
        frontier_count = 1;
        const Key id = Keys::of(frontier.data(), n);
        if (two_layer) cur.insert(id); else seen.insert(id);
    }

    // One BFS step: returns the size of the next layer and makes it the frontier.
    uint64_t step() {
        std::vector<uint8_t> next;
        typename Keys::Set next_set;
        std::vector<uint8_t> t(n);
        for (uint64_t s = 0; s < frontier_count; ++s) {
            const uint8_t* st = &frontier[s * n];
            for (int j = 0; j < k; ++j) {
                apply(st, gens + j * n, t.data(), n);
                const Key key = Keys::of(t.data(), n);
                bool fresh;
                if (two_layer) {
                    // Only valid for inverse-closed sets: every neighbour of layer r lies in
                    // layer r-1, r or r+1.
                    fresh = !prev.count(key) && !cur.count(key) && next_set.insert(key).second;
                } else {
                    fresh = seen.insert(key).second;
                }
                if (fresh) next.insert(next.end(), t.begin(), t.end());
            }
        }
        uint64_t count = next.size() / (size_t)n;
        frontier.swap(next);
        frontier_count = count;
        if (two_layer) {
            prev.swap(cur);
            cur.swap(next_set);
        }
        ++radius;
        return count;
    }
};

using Bfs = BfsT<NarrowKeys>;

template <class B>
int run_growth(B& bfs, int max_radius, uint64_t stop_above, uint64_t* out, int cap, int* num_layers) {
    std::vector<uint64_t> layers{1};
    int rc = 0;
    while (true) {
        if (max_radius >= 0 && bfs.radius >= max_radius) { rc = 1; break; }
        if (stop_above > 0 && layers.back() > stop_above) { rc = 1; break; }
        uint64_t c = bfs.step();
        if (c == 0) break;
        layers.push_back(c);
    }
    *num_layers = (int)layers.size();
    for (int r = 0; r < (int)layers.size() && r < cap; ++r) out[r] = layers[r];
    if ((int)layers.size() > cap) return -2;
    return rc;
}

}  // namespace

extern "C" {

/*
 * Growth vector of <gens> from the identity (oracle_growth, n <= 32) or from the vector `start`
 * (oracle_growth_from; n <= 64 values in 0..15, repeats allowed).
 *   two_layer   0: full visited set (any generating set); 1: keep only layers r-1 and r
 *               (correct only for inverse-closed sets; the tests check it against mode 0).
 *   max_radius  < 0: unlimited; else stop after layer max_radius.
 *   stop_above  > 0: stop after the first layer whose size exceeds this value.
 * Writes gamma(0..R) to out[0..cap) and R+1 to *num_layers.
 * Returns 0 when the growth ended (empty next layer), 1 when stopped by max_radius or
 * stop_above, -1 on invalid input, -2 when cap was too small (*num_layers still exact).
 */
int oracle_growth_from(int n, int k, const uint8_t* gens, const uint8_t* start, int two_layer,
                       int max_radius, uint64_t stop_above, uint64_t* out, int cap, int* num_layers) {
    // n up to 64 when a start vector is given (values below 16), up to 32 from the identity
    if (!valid_gens(n, k, gens, start ? 64 : 32) || num_layers == nullptr) return -1;
    if (start)
        for (int i = 0; i < n; ++i)
            if (start[i] > 15) return -1;
    if (n <= 16) {
        BfsT<NarrowKeys> bfs(n, k, gens, two_layer != 0, start);
        return run_growth(bfs, max_radius, stop_above, out, cap, num_layers);
    }
    if (!start) {
        BfsT<ByteKeys> bfs(n, k, gens, two_layer != 0, start);
        return run_growth(bfs, max_radius, stop_above, out, cap, num_layers);
    }
    BfsT<WideKeys> bfs(n, k, gens, two_layer != 0, start);
    return run_growth(bfs, max_radius, stop_above, out, cap, num_layers);
}

int oracle_growth(int n, int k, const uint8_t* gens, int two_layer, int max_radius,
                  uint64_t stop_above, uint64_t* out, int cap, int* num_layers) {
    return oracle_growth_from(n, k, gens, nullptr, two_layer, max_radius, stop_above, out, cap,
                              num_layers);
}

/*
 * The states of layer <radius> as packed keys (element i in bits [4i, 4i+4)), sorted
 * ascending.  Returns 0, -1 on invalid input, -2 if cap is too small (*count still exact),
 * -3 if the layer is empty (radius beyond the diameter).
 */
int oracle_layer_keys(int n, int k, const uint8_t* gens, int radius, uint64_t* keys_out,
                      uint64_t cap, uint64_t* count) {
    if (!valid_gens(n, k, gens) || radius < 0 || count == nullptr) return -1;
    Bfs bfs(n, k, gens, false);
    while (bfs.radius < radius) {
        if (bfs.step() == 0) { *count = 0; return -3; }
    }
    std::vector<uint64_t> keys(bfs.frontier_count);
    for (uint64_t s = 0; s < bfs.frontier_count; ++s) keys[s] = key_of(&bfs.frontier[s * n], n);
    std::sort(keys.begin(), keys.end());
    *count = keys.size();
    if (keys.size() > cap) return -2;
    std::copy(keys.begin(), keys.end(), keys_out);
    return 0;
}

/*
 * Word-metric distance from the identity to <target> (one-line bytes), searching layers
 * up to max_radius.  Returns the distance, -1 if not found within max_radius or not in the
 * group, -2 on invalid input.
 */
int oracle_distance(int n, int k, const uint8_t* gens, const uint8_t* target, int max_radius) {
    if (!valid_gens(n, k, gens) || target == nullptr) return -2;
    uint64_t want = key_of(target, n);
    Bfs bfs(n, k, gens, false);
    if (key_of(bfs.frontier.data(), n) == want) return 0;
    while (max_radius < 0 || bfs.radius < max_radius) {
        if (bfs.step() == 0) return -1;
        for (uint64_t s = 0; s < bfs.frontier_count; ++s)
            if (key_of(&bfs.frontier[s * n], n) == want) return bfs.radius;
    }
    return -1;
}

}  // extern "C"
