/*
 * ORACLE B (test infrastructure only): growth of a permutation Cayley graph by breadth-first
 * search with a visited bitmap over all n! permutations, for groups too large for the
 * unordered_set oracle (growth_ref.cpp) to hold in host memory.
 *
 * Same definition as oracle A (Section 2.1, Def. "Growth"; BFS of Sections 3.1.2-3.1.3):
 * layer r+1 = the states reached from layer r by one generator that were never seen before.
 * The visited set is one bit per element of S_n, at index = Lehmer rank, computed directly from
 * its definition: digit c_i = #{ j > i : p[j] < p[i] }, rank = sum_i c_i (n-1-i)!.  The frontier
 * is a list of permutations (one byte per element); the expansion is split over threads, each
 * claiming bits with an atomic fetch-or.  Checked against oracle A in tests/test_oracle_pins.py.
 *
 * ORACLE C (oracle_growth_bitmask, same file): the same BFS with the frontier too kept as a
 * bitmap over the n! ranks (the paper's bitmask BFS of Section 3.1.3: bits per element of the
 * group instead of a list of states), so that the whole of S_14 (87,178,291,200 states) fits in
 * host memory: three bitmaps of n!/8 bytes (seen, current layer, next layer), 32.7 GB for n = 14.
 * Each layer step visits the set bits of the current layer in rank order, unranks each (the
 * factorial-base digits, each picking the d-th smallest unused value), applies every generator,
 * ranks the image and claims its bit in `seen`; a new state also sets its bit in the next layer.
 * Its index is the position-major Lehmer rank (posmajor_rank), under which the images of a state
 * by short-support generators lie near it, so the bit updates of neighbouring states share
 * cache lines.
 * Pinned to oracle A and oracle B in tests/test_oracle_pins.py.
 *
 * Only tests/ and the committed golden-value script may call this code.
 */
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

bool valid(int n, int k, const uint8_t* gens) {
    if (n < 1 || n > 16 || k < 1 || !gens) return false;
    for (int j = 0; j < k; ++j) {
        unsigned seen = 0;
        for (int i = 0; i < n; ++i) {
            const int v = gens[j * n + i];
            if (v >= n || (seen >> v) & 1u) return false;
            seen |= 1u << v;
        }
    }
    return true;
}

uint64_t factorial(int m) {
    uint64_t f = 1;
    for (int i = 2; i <= m; ++i) f *= (uint64_t)i;
    return f;
}

// Lehmer rank by its definition.
uint64_t lehmer_rank(const uint8_t* p, int n, const uint64_t* fact) {
    uint64_t r = 0;
    for (int i = 0; i < n; ++i) {
        uint64_t c = 0;
        for (int j = i + 1; j < n; ++j)
            if (p[j] < p[i]) ++c;
        r += c * fact[n - 1 - i];
    }
    return r;
}

// Inverse of lehmer_rank: digit c_i = (r / (n-1-i)!) mod (n-i); position i takes the c_i-th
// smallest of the values not yet used.
void lehmer_unrank(uint64_t r, int n, const uint64_t* fact, uint8_t* p) {
    unsigned unused = (1u << n) - 1u;
    for (int i = 0; i < n; ++i) {
        const uint64_t w = fact[n - 1 - i];
        unsigned c = (unsigned)(r / w);
        r -= (uint64_t)c * w;
        int v = 0;
        for (;; ++v) {
            if ((unused >> v) & 1u) {
                if (c == 0) break;
                --c;
            }
        }
        p[i] = (uint8_t)v;
        unused &= ~(1u << v);
    }
}

// lehmer_rank with the count of smaller elements to the right taken from a bit mask of the
// values at positions > i (the same definition, c_i = #{ j > i : p[j] < p[i] }).
uint64_t lehmer_rank_mask(const uint8_t* p, int n, const uint64_t* fact) {
    uint64_t r = 0;
    unsigned right = 0;
    for (int i = n - 1; i >= 0; --i) {
        const unsigned c = (unsigned)__builtin_popcount(right & ((1u << p[i]) - 1u));
        right |= 1u << p[i];
        r += (uint64_t)c * fact[n - 1 - i];
    }
    return r;
}

// Position-major Lehmer rank, rank(p) = sum_{i>=1} d_i i!, d_i = #{ j < i : p[j] < p[i] }: another
// bijection S_n -> [0, n!), used by oracle C because a generator that moves only positions
// below j changes only the digits below j, keeping its image within j! ranks (cache-friendly
// for prefix reversals and adjacent transpositions).  Digits from the top position down: d_i is
// p[i] minus the smaller values at positions above i.
uint64_t posmajor_rank(const uint8_t* p, int n, const uint64_t* fact) {
    uint64_t r = 0;
    unsigned above = 0;
    for (int i = n - 1; i >= 1; --i) {
        const unsigned d = p[i] - (unsigned)__builtin_popcount(above & ((1u << p[i]) - 1u));
        above |= 1u << p[i];
        r += (uint64_t)d * fact[i];
    }
    return r;
}

// Inverse: from the top position down, position i takes the d_i-th smallest unused value.
void posmajor_unrank(uint64_t r, int n, const uint64_t* fact, uint8_t* p) {
    unsigned unused = (1u << n) - 1u;
    for (int i = n - 1; i >= 1; --i) {
        unsigned d = (unsigned)(r / fact[i]);
        r -= (uint64_t)d * fact[i];
        int v = 0;
        for (;; ++v) {
            if ((unused >> v) & 1u) {
                if (d == 0) break;
                --d;
            }
        }
        p[i] = (uint8_t)v;
        unused &= ~(1u << v);
    }
    p[0] = (uint8_t)__builtin_ctz(unused);
}

}  // namespace

extern "C" {

/*
 * Growth from the identity, as oracle_growth (max_radius < 0: unlimited; stop_above > 0: stop
 * after the first layer larger than it).  threads <= 0: use the hardware concurrency.
 * Returns 0 (ended), 1 (stopped by a limit), -1 invalid input or n > 14 (bitmap too large),
 * -2 cap too small (*num_layers still exact), -3 out of memory.
 */
int oracle_growth_bitmap(int n, int k, const uint8_t* gens, int max_radius, uint64_t stop_above,
                         int threads, uint64_t* out, int cap, int* num_layers) {
    if (!valid(n, k, gens) || !num_layers || n > 14) return -1;
    uint64_t fact[17];
    for (int i = 0; i <= 16; ++i) fact[i] = factorial(i);
    const uint64_t total = fact[n];
    const uint64_t words = (total + 63) / 64;
    std::vector<std::atomic<uint64_t>> seen;
    try {
        seen = std::vector<std::atomic<uint64_t>>(words);
    } catch (...) {
        return -3;
    }
    for (auto& w : seen) w.store(0, std::memory_order_relaxed);
    if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());

    std::vector<uint8_t> frontier(n);
    for (int i = 0; i < n; ++i) frontier[i] = (uint8_t)i;
    {
        const uint64_t r0 = lehmer_rank(frontier.data(), n, fact);
        seen[r0 / 64].fetch_or(1ull << (r0 % 64));
    }
    std::vector<uint64_t> layers{1};
    int rc = 0;
    int radius = 0;
    for (;;) {
        if (max_radius >= 0 && radius >= max_radius) { rc = 1; break; }
        if (stop_above > 0 && layers.back() > stop_above) { rc = 1; break; }
        const uint64_t F = frontier.size() / (size_t)n;
        // The step that produces the last layer max_radius allows only counts its new states.
        const bool store = !(max_radius >= 0 && radius + 1 >= max_radius);
        std::vector<std::vector<uint8_t>> parts(threads);
        std::vector<uint64_t> counts(threads, 0);
        std::vector<std::thread> pool;
        for (int t = 0; t < threads; ++t) {
            pool.emplace_back([&, t]() {
                const uint64_t lo = F * (uint64_t)t / (uint64_t)threads;
                const uint64_t hi = F * (uint64_t)(t + 1) / (uint64_t)threads;
                std::vector<uint8_t> nb(n);
                auto& mine = parts[t];
                for (uint64_t s = lo; s < hi; ++s) {
                    const uint8_t* st = &frontier[s * (size_t)n];
                    for (int j = 0; j < k; ++j) {
                        for (int i = 0; i < n; ++i) nb[i] = st[gens[j * n + i]];   // t[i] = s[g[i]]
                        const uint64_t r = lehmer_rank(nb.data(), n, fact);
                        const uint64_t bit = 1ull << (r % 64);
                        if (!(seen[r / 64].fetch_or(bit) & bit)) {
                            ++counts[t];
                            if (store) mine.insert(mine.end(), nb.begin(), nb.end());
                        }
                    }
                }
            });
        }
        for (auto& th : pool) th.join();
        uint64_t count = 0;
        for (auto c : counts) count += c;
        if (count == 0) break;
        if (!store) {
            layers.push_back(count);
            ++radius;
            rc = 1;
            break;
        }
        std::vector<uint8_t> next;
        try {
            next.reserve(count * (size_t)n);
        } catch (...) {
            return -3;
        }
        for (auto& p : parts) {
            next.insert(next.end(), p.begin(), p.end());
            std::vector<uint8_t>().swap(p);
        }
        frontier.swap(next);
        layers.push_back(count);
        ++radius;
    }
    *num_layers = (int)layers.size();
    for (int r = 0; r < (int)layers.size() && r < cap; ++r) out[r] = layers[r];
    if ((int)layers.size() > cap) return -2;
    return rc;
}

/*
 * Oracle C: growth from the identity with the visited set and the current and next layers as
 * bitmaps over the n! Lehmer ranks.  Arguments and return codes as oracle_growth_bitmap.
 * progress, when not NULL, is called after each layer with its radius and size.
 */
int oracle_growth_bitmask(int n, int k, const uint8_t* gens, int max_radius, uint64_t stop_above,
                          int threads, uint64_t* out, int cap, int* num_layers,
                          void (*progress)(int, uint64_t)) {
    if (!valid(n, k, gens) || !num_layers || n > 14) return -1;
    uint64_t fact[17];
    for (int i = 0; i <= 16; ++i) fact[i] = factorial(i);
    const uint64_t total = fact[n];
    const uint64_t words = (total + 63) / 64;
    std::vector<std::atomic<uint64_t>> seen, cur, nxt;
    try {
        seen = std::vector<std::atomic<uint64_t>>(words);
        cur = std::vector<std::atomic<uint64_t>>(words);
        nxt = std::vector<std::atomic<uint64_t>>(words);
    } catch (...) {
        return -3;
    }
    if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());
    auto parallel = [&](auto&& body) {   // body(word_begin, word_end) over chunks of the words
        std::atomic<uint64_t> next_chunk{0};
        const uint64_t chunk = 1u << 14;
        std::vector<std::thread> pool;
        for (int t = 0; t < threads; ++t)
            pool.emplace_back([&]() {
                for (;;) {
                    const uint64_t c = next_chunk.fetch_add(1);
                    const uint64_t b = c * chunk;
                    if (b >= words) break;
                    body(b, std::min(words, b + chunk));
                }
            });
        for (auto& th : pool) th.join();
    };
    parallel([&](uint64_t b, uint64_t e) {
        for (uint64_t w = b; w < e; ++w) {
            seen[w].store(0, std::memory_order_relaxed);
            cur[w].store(0, std::memory_order_relaxed);
            nxt[w].store(0, std::memory_order_relaxed);
        }
    });
    {
        std::vector<uint8_t> id(n);
        for (int i = 0; i < n; ++i) id[i] = (uint8_t)i;
        const uint64_t r0 = posmajor_rank(id.data(), n, fact);
        seen[r0 / 64].fetch_or(1ull << (r0 % 64));
        cur[r0 / 64].fetch_or(1ull << (r0 % 64));
    }
    std::vector<uint64_t> layers{1};
    int rc = 0;
    int radius = 0;
    for (;;) {
        if (max_radius >= 0 && radius >= max_radius) { rc = 1; break; }
        if (stop_above > 0 && layers.back() > stop_above) { rc = 1; break; }
        std::atomic<uint64_t> count{0};
        parallel([&](uint64_t b, uint64_t e) {
            std::vector<uint8_t> s(n), t(n);
            uint64_t mine = 0;
            for (uint64_t w = b; w < e; ++w) {
                uint64_t bits = cur[w].load(std::memory_order_relaxed);
                while (bits) {
                    const int bit = __builtin_ctzll(bits);
                    bits &= bits - 1;
                    posmajor_unrank(w * 64 + (uint64_t)bit, n, fact, s.data());
                    for (int j = 0; j < k; ++j) {
                        for (int i = 0; i < n; ++i) t[i] = s[gens[j * n + i]];   // t[i] = s[g[i]]
                        const uint64_t r = posmajor_rank(t.data(), n, fact);
                        const uint64_t m = 1ull << (r % 64);
                        if (!(seen[r / 64].fetch_or(m, std::memory_order_relaxed) & m)) {
                            nxt[r / 64].fetch_or(m, std::memory_order_relaxed);
                            ++mine;
                        }
                    }
                }
            }
            count.fetch_add(mine);
        });
        const uint64_t c = count.load();
        if (c == 0) break;
        layers.push_back(c);
        ++radius;
        if (progress) progress(radius, c);
        // the next layer becomes the current one; the old current layer is cleared
        cur.swap(nxt);
        parallel([&](uint64_t b, uint64_t e) {
            for (uint64_t w = b; w < e; ++w) nxt[w].store(0, std::memory_order_relaxed);
        });
    }
    *num_layers = (int)layers.size();
    for (int r = 0; r < (int)layers.size() && r < cap; ++r) out[r] = layers[r];
    if ((int)layers.size() > cap) return -2;
    return rc;
}

}  // extern "C"
