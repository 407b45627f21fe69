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

}  // extern "C"
