// Device-side building blocks of the growth kernels: the generator action on packed keys,
// the key hash, the open-addressing insert, and a bounded grid-wide barrier.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "cg_internal.h"
#include "../../include/cg_growth.h"

namespace cg {

// Rotation of the 64-bit word hi:lo left by r (0..63), as two 32-bit funnel shifts: the halves
// trade places when r >= 32, then each result half is the top word of a 64-bit concatenation
// shifted left by r mod 32.  (A 64-bit rotate by a run-time amount costs several times this.)
__device__ __forceinline__ void rotl_halves(uint32_t lo, uint32_t hi, unsigned r, uint32_t& rlo,
                                            uint32_t& rhi) {
    const bool swap = (r & 32u) != 0;
    const uint32_t a = swap ? hi : lo, b = swap ? lo : hi;
    rhi = __funnelshift_l(a, b, r);
    rlo = __funnelshift_l(b, a, r);
}

// t[i] = s[g[i]] on packed keys (see GenSM): a range reversal by bit reversal, otherwise a union
// of rotated, masked copies of s, built on 32-bit halves.  kRev = false compiles the
// shift-and-mask form only: for kernels that run generators of at most 16 elements, where
// reversals are in that form.
template <bool kRev = true>
__device__ __forceinline__ uint64_t apply_gen(const GenSM& g, uint64_t s) {
    if (kRev && g.kind == 1) {
        uint64_t r = __brevll(s);
        if (g.width >= 2) r = ((r >> 1) & 0x5555555555555555ull) | ((r & 0x5555555555555555ull) << 1);
        if (g.width == 4) r = ((r >> 2) & 0x3333333333333333ull) | ((r & 0x3333333333333333ull) << 2);
        const int sh = g.rev_shift;
        r = sh >= 0 ? (r >> sh) : (r << -sh);
        return (s & ~g.mask[0]) | (r & g.mask[0]);
    }
    const uint32_t lo = (uint32_t)s, hi = (uint32_t)(s >> 32);
    uint32_t tlo = 0, thi = 0;
    const uint32_t nt = g.nterms;
#pragma unroll 2
    for (uint32_t i = 0; i < nt; ++i) {
        uint32_t rlo, rhi;
        rotl_halves(lo, hi, g.rot[i], rlo, rhi);
        const uint64_t m = g.mask[i];
        tlo |= rlo & (uint32_t)m;
        thi |= rhi & (uint32_t)(m >> 32);
    }
    return ((uint64_t)thi << 32) | tlo;
}

// 64-bit finaliser of MurmurHash3 (A. Appleby, public domain): a bijection of uint64.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

// Relaxed load served by L2 (never a stale L1 line): used for data other SMs write.
__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_ull(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ int ld_relaxed_int(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Insert-if-absent with linear probing.  Returns 1 if this call inserted the key, 0 if it was
// present (or inserted concurrently by another thread), -1 if `max_probe` slots were visited
// without finding the key or an empty slot.
__device__ __forceinline__ int table_insert(uint64_t* table, uint64_t mask, uint64_t key,
                                            uint64_t max_probe) {
    uint64_t h = mix64(key) & mask;
    for (uint64_t p = 0; p < max_probe; ++p) {
        uint64_t cur = ld_relaxed(table + h);
        if (cur == key) return 0;
        if (cur == kEmpty) {
            unsigned long long prev = atomicCAS(reinterpret_cast<unsigned long long*>(table + h),
                                                (unsigned long long)kEmpty,
                                                (unsigned long long)key);
            if (prev == kEmpty) return 1;
            if (prev == key) return 0;
        }
        h = (h + 1) & mask;
    }
    return -1;
}

// Two 16-byte loads served by L2 (cache-global, never a stale L1 line) covering one aligned
// 32-byte sector = 4 table slots.  Weak loads are enough: a slot, once written, never changes,
// and a stale "empty" is caught by the CAS that follows.
__device__ __forceinline__ void ld_sector(const uint64_t* p, uint64_t (&v)[4]) {
    const ulonglong2 a = __ldcg(reinterpret_cast<const ulonglong2*>(p));
    const ulonglong2 b = __ldcg(reinterpret_cast<const ulonglong2*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// G independent insert-if-absent sequences (linear probing) advanced together, so that one
// thread keeps G sector loads (and CASes) in flight.  Each step reads the aligned 4-slot
// sector holding the current slot and scans it from that slot on: a match ends the sequence
// (already present); the first empty slot gets a CAS; a full sector moves on to the next.
// res[i] as for table_insert; entries whose bit in vmask is clear are left at 0.
template <int G>
__device__ __forceinline__ void table_insert_multi_sector(uint64_t* table, uint64_t mask,
                                                          const uint64_t (&key)[G], int (&res)[G],
                                                          unsigned vmask, uint64_t max_steps) {
    uint64_t h[G];
    unsigned pend = vmask;   // bit i: sequence i still probing
#pragma unroll
    for (int i = 0; i < G; ++i) {
        res[i] = 0;
        h[i] = mix64(key[i]) & mask;
    }
    for (uint64_t step = 0; pend && step < max_steps; ++step) {
        uint64_t v[G][4];
#pragma unroll
        for (int i = 0; i < G; ++i)
            if (pend >> i & 1u) ld_sector(table + (h[i] & ~3ull), v[i]);
        unsigned cas = 0;
        uint64_t old[G];
#pragma unroll
        for (int i = 0; i < G; ++i) {
            if (!(pend >> i & 1u)) continue;
            const unsigned off = (unsigned)(h[i] & 3u);
            int hit = -1, empty = -1;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if ((unsigned)q >= off && hit < 0 && empty < 0) {
                    if (v[i][q] == key[i]) hit = q;
                    else if (v[i][q] == kEmpty) empty = q;
                }
            }
            if (hit >= 0) {
                pend &= ~(1u << i);
            } else if (empty >= 0) {
                h[i] = (h[i] & ~3ull) | (unsigned)empty;
                cas |= 1u << i;
                old[i] = atomicCAS(reinterpret_cast<unsigned long long*>(table + h[i]),
                                   (unsigned long long)kEmpty, (unsigned long long)key[i]);
            } else {
                h[i] = ((h[i] | 3ull) + 1) & mask;   // next sector
            }
        }
#pragma unroll
        for (int i = 0; i < G; ++i) {
            if (cas >> i & 1u) {
                if (old[i] == kEmpty) { res[i] = 1; pend &= ~(1u << i); }
                else if (old[i] == key[i]) { pend &= ~(1u << i); }
                else h[i] = (h[i] + 1) & mask;       // lost the slot: continue after it
            }
        }
    }
#pragma unroll
    for (int i = 0; i < G; ++i)
        if (pend >> i & 1u) res[i] = -1;
}

// As table_insert_multi_sector, but each step reads the single current slot (8 bytes).
template <int G>
__device__ __forceinline__ void table_insert_multi_slot(uint64_t* table, uint64_t mask,
                                                        const uint64_t (&key)[G], int (&res)[G],
                                                        unsigned vmask, uint64_t max_steps) {
    uint64_t h[G];
    unsigned pend = vmask;
#pragma unroll
    for (int i = 0; i < G; ++i) {
        res[i] = 0;
        h[i] = mix64(key[i]) & mask;
    }
    for (uint64_t step = 0; pend && step < max_steps; ++step) {
        uint64_t v[G];
#pragma unroll
        for (int i = 0; i < G; ++i)
            if (pend >> i & 1u) v[i] = __ldcg(table + h[i]);
        unsigned cas = 0;
#pragma unroll
        for (int i = 0; i < G; ++i) {
            if (pend >> i & 1u) {
                if (v[i] == key[i]) {
                    pend &= ~(1u << i);
                } else if (v[i] == kEmpty) {
                    cas |= 1u << i;
                    v[i] = atomicCAS(reinterpret_cast<unsigned long long*>(table + h[i]),
                                     (unsigned long long)kEmpty, (unsigned long long)key[i]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < G; ++i) {
            if (cas >> i & 1u) {
                if (v[i] == kEmpty) { res[i] = 1; pend &= ~(1u << i); }
                else if (v[i] == key[i]) { pend &= ~(1u << i); }
            }
            if (pend >> i & 1u) h[i] = (h[i] + 1) & mask;
        }
    }
#pragma unroll
    for (int i = 0; i < G; ++i)
        if (pend >> i & 1u) res[i] = -1;
}

// Index of a permutation in a bitmap over S_n: the position-major Lehmer rank
//     rank(s) = sum_{i=1}^{n-1} d_i * i!,   d_i = #{ j < i : s_j < s_i },
// a bijection onto [0, n!) (identity -> n!-1, full reversal -> 0).  A generator that moves only
// positions below j changes only the digits below j, so the image of a state lies within j!
// ranks of it: the probes of prefix reversals and other short-support generators of one state
// share cache lines.  Digits are taken from the top position down, d_i = s_i - #{j > i : s_j <
// s_i}; the digits of positions 12.. and 1..11 form two 32-bit Horner sums, then joined.
template <int N>
__device__ __forceinline__ uint64_t perm_rank_n(uint64_t key) {
    unsigned right = 0, top = 0, low = 0;
#pragma unroll
    for (int i = N - 1; i >= 1; --i) {
        const unsigned v = (unsigned)(key >> (4 * i)) & 15u;
        const unsigned d = v - __popc(right & ((1u << v) - 1u));
        right |= 1u << v;
        if (i >= 12) top = top * (unsigned)(i + 1) + d;
        else low = low * (unsigned)(i + 1) + d;
    }
    if (N > 12) return (uint64_t)top * 479001600ull + low;   // 12!
    return low;
}

// The same rank with n known only at run time (n <= 16).
__device__ __forceinline__ uint64_t perm_rank(uint64_t key, int n) {
    unsigned right = 0, top = 0, low = 0;
#pragma unroll
    for (int i = 15; i >= 1; --i) {
        if (i < n) {
            const unsigned v = (unsigned)(key >> (4 * i)) & 15u;
            const unsigned d = v - __popc(right & ((1u << v) - 1u));
            right |= 1u << v;
            if (i >= 12) top = top * (unsigned)(i + 1) + d;
            else low = low * (unsigned)(i + 1) + d;
        }
    }
    return (uint64_t)top * 479001600ull + low;
}

// The rank with n known at run time but the same for a whole warp (one job): the loop compiled
// for that n, through a switch.
__device__ __forceinline__ uint64_t perm_rank_uniform(uint64_t key, int n) {
    switch (n) {
        case 2: return perm_rank_n<2>(key);
        case 3: return perm_rank_n<3>(key);
        case 4: return perm_rank_n<4>(key);
        case 5: return perm_rank_n<5>(key);
        case 6: return perm_rank_n<6>(key);
        case 7: return perm_rank_n<7>(key);
        case 8: return perm_rank_n<8>(key);
        case 9: return perm_rank_n<9>(key);
        case 10: return perm_rank_n<10>(key);
        case 11: return perm_rank_n<11>(key);
        case 12: return perm_rank_n<12>(key);
        case 13: return perm_rank_n<13>(key);
        case 14: return perm_rank_n<14>(key);
        default: return perm_rank(key, n);
    }
}

// Visited test-and-set of G keys in a rank-indexed bitmap (one bit per element of S_n): one
// atomicOr per key, whose returned word says whether the bit was already set (a single L2
// round trip whether the key is new or not).  res[i] = 1 if this call set the bit, 0 if it
// was set, -1 if the rank fell outside the bitmap (not a permutation of 0..n-1).
template <int G, int N = 0>
__device__ __forceinline__ void bitmap_insert_multi(unsigned* bm, uint64_t words, int n,
                                                    const uint64_t (&key)[G], int (&res)[G],
                                                    unsigned vmask) {
    uint64_t w[G];
    unsigned bit[G], old[G];
#pragma unroll
    for (int i = 0; i < G; ++i) {
        res[i] = 0;
        const uint64_t r = N > 0 ? perm_rank_n<(N > 0 ? N : 1)>(key[i]) : perm_rank_uniform(key[i], n);
        w[i] = r >> 5;
        bit[i] = 1u << (unsigned)(r & 31u);
        if ((vmask >> i & 1u) && w[i] >= words) res[i] = -1;
    }
#pragma unroll
    for (int i = 0; i < G; ++i)
        if ((vmask >> i & 1u) && res[i] == 0) old[i] = atomicOr(bm + w[i], bit[i]);
#pragma unroll
    for (int i = 0; i < G; ++i)
        if ((vmask >> i & 1u) && res[i] == 0) res[i] = (old[i] & bit[i]) ? 0 : 1;
}

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned long long ld_acquire_ull(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_ull(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.b64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}

// Arrival half of a grid barrier whose last arriving block does some work before releasing
// the others (cooperative launch: all blocks co-resident).  `gen` is the number of barriers
// this block has passed in the launch (every block passes the same ones).  Returns 1 in every
// thread of the block that arrived last (it must call grid_release after its work), 0 in the
// other blocks once the last block has released them, -1 on error (timeout or an error word
// set by another block: the caller returns from the kernel).  `word` receives the barrier word:
// for the last block the one it arrived on (pass it to grid_release), for the others the one
// the release wrote, whose payload is word >> kGenBits.
// Ordering: every arrival is an acquire-release atomic (the block's writes before it, ordered
// by the block's own barrier, are visible to whoever observes it later, and the last arrival
// acquires everything released before), and the waiters' poll of the barrier word is an
// acquire of the closing block's work.
__device__ __forceinline__ int grid_arrive(Ctl* ctl, uint64_t timeout_ns, unsigned long long& word,
                                           unsigned gen) {
    __shared__ int s_state;
    __shared__ unsigned long long s_word;
    __syncthreads();
    if (threadIdx.x == 0) {
        gen &= (unsigned)kGenMask;
        const unsigned g = blockIdx.x % kBarGroups;
        const unsigned gsize = (gridDim.x - g + kBarGroups - 1) / kBarGroups;
        const unsigned ngroups = gridDim.x < (unsigned)kBarGroups ? gridDim.x : (unsigned)kBarGroups;
        int state = 0;
        unsigned long long w = gen;
        // The counters only grow (zeroed before each launch): barrier `gen` is complete in a
        // group when its counter reaches gsize * (gen + 1), so nothing is reset on the way.
        if (atom_add_acq_rel(&ctl->group[g].count, 1u) == gsize * (gen + 1) - 1) {
            if (atom_add_acq_rel(&ctl->bar_count, 1u) == ngroups * (gen + 1) - 1) state = 1;
        }
        if (state == 0) {
            const uint64_t t0 = globaltimer_ns();
            unsigned spins = 0;
            while (((w = ld_acquire_ull(&ctl->bar_word)) & kGenMask) == gen) {
                if ((++spins & 63u) == 0) {
                    if (*(volatile int*)&ctl->err != 0) { state = -1; break; }
                    if (globaltimer_ns() - t0 > timeout_ns) {
                        atomicCAS(&ctl->err, 0, CG_ETIMEOUT);
                        state = -1;
                        break;
                    }
                }
                __nanosleep(spins < 64 ? 32 : 256);
            }
        }
        s_state = state;
        s_word = w;
    }
    __syncthreads();
    word = s_word;
    return s_state;
}

// Release half: called by every thread of the last arriving block after its work, with the
// word grid_arrive gave it and the payload for every block (below 2^(64 - kGenBits)).
__device__ __forceinline__ void grid_release(Ctl* ctl, unsigned long long word, unsigned long long payload) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long gen = ((word & kGenMask) + 1) & kGenMask;
        st_release_ull(&ctl->bar_word, gen | (payload << kGenBits));
    }
}

}  // namespace cg
