// Sort strategy of the growth library: sorted layers, radix sort + unique of the candidates,
// set difference against the two previous layers, compaction.
//
// For an inverse-closed generating set every neighbour of layer r lies in layer r-1, r or r+1,
// so layer r+1 = unique(candidates) \ (L_r U L_{r-1}) needs only the two previous layers
// (Section 3.4: undirected graphs are those with inverse-closed generators).  Layers are kept
// as arrays of packed keys sorted ascending.  One layer step is:
//   histograms    one read of the candidates -- generated on the fly from L_r (every generator
//                 on every state: the expand is fused, candidates are never written unsorted)
//                 -- counts the 8-bit digits of every pass at once
//   radix passes  LSD over the w n significant key bits, one kernel per pass: each 4096-key
//                 tile ranks its keys by digit (warp match_any, per-warp digit counts in shared
//                 memory), finds each digit's offset among the earlier tiles by a decoupled
//                 look-back per digit, and writes its keys digit run by digit run (coalesced)
//                 from a shared-memory staging copy; stable, so the passes compose
//   difference    one kernel: a candidate survives when it is the first of its run and absent
//                 from L_r and L_{r-1} (a galloping walk through each sorted layer from the
//                 thread's first key), and the survivors are compacted in order with a
//                 decoupled look-back over tiles: layer r+1, sorted, and its size
// The same primitives back the step-level entry points cg_sort_unique and cg_set_difference.
#include <cstdint>

#include "cg_device.cuh"
#include "sort_kernels.h"

namespace cg {

namespace {

constexpr int kBlock = 256;
constexpr int kItems = 16;                       // keys per thread per tile
constexpr int kTile = kBlock * kItems;           // 4096 keys per tile
constexpr int kWarps = kBlock / 32;
constexpr int kRadixBits = 8;
constexpr int kDigits = 1 << kRadixBits;
constexpr uint64_t kSpinTimeoutNs = 5ull * 1000 * 1000 * 1000;

// ---- decoupled look-back ---------------------------------------------------------------------
// Descriptor: bits 60-63 epoch (which pass wrote it; the region is cleared once per sort),
// bits 58-59 status (1 aggregate of the tile, 2 inclusive prefix), bits 0-57 value.  Tiles take
// tickets in start order, so every predecessor a tile waits on is running.
constexpr unsigned long long kValMask = (1ull << 58) - 1;

__device__ __forceinline__ unsigned long long make_desc(unsigned epoch, unsigned status, unsigned long long v) {
    return ((unsigned long long)epoch << 60) | ((unsigned long long)status << 58) | (v & kValMask);
}

// Exclusive prefix of `agg` over the tiles before `tile`, for one lane of descriptors
// (desc[t * stride]).  The walk back reads kWindow predecessors' descriptors per round trip
// (independent loads), sums aggregates in order and stops at the first inclusive prefix; a
// window with an unpublished descriptor is read again from there.  Sets *err and returns 0 if
// a predecessor never publishes in time.
constexpr int kWindow = 8;

__device__ unsigned long long look_back(unsigned long long* desc, int stride, int tile, unsigned long long agg,
                                        unsigned epoch, int* err) {
    if (tile == 0) {
        atomicExch(desc, make_desc(epoch, 2, agg));
        return 0;
    }
    atomicExch(desc + (size_t)tile * stride, make_desc(epoch, 1, agg));
    unsigned long long prefix = 0;
    int t = tile - 1;
    const uint64_t t0 = globaltimer_ns();
    unsigned spins = 0;
    bool done = false;
    while (!done) {
        unsigned long long d[kWindow];
#pragma unroll
        for (int i = 0; i < kWindow; ++i)
            d[i] = t - i >= 0 ? ld_relaxed_ull(desc + (size_t)(t - i) * stride) : 0;
        int used = 0;
        bool stalled = false;
#pragma unroll
        for (int i = 0; i < kWindow; ++i) {
            if (done || stalled || t - i < 0) continue;
            const unsigned st = (unsigned)(d[i] >> 58) & 3u;
            if ((unsigned)(d[i] >> 60) != epoch || st == 0) { stalled = true; continue; }
            prefix += d[i] & kValMask;
            ++used;
            if (st == 2) done = true;
        }
        t -= used;
        if (t < 0) done = true;            // never reached: tile 0 publishes an inclusive prefix
        if (!done && stalled && (++spins & 7u) == 0) {
            if (*(volatile int*)err != 0) return 0;
            if (globaltimer_ns() - t0 > kSpinTimeoutNs) {
                atomicCAS(err, 0, CG_ETIMEOUT);
                return 0;
            }
        }
    }
    atomicExch(desc + (size_t)tile * stride, make_desc(epoch, 2, prefix + agg));
    return prefix;
}

// Block-wide exclusive scan of one value per thread (kBlock threads); *total = block sum.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* total) {
    __shared__ T s_w[kWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
        T s = lane < kWarps ? s_w[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kWarps) s_w[lane] = s;
    }
    __syncthreads();
    const T excl = (w ? s_w[w - 1] : T(0)) + x - v;
    *total = s_w[kWarps - 1];
    __syncthreads();
    return excl;
}

__device__ __forceinline__ uint64_t gen_candidate(const ExpandSrc& src, unsigned long long i) {
    const unsigned g = (unsigned)(i / src.F);
    return apply_gen(src.gens[g], src.frontier[i - (unsigned long long)g * src.F]);
}

// ---- expand (standalone: the step-level cg_expand and the memory hand-off) ----------------
constexpr size_t kExpandSmem = 32 << 10;

template <bool kSmem>
__global__ void expand_all_kernel(const GenSM* __restrict__ gens, int k, const uint64_t* __restrict__ in,
                                  unsigned long long F, uint64_t* __restrict__ out) {
    extern __shared__ GenSM s_gens[];
    const GenSM* g = gens;
    if (kSmem) {
        for (int j = threadIdx.x; j < k; j += blockDim.x) s_gens[j] = gens[j];
        __syncthreads();
        g = s_gens;
    }
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < F; i += stride) {
        const uint64_t s = in[i];
        for (int j = 0; j < k; ++j) out[(unsigned long long)j * F + i] = apply_gen(g[j], s);
    }
}

// ---- digit histograms of every pass in one read ------------------------------------------
template <bool kGen>
__global__ void __launch_bounds__(kBlock)
hist_all_kernel(const uint64_t* __restrict__ keys, ExpandSrc src, unsigned long long n, int passes, int lo,
                unsigned long long* __restrict__ ghist) {
    __shared__ unsigned s_h[kSortMaxPasses][kDigits];
    for (int i = threadIdx.x; i < kSortMaxPasses * kDigits; i += kBlock) (&s_h[0][0])[i] = 0;
    __syncthreads();
    const unsigned long long stride = (unsigned long long)gridDim.x * kBlock;
    for (unsigned long long i = blockIdx.x * (unsigned long long)kBlock + threadIdx.x; i < n; i += stride) {
        const uint64_t key = kGen ? gen_candidate(src, i) : keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&s_h[p][(key >> (lo + kRadixBits * p)) & (kDigits - 1)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kDigits; i += kBlock) {
        const unsigned c = (&s_h[0][0])[i];
        if (c) atomicAdd(ghist + i, (unsigned long long)c);
    }
}

// ---- one LSD pass: rank, look-back per digit, staged coalesced scatter ---------------------
// Warp w of a tile holds the tile's keys w*512 + r*32 + lane (r < kItems), so row-major order
// is input order and the ranks are stable.
template <bool kGen>
__global__ void __launch_bounds__(kBlock, 2)
onesweep_kernel(const uint64_t* __restrict__ in, ExpandSrc src, uint64_t* __restrict__ out, unsigned long long n,
                int shift, const unsigned long long* __restrict__ ghist_p, unsigned long long* desc,
                unsigned* ticket, unsigned epoch, int* err) {
    __shared__ unsigned s_whist[kWarps][kDigits];
    __shared__ unsigned s_lstart[kDigits];
    __shared__ unsigned long long s_base[kDigits];
    __shared__ uint64_t s_stage[kTile];
    __shared__ int s_tile;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) s_tile = (int)atomicAdd(ticket, 1u);
    for (int i = tid; i < kWarps * kDigits; i += kBlock) (&s_whist[0][0])[i] = 0;
    __syncthreads();
    const int tile = s_tile;
    const unsigned long long base = (unsigned long long)tile * kTile;
    uint64_t key[kItems];
    unsigned rank[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const unsigned long long idx = base + (unsigned)(wid * (kItems * 32) + r * 32 + lane);
        key[r] = idx < n ? (kGen ? gen_candidate(src, idx) : in[idx]) : 0;
    }
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const unsigned long long idx = base + (unsigned)(wid * (kItems * 32) + r * 32 + lane);
        const unsigned d = idx < n ? (unsigned)(key[r] >> shift) & (kDigits - 1) : (unsigned)kDigits;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned lt = __popc(peers & lanemask_lt());
        const unsigned run = d < (unsigned)kDigits ? s_whist[wid][d] : 0u;
        rank[r] = run + lt;
        __syncwarp();
        if (d < (unsigned)kDigits && lt == 0) s_whist[wid][d] = run + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // thread d: the tile's count of digit d, exclusive over warps in place
    unsigned cnt = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const unsigned c = s_whist[w][tid];
        s_whist[w][tid] = cnt;
        cnt += c;
    }
    unsigned tile_total = 0;
    s_lstart[tid] = block_excl_scan<unsigned>(cnt, &tile_total);
    unsigned long long all = 0;
    const unsigned long long goff = block_excl_scan<unsigned long long>(ghist_p[tid], &all);
    s_base[tid] = goff + look_back(desc + tid, kDigits, tile, cnt, epoch, err);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const unsigned long long idx = base + (unsigned)(wid * (kItems * 32) + r * 32 + lane);
        if (idx < n) {
            const unsigned d = (unsigned)(key[r] >> shift) & (kDigits - 1);
            s_stage[s_lstart[d] + s_whist[wid][d] + rank[r]] = key[r];
        }
    }
    __syncthreads();
    const unsigned tile_n = (unsigned)(n - base < (unsigned long long)kTile ? n - base : (unsigned long long)kTile);
    for (unsigned i = tid; i < tile_n; i += kBlock) {
        const uint64_t k = s_stage[i];
        const unsigned d = (unsigned)(k >> shift) & (kDigits - 1);
        const unsigned long long pos = s_base[d] + (i - s_lstart[d]);
        if (pos < n) out[pos] = k;            // always, unless a look-back gave up (error word set)
    }
}

// ---- first of run, set difference and compaction in one pass -------------------------------
// Lower bound of key in b[j, nb), galloping from j (the keys a thread asks for ascend).
__device__ __forceinline__ unsigned long long gallop(const uint64_t* __restrict__ b, unsigned long long nb,
                                                     unsigned long long j, uint64_t key) {
    if (j >= nb || b[j] >= key) return j;
    unsigned long long lo = j, step = 1;        // b[lo] < key
    while (lo + step < nb && b[lo + step] < key) {
        lo += step;
        step <<= 1;
    }
    unsigned long long hi = lo + step < nb ? lo + step : nb;   // b[hi] >= key or hi = nb
    while (hi - lo > 1) {
        const unsigned long long mid = lo + ((hi - lo) >> 1);
        if (b[mid] < key) lo = mid; else hi = mid;
    }
    return hi;
}

// First index j of sorted b[0, nb) with b[j] >= key (nb if none), found by one warp: each step
// probes 32 evenly spaced positions of the remaining interval at once (one round trip) and keeps
// the part between the last probe below key and the first one at or above it.
__device__ unsigned long long warp_lower_bound(const uint64_t* __restrict__ b, unsigned long long nb, uint64_t key,
                                               int lane) {
    unsigned long long lo = 0, hi = nb;         // the answer lies in [lo, hi]
    while (hi - lo > 32) {
        const unsigned long long span = hi - lo;
        const unsigned long long p = lo + span * (unsigned long long)(lane + 1) / 33;   // in [lo, hi)
        const int c = __popc(__ballot_sync(0xffffffffu, b[p] < key));                  // lanes 0..c-1
        const unsigned long long nlo = c ? lo + span * (unsigned long long)c / 33 + 1 : lo;
        const unsigned long long nhi = c < 32 ? lo + span * (unsigned long long)(c + 1) / 33 : hi;
        lo = nlo;
        hi = nhi;
    }
    const unsigned long long p = lo + (unsigned)lane;
    return lo + __popc(__ballot_sync(0xffffffffu, p < hi && b[p] < key));
}

// Lower bound of key in the shared-memory slice s[j, ns), galloping from j.
__device__ __forceinline__ unsigned gallop_smem(const uint64_t* s, unsigned ns, unsigned j, uint64_t key) {
    if (j >= ns || s[j] >= key) return j;
    unsigned lo = j, step = 1;
    while (lo + step < ns && s[lo + step] < key) {
        lo += step;
        step <<= 1;
    }
    unsigned hi = lo + step < ns ? lo + step : ns;
    while (hi - lo > 1) {
        const unsigned mid = lo + ((hi - lo) >> 1);
        if (s[mid] < key) lo = mid; else hi = mid;
    }
    return hi;
}

// The keys of b0 and b1 that can match a tile's keys (those within the tile's first and last
// key) are staged in shared memory when there are at most kSlice of them; each thread then walks
// the staged slices instead of L2.  A slice larger than that falls back to the global walk.
constexpr int kSlice = 2048;

__global__ void __launch_bounds__(kBlock)
unique_diff_kernel(const uint64_t* __restrict__ a, unsigned long long na, const uint64_t* __restrict__ b0,
                   unsigned long long nb0, const uint64_t* __restrict__ b1, unsigned long long nb1,
                   int first_of_run, uint64_t* __restrict__ out, unsigned long long* d_count,
                   unsigned long long* desc, unsigned* ticket, int ntiles, unsigned epoch, int* err) {
    // the staged slices are done with before the survivors are staged for the output
    __shared__ union {
        uint64_t stage[kTile];
        uint64_t slice[2][kSlice];
    } s_m;
    __shared__ int s_tile;
    __shared__ unsigned long long s_prefix;
    __shared__ unsigned long long s_j[2][2], s_lo[2], s_n[2];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) s_tile = (int)atomicAdd(ticket, 1u);
    __syncthreads();
    const int tile = s_tile;
    const unsigned long long t0 = (unsigned long long)tile * kTile;
    const unsigned long long t1 = t0 + kTile < na ? t0 + kTile : na;
    // warps 0-3, in parallel: the slice of b0 (warps 0, 1) and b1 (warps 2, 3) holding the keys
    // in [a[t0], a[t1 - 1]]: its first index (lower bound of a[t0]) and its end (lower bound of
    // a[t1 - 1] + 1)
    if (wid < 4) {
        const int q = wid >> 1, end = wid & 1;
        const uint64_t* b = q ? b1 : b0;
        const unsigned long long nb = q ? nb1 : nb0;
        const uint64_t key = end ? a[t1 - 1] : a[t0];
        const unsigned long long j = (end && key == ~0ull) ? nb : warp_lower_bound(b, nb, key + (end ? 1 : 0), lane);
        if (lane == 0) s_j[q][end] = j;
    }
    __syncthreads();
    if (tid < 2) {
        s_lo[tid] = s_j[tid][0];
        s_n[tid] = s_j[tid][1] - s_j[tid][0];
    }
    __syncthreads();
    bool staged[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        staged[q] = s_n[q] <= (unsigned long long)kSlice;
        if (staged[q]) {
            const uint64_t* b = q ? b1 : b0;
            for (unsigned i = tid; i < (unsigned)s_n[q]; i += kBlock) s_m.slice[q][i] = b[s_lo[q] + i];
        }
    }
    __syncthreads();
    const unsigned long long p0 = t0 + (unsigned long long)tid * kItems;
    uint64_t key[kItems];
    unsigned keep = 0, cnt = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) key[i] = p0 + i < na ? a[p0 + i] : 0;
    uint64_t prev = (p0 > 0 && p0 - 1 < na) ? a[p0 - 1] : 0;
    bool has_prev = p0 > 0;
    unsigned long long j0 = 0, j1 = 0;         // global walks (slices too large)
    unsigned k0 = 0, k1 = 0;                   // walks in the staged slices
    if (p0 < na) {
        if (!staged[0]) j0 = gallop(b0, nb0, s_lo[0], key[0]);
        if (!staged[1]) j1 = gallop(b1, nb1, s_lo[1], key[0]);
    }
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        if (p0 + i >= na) break;
        bool k = !(first_of_run && has_prev && prev == key[i]);
        if (staged[0]) {
            k0 = gallop_smem(s_m.slice[0], (unsigned)s_n[0], k0, key[i]);
            if (k0 < (unsigned)s_n[0] && s_m.slice[0][k0] == key[i]) k = false;
        } else {
            j0 = gallop(b0, nb0, j0, key[i]);
            if (j0 < nb0 && b0[j0] == key[i]) k = false;
        }
        if (staged[1]) {
            k1 = gallop_smem(s_m.slice[1], (unsigned)s_n[1], k1, key[i]);
            if (k1 < (unsigned)s_n[1] && s_m.slice[1][k1] == key[i]) k = false;
        } else {
            j1 = gallop(b1, nb1, j1, key[i]);
            if (j1 < nb1 && b1[j1] == key[i]) k = false;
        }
        keep |= (unsigned)k << i;
        cnt += k;
        prev = key[i];
        has_prev = true;
    }
    unsigned total = 0;
    const unsigned excl = block_excl_scan<unsigned>(cnt, &total);   // ends with __syncthreads
    if (tid == 0) {
        s_prefix = look_back(desc, 1, tile, total, epoch, err);
        if (tile == ntiles - 1 && *(volatile int*)err == 0) *d_count = s_prefix + total;
    }
    unsigned pos = excl;
#pragma unroll
    for (int i = 0; i < kItems; ++i)
        if (keep >> i & 1u) s_m.stage[pos++] = key[i];
    __syncthreads();
    const unsigned long long o = s_prefix;
    for (unsigned i = tid; i < total; i += kBlock)
        if (o + i < na) out[o + i] = s_m.stage[i];
}

// ---- key-range chunks of a layer's candidates -----------------------------------------------
// Append the candidates whose top digit (bits [shift, shift + 8)) lies in [d0, d1) to out, in
// no particular order (one atomic per warp and step); *count must start at 0.
__global__ void __launch_bounds__(kBlock)
expand_filter_kernel(ExpandSrc src, int shift, unsigned d0, unsigned d1, uint64_t* __restrict__ out,
                     unsigned long long cap, unsigned long long* count, int* err) {
    const unsigned long long n = src.F * (unsigned long long)src.k;
    const int lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)gridDim.x * kBlock;
    for (unsigned long long w = blockIdx.x * (unsigned long long)kBlock + (threadIdx.x & ~31u); w < n; w += stride) {
        const unsigned long long i = w + lane;
        uint64_t t = 0;
        bool in = false;
        if (i < n) {
            t = gen_candidate(src, i);
            const unsigned d = (unsigned)(t >> shift) & (kDigits - 1);
            in = d >= d0 && d < d1;
        }
        const unsigned m = __ballot_sync(0xffffffffu, in);
        if (!m) continue;
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(count, (unsigned long long)__popc(m));
        b = __shfl_sync(0xffffffffu, b, 0);
        if (in) {
            const unsigned long long pos = b + __popc(m & lanemask_lt());
            if (pos < cap) out[pos] = t;
            else atomicExch(err, CG_EDEVICE);
        }
    }
}

__global__ void mask_keys_kernel(uint64_t* keys, unsigned long long n, uint64_t mask) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x)
        keys[i] &= mask;
}

// ---- small layer steps in one block ----------------------------------------------------------
constexpr int kSmallBlock = 1024;
constexpr int kSmallPer = kSmallStep / kSmallBlock;     // candidates per thread

__device__ __forceinline__ unsigned small_lower_bound(const uint64_t* s, unsigned n, uint64_t key) {
    unsigned lo = 0, hi = n;
    while (lo < hi) {
        const unsigned mid = (lo + hi) >> 1;
        if (s[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// One block; dynamic shared memory: candidates | L_r | L_{r-1}, kSmallStep keys each.
__global__ void __launch_bounds__(kSmallBlock)
small_steps_kernel(const GenSM* __restrict__ gens, int k, uint64_t* L0, uint64_t* L1, uint64_t* L2,
                   int max_radius, unsigned long long stop_above, int layers_done, SmallSteps* S) {
    extern __shared__ uint64_t s_small[];
    uint64_t* A = s_small;
    uint64_t* Lc = s_small + kSmallStep;
    uint64_t* Lp = s_small + 2 * kSmallStep;
    __shared__ unsigned s_w[kSmallBlock / 32];
    uint64_t* L[3] = {L0, L1, L2};
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int cur = S->cur, prev = S->prev, radius = S->radius, nsteps = 0, status = kRunning;
    unsigned long long Fcur = S->Fcur, Fprev = S->Fprev;
    for (;;) {
        // the host loop's tests, in its order
        if (max_radius >= 0 && radius >= max_radius) { status = kTruncRadius; break; }
        const unsigned long long C = (unsigned long long)k * Fcur;
        if (C > (unsigned long long)kSmallStep || Fprev > (unsigned long long)kSmallStep || C == 0 ||
            nsteps >= kSmallMaxSteps)
            break;
        const int nxt = 3 - cur - prev;
        const unsigned nc = (unsigned)C, fc = (unsigned)Fcur, fp = (unsigned)Fprev;
        unsigned P = 1;
        while (P < nc) P <<= 1;
        for (unsigned i = tid; i < fc; i += kSmallBlock) Lc[i] = L[cur][i];
        for (unsigned i = tid; i < fp; i += kSmallBlock) Lp[i] = L[prev][i];
        __syncthreads();
        // candidate i: generator i / F on state i mod F; padding sorts last
        for (unsigned i = tid; i < P; i += kSmallBlock) {
            if (i < nc) {
                const unsigned g = i / fc;
                A[i] = apply_gen(gens[g], Lc[i - g * fc]);
            } else {
                A[i] = ~0ull;
            }
        }
        __syncthreads();
        // bitonic sort of A[0, P)
        for (unsigned kk = 2; kk <= P; kk <<= 1) {
            for (unsigned j = kk >> 1; j > 0; j >>= 1) {
                for (unsigned i = tid; i < P; i += kSmallBlock) {
                    const unsigned p = i ^ j;
                    if (p > i) {
                        const uint64_t a = A[i], b = A[p];
                        if ((a > b) == ((i & kk) == 0)) {
                            A[i] = b;
                            A[p] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
        // thread t: candidates [t kSmallPer, (t + 1) kSmallPer): first of run, not in L_r, L_{r-1}
        unsigned keep = 0, cnt = 0;
#pragma unroll
        for (int q = 0; q < kSmallPer; ++q) {
            const unsigned i = (unsigned)tid * kSmallPer + q;
            if (i < nc) {
                const uint64_t key = A[i];
                bool kp = i == 0 || A[i - 1] != key;
                if (kp) {
                    const unsigned a = small_lower_bound(Lc, fc, key);
                    if (a < fc && Lc[a] == key) kp = false;
                }
                if (kp) {
                    const unsigned b = small_lower_bound(Lp, fp, key);
                    if (b < fp && Lp[b] == key) kp = false;
                }
                keep |= (unsigned)kp << q;
                cnt += kp;
            }
        }
        // exclusive scan of the counts over threads (thread order = candidate order)
        unsigned x = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[wid] = x;
        __syncthreads();
        if (wid == 0) {
            unsigned v = lane < kSmallBlock / 32 ? s_w[lane] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            if (lane < kSmallBlock / 32) s_w[lane] = v;
        }
        __syncthreads();
        unsigned pos = (wid ? s_w[wid - 1] : 0u) + x - cnt;
        const unsigned Fn = s_w[kSmallBlock / 32 - 1];
#pragma unroll
        for (int q = 0; q < kSmallPer; ++q)
            if (keep >> q & 1u) L[nxt][pos++] = A[(unsigned)tid * kSmallPer + q];
        __syncthreads();                        // A, Lc, Lp and s_w are reused by the next step
        if (Fn == 0) { status = kDone; break; }
        if (tid == 0) S->sizes[nsteps] = Fn;
        ++nsteps;
        ++radius;
        prev = cur;
        cur = nxt;
        Fprev = Fcur;
        Fcur = Fn;
        if (stop_above > 0 && Fn > stop_above) { status = kTruncAbove; break; }
        if (layers_done + nsteps >= kMaxLayers) { status = kTruncRadius; break; }
        // the new layer is read back by every thread next step: its writes must be visible
        __threadfence_block();
        __syncthreads();
    }
    if (tid == 0) {
        S->cur = cur;
        S->prev = prev;
        S->radius = radius;
        S->status = status;
        S->Fcur = Fcur;
        S->Fprev = Fprev;
        S->nsteps = nsteps;
    }
}

int tiles_of(unsigned long long n) { return (int)((n + kTile - 1) / kTile); }

int passes_of(int bits) { return (bits + kRadixBits - 1) / kRadixBits; }

size_t al(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// ---- host-side launchers ---------------------------------------------------------------------------

// Layout: keys_tmp | error word (256 B) | digit histograms | tickets (256 B) | descriptors.
// A sort clears histograms, tickets and descriptors with one memset (never the error word,
// which the caller clears once per operation and reads at its end).
size_t sort_scratch_bytes(unsigned long long n) {
    const unsigned long long nt = (unsigned long long)tiles_of(n ? n : 1);
    return al(n * 8) + 256 + al(sizeof(unsigned long long) * kSortMaxPasses * kDigits) + 256 +
           al(nt * kDigits * 8);
}

SortScratch carve_sort_scratch(void* scratch, unsigned long long n) {
    SortScratch s{};
    char* p = static_cast<char*>(scratch);
    const unsigned long long nt = (unsigned long long)tiles_of(n ? n : 1);
    s.keys_tmp = reinterpret_cast<uint64_t*>(p);
    p += al(n * 8);
    s.err = reinterpret_cast<int*>(p);
    p += 256;
    s.ghist = reinterpret_cast<unsigned long long*>(p);
    p += al(sizeof(unsigned long long) * kSortMaxPasses * kDigits);
    s.ctl = reinterpret_cast<unsigned*>(p);           // tile tickets: [p] pass p, [15] compaction
    p += 256;
    s.desc = reinterpret_cast<unsigned long long*>(p);
    s.n = n;
    s.reset_bytes = al(sizeof(unsigned long long) * kSortMaxPasses * kDigits) + 256 + al(nt * kDigits * 8);
    return s;
}

cudaError_t launch_expand_all(const GenSM* d_gens, int k, const uint64_t* in, unsigned long long F,
                              uint64_t* out, cudaStream_t st) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    if (F == 0) return cudaSuccess;
    unsigned long long blocks = (F + kBlock - 1) / kBlock;
    if (blocks > 152ull * 16) blocks = 152ull * 16;
    const size_t smem = sizeof(GenSM) * (size_t)k;
    if (smem <= kExpandSmem)
        expand_all_kernel<true><<<(unsigned)blocks, kBlock, smem, st>>>(d_gens, k, in, F, out);
    else
        expand_all_kernel<false><<<(unsigned)blocks, kBlock, 0, st>>>(d_gens, k, in, F, out);
    return cudaGetLastError();
}

namespace {

// The passes of one sort, over key bits [lo, bits).  Input: `in` keys, or the candidates of src
// (gen).  Pass p writes bufs[(P - 1 - p) & 1], so the last pass writes bufs[0].  The error word
// and the descriptors are cleared first (one memset); the caller zeroes nothing.
cudaError_t radix_passes(const uint64_t* in, const ExpandSrc* src, unsigned long long n, int bits, int lo,
                         uint64_t* const bufs[2], const SortScratch& s, cudaStream_t st) {
    const int P = passes_of(bits - lo < 1 ? 1 : bits - lo);
    const int nt = tiles_of(n);
    const size_t reset = al(sizeof(unsigned long long) * kSortMaxPasses * kDigits) + 256 + al((size_t)nt * kDigits * 8);
    cudaError_t e = cudaMemsetAsync(s.ghist, 0, reset, st);
    if (e != cudaSuccess) return e;
    const ExpandSrc none{};
    unsigned long long hb = (n + kBlock - 1) / kBlock;
    if (hb > 152ull * 4) hb = 152ull * 4;
    if (src) hist_all_kernel<true><<<(unsigned)hb, kBlock, 0, st>>>(nullptr, *src, n, P, lo, s.ghist);
    else hist_all_kernel<false><<<(unsigned)hb, kBlock, 0, st>>>(in, none, n, P, lo, s.ghist);
    const uint64_t* cur = in;
    for (int p = 0; p < P; ++p) {
        uint64_t* dst = bufs[(P - 1 - p) & 1];
        if (p == 0 && src)
            onesweep_kernel<true><<<nt, kBlock, 0, st>>>(nullptr, *src, dst, n, lo + kRadixBits * p,
                                                         s.ghist + p * kDigits, s.desc, s.ctl + p,
                                                         (unsigned)(p + 1), s.err);
        else
            onesweep_kernel<false><<<nt, kBlock, 0, st>>>(cur, none, dst, n, lo + kRadixBits * p,
                                                          s.ghist + p * kDigits, s.desc, s.ctl + p,
                                                          (unsigned)(p + 1), s.err);
        cur = dst;
    }
    return cudaGetLastError();
}

}  // namespace

// Sort keys[0, n) ascending on their bits [lo, bits) (higher bits must be zero; lower bits
// decided by the others), in place; an odd number of 8-bit passes ends with one copy back.
cudaError_t launch_radix_sort(uint64_t* keys, unsigned long long n, int bits, const SortScratch& s,
                              cudaStream_t st, int lo) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    if (n <= 1) return cudaSuccess;
    const int P = passes_of(bits - lo < 1 ? 1 : bits - lo);
    uint64_t* bufs[2];
    if (P % 2 == 0) { bufs[0] = keys; bufs[1] = s.keys_tmp; }
    else { bufs[0] = s.keys_tmp; bufs[1] = keys; }
    cudaError_t e = radix_passes(keys, nullptr, n, bits, lo, bufs, s, st);
    if (e == cudaSuccess && P % 2 == 1)
        e = cudaMemcpyAsync(keys, s.keys_tmp, n * 8, cudaMemcpyDeviceToDevice, st);
    return e;
}

cudaError_t launch_expand_sort(const ExpandSrc& src, uint64_t* out, int bits, const SortScratch& s,
                               cudaStream_t st, int lo) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    const unsigned long long n = src.F * (unsigned long long)src.k;
    if (n == 0) return cudaSuccess;
    uint64_t* bufs[2] = {out, s.keys_tmp};
    return radix_passes(nullptr, &src, n, bits, lo, bufs, s, st);
}

// out = keys of sorted a that are first of their run and absent from every sorted b_j,
// compacted in order; *d_count = their number.
cudaError_t launch_unique_difference(const uint64_t* a, unsigned long long na, const uint64_t* const* bs,
                                     const unsigned long long* nbs, int nb_sets, uint64_t* out,
                                     unsigned long long* d_count, const SortScratch& s, cudaStream_t st) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    if (na == 0) return cudaMemsetAsync(d_count, 0, 8, st);
    const int nt = tiles_of(na);
    // its own ticket and descriptors (epoch 15): clear the tickets and one descriptor per tile
    cudaError_t e = cudaMemsetAsync(s.ctl, 0, 256 + al((size_t)nt * 8), st);
    if (e != cudaSuccess) return e;
    const uint64_t* b0 = nb_sets > 0 ? bs[0] : a;
    const uint64_t* b1 = nb_sets > 1 ? bs[1] : a;
    const unsigned long long n0 = nb_sets > 0 ? nbs[0] : 0, n1 = nb_sets > 1 ? nbs[1] : 0;
    unique_diff_kernel<<<nt, kBlock, 0, st>>>(a, na, b0, n0, b1, n1, 1, out, d_count, s.desc, s.ctl + 15,
                                              nt, 15u, s.err);
    return cudaGetLastError();
}

cudaError_t launch_candidate_hist(const ExpandSrc& src, int bits, const SortScratch& s, cudaStream_t st,
                                  int lo) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    const unsigned long long n = src.F * (unsigned long long)src.k;
    cudaError_t e = cudaMemsetAsync(s.ghist, 0, sizeof(unsigned long long) * kSortMaxPasses * kDigits, st);
    if (e != cudaSuccess || n == 0) return e;
    unsigned long long hb = (n + kBlock - 1) / kBlock;
    if (hb > 152ull * 4) hb = 152ull * 4;
    hist_all_kernel<true><<<(unsigned)hb, kBlock, 0, st>>>(nullptr, src, n, passes_of(bits - lo < 1 ? 1 : bits - lo),
                                                          lo, s.ghist);
    return cudaGetLastError();
}

cudaError_t launch_expand_filter(const ExpandSrc& src, int shift, unsigned d0, unsigned d1, uint64_t* out,
                                 unsigned long long cap, unsigned long long* d_count, int* d_err,
                                 cudaStream_t st) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    cudaError_t e = cudaMemsetAsync(d_count, 0, 8, st);
    if (e != cudaSuccess || src.F == 0) return e;
    expand_filter_kernel<<<152 * 8, kBlock, 0, st>>>(src, shift, d0, d1, out, cap, d_count, d_err);
    return cudaGetLastError();
}

cudaError_t launch_mask_keys(uint64_t* keys, unsigned long long n, uint64_t mask, cudaStream_t st) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    if (n == 0) return cudaSuccess;
    unsigned long long blocks = (n + 255) / 256;
    if (blocks > 152ull * 8) blocks = 152ull * 8;
    mask_keys_kernel<<<(unsigned)blocks, 256, 0, st>>>(keys, n, mask);
    return cudaGetLastError();
}

int sort_passes(int bits, int lo) { return passes_of(bits - lo < 1 ? 1 : bits - lo); }

cudaError_t launch_small_steps(const GenSM* d_gens, int k, uint64_t* L0, uint64_t* L1, uint64_t* L2,
                               int max_radius, unsigned long long stop_above, int layers_done,
                               SmallSteps* d_state, cudaStream_t st) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    const size_t smem = 3 * (size_t)kSmallStep * sizeof(uint64_t);
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 64 && !attr_set[dev]) {
        e = cudaFuncSetAttribute(small_steps_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    small_steps_kernel<<<1, kSmallBlock, smem, st>>>(d_gens, k, L0, L1, L2, max_radius, stop_above, layers_done,
                                                      d_state);
    return cudaGetLastError();
}

}  // namespace cg
