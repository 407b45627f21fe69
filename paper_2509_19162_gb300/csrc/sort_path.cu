// Sort strategy of the growth library: sorted layers, radix sort + unique of the candidates,
// merge-path set difference against the two previous layers, compaction.
//
// For an inverse-closed generating set every neighbour of layer r lies in layer r-1, r or r+1,
// so layer r+1 = unique(candidates) \ (L_r U L_{r-1}) needs only the two previous layers
// (Section 3.4: undirected graphs are those with inverse-closed generators).  Layers are kept
// as arrays of packed keys sorted ascending.  Per layer step:
//   expand        candidates = every generator applied to every state of L_r
//   radix sort    LSD, 8-bit digits over the w n significant key bits (w = 4 bits per element
//                 for permutations, 1 or 2 for narrow coset vectors); per pass: per-tile digit
//                 histograms, one device-wide scan (decoupled look-back), stable scatter with
//                 warp match_any ranking
//   unique + diff one merge-path kernel per previous layer flags the candidates that are the
//                 first of their run and absent from that layer
//   compaction    single-pass decoupled look-back over tiles; the flagged keys, in order, are
//                 layer r+1 (still sorted) and their number is |L_{r+1}|
// The same primitives back the step-level entry points cg_sort_unique and cg_set_difference.
#include <cstdint>

#include "cg_device.cuh"
#include "sort_kernels.h"

namespace cg {

namespace {

constexpr int kBlock = 256;
constexpr int kItems = 16;                       // keys per thread per tile
constexpr int kTile = kBlock * kItems;           // 4096 keys per tile
constexpr int kRadixBits = 8;
constexpr int kDigits = 1 << kRadixBits;
constexpr uint64_t kSpinTimeoutNs = 5ull * 1000 * 1000 * 1000;

// ---- decoupled look-back ---------------------------------------------------------------------
// Tile descriptor: bits 62-63 = status (0 none, 1 aggregate, 2 inclusive prefix), bits 0-61 =
// value.  Tiles take tickets in start order, so every predecessor a tile waits on is running.
constexpr unsigned long long kStatusShift = 62;
constexpr unsigned long long kValueMask = (1ull << 62) - 1;

__device__ __forceinline__ void publish(unsigned long long* desc, int tile, unsigned long long status,
                                        unsigned long long value) {
    __threadfence();
    atomicExch(desc + tile, (status << kStatusShift) | (value & kValueMask));
}

// Exclusive prefix of `aggregate` over tiles [0, tile); called by one thread.  Returns false
// (and sets *err) if a predecessor never published within the time limit.
__device__ bool look_back(unsigned long long* desc, int tile, unsigned long long aggregate,
                          unsigned long long* prefix_out, int* err) {
    if (tile == 0) {
        publish(desc, 0, 2, aggregate);
        *prefix_out = 0;
        return true;
    }
    publish(desc, tile, 1, aggregate);
    unsigned long long prefix = 0;
    int t = tile - 1;
    const uint64_t t0 = globaltimer_ns();
    while (t >= 0) {
        const unsigned long long d = ld_relaxed_ull(desc + t);
        const unsigned long long st = d >> kStatusShift;
        if (st == 0) {
            if (globaltimer_ns() - t0 > kSpinTimeoutNs) {
                atomicCAS(err, 0, CG_ETIMEOUT);
                return false;
            }
            if (*(volatile int*)err != 0) return false;
            __nanosleep(64);
            continue;
        }
        prefix += d & kValueMask;
        if (st == 2) break;
        --t;
    }
    __threadfence();
    publish(desc, tile, 2, prefix + aggregate);
    *prefix_out = prefix;
    return true;
}

// Block-wide exclusive scan of one value per thread (kBlock threads).  Returns the exclusive
// prefix; *total receives the block sum.
__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned* total) {
    __shared__ unsigned s_w[kBlock / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned s = lane < kBlock / 32 ? s_w[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kBlock / 32) s_w[lane] = s;
    }
    __syncthreads();
    const unsigned excl = (w ? s_w[w - 1] : 0) + x - v;
    *total = s_w[kBlock / 32 - 1];
    __syncthreads();
    return excl;
}

// ---- expand ------------------------------------------------------------------------------------
// out[j*F + i] = gens[j](in[i]).  The generators are staged in shared memory when they fit in
// kExpandSmem bytes, else read through L1.
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

// ---- radix sort --------------------------------------------------------------------------------
// Digit histogram of each tile, stored digit-major: hist[d * ntiles + tile].
__global__ void __launch_bounds__(kBlock)
radix_hist_kernel(const uint64_t* __restrict__ keys, unsigned long long n, int shift,
                  unsigned* __restrict__ hist, int ntiles) {
    __shared__ unsigned s_h[kDigits];
    for (int d = threadIdx.x; d < kDigits; d += kBlock) s_h[d] = 0;
    __syncthreads();
    const unsigned long long base = (unsigned long long)blockIdx.x * kTile;
#pragma unroll 4
    for (int i = 0; i < kItems; ++i) {
        const unsigned long long e = base + (unsigned long long)i * kBlock + threadIdx.x;
        if (e < n) atomicAdd(&s_h[(keys[e] >> shift) & (kDigits - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kDigits; d += kBlock) hist[(size_t)d * ntiles + blockIdx.x] = s_h[d];
}

// Exclusive scan in place of a u32 array of length n (< 2^32 total), tiles of kTile entries,
// decoupled look-back.  desc must be zeroed (one entry per tile); ticket zeroed.
__global__ void __launch_bounds__(kBlock)
scan_u32_kernel(unsigned* data, unsigned long long n, unsigned long long* desc, unsigned* ticket,
                int* err) {
    __shared__ int s_tile;
    __shared__ unsigned long long s_prefix;
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(ticket, 1u);
    __syncthreads();
    const int tile = s_tile;
    const unsigned long long base = (unsigned long long)tile * kTile + (unsigned long long)threadIdx.x * kItems;
    unsigned v[kItems];
    unsigned sum = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        v[i] = (base + i < n) ? data[base + i] : 0u;
        sum += v[i];
    }
    unsigned total = 0;
    const unsigned excl = block_exclusive_scan(sum, &total);
    if (threadIdx.x == 0) {
        unsigned long long p = 0;
        if (!look_back(desc, tile, total, &p, err)) p = 0;
        s_prefix = p;
    }
    __syncthreads();
    unsigned run = (unsigned)s_prefix + excl;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        if (base + i < n) data[base + i] = run;
        run += v[i];
    }
}

// Stable scatter of one LSD pass.  Keys are taken in tile order (round r covers keys
// [tile*kTile + r*kBlock, +kBlock), lane order within a warp); a key's rank within its tile and
// digit is the count of equal digits before it in that order, so equal digits keep their
// relative order (the pass is stable).
__global__ void __launch_bounds__(kBlock)
radix_scatter_kernel(const uint64_t* __restrict__ in, uint64_t* __restrict__ out, unsigned long long n,
                     int shift, const unsigned* __restrict__ offsets, int ntiles) {
    __shared__ unsigned s_run[kDigits];              // running count per digit within the tile
    __shared__ unsigned s_warp[kBlock / 32][kDigits];
    const int w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kDigits; d += kBlock) s_run[d] = 0;
    const unsigned long long base = (unsigned long long)blockIdx.x * kTile;
    for (int r = 0; r < kItems; ++r) {
        for (int i = threadIdx.x; i < (kBlock / 32) * kDigits; i += kBlock) (&s_warp[0][0])[i] = 0;
        __syncthreads();
        const unsigned long long e = base + (unsigned long long)r * kBlock + threadIdx.x;
        const bool valid = e < n;
        const uint64_t key = valid ? in[e] : 0;
        const unsigned d = valid ? (unsigned)((key >> shift) & (kDigits - 1)) : (unsigned)kDigits;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned lane_rank = __popc(peers & lanemask_lt());
        if (valid && lane_rank == 0) s_warp[w][d] = __popc(peers);
        __syncthreads();
        // per digit: exclusive prefix over warps, continued from earlier rounds
        for (int dd = threadIdx.x; dd < kDigits; dd += kBlock) {
            unsigned run = s_run[dd];
#pragma unroll
            for (int ww = 0; ww < kBlock / 32; ++ww) {
                const unsigned c = s_warp[ww][dd];
                s_warp[ww][dd] = run;
                run += c;
            }
            s_run[dd] = run;
        }
        __syncthreads();
        if (valid) {
            const unsigned pos = offsets[(size_t)d * ntiles + blockIdx.x] + s_warp[w][d] + lane_rank;
            if (pos < n) out[pos] = key;   // always true unless the offset scan failed (error word set)
        }
        __syncthreads();
    }
}

// ---- unique + merge-path set difference ------------------------------------------------------
// Number of elements of a among the first `diag` elements of the merge of a and b, where an
// element of a goes before an equal element of b.
__device__ __forceinline__ unsigned long long merge_path(const uint64_t* a, unsigned long long na,
                                                         const uint64_t* b, unsigned long long nb,
                                                         unsigned long long diag) {
    unsigned long long lo = diag > nb ? diag - nb : 0;
    unsigned long long hi = diag < na ? diag : na;
    while (lo < hi) {
        const unsigned long long mid = (lo + hi) >> 1;   // candidate count of a-elements
        // a[mid] goes before b[diag - mid - 1] iff a[mid] <= b[diag - mid - 1]
        if (a[mid] <= b[diag - mid - 1]) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// flags[i] &= (a[i] is absent from b) [and, if first_of_run, a[i] != a[i-1]].  a sorted
// (duplicates allowed), b sorted.  Each thread walks kItems steps of the merge of a and b.
__global__ void __launch_bounds__(kBlock)
setdiff_flags_kernel(const uint64_t* __restrict__ a, unsigned long long na, const uint64_t* __restrict__ b,
                     unsigned long long nb, unsigned char* __restrict__ flags, int first_of_run, int init) {
    const unsigned long long total = na + nb;
    const unsigned long long diag = ((unsigned long long)blockIdx.x * kBlock + threadIdx.x) * kItems;
    if (diag >= total) return;
    unsigned long long ai = merge_path(a, na, b, nb, diag);
    unsigned long long bi = diag - ai;
    const unsigned long long end = diag + kItems < total ? diag + kItems : total;
    for (unsigned long long step = diag; step < end; ++step) {
        if (ai < na && (bi >= nb || a[ai] <= b[bi])) {
            const uint64_t x = a[ai];
            bool keep = !(bi < nb && b[bi] == x);
            if (first_of_run && ai > 0 && a[ai - 1] == x) keep = false;
            if (init) flags[ai] = keep ? 1 : 0;
            else if (!keep) flags[ai] = 0;
            ++ai;
        } else {
            ++bi;
        }
    }
}

// ---- compaction ----------------------------------------------------------------------------------
// out[...] = in[i] for flags[i] != 0, in order; *count = number kept.  Single pass, decoupled
// look-back over tiles (desc zeroed, ticket zeroed).
__global__ void __launch_bounds__(kBlock)
compact_kernel(const uint64_t* __restrict__ in, const unsigned char* __restrict__ flags, unsigned long long n,
               uint64_t* __restrict__ out, unsigned long long* count, unsigned long long* desc,
               unsigned* ticket, int ntiles, int* err) {
    __shared__ int s_tile;
    __shared__ unsigned long long s_prefix;
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(ticket, 1u);
    __syncthreads();
    const int tile = s_tile;
    const unsigned long long base = (unsigned long long)tile * kTile + (unsigned long long)threadIdx.x * kItems;
    unsigned keepmask = 0, cnt = 0;
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const bool k = (base + i < n) && flags[base + i];
        keepmask |= (unsigned)k << i;
        cnt += k;
    }
    unsigned total = 0;
    const unsigned excl = block_exclusive_scan(cnt, &total);
    if (threadIdx.x == 0) {
        unsigned long long p = 0;
        if (!look_back(desc, tile, total, &p, err)) p = 0;
        s_prefix = p;
        if (tile == ntiles - 1 && *(volatile int*)err == 0) *count = p + total;
    }
    __syncthreads();
    unsigned long long pos = s_prefix + excl;
#pragma unroll
    for (int i = 0; i < kItems; ++i)
        if ((keepmask >> i & 1u) && pos < n) out[pos++] = in[base + i];
}

int tiles_of(unsigned long long n) { return (int)((n + kTile - 1) / kTile); }

}  // namespace

// ---- host-side launchers ---------------------------------------------------------------------------

size_t sort_scratch_bytes(unsigned long long n) {
    const unsigned long long nt = (unsigned long long)tiles_of(n ? n : 1);
    const unsigned long long hist = (unsigned long long)kDigits * nt;           // u32
    const unsigned long long scan_tiles = (hist + kTile - 1) / kTile + 1;
    size_t b = 0;
    b += ((n * 8 + 255) / 256) * 256;                       // ping-pong keys
    b += ((hist * 4 + 255) / 256) * 256;                    // histograms / offsets
    b += ((scan_tiles * 8 + 255) / 256) * 256;              // scan descriptors
    b += ((nt * 8 + 255) / 256) * 256;                      // compaction descriptors
    b += ((n + 255) / 256) * 256;                           // flags
    b += 256;                                               // tickets, error word
    return b;
}

SortScratch carve_sort_scratch(void* scratch, unsigned long long n) {
    SortScratch s{};
    char* p = static_cast<char*>(scratch);
    const unsigned long long nt = (unsigned long long)tiles_of(n ? n : 1);
    const unsigned long long hist = (unsigned long long)kDigits * nt;
    const unsigned long long scan_tiles = (hist + kTile - 1) / kTile + 1;
    auto take = [&](size_t bytes) { char* r = p; p += ((bytes + 255) / 256) * 256; return r; };
    s.keys_tmp = reinterpret_cast<uint64_t*>(take(n * 8));
    s.hist = reinterpret_cast<unsigned*>(take(hist * 4));
    s.scan_desc = reinterpret_cast<unsigned long long*>(take(scan_tiles * 8));
    s.compact_desc = reinterpret_cast<unsigned long long*>(take(nt * 8));
    s.flags = reinterpret_cast<unsigned char*>(take(n));
    char* small = take(256);
    s.tickets = reinterpret_cast<unsigned*>(small);            // [0] scan, [1] compaction
    s.err = reinterpret_cast<int*>(small + 64);
    s.n = n;
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

// Sort keys[0, n) ascending on their low `bits` bits (higher bits must be zero), in place; the
// number of 8-bit passes is ceil(bits / 8), an odd count ends with one extra copy.
cudaError_t launch_radix_sort(uint64_t* keys, unsigned long long n, int bits, const SortScratch& s,
                              cudaStream_t st) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    if (n <= 1) return cudaSuccess;
    const int nt = tiles_of(n);
    const unsigned long long hist_n = (unsigned long long)kDigits * nt;
    const int scan_tiles = tiles_of(hist_n);
    uint64_t* src = keys;
    uint64_t* dst = s.keys_tmp;
    const int passes = (bits + kRadixBits - 1) / kRadixBits;
    cudaError_t e = cudaSuccess;
    for (int p = 0; p < passes && e == cudaSuccess; ++p) {
        const int shift = p * kRadixBits;
        radix_hist_kernel<<<nt, kBlock, 0, st>>>(src, n, shift, s.hist, nt);
        if ((e = cudaMemsetAsync(s.scan_desc, 0, (size_t)scan_tiles * 8, st)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(s.tickets, 0, 4, st)) != cudaSuccess) break;
        scan_u32_kernel<<<scan_tiles, kBlock, 0, st>>>(s.hist, hist_n, s.scan_desc, s.tickets, s.err);
        radix_scatter_kernel<<<nt, kBlock, 0, st>>>(src, dst, n, shift, s.hist, nt);
        e = cudaGetLastError();
        uint64_t* t = src; src = dst; dst = t;
    }
    if (e == cudaSuccess && src != keys)
        e = cudaMemcpyAsync(keys, src, n * 8, cudaMemcpyDeviceToDevice, st);
    return e;
}

// flags[i] = a[i] is the first of its run and absent from every b_j; then compaction of a into
// out, count into *d_count.  a sorted; each b_j sorted.
cudaError_t launch_unique_difference(const uint64_t* a, unsigned long long na, const uint64_t* const* bs,
                                     const unsigned long long* nbs, int nb_sets, uint64_t* out,
                                     unsigned long long* d_count, const SortScratch& s, cudaStream_t st) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    if (na == 0) return cudaMemsetAsync(d_count, 0, 8, st);
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < (nb_sets > 0 ? nb_sets : 1) && e == cudaSuccess; ++j) {
        const uint64_t* b = nb_sets > 0 ? bs[j] : a;
        const unsigned long long nb = nb_sets > 0 ? nbs[j] : 0;
        const unsigned long long total = na + nb;
        const unsigned long long threads = (total + kItems - 1) / kItems;
        const unsigned blocks = (unsigned)((threads + kBlock - 1) / kBlock);
        setdiff_flags_kernel<<<blocks, kBlock, 0, st>>>(a, na, b, nb, s.flags, j == 0 ? 1 : 0,
                                                        j == 0 ? 1 : 0);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    const int nt = tiles_of(na);
    if ((e = cudaMemsetAsync(s.compact_desc, 0, (size_t)nt * 8, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(s.tickets + 1, 0, 4, st)) != cudaSuccess) return e;
    compact_kernel<<<nt, kBlock, 0, st>>>(a, s.flags, na, out, d_count, s.compact_desc, s.tickets + 1,
                                          nt, s.err);
    return cudaGetLastError();
}

}  // namespace cg
