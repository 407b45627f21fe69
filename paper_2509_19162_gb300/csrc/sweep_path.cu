// Sweep strategy of the growth library: breadth-first growth with the visited set and the
// layers held as bitmaps over S_n, the paper's bitmask BFS (Section 3.1.3: a few bits per
// element of the group instead of a list of states).  Nothing per state is stored but bits --
// the visited set and two layers, 3 bits per element of S_n -- so a growth needs 3 n!/8 bytes
// (plus about 1 % for block lists) whatever its layers hold: 33.4 GB for all of S_14.
//
// Index of a permutation: the position-major Lehmer rank
//     rank(s) = sum_{i=1}^{n-1} d_i * i!,   d_i = #{ j < i : s_j < s_i },
// a bijection S_n -> [0, n!).  A generator that moves only positions below j changes only the
// digits below j, so its image lies within j! ranks of the state: prefix reversals, adjacent
// transpositions and other short-support generators keep their visited-set accesses close to
// the block being expanded, which the L2 serves.
//
// One round (layer step) of the persistent cooperative kernel:
//   the listed blocks of layer r-1 are cleared (F and S), and after a grid barrier its buffers,
//   empty, receive layer r+1;
//   the nonempty 1024-rank blocks of layer r are expanded: their states are unranked, every
//   generator applied, the images ranked and test-and-set in V (one atomicOr each); a new state
//   sets its bit in F_{r+1}, the first bit of a block enters the block in L_{r+1} (per-warp
//   staging, one atomic per 32 entries).  Dense layers are taken in rank order (found from the
//   per-block bits), sparse ones in the order of the block list L_r;
//   grid barrier; the last block to arrive records |L_{r+1}| and the stop tests.
// Warps draw the work units from one counter.
#include <cstdio>
#include <utility>

#include "cg_device.cuh"
#include "cg_kernels.h"

namespace cg {

namespace {

constexpr int kSweepBlock = 256;
constexpr int kSweepWarps = kSweepBlock / 32;
constexpr int kSweepSmemGens = 32;
constexpr int kListStage = 64;   // staged block-list entries per warp
constexpr unsigned long long kUnitStates = 256;  // rank order: target states per work unit
constexpr unsigned long long kRankFill = 4;      // auto order: rank order from 1/4 of blocks

__host__ __device__ constexpr uint64_t fact(int i) { return i <= 1 ? 1ull : (uint64_t)i * fact(i - 1); }

// Digit weights of the two halves of the rank, as 32-bit constants: i! for positions below 12,
// i!/12! for positions 12..15.  Called with unrolled-loop constants, so every division by a
// weight below is by a compile-time constant.
__host__ __device__ constexpr unsigned weight_low(int i) { return (unsigned)fact(i); }
__host__ __device__ constexpr unsigned weight_top(int i) { return (unsigned)(fact(i) / fact(12)); }

// The rank of the bitmaps is perm_rank_n / perm_rank (cg_device.cuh), the position-major Lehmer
// rank.
template <int N>
__device__ __forceinline__ uint64_t pos_rank(uint64_t key) { return perm_rank_n<N>(key); }

// Inverse of the rank: from the top position down, position i holds the d_i-th smallest of the
// values not yet placed.  The unplaced values are kept sorted in the nibbles of `avail`.
template <int N>
__device__ __forceinline__ uint64_t pos_unrank(uint64_t r) {
    unsigned top = 0, low = (unsigned)r;
    if (N > 12) {
        top = (unsigned)(r / fact(12));
        low = (unsigned)(r - (uint64_t)top * fact(12));
    }
    uint64_t avail = 0xFEDCBA9876543210ull;
    uint64_t key = 0;
#pragma unroll
    for (int i = N - 1; i >= 1; --i) {
        unsigned d;
        if (i >= 12) {
            d = top / weight_top(i);
            top -= d * weight_top(i);
        } else {
            d = low / weight_low(i);
            low -= d * weight_low(i);
        }
        const unsigned sh = 4u * d;
        const uint64_t below = (1ull << sh) - 1ull;
        key |= ((avail >> sh) & 15ull) << (4 * i);
        avail = (avail & below) | ((avail >> 4) & ~below);
    }
    return key | (avail & 15ull);
}

// Append block index b (lanes with `want`) to the warp's staging buffer; flush to the global
// list with one atomic when it holds at least 32 entries.
__device__ __forceinline__ void list_stage(unsigned* buf, int& cnt, bool want, unsigned b,
                                           unsigned* list, unsigned long long* lcount, int lane) {
    const unsigned m = __ballot_sync(0xffffffffu, want);
    if (want) buf[cnt + __popc(m & lanemask_lt())] = b;
    cnt += __popc(m);
    __syncwarp();
    if (cnt >= kListStage - 32) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(lcount, (unsigned long long)cnt);
        base = __shfl_sync(0xffffffffu, base, 0);
        for (int i = lane; i < cnt; i += 32) list[base + i] = buf[i];
        cnt = 0;
        __syncwarp();
    }
}

__device__ __forceinline__ void list_flush(unsigned* buf, int& cnt, unsigned* list,
                                           unsigned long long* lcount, int lane) {
    if (cnt == 0) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(lcount, (unsigned long long)cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int i = lane; i < cnt; i += 32) list[base + i] = buf[i];
    cnt = 0;
    __syncwarp();
}

// Clear block blk of a layer that is no longer needed: its 32 words and its block-bit word.
__device__ __forceinline__ void clear_block(unsigned* F, unsigned* S, unsigned blk) {
    uint4* pw = reinterpret_cast<uint4*>(F + (uint64_t)blk * 32);
#pragma unroll
    for (int j = 0; j < 8; ++j) pw[j] = make_uint4(0u, 0u, 0u, 0u);
    S[blk >> 5] = 0u;
}

// Expand one state (lanes with `active`): apply every generator, test-and-set the images in V,
// record the new ones in the next layer.
template <int kILP, int kN>
__device__ __forceinline__ void sweep_state(const GenSM* gens, int k, unsigned* V, unsigned* N,
                                            unsigned* SN, unsigned* list, unsigned long long* lcount,
                                            unsigned* lbuf, int& lcnt, bool active, uint64_t rank,
                                            unsigned& fresh, int lane) {
    const uint64_t s = active ? pos_unrank<kN>(rank) : 0;
    for (int g0 = 0; g0 < k; g0 += kILP) {
        uint64_t rt[kILP];
        unsigned old[kILP];
#pragma unroll
        for (int i = 0; i < kILP; ++i)
            if (active && g0 + i < k) rt[i] = pos_rank<kN>(apply_gen<false>(gens[g0 + i], s));
#pragma unroll
        for (int i = 0; i < kILP; ++i)
            if (active && g0 + i < k) old[i] = atomicOr(V + (rt[i] >> 5), 1u << (unsigned)(rt[i] & 31u));
#pragma unroll
        for (int i = 0; i < kILP; ++i) {
            bool first_in_block = false;
            unsigned blk = 0;
            if (active && g0 + i < k) {
                const unsigned bit = 1u << (unsigned)(rt[i] & 31u);
                if (!(old[i] & bit)) {
                    ++fresh;
                    if (atomicOr(N + (rt[i] >> 5), bit) == 0u) {
                        blk = (unsigned)(rt[i] >> 10);
                        const unsigned sb = 1u << (blk & 31u);
                        first_in_block = !(atomicOr(SN + (blk >> 5), sb) & sb);
                    }
                }
            }
            if (__any_sync(0xffffffffu, first_in_block))
                list_stage(lbuf, lcnt, first_in_block, blk, list, lcount, lane);
        }
    }
}

// Close a round (one thread of the last block to arrive).
__device__ void sweep_close(SweepDev& D, Ctl* ctl) {
    volatile SweepDev& W = D;
    const int r = W.radius;
    const unsigned long long fresh = ld_relaxed_ull(&D.fresh);
    if (fresh == 0) {
        W.status = kDone;
    } else {
        const int r1 = r + 1;
        D.layer_sizes[r1] = fresh;
        W.radius = r1;
        if (D.max_radius >= 0 && r1 >= D.max_radius) W.status = kTruncRadius;
        else if (D.stop_above > 0 && fresh > D.stop_above) W.status = kTruncAbove;
        else if (r1 + 1 >= D.layers_cap) W.status = kTruncRadius;
    }
    W.fresh = 0;
    W.grab = 0;
    *(volatile int*)&ctl->rounds += 1;
    __threadfence();
}

template <int kILP, int kN>
__global__ void __launch_bounds__(kSweepBlock, 4)
sweep_grow_kernel(SweepDev* Dp, Ctl* ctl, int max_rounds, uint64_t timeout_ns, int order) {
    __shared__ unsigned short s_off[kSweepWarps][1024];
    __shared__ uint64_t s_carry[kSweepWarps][32];
    __shared__ unsigned s_list[kSweepWarps][kListStage];
    __shared__ GenSM s_gens[kSweepSmemGens];
    __shared__ unsigned long long s_fresh;
    SweepDev& D = *Dp;
    const int k = D.k;
    const GenSM* gens = D.gens;
    if (k <= kSweepSmemGens) {
        for (int j = threadIdx.x; j < k; j += blockDim.x) s_gens[j] = D.gens[j];
        gens = s_gens;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned short* off = s_off[wid];
    uint64_t* carry = s_carry[wid];
    unsigned* lbuf = s_list[wid];
    const unsigned long long nwarps = (unsigned long long)gridDim.x * kSweepWarps;

    unsigned nbar = 0;                      // grid barriers this block has passed
    for (int round = 0; round < max_rounds; ++round) {
        if (ld_relaxed_int(&D.status) != kRunning) break;
        const int r = ld_relaxed_int(&D.radius);
        // Layer r is F[r & 1]; layer r + 1 goes to the other bitmap, which still holds layer
        // r - 1 (3 bits per element of S_n: V and two layers).  That layer is cleared first --
        // its listed blocks, one per thread -- and after a grid barrier the round expands layer r.
        const int cur = r & 1, nxt = cur ^ 1;
        unsigned* F = D.F[cur];
        unsigned* N = D.F[nxt];
        unsigned* SN = D.S[nxt];
        const unsigned* Lc = D.L[cur];
        unsigned* Ln = D.L[nxt];
        unsigned long long* ln_count = &D.lcount[nxt];
        // (r > 0 decides the clearing phase for every block alike: the other list's count is
        // read before the barrier, and blocks append to it only after it)
        if (r > 0) {
            const unsigned long long nprv = ld_relaxed_ull(&D.lcount[nxt]);
            const unsigned long long nth = (unsigned long long)gridDim.x * kSweepBlock;
            for (unsigned long long e = blockIdx.x * (unsigned long long)kSweepBlock + threadIdx.x; e < nprv; e += nth)
                clear_block(N, SN, __ldcg(Ln + e));
            unsigned long long word = 0;
            const int arrive = grid_arrive(ctl, timeout_ns, word, nbar++);
            if (arrive < 0) return;
            if (arrive == 1) {
                if (threadIdx.x == 0) *(volatile unsigned long long*)ln_count = 0;   // receives layer r + 1
                grid_release(ctl, word, 0);
            }
        }
        if (threadIdx.x == 0) s_fresh = 0;
        __syncthreads();

        // Work units.  A warp fetches the 32 words of a 1024-rank block of layer r (one per
        // lane), or 32 words of several blocks, and queues the ranks of their set bits; it
        // expands them 32 at a time, carrying fewer than 32 over to the next fetch, so every
        // chunk but the warp's last fills all lanes.  The blocks come in one of two orders:
        //   rank order (layers whose nonempty blocks fill at least 1/kRankFill of S_n): units
        //       are drawn one at a time from one counter and cover S_n in rank
        //       order, 2^lc blocks each, lc chosen so that a unit holds about kUnitStates
        //       states when they are spread evenly, and the warp finds their nonempty blocks
        //       from the block bits of layer r.  The warps of the grid then work within a
        //       narrow range of ranks, near which the images of their states under
        //       short-support generators fall, so those visited-set accesses hit L2;
        //   discovery order (sparser layers, which may crowd into few ranges of S_n, and every
        //       layer when the visited bitmap fits L2 anyway): units
        //       are the 32 |L_r| words of the listed blocks of layer r, drawn in chunks of a
        //       quarter of the remaining units' share of one warp (at least 32).
        const unsigned long long ncur = ld_relaxed_ull(&D.lcount[cur]);
        const bool by_rank =
            order == kSweepOrderRank || (order == kSweepOrderAuto && ncur * kRankFill >= D.nblocks);
        const unsigned long long fsize =
            ld_relaxed_ull(reinterpret_cast<const unsigned long long*>(D.layer_sizes + r));
        const unsigned long long want = fsize ? (kUnitStates * D.nblocks) / fsize : 1024ull;
        int lc = 0;
        while (lc < 10 && (1ull << lc) < want) ++lc;
        const unsigned long long xunits = ncur * 32;
        const unsigned long long units = by_rank ? (D.nblocks + (1ull << lc) - 1) >> lc : xunits;
        const unsigned* S = D.S[cur];
        unsigned fresh = 0;
        int lcnt = 0;
        unsigned ncarry = 0, T = 0, i = 0;  // queue: [0, ncarry) in carry, [ncarry, T) in off
        uint64_t lbase = 0;                 // first rank of this lane's fetched word
        bool have = false;                  // rank order: a unit's block bits are held in sw
        unsigned sw = 0;                    //   lane l: block bits (32 blocks) of word wb + l
        unsigned long long wb = 0;
        unsigned long long ua = 0, ub = 0;  // discovery order: grabbed, not yet fetched units
        unsigned long long seen = 0;
        bool exhausted = false;
        const uint64_t t_round = globaltimer_ns();
        unsigned guard = 0;
        for (;;) {
            // a round that runs past the wait limit is abandoned with an error (never expected:
            // the loop ends when the round's units are used up)
            if ((++guard & 1023u) == 0 &&
                __any_sync(0xffffffffu, globaltimer_ns() - t_round > timeout_ns)) {
                if (lane == 0) atomicCAS(&ctl->err, 0, CG_ETIMEOUT);
                break;
            }
            if (i + 32 <= T || (exhausted && i < T)) {
                const unsigned q = i + lane;
                const bool active = q < T;
                const unsigned o = (active && q >= ncarry) ? off[q - ncarry] : 0u;
                const uint64_t b = __shfl_sync(0xffffffffu, lbase, o >> 5);
                const uint64_t rank = !active ? 0ull : q < ncarry ? carry[q] : b + (o & 31u);
                sweep_state<kILP, kN>(gens, k, D.V, N, SN, Ln, ln_count, lbuf, lcnt, active, rank,
                                      fresh, lane);
                i += 32;
                continue;
            }
            if (exhausted) break;
            {   // keep the queue's remainder (< 32 ranks) in carry
                const unsigned q = i + lane;
                const unsigned o = (q < T && q >= ncarry) ? off[q - ncarry] : 0u;
                const uint64_t b = __shfl_sync(0xffffffffu, lbase, o >> 5);
                const uint64_t keep = q >= T ? 0ull : q < ncarry ? carry[q] : b + (o & 31u);
                __syncwarp();
                if (q < T) carry[lane] = keep;
                ncarry = T > i ? T - i : 0u;
                T = ncarry;
                i = 0;
                __syncwarp();
            }
            unsigned fw = 0;
            lbase = 0;
            if (by_rank) {
                if (!have) {
                    unsigned long long u = 0;
                    if (lane == 0) u = atomicAdd(&D.grab, 1ull);
                    u = __shfl_sync(0xffffffffu, u, 0);
                    if (u >= units) {
                        exhausted = true;
                        continue;
                    }
                    // blocks [b0, b1) of S_n: lane l holds the bits of blocks 32 (wb + l) ..
                    // 32 (wb + l) + 31 that fall in the range (at most 32 words: 2^lc <= 1024)
                    const unsigned long long b0 = u << lc;
                    const unsigned long long b1 =
                        b0 + (1ull << lc) < D.nblocks ? b0 + (1ull << lc) : D.nblocks;
                    wb = b0 >> 5;
                    const unsigned long long w0 = (wb + lane) << 5;
                    sw = w0 < b1 ? __ldcg(S + wb + lane) : 0u;
                    if (lane == 0) sw &= ~((1u << (unsigned)(b0 & 31u)) - 1u);
                    if (w0 < b1 && w0 + 32 > b1) sw &= (1u << (unsigned)(b1 - w0)) - 1u;
                    have = true;
                }
                const unsigned nz = __ballot_sync(0xffffffffu, sw != 0u);
                if (nz == 0u) {
                    have = false;
                    continue;
                }
                const int l = __ffs(nz) - 1;
                const unsigned bits = __shfl_sync(0xffffffffu, sw, l);
                if (lane == l) sw &= sw - 1u;
                const unsigned long long blk = ((wb + (unsigned)l) << 5) + (unsigned)(__ffs(bits) - 1);
                fw = __ldcg(F + blk * 32 + lane);
                lbase = (blk << 10) | ((unsigned long long)lane << 5);
            } else {
                if (ua >= ub) {
                    unsigned long long a = 0, g = 0;
                    if (lane == 0) {
                        const unsigned long long rem = seen < units ? units - seen : 0;
                        g = rem / (4 * nwarps);
                        if (g < 32) g = 32;
                        a = atomicAdd(&D.grab, g);
                    }
                    a = __shfl_sync(0xffffffffu, a, 0);
                    g = __shfl_sync(0xffffffffu, g, 0);
                    if (a >= units) {
                        exhausted = true;
                        continue;
                    }
                    ua = a;
                    ub = a + g < units ? a + g : units;
                    seen = ub;
                }
                const unsigned long long u = ua + lane;
                if (u < ub) {
                    const unsigned blk = __ldcg(Lc + (u >> 5));
                    const unsigned w = (unsigned)(u & 31u);
                    fw = __ldcg(F + (uint64_t)blk * 32 + w);
                    lbase = ((uint64_t)blk << 10) | (w << 5);
                }
                ua = ua + 32 < ub ? ua + 32 : ub;
            }
            // append the fetched ranks to the queue: offsets (lane << 5 | bit) after the carry
            const unsigned c = __popc(fw);
            unsigned incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
            unsigned pos = incl - c;
            for (unsigned m = fw; m; m &= m - 1) off[pos++] = (unsigned short)((lane << 5) | (__ffs(m) - 1));
            __syncwarp();
            T = ncarry + total;
        }
        list_flush(lbuf, lcnt, Ln, ln_count, lane);
        // states found by the block
#pragma unroll
        for (int o = 16; o; o >>= 1) fresh += __shfl_xor_sync(0xffffffffu, fresh, o);
        if (lane == 0 && fresh) atomicAdd(&s_fresh, (unsigned long long)fresh);
        __syncthreads();
        if (threadIdx.x == 0 && s_fresh) atomicAdd(&D.fresh, s_fresh);

        unsigned long long word = 0;
        const int arrive = grid_arrive(ctl, timeout_ns, word, nbar++);
        if (arrive < 0) return;
        if (arrive == 1) {
            if (threadIdx.x == 0) sweep_close(D, ctl);
            grid_release(ctl, word, 0);
        }
    }
}

using sweep_fn_t = void (*)(SweepDev*, Ctl*, int, uint64_t, int);

// The sweep kernel is compiled for every n (its rank arithmetic unrolls over n) and for one or
// two generators in flight per thread.
template <int kILP, int... Ns>
sweep_fn_t sweep_pick(int n, std::integer_sequence<int, Ns...>) {
    sweep_fn_t f = nullptr;
    (void)((n == Ns + 2 ? (f = sweep_grow_kernel<kILP, Ns + 2>, 0) : 0) + ...);
    return f;
}

sweep_fn_t sweep_fn(int ilp, int n) {
    if (n < 2 || n > 14) return nullptr;
    return ilp <= 1 ? sweep_pick<1>(n, std::make_integer_sequence<int, 13>{})
                    : sweep_pick<2>(n, std::make_integer_sequence<int, 13>{});
}

// Start state: its bit in V and F[0], its block in S[0] and L[0].
__global__ void sweep_init_kernel(SweepDev* Dp) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    SweepDev& D = *Dp;
    const uint64_t r = D.start_rank;
    const unsigned bit = 1u << (unsigned)(r & 31u);
    const unsigned blk = (unsigned)(r >> 10);
    D.V[r >> 5] |= bit;
    D.F[0][r >> 5] |= bit;
    D.S[0][blk >> 5] |= 1u << (blk & 31u);
    D.L[0][0] = blk;
    D.lcount[0] = 1;
    D.lcount[1] = 0;
    D.layer_sizes[0] = 1;
    D.grab = 0;
    D.fresh = 0;
    D.radius = 0;
    D.status = D.max_radius == 0 ? kTruncRadius : kRunning;
}

// Keys of layer `which` (its bitmap F and block list L[0, nlist)): every set bit unranked and
// written to out at a position from one counter (order unspecified).  Writes at most cap keys;
// *count receives the number of states.
template <int kN>
__global__ void sweep_export_kernel(const unsigned* F, const unsigned* L, unsigned long long nlist,
                                    uint64_t* out, unsigned long long cap, unsigned long long* count) {
    const int lane = threadIdx.x & 31;
    const unsigned long long w = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    for (unsigned long long it = w; it < nlist; it += nw) {
        const unsigned blk = L[it];
        const unsigned fw = F[(uint64_t)blk * 32 + lane];
        const unsigned c = __popc(fw);
        unsigned incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long base = 0;
        if (lane == 0 && total) base = atomicAdd(count, (unsigned long long)total);
        base = __shfl_sync(0xffffffffu, base, 0) + (incl - c);
        for (unsigned m = fw; m; m &= m - 1) {
            const uint64_t rank = ((uint64_t)blk << 10) + lane * 32 + __ffs(m) - 1;
            if (base < cap) out[base] = pos_unrank<kN>(rank);
            ++base;
        }
    }
}

template <int kN>
__global__ void pos_rank_kernel(const uint64_t* keys, unsigned long long count, uint64_t* out) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < count;
         i += (unsigned long long)gridDim.x * blockDim.x)
        out[i] = pos_rank<kN>(keys[i]);
}

template <int kN>
__global__ void pos_unrank_kernel(const uint64_t* ranks, unsigned long long count, uint64_t* out) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < count;
         i += (unsigned long long)gridDim.x * blockDim.x)
        out[i] = pos_unrank<kN>(ranks[i]);
}

// Launch K<n> for a runtime n in 1..16 with the given arguments.
template <template <int> class K, int... Ns, typename... A>
cudaError_t launch_by_n_impl(std::integer_sequence<int, Ns...>, int n, int grid, cudaStream_t st,
                             A... args) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    cudaError_t e = cudaErrorInvalidValue;
    (void)((n == Ns + 1 ? (K<Ns + 1>::launch(grid, st, args...), e = cudaGetLastError(), 0) : 0) + ...);
    return e;
}

template <template <int> class K, typename... A>
cudaError_t launch_by_n(int n, int grid, cudaStream_t st, A... args) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    return launch_by_n_impl<K>(std::make_integer_sequence<int, 16>{}, n, grid, st, args...);
}

template <int kN> struct RankK {
    static void launch(int grid, cudaStream_t st, const uint64_t* a, unsigned long long c, uint64_t* o) {
        pos_rank_kernel<kN><<<grid, 256, 0, st>>>(a, c, o);
    }
};
template <int kN> struct UnrankK {
    static void launch(int grid, cudaStream_t st, const uint64_t* a, unsigned long long c, uint64_t* o) {
        pos_unrank_kernel<kN><<<grid, 256, 0, st>>>(a, c, o);
    }
};
template <int kN> struct ExportK {
    static void launch(int grid, cudaStream_t st, const unsigned* F, const unsigned* L,
                       unsigned long long nl, uint64_t* out, unsigned long long cap,
                       unsigned long long* count) {
        sweep_export_kernel<kN><<<grid, 256, 0, st>>>(F, L, nl, out, cap, count);
    }
};

}  // namespace

int sweep_max_grid(int device, int ilp, int n) {
    int sms = 0, per_sm = 0;
    const sweep_fn_t f = sweep_fn(ilp, n);
    if (!f) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kSweepBlock, 0) != cudaSuccess)
        return -1;
    return sms * per_sm;
}

cudaError_t launch_sweep_init(SweepDev* d, cudaStream_t st) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    sweep_init_kernel<<<1, 32, 0, st>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_sweep_grow(SweepDev* d, Ctl* ctl, int grid, int max_rounds, uint64_t timeout_ns,
                              int ilp, int n, int order, cudaStream_t st) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    const sweep_fn_t f = sweep_fn(ilp, n);
    if (!f) return cudaErrorInvalidValue;
    // Rank order pays for itself through L2 hits on a visited bitmap larger than L2; when the
    // bitmap (n!/8 bytes) fits, every layer is taken in order of discovery (S_12 Coxeter: 61 ms,
    // against 66 ms with its dense layers in rank order).
    if (order == kSweepOrderAuto) {
        int dev = 0, l2 = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess && l2 > 0 &&
            fact(n) / 8 <= (uint64_t)l2)
            order = kSweepOrderList;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kSweepBlock);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, f, d, ctl, max_rounds, timeout_ns, order);
}

cudaError_t launch_sweep_export(const unsigned* F, const unsigned* L, unsigned long long nlist, int n,
                                uint64_t* out, unsigned long long cap, unsigned long long* count,
                                int grid, cudaStream_t st) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    if (nlist == 0) return cudaSuccess;
    return launch_by_n<ExportK>(n, grid, st, F, L, nlist, out, cap, count);
}

cudaError_t launch_pos_rank(const uint64_t* keys, unsigned long long count, int n, uint64_t* out,
                            int grid, cudaStream_t st) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    if (count == 0) return cudaSuccess;
    return launch_by_n<RankK>(n, grid, st, keys, count, out);
}

cudaError_t launch_pos_unrank(const uint64_t* ranks, unsigned long long count, int n, uint64_t* out,
                              int grid, cudaStream_t st) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    if (count == 0) return cudaSuccess;
    return launch_by_n<UnrankK>(n, grid, st, ranks, count, out);
}

}  // namespace cg
