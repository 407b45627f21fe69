// Hash strategy of the growth library: every layer step of every job in one persistent,
// cooperative launch.
//
// One round = one BFS layer step (Section 3.1.2) for every running job:
//   phase A  (all warps)  for each (job, generator, 32 frontier states):  t = g(s)  [expand],
//            insert-if-absent of t into the job's visited table  [dedup + visited probe],
//            warp-aggregated append of the winners to the job's key array  [compaction];
//   barrier
//   phase B  (block 0)    per job: |L_{r+1}| = tail - hi  [layer count], stop tests, and the
//            exclusive scan of next-round work units over jobs;
//   barrier.
// The visited table holds every state seen so far, which is what a directed generating set
// needs; for an inverse-closed set it is a superset of the two layers that suffice.
#include <cooperative_groups.h>
#include <cstdio>
#include <utility>

#include "cg_device.cuh"
#include "cg_kernels.h"

namespace cg {

__device__ void init_job(JobDev& J);

namespace {

constexpr int kGrowBlock = 256;
// Probe steps of one insert before the job is treated as full.  At the table's load limit
// (0.5) a linear-probing sequence longer than a few dozen slots essentially never occurs; a job
// whose layer overflows its state array keeps inserting, though, and would otherwise fill the
// table and scan it.  Hitting the limit marks the job full: the host grows its buffers and
// redoes the layer, or reports the exact layers so far (CG_TRUNC_MEMCAP).
constexpr uint64_t kMaxProbe = 64;
// Bound for re-inserting stored states into a fresh table (load <= 0.5 by construction).
constexpr uint64_t kMaxProbeRebuild = 1ull << 16;

// Largest j with ubeg[j] <= u (ubeg ascending, ubeg[0] = 0).
__device__ __forceinline__ int find_job(const unsigned long long* ubeg, int njobs,
                                        unsigned long long u) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (ld_relaxed_ull(ubeg + mid) <= u) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Units of a round handed out in equal contiguous ranges per block; the rest (half of them) is
// drawn dynamically by the blocks that finish first (a half measured better than a quarter).
__host__ __device__ __forceinline__ unsigned long long static_units(unsigned long long total) {
    return total - total / 2;
}

// Phase B, executed by the block that arrives last at the round's barrier: close the layer of
// every running job and lay out the work of the next round.  ubeg has njobs + 1 entries.
__device__ void close_round(JobDev* jobs, int njobs, unsigned long long* ubeg, Ctl* ctl) {
    __shared__ unsigned long long s_warp[kGrowBlock / 32];
    __shared__ unsigned long long s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < njobs; base += blockDim.x) {
        const int j = base + threadIdx.x;
        unsigned long long units = 0;
        if (j < njobs) {
            // The previous round may have been closed by another SM: the fields that change
            // during a run are read through L2 (relaxed loads, never this SM's L1), all in one
            // round trip, and nothing is read back after a write.
            JobDev& J = jobs[j];
            unsigned long long lo, hi, tail, rs;
            asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(lo), "=l"(hi) : "l"(&J.lo));
            asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(tail), "=l"(rs) : "l"(&J.tail));
            const int overflow = ld_relaxed_int(&J.overflow);
            int radius = (int)(unsigned)(rs & 0xffffffffull);
            int status = (int)(unsigned)(rs >> 32);
            if (status == kRunning) {
                volatile JobDev& V = jobs[j];
                if (overflow) {
                    status = kNeedMem;
                } else {
                    const unsigned long long fresh = tail - hi;
                    if (fresh == 0) {
                        status = kDone;
                    } else {
                        radius += 1;
                        J.layer_sizes[radius] = fresh;
                        V.radius = radius;
                        V.lo = hi;
                        V.hi = tail;
                        if (J.max_radius >= 0 && radius >= J.max_radius) status = kTruncRadius;
                        else if (J.stop_above > 0 && fresh > J.stop_above) status = kTruncAbove;
                        else if (radius + 1 >= J.layers_cap) status = kTruncRadius;
                        if (status == kRunning) units = (fresh + 31) >> 5;
                    }
                }
                if (status != kRunning) V.status = status;
            }
            (void)lo;
        }
        // block-wide exclusive scan of units
        unsigned long long v = units;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long n = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += n;
        }
        if (lane == 31) s_warp[wid] = v;
        __syncthreads();
        if (wid == 0) {
            unsigned long long w = (lane < (int)(blockDim.x >> 5)) ? s_warp[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long n = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += n;
            }
            if (lane < (int)(blockDim.x >> 5)) s_warp[lane] = w;
        }
        __syncthreads();
        const unsigned long long before = (wid ? s_warp[wid - 1] : 0) + (v - units) + s_carry;
        if (j < njobs) ubeg[j] = before;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry = before + units;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ubeg[njobs] = s_carry;
        ctl->total_units = s_carry;
        ctl->dyn_next = static_units(s_carry);
        atomicAdd(&ctl->rounds, 1);
    }
}

// Block-wide inclusive scan of one 64-bit value per thread (blockDim.x = kGrowBlock); returns
// the inclusive prefix, *total the block's sum.  Called by every thread of the block.
__device__ __forceinline__ unsigned long long block_scan_incl(unsigned long long v, unsigned long long* total) {
    __shared__ unsigned long long s_part[kGrowBlock / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) s_part[wid] = v;
    __syncthreads();
    if (wid == 0) {
        unsigned long long w = lane < kGrowBlock / 32 ? s_part[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kGrowBlock / 32) s_part[lane] = w;
    }
    __syncthreads();
    const unsigned long long r = v + (wid ? s_part[wid - 1] : 0);
    *total = s_part[kGrowBlock / 32 - 1];
    __syncthreads();
    return r;
}

// Phase B of a batch launch (AdmitDev), executed by the block that arrives last: close the
// layer of every active job, drop the jobs that ended from the active list (order kept), admit
// the next jobs while the window allows, set them up, and lay out the next round's work units
// over the active list (ubeg[slot], ubeg[nactive] = total).  With no active job and none left
// to admit the total is 0 and the launch ends.  Also run by one block before the launch
// (admit_first_kernel) to admit the first jobs.
__device__ void close_round_admit(JobDev* jobs, unsigned long long* ubeg, Ctl* ctl, const AdmitDev* A) {
    __shared__ unsigned long long s_units, s_freed, s_used, s_next;
    __shared__ int s_kept, s_new;
    const int sel = ld_relaxed_int(&ctl->adm.act_sel);
    const int nact = ld_relaxed_int(&ctl->adm.nactive);
    const int* cur = A->act[sel];
    int* nxt = A->act[sel ^ 1];
    const unsigned long long per_unit = 32ull * (unsigned long long)A->unit_mult;
    if (threadIdx.x == 0) { s_units = 0; s_freed = 0; s_kept = 0; }
    __syncthreads();
    for (int base = 0; base < nact; base += blockDim.x) {
        const int a = base + threadIdx.x;
        unsigned long long units = 0, keep = 0;
        int j = -1;
        if (a < nact) {
            j = __ldcg(cur + a);
            JobDev& J = jobs[j];
            unsigned long long lo, hi, tail, rs;
            asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(lo), "=l"(hi) : "l"(&J.lo));
            asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(tail), "=l"(rs) : "l"(&J.tail));
            const int overflow = ld_relaxed_int(&J.overflow);
            int radius = (int)(unsigned)(rs & 0xffffffffull);
            int status = (int)(unsigned)(rs >> 32);
            (void)lo;
            if (status == kRunning) {
                volatile JobDev& V = jobs[j];
                if (overflow) {
                    status = kNeedMem;
                } else {
                    const unsigned long long fresh = tail - hi;
                    if (fresh == 0) {
                        status = kDone;
                    } else {
                        radius += 1;
                        J.layer_sizes[radius] = fresh;
                        V.radius = radius;
                        V.lo = hi;
                        V.hi = tail;
                        if (J.max_radius >= 0 && radius >= J.max_radius) status = kTruncRadius;
                        else if (J.stop_above > 0 && fresh > J.stop_above) status = kTruncAbove;
                        else if (radius + 1 >= J.layers_cap) status = kTruncRadius;
                        if (status == kRunning) units = (fresh + per_unit - 1) / per_unit;
                    }
                }
                if (status != kRunning) V.status = status;
            }
            if (status == kRunning) keep = 1;
            else atomicAdd(&s_freed, (unsigned long long)A->vis[j]);
        }
        unsigned long long tk = 0, tu = 0;
        const unsigned long long pk = block_scan_incl(keep, &tk);
        const unsigned long long pu = block_scan_incl(units, &tu);
        if (keep) {
            const int slot = s_kept + (int)(pk - 1);
            nxt[slot] = j;
            ubeg[slot] = s_units + pu - units;
        }
        __syncthreads();
        if (threadIdx.x == 0) { s_kept += (int)tk; s_units += tu; }
        __syncthreads();
    }
    // admission, by warp 0: 32 candidates per step, in job order, while the window and the
    // active list allow (a job is always admitted when nothing else is active)
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        unsigned long long used = ld_relaxed_ull(&ctl->adm.vis_used) - s_freed;
        unsigned long long next = ld_relaxed_ull(&ctl->adm.next_admit);
        const int kept = s_kept;
        int nnew = 0;
        while (next < (unsigned long long)A->njobs && kept + nnew < A->max_active) {
            const unsigned long long c = next + lane;
            const bool valid = c < (unsigned long long)A->njobs && kept + nnew + lane < A->max_active;
            const unsigned long long v = valid ? A->vis[c] : 0;
            unsigned long long pre = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, pre, o);
                if (lane >= o) pre += y;
            }
            const bool fits = valid && (used + pre <= A->window || (kept + nnew == 0 && lane == 0));
            const unsigned fail = __ballot_sync(0xffffffffu, !fits);
            const int cnt = fail ? __ffs(fail) - 1 : 32;
            if (lane < cnt) nxt[kept + nnew + lane] = (int)c;
            if (cnt > 0) used += __shfl_sync(0xffffffffu, pre, cnt - 1);
            next += (unsigned long long)cnt;
            nnew += cnt;
            if (cnt < 32) break;
        }
        if (lane == 0) {
            s_used = used;
            s_next = next;
            s_new = nnew;
        }
    }
    __syncthreads();
    const int kept = s_kept, nnew = s_new;
    // set up the admitted jobs: one work unit each (their frontier is the start state)
    for (int i = threadIdx.x; i < nnew; i += blockDim.x) {
        JobDev& J = jobs[nxt[kept + i]];
        init_job(J);
        ubeg[kept + i] = s_units + (unsigned long long)i;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long total = s_units + (unsigned long long)nnew;
        ubeg[kept + nnew] = total;
        ctl->adm.vis_used = s_used;
        ctl->adm.next_admit = s_next;
        ctl->adm.nactive = kept + nnew;
        ctl->adm.act_sel = sel ^ 1;
        ctl->total_units = total;
        ctl->dyn_next = static_units(total);
        atomicAdd(&ctl->rounds, 1);
        __threadfence();
    }
    __syncthreads();
}

// close_round for a launch with one job, by one thread (no block-wide scan).  Called by every
// thread of the closing block.

// The closing block's thread 0 also receives the next frontier: *next_fresh = its size (0 when
// the growth stops), *next_lo/*next_hi its bounds in the key array.
__device__ void close_round_single(JobDev* jobs, unsigned long long* ubeg, Ctl* ctl,
                                   unsigned long long* next_fresh, unsigned long long* next_lo,
                                   unsigned long long* next_hi) {
    if (threadIdx.x == 0) {
        JobDev& J = jobs[0];
        // The round's state in one round trip: (lo, hi), (tail, radius | status << 32), overflow
        // and the static limits are loaded together; nothing is read back after a write.
        unsigned long long lo, hi, tail, rs;
        asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(lo), "=l"(hi) : "l"(&J.lo));
        asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(tail), "=l"(rs) : "l"(&J.tail));
        const int overflow = ld_relaxed_int(&J.overflow);
        const int max_radius = J.max_radius, layers_cap = J.layers_cap;
        const uint64_t stop_above = J.stop_above;
        int radius = (int)(unsigned)(rs & 0xffffffffull);
        int status = (int)(unsigned)(rs >> 32);
        unsigned long long units = 0;
        if (status == kRunning) {
            volatile JobDev& V = jobs[0];
            if (overflow) {
                status = kNeedMem;
            } else {
                const unsigned long long fresh = tail - hi;
                if (fresh == 0) {
                    status = kDone;
                } else {
                    radius += 1;
                    J.layer_sizes[radius] = fresh;
                    V.radius = radius;
                    V.lo = hi;
                    V.hi = tail;
                    if (max_radius >= 0 && radius >= max_radius) status = kTruncRadius;
                    else if (stop_above > 0 && fresh > stop_above) status = kTruncAbove;
                    else if (radius + 1 >= layers_cap) status = kTruncRadius;
                    if (status == kRunning) units = (fresh + 31) >> 5;
                }
            }
            if (status != kRunning) V.status = status;
        }
        ubeg[0] = 0;
        ubeg[1] = units;
        *(volatile unsigned long long*)&ctl->total_units = units;
        *(volatile unsigned long long*)&ctl->dyn_next = static_units(units);
        atomicAdd(&ctl->rounds, 1);           // result unused: a reduction, no round trip
        *next_fresh = units ? tail - hi : 0;
        *next_lo = hi;
        *next_hi = tail;
        // The release of the barrier (grid_release) makes these writes visible to the blocks
        // it wakes; rounds this block runs alone see them after its own __syncthreads.
    }
    __syncthreads();
}

// Per-warp staging of newly found states in shared memory: a warp appends its winners to
// its own buffer and reserves room in the job's key array with one atomic per flush, which
// turns a per-unit atomic on one global counter into one per ~kStage/32 units and writes the
// keys out coalesced.
constexpr int kStage = 512;

// The static fields of one job as the work loops use them.  A single-job launch receives them
// as a kernel parameter (read from the constant bank: no load, no register, nothing to reload
// after the atomics of a round); launches of several jobs read them from the job's descriptor
// when a warp moves to another job.
struct JobConst {
    uint64_t* keys;
    unsigned long long keys_cap;
    uint64_t* table;
    uint64_t table_mask;
    unsigned long long bitmap_words;
    int k;
    int n;
    int tagged;
    int mode;
    int closed;
};

__device__ __forceinline__ JobConst job_const(const JobDev* J) {
    JobConst c;
    c.keys = J->keys;
    c.keys_cap = J->keys_cap;
    c.table = J->table;
    c.table_mask = J->table_mask;
    c.bitmap_words = J->bitmap_words;
    c.k = J->k;
    c.n = J->n;
    c.tagged = J->tagged;
    c.mode = J->mode;
    c.closed = J->closed;
    return c;
}

__device__ __forceinline__ void stage_flush(uint64_t* buf, int& cnt, JobDev* J, const JobConst& c,
                                            int lane) {
    if (cnt == 0) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&J->tail, (unsigned long long)cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    uint64_t* keys = c.keys;
    const unsigned long long cap = c.keys_cap;
    bool over = false;
    for (int i = lane; i < cnt; i += 32) {
        const unsigned long long pos = base + i;
        if (pos < cap) keys[pos] = buf[i];
        else over = true;
    }
    if (__any_sync(0xffffffffu, over) && lane == 0) atomicExch(&J->overflow, 1);
    cnt = 0;
    __syncwarp();
}

// End-of-round flush of a single job's staged states: one atomicAdd on the job's tail for the
// whole block (warps take their offsets from a block-level prefix of their counts) instead of
// one per warp, since same-address atomics serialise at one L2 slice.  Called by every thread
// of the block.
__device__ __forceinline__ void stage_flush_block(uint64_t* buf, int& cnt, JobDev* J, const JobConst& c,
                                                  int lane) {
    __shared__ unsigned s_cnt[kGrowBlock / 32];
    __shared__ unsigned long long s_base;
    const int w = threadIdx.x >> 5;
    if (lane == 0) s_cnt[w] = (unsigned)cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long total = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            const unsigned c = s_cnt[i];
            s_cnt[i] = (unsigned)total;
            total += c;
        }
        s_base = total ? atomicAdd(&J->tail, total) : 0;
    }
    __syncthreads();
    const unsigned long long base = s_base + s_cnt[w];
    uint64_t* keys = c.keys;
    const unsigned long long cap = c.keys_cap;
    bool over = false;
    for (int i = lane; i < cnt; i += 32) {
        const unsigned long long pos = base + i;
        if (pos < cap) keys[pos] = buf[i];
        else over = true;
    }
    if (__any_sync(0xffffffffu, over) && lane == 0) atomicExch(&J->overflow, 1);
    cnt = 0;
    __syncwarp();
}

// One unit = 32 frontier states (one per lane) of job J, every generator applied to each:
// expand, insert-if-absent into the visited table, stage the winners.  kProbeILP generators
// are handled together (that many independent probe sequences in flight per thread).
// A state found through generator g carries the tag 1 + (index of g's inverse); that inverse
// leads back to its parent, which is already visited.  When every active lane of the warp holds
// a tagged state, each lane runs only the other k - 1 generators (the generator index depends on
// the lane), so the parent edge costs neither a probe nor the expansion and index arithmetic.
template <int kProbeILP, int kMode, int kN = 0>
__device__ __forceinline__ void do_unit(JobDev* J, const JobConst& c, const GenSM* gens,
                                        unsigned long long idx, unsigned long long hi, uint64_t* buf,
                                        int& cnt, int lane, bool& overflow_seen, uint64_t s) {
    const bool active = idx < hi;
    const int n = c.n;
    const bool tagged = c.tagged != 0;
    unsigned tag = 0;                       // 1 + generator that leads back to the parent
    if (tagged) {
        tag = (unsigned)(s >> 60);
        s &= kKeyBits60;
    }
    const int k = c.k;
    const bool skip = tagged && __all_sync(0xffffffffu, !active || tag != 0);
    const int iters = skip ? k - 1 : k;
    for (int j0 = 0; j0 < iters; j0 += kProbeILP) {
        const int ng = min(kProbeILP, iters - j0);
        uint64_t t[kProbeILP];
        int res[kProbeILP];
        int gi[kProbeILP];
        unsigned vmask = 0;
#pragma unroll
        for (int i = 0; i < kProbeILP; ++i) {
            const int j = j0 + i;
            // skipping: generators 0..tag-2 keep their slot, the rest move up by one (inactive
            // lanes have tag 0 and take j + 1 <= k - 1)
            gi[i] = (skip && (int)tag - 1 <= j) ? j + 1 : j;
            t[i] = (i < ng) ? apply_gen<kMode != kVisitBitmap>(gens[gi[i]], s) : 0;
            if (active && i < ng && tag != (unsigned)(gi[i] + 1)) vmask |= 1u << i;
        }
        if (kMode == kVisitBitmap)
            bitmap_insert_multi<kProbeILP, kN>(reinterpret_cast<unsigned*>(c.table), c.bitmap_words,
                                               n, t, res, vmask);
        else if (kMode == 1)
            table_insert_multi_sector<kProbeILP>(c.table, c.table_mask, t, res, vmask, kMaxProbe);
        else
            table_insert_multi_slot<kProbeILP>(c.table, c.table_mask, t, res, vmask, kMaxProbe);
        bool bad = false;
#pragma unroll
        for (int i = 0; i < kProbeILP; ++i) bad |= (res[i] < 0);
        if (__any_sync(0xffffffffu, bad)) {
            overflow_seen = true;
            if (lane == 0) atomicExch(&J->overflow, 1);
        }
#pragma unroll
        for (int i = 0; i < kProbeILP; ++i) {
            const unsigned fresh = __ballot_sync(0xffffffffu, res[i] == 1);
            if (res[i] == 1) {
                const uint64_t itag = tagged ? (uint64_t)gens[gi[i]].inv_tag << 60 : 0;
                buf[cnt + __popc(fresh & lanemask_lt())] = t[i] | itag;
            }
            cnt += __popc(fresh);
            __syncwarp();
            if (cnt > kStage - 32) stage_flush(buf, cnt, J, c, lane);
        }
    }
}

// The same work with a lane per (state, generator) pair instead of per state, for rounds in which
// every warp has at most one unit: a unit is sp = 32 / (k - 1) states, lane l takes state l / (k - 1)
// and its non-parent generator number l mod (k - 1) (lslot), so that the k - 1 probes of a state
// are in flight together rather than one after the other.  Every state must carry its parent-edge
// tag (the set is closed under inverses and the frontier is not the start).
template <int kMode, int kN = 0>
__device__ __forceinline__ void do_unit_split(JobDev* J, const JobConst& c, const GenSM* gens, bool active,
                                              uint64_t s, int lslot, uint64_t* buf, int& cnt, int lane,
                                              bool& overflow_seen) {
    const unsigned tag = (unsigned)(s >> 60);   // 1 + generator that leads back to the parent
    s &= kKeyBits60;
    // generators 0..tag-2 keep their number, the rest move up by one (idle lanes: lslot itself)
    const int gi = (active && lslot >= (int)tag - 1) ? lslot + 1 : lslot;
    uint64_t t[1];
    int res[1];
    t[0] = apply_gen<kMode != kVisitBitmap>(gens[gi], s);
    const unsigned vmask = active ? 1u : 0u;
    if (kMode == kVisitBitmap)
        bitmap_insert_multi<1, kN>(reinterpret_cast<unsigned*>(c.table), c.bitmap_words, c.n, t, res, vmask);
    else if (kMode == 1)
        table_insert_multi_sector<1>(c.table, c.table_mask, t, res, vmask, kMaxProbe);
    else
        table_insert_multi_slot<1>(c.table, c.table_mask, t, res, vmask, kMaxProbe);
    if (__any_sync(0xffffffffu, res[0] < 0)) {
        overflow_seen = true;
        if (lane == 0) atomicExch(&J->overflow, 1);
    }
    const unsigned fresh = __ballot_sync(0xffffffffu, res[0] == 1);
    if (res[0] == 1) buf[cnt + __popc(fresh & lanemask_lt())] = t[0] | (uint64_t)gens[gi].inv_tag << 60;
    cnt += __popc(fresh);
    __syncwarp();
    if (cnt > kStage - 32) stage_flush(buf, cnt, J, c, lane);
}

// Next work unit of the block for the calling warp (one shared-memory atomic per warp).
__device__ __forceinline__ unsigned long long draw_unit(unsigned long long& counter, int lane) {
    unsigned long long u = 0;
    if (lane == 0) u = atomicAdd(&counter, 1ull);
    return __shfl_sync(0xffffffffu, u, 0);
}

// The work phase of a round of a single job: the warp takes units w0, w0 + W, w0 + 2W, ... of
// the frontier keys[lo, hi) (W = warps taking part, w0 = this warp's place among them), so the
// units are dealt out with no atomics and the warp knows its next unit in advance: the next
// unit's frontier key is loaded while the current one is processed.  Ends with the block's
// flush of newly found states (every thread of the block calls this).  The job's overflow flag
// (buffers full: the host grows them and redoes the layer) is read every 16 units, one unit
// before its value is needed.
template <int kProbeILP, int kMode, int kN = 0>
__device__ __forceinline__ void phase_single(JobDev* J, const JobConst& c, const GenSM* gens,
                                             unsigned long long w0, unsigned long long W, uint64_t* buf,
                                             int lane, unsigned long long lo, unsigned long long hi) {
    int cnt = 0;
    bool overflow_seen = false;
    const unsigned long long total = (hi - lo + 31) >> 5;
    const int m = c.k - 1;                      // generators a tagged state expands
    if (total <= W && c.tagged && c.closed && lo > 0 && m >= 1 && m <= 32) {
        // a small round (at most one unit a warp): a lane per (state, generator) pair
        const int sp = 32 / m;
        const int lstate = lane / m, lslot = lane - lstate * m;
        const unsigned long long ts = (hi - lo + (unsigned long long)sp - 1) / (unsigned long long)sp;
        for (unsigned long long u = w0; u < ts; u += W) {
            const unsigned long long idx = lo + u * (unsigned long long)sp + (unsigned long long)lstate;
            const bool active = lstate < sp && idx < hi;
            const uint64_t s = active ? __ldcg(c.keys + idx) : 0;
            do_unit_split<kMode, kN>(J, c, gens, active, s, lslot, buf, cnt, lane, overflow_seen);
            if (overflow_seen) break;
        }
        stage_flush_block(buf, cnt, J, c, lane);
        return;
    }
    unsigned long long u = w0;
    uint64_t s_next = (u < total && lo + (u << 5) + lane < hi) ? __ldcg(c.keys + lo + (u << 5) + lane) : 0;
    int ov = 0;
    for (unsigned iter = 0; u < total; ++iter) {
        const uint64_t s_cur = s_next;
        const unsigned long long nu = u + W;
        s_next = (nu < total && lo + (nu << 5) + lane < hi) ? __ldcg(c.keys + lo + (nu << 5) + lane) : 0;
        const bool check = (iter & 15u) == 15u;
        if ((iter & 15u) == 14u) ov = ld_relaxed_int(&J->overflow);
        do_unit<kProbeILP, kMode, kN>(J, c, gens, lo + (u << 5) + lane, hi, buf, cnt, lane, overflow_seen, s_cur);
        if (check && __any_sync(0xffffffffu, ov)) overflow_seen = true;
        if (overflow_seen) break;
        u = nu;
    }
    stage_flush_block(buf, cnt, J, c, lane);
}

// Barrier payload of a single-job round: the next frontier's size, with this bit set when the
// releasing block ran rounds alone before releasing (the other blocks reload the bounds).
constexpr unsigned long long kReloadFlag = 1ull << 42;

// Rounds of at most this many units (one per warp of a block) are run by one block alone.
constexpr unsigned long long kSoloUnits = kGrowBlock / 32;

// Generators of a single job kept in shared memory when there are at most this many.
constexpr int kSmemGens = 32;
// Several jobs: each warp keeps the generators of its current job in shared memory when the job
// has at most this many.
constexpr int kWarpGens = 10;

// kMulti = false: the launch has exactly one job (the single-job path only is compiled, which
// keeps registers low), whose static fields are `jc`; true: any number of jobs (`jc` unused).
template <int kProbeILP, int kMode, bool kMulti, int kN = 0>
__global__ void __launch_bounds__(kGrowBlock, kMode == 2 ? 4 : ((kMode == 1 && kProbeILP >= 3) ? 2 : 3))
hash_grow_kernel(JobDev* jobs, int njobs, unsigned long long* ubeg, Ctl* ctl, int max_rounds,
                 uint64_t timeout_ns, const AdmitDev* adm, const JobConst jc) {
    __shared__ uint64_t s_stage[kGrowBlock / 32][kStage];
    __shared__ GenSM s_gens[kSmemGens];
    __shared__ unsigned long long s_unit;
    __shared__ JobConst s_jc[kMulti ? kGrowBlock / 32 : 1];
    __shared__ GenSM s_wgens[kMulti ? kGrowBlock / 32 : 1][kMulti ? kWarpGens : 1];
    const GenSM* single_gens = jobs[0].gens;
    if (!kMulti && jobs[0].k <= kSmemGens) {
        for (int j = threadIdx.x; j < jobs[0].k; j += blockDim.x) s_gens[j] = jobs[0].gens[j];
        __syncthreads();
        single_gens = s_gens;
    }
    const int lane = threadIdx.x & 31;
    uint64_t* buf = s_stage[threadIdx.x >> 5];
    // One job: every block keeps the frontier bounds itself.  They are read once here; after
    // each barrier the releasing block hands every block the size of the next frontier in the
    // barrier word, so no block reloads them.  (Several jobs: the round's layout is read from
    // the control block each round.)
    __shared__ unsigned long long s_lo, s_hi, s_total, s_fresh;
    __shared__ int s_nact, s_sel;
    if (threadIdx.x == 0 && !kMulti) {
        const bool running = ld_relaxed_int(&jobs[0].status) == kRunning;
        s_lo = ld_relaxed_ull(&jobs[0].lo);
        s_hi = running ? ld_relaxed_ull(&jobs[0].hi) : s_lo;
    }

    unsigned nbar = 0;                      // grid barriers this block has passed
    for (int round = 0; round < max_rounds; ++round) {
        if (threadIdx.x == 0) {
            s_total = kMulti ? ld_relaxed_ull(&ctl->total_units) : (s_hi - s_lo + 31) >> 5;
            if (kMulti && adm) {
                s_nact = ld_relaxed_int(&ctl->adm.nactive);
                s_sel = ld_relaxed_int(&ctl->adm.act_sel);
            }
        }
        __syncthreads();
        const unsigned long long total = s_total;
        const unsigned long long lo = s_lo, hi = s_hi;
        if (total == 0) break;
        // Rounds of at least 16 units per block share their second half (blocks that finish
        // their range early take from it); smaller rounds are split in equal ranges only.
        const bool shared_tail = total >= 16ull * gridDim.x;
        const unsigned long long stat = shared_tail ? static_units(total) : total;
        if (kMulti) {
            if (threadIdx.x == 0) s_unit = stat * blockIdx.x / gridDim.x;   // this block's first unit
            __syncthreads();
        }
        int cnt = 0;
        bool overflow_seen = false;
        if (!kMulti) {
            // unit u goes to block u mod grid, so that a small round spreads over every SM
            const unsigned long long W = (unsigned long long)gridDim.x * (blockDim.x >> 5);
            const unsigned long long w0 = (unsigned long long)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
            phase_single<kProbeILP, kMode, kN>(jobs, jc, single_gens, w0, W, buf, lane, lo, hi);
        } else {
            int cur = -1;
            JobDev* J = nullptr;
            // the current job's static fields, one copy per warp in shared memory (read where
            // used, which keeps them out of the registers)
            JobConst& c = s_jc[threadIdx.x >> 5];
            const GenSM* jg = nullptr;              // the current job's generators
            int ovf = 0;                            // the current job's overflow flag, read a unit ago
            unsigned long long lo = 0, hi = 0, u0 = 0;
            const unsigned long long ue = stat * (blockIdx.x + 1) / gridDim.x;
            unsigned long long pending = ~0ull;
            // a batch launch (adm): units map to slots of the active list, 32 * unit_mult
            // frontier states each; otherwise to jobs, 32 states each
            const int nj = adm ? s_nact : njobs;
            const int* act = adm ? adm->act[s_sel] : nullptr;
            const int umult = adm ? adm->unit_mult : 1;
            // the block's range, then (large rounds) the shared half, two units per draw
            auto next_unit = [&]() -> unsigned long long {
                const unsigned long long u = draw_unit(s_unit, lane);
                if (u < ue) return u;
                if (pending != ~0ull) {
                    const unsigned long long p = pending;
                    pending = ~0ull;
                    return p;
                }
                if (!shared_tail) return ~0ull;
                unsigned long long d = 0;
                if (lane == 0) d = atomicAdd(&ctl->dyn_next, 2ull);
                d = __shfl_sync(0xffffffffu, d, 0);
                if (d >= total) return ~0ull;
                if (d + 1 < total) pending = d + 1;
                return d;
            };
            unsigned long long u1 = 0;              // units of slot cur: [u0, u1)
            for (unsigned long long u = next_unit(); u != ~0ull; u = next_unit()) {
                // a warp's units mostly stay within one job: search the table only on leaving it
                if (cur >= 0 && u >= u0 && u < u1) {
                    // same job as the previous unit
                } else {
                    const int slot = find_job(ubeg, nj, u);
                    if (J) stage_flush(buf, cnt, J, c, lane);
                    cur = slot;
                    J = jobs + (act ? __ldcg(act + slot) : slot);
                    if (lane == 0) c = job_const(J);
                    __syncwarp();
                    ovf = 0;
                    jg = J->gens;
                    if (kMulti && c.k <= kWarpGens) {
                        // copy them into this warp's shared slots, word by word across the lanes
                        GenSM* dst = s_wgens[threadIdx.x >> 5];
                        const unsigned words = (unsigned)c.k * (unsigned)(sizeof(GenSM) / 4);
                        const unsigned* from = reinterpret_cast<const unsigned*>(jg);
                        unsigned* to = reinterpret_cast<unsigned*>(dst);
                        for (unsigned i = lane; i < words; i += 32) to[i] = from[i];
                        __syncwarp();
                        jg = dst;
                    }
                    lo = ld_relaxed_ull(&J->lo);
                    hi = ld_relaxed_ull(&J->hi);
                    u0 = ld_relaxed_ull(ubeg + slot);
                    u1 = ld_relaxed_ull(ubeg + slot + 1);
                }
                // A job whose buffers ran full stops expanding (the host grows them or reports
                // the exact layers so far): its flag, read while the previous unit of the same
                // job ran, skips the rest of its units.
                if (__any_sync(0xffffffffu, ovf)) continue;
                ovf = ld_relaxed_int(&J->overflow);
                // the unit's unit_mult groups of 32 states, the next group's keys loaded while one
                // is expanded
                unsigned long long first = lo + (((u - u0) * (unsigned long long)umult) << 5);
                uint64_t s_nx = first + lane < hi ? __ldcg(c.keys + first + lane) : 0;
                for (int sub = 0; sub < umult && first < hi; ++sub) {
                    const unsigned long long idx = first + lane;
                    const uint64_t s0 = s_nx;
                    const unsigned long long nf = first + 32;
                    s_nx = (sub + 1 < umult && nf + lane < hi) ? __ldcg(c.keys + nf + lane) : 0;
                    // In the rank-bitmap variant a launch may mix jobs of both visited-set kinds.
                    if (kMode == kVisitBitmap && c.mode != kVisitBitmap)
                        do_unit<kProbeILP, kVisitHash>(J, c, jg, idx, hi, buf, cnt, lane, overflow_seen, s0);
                    else
                        do_unit<kProbeILP, kMode>(J, c, jg, idx, hi, buf, cnt, lane, overflow_seen, s0);
                    first = nf;
                }
            }
            if (J) stage_flush(buf, cnt, J, c, lane);
        }
        // One barrier per round: the last block to finish the round closes it (layer counts,
        // stop tests, next round's work layout) and then releases the others.
        unsigned long long word = 0;
        const int arrive = grid_arrive(ctl, timeout_ns, word, nbar++);
        if (arrive < 0) return;
        if (arrive == 1) {
            if (!kMulti) {
                close_round_single(jobs, ubeg, ctl, &s_fresh, &s_lo, &s_hi);
                // While the frontier stays small this block runs the next rounds alone, with
                // __syncthreads for a barrier; the other blocks wait until it releases them.
                bool solo = false;
                for (;;) {
                    const unsigned long long t = (s_fresh + 31) >> 5;
                    if (t == 0 || t > kSoloUnits || round + 1 >= max_rounds) break;
                    ++round;
                    solo = true;
                    const unsigned long long slo = s_lo, shi = s_hi;
                    phase_single<kProbeILP, kMode, kN>(jobs, jc, single_gens, threadIdx.x >> 5,
                                                       blockDim.x >> 5, buf, lane, slo, shi);
                    __syncthreads();
                    close_round_single(jobs, ubeg, ctl, &s_fresh, &s_lo, &s_hi);
                }
                if (threadIdx.x == 0 && s_fresh == 0) s_hi = s_lo;   // stop: empty frontier
                // payload: the next frontier's size, and whether this block ran rounds alone (the
                // others' bounds are then stale and they reload them)
                grid_release(ctl, word, s_fresh | (solo ? kReloadFlag : 0ull));
            } else {
                if (adm) close_round_admit(jobs, ubeg, ctl, adm);
                else close_round(jobs, njobs, ubeg, ctl);
                grid_release(ctl, word, 0);
            }
        } else if (!kMulti && threadIdx.x == 0) {
            // the next frontier follows this one in the key array (size 0: the growth stops)
            const unsigned long long payload = word >> kGenBits;
            const unsigned long long fresh = payload & ~kReloadFlag;
            if (fresh == 0) {
                s_lo = s_hi;
            } else if (payload & kReloadFlag) {
                s_lo = ld_relaxed_ull(&jobs[0].lo);
                s_hi = ld_relaxed_ull(&jobs[0].hi);
            } else {
                s_lo = s_hi;
                s_hi = s_hi + fresh;
            }
        }
    }
}

}  // namespace

// Set up one job for a run from the identity (or its start state): its visited set must already
// be cleared.
__device__ void init_job(JobDev& J) {
    uint64_t id = 0;
    for (int i = 0; i < J.n; ++i) id |= (uint64_t)i << (4 * i);
    if (J.use_start) id = J.start_key;      // a central state: the growth of its orbit
    J.keys[0] = id;
    if (J.mode == kVisitBitmap) {
        const uint64_t r = perm_rank(id, J.n);
        atomicOr(reinterpret_cast<unsigned*>(J.table) + (r >> 5), 1u << (unsigned)(r & 31u));
    } else {
        table_insert(J.table, J.table_mask, id, kMaxProbe);
    }
    J.layer_sizes[0] = 1;
    J.lo = 0;
    J.hi = 1;
    J.tail = 1;
    J.radius = 0;
    J.overflow = 0;
    J.status = kRunning;
    if (J.max_radius == 0) J.status = kTruncRadius;
}

namespace {

__global__ void init_jobs_kernel(JobDev* jobs, int njobs, int only_fresh) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= njobs) return;
    JobDev& J = jobs[j];
    if (only_fresh && J.status != kFresh) return;
    init_job(J);
}

// Work layout of the first round (after init, or after the host resized a job's buffers):
// one warp unit per 32 frontier states of every running job.
__global__ void init_units_kernel(JobDev* jobs, int njobs, unsigned long long* ubeg, Ctl* ctl) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    unsigned long long acc = 0;
    for (int j = 0; j < njobs; ++j) {
        ubeg[j] = acc;
        if (jobs[j].status == kRunning) acc += (jobs[j].hi - jobs[j].lo + 31) >> 5;
    }
    ubeg[njobs] = acc;
    ctl->total_units = acc;
    ctl->dyn_next = static_units(acc);
    ctl->rounds = 0;
    ctl->bar_count = 0;
    ctl->bar_word = 0;
    for (int g = 0; g < kBarGroups; ++g) ctl->group[g].count = 0;   // the barrier counters only grow
    ctl->err = 0;
}

// First admission of a batch launch (one block): admit the first jobs and lay out their work.
__global__ void __launch_bounds__(kGrowBlock) admit_first_kernel(JobDev* jobs, unsigned long long* ubeg,
                                                                 Ctl* ctl, const AdmitDev* adm) {
    close_round_admit(jobs, ubeg, ctl, adm);
}

// Re-insert keys[0, count) of one job into its (cleared) table; used after the key array
// grew.  Dups cannot occur: the keys are distinct.
__global__ void rebuild_table_kernel(const uint64_t* keys, unsigned long long count,
                                     uint64_t* table, uint64_t mask, uint64_t key_mask, int* err) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
         i < count; i += (unsigned long long)gridDim.x * blockDim.x) {
        if (table_insert(table, mask, __ldcg(keys + i) & key_mask, kMaxProbeRebuild) < 0)
            atomicExch(err, CG_EDEVICE);
    }
}

// Set the bits of keys[0, count) in a (cleared) rank bitmap; used after the key array grew.
__global__ void rebuild_bitmap_kernel(const uint64_t* keys, unsigned long long count, unsigned* bm,
                                      uint64_t words, int n, int* err) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
         i < count; i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint64_t r = perm_rank(__ldcg(keys + i) & (n <= 15 ? kKeyBits60 : ~0ull), n);
        if ((r >> 5) < words) atomicOr(bm + (r >> 5), 1u << (unsigned)(r & 31u));
        else atomicExch(err, CG_EDEVICE);
    }
}

__global__ void expand_kernel(const GenSM* __restrict__ gens, int k, const uint64_t* __restrict__ in,
                              unsigned long long F, uint64_t* __restrict__ out) {
    const unsigned long long total = F * (unsigned long long)k;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < total;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned g = (unsigned)(i / F);
        const unsigned long long s = i - (unsigned long long)g * F;
        out[i] = apply_gen(gens[g], in[s]);
    }
}

__global__ void hash_insert_kernel(uint64_t* table, uint64_t mask, const uint64_t* __restrict__ keys,
                                   unsigned long long N, uint64_t* out,
                                   unsigned long long* count, int* fail) {
    const int lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long warp = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nw = stride >> 5;
    for (unsigned long long w = warp; (w << 5) < N; w += nw) {
        const unsigned long long idx = (w << 5) + lane;
        int ins = 0;
        uint64_t t = 0;
        if (idx < N) {
            t = keys[idx];
            ins = table_insert(table, mask, t, mask + 1);
        }
        if (__any_sync(0xffffffffu, ins < 0) && lane == 0) atomicExch(fail, 1);
        const unsigned fresh = __ballot_sync(0xffffffffu, ins == 1);
        if (fresh) {
            unsigned long long b = 0;
            if (lane == 0) b = atomicAdd(count, (unsigned long long)__popc(fresh));
            b = __shfl_sync(0xffffffffu, b, 0);
            if (ins == 1) out[b + __popc(fresh & lanemask_lt())] = t;
        }
    }
}

__global__ void finish_insert_count_kernel(unsigned long long* count, const int* fail) {
    if (*fail) *count = ~0ull;
}

}  // namespace

int hash_grow_block() { return kGrowBlock; }

namespace {
using GrowFn = void (*)(JobDev*, int, unsigned long long*, Ctl*, int, uint64_t, const AdmitDev*, const JobConst);
// Kernel variants: `ilp` generators per thread (1..4); +8 selects whole-sector table probing,
// +16 the rank bitmap; multi = launches of several jobs.
template <bool M>
GrowFn grow_fn_t(int variant) {
    switch (variant) {
        case 1: return hash_grow_kernel<1, 0, M>;
        case 2: return hash_grow_kernel<2, 0, M>;
        case 3: return hash_grow_kernel<3, 0, M>;
        case 4: return hash_grow_kernel<4, 0, M>;
        case 9: return hash_grow_kernel<1, 1, M>;
        case 10: return hash_grow_kernel<2, 1, M>;
        case 11: return hash_grow_kernel<3, 1, M>;
        case 12: return hash_grow_kernel<4, 1, M>;
        case 17: return hash_grow_kernel<1, 2, M>;
        case 18: return hash_grow_kernel<2, 2, M>;
        case 19: return hash_grow_kernel<3, 2, M>;
        default: return hash_grow_kernel<4, 2, M>;
    }
}

GrowFn grow_fn(int variant, bool multi) { return multi ? grow_fn_t<true>(variant) : grow_fn_t<false>(variant); }

// The single-job rank-bitmap kernel with one generator in flight per thread (the default for
// S_n, n <= 14) is also compiled per n, so its rank arithmetic unrolls with constants.
template <int kILP, int... Ns>
GrowFn grow_fn_bitmap_n(int n, std::integer_sequence<int, Ns...>) {
    GrowFn f = nullptr;
    (void)((n == Ns + 2 ? (f = hash_grow_kernel<kILP, 2, false, Ns + 2>, 0) : 0) + ...);
    return f;
}

GrowFn grow_fn(int variant, bool multi, int n) {
    if (variant == 17 && !multi && n >= 2 && n <= 14)
        return grow_fn_bitmap_n<1>(n, std::make_integer_sequence<int, 13>{});
    return grow_fn(variant, multi);
}
}  // namespace

int hash_grow_max_grid(int device, int ilp, bool multi) {
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grow_fn(ilp, multi), kGrowBlock, 0) !=
        cudaSuccess)
        return 0;
    return sms * per_sm;
}

cudaError_t launch_init_jobs(JobDev* d_jobs, int njobs, unsigned long long* d_ubeg, Ctl* d_ctl,
                             cudaStream_t st, int only_fresh) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    init_jobs_kernel<<<(njobs + 255) / 256, 256, 0, st>>>(d_jobs, njobs, only_fresh);
    init_units_kernel<<<1, 1, 0, st>>>(d_jobs, njobs, d_ubeg, d_ctl);
    return cudaGetLastError();
}

cudaError_t launch_resume_units(JobDev* d_jobs, int njobs, unsigned long long* d_ubeg, Ctl* d_ctl,
                                cudaStream_t st) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    init_units_kernel<<<1, 1, 0, st>>>(d_jobs, njobs, d_ubeg, d_ctl);
    return cudaGetLastError();
}

cudaError_t launch_admit_first(JobDev* d_jobs, unsigned long long* d_ubeg, Ctl* d_ctl,
                               const AdmitDev* d_adm, cudaStream_t st) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    admit_first_kernel<<<1, kGrowBlock, 0, st>>>(d_jobs, d_ubeg, d_ctl, d_adm);
    return cudaGetLastError();
}

cudaError_t launch_hash_grow(JobDev* d_jobs, int njobs, unsigned long long* d_ubeg, Ctl* d_ctl,
                             int grid, int max_rounds, uint64_t timeout_ns, int ilp, cudaStream_t st,
                             int n, const AdmitDev* d_adm, const JobDev* host_job) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    // The single-job kernels take the job's static fields as a parameter: without the host's
    // copy of them, one job runs through the general kernel.
    const bool multi = njobs > 1 || d_adm != nullptr || host_job == nullptr;
    JobConst jc = {};
    if (!multi) {
        jc.keys = host_job->keys;
        jc.keys_cap = host_job->keys_cap;
        jc.table = host_job->table;
        jc.table_mask = host_job->table_mask;
        jc.bitmap_words = host_job->bitmap_words;
        jc.k = host_job->k;
        jc.n = host_job->n;
        jc.tagged = host_job->tagged;
        jc.mode = host_job->mode;
        jc.closed = host_job->closed;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kGrowBlock);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, grow_fn(ilp, multi, n), d_jobs, njobs, d_ubeg, d_ctl, max_rounds,
                              timeout_ns, d_adm, jc);
}

cudaError_t launch_rebuild_table(const uint64_t* keys, unsigned long long count, uint64_t* table,
                                 uint64_t mask, uint64_t key_mask, int* d_err, int grid,
                                 cudaStream_t st) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    if (count == 0) return cudaSuccess;
    rebuild_table_kernel<<<grid, 256, 0, st>>>(keys, count, table, mask, key_mask, d_err);
    return cudaGetLastError();
}

cudaError_t launch_rebuild_bitmap(const uint64_t* keys, unsigned long long count, unsigned* bm,
                                  uint64_t words, int n, int* d_err, int grid, cudaStream_t st) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    if (count == 0) return cudaSuccess;
    rebuild_bitmap_kernel<<<grid, 256, 0, st>>>(keys, count, bm, words, n, d_err);
    return cudaGetLastError();
}

cudaError_t launch_expand(const GenSM* d_gens, int k, const uint64_t* in, unsigned long long F,
                          uint64_t* out, int grid, cudaStream_t st) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    if (F == 0) return cudaSuccess;
    expand_kernel<<<grid, 256, 0, st>>>(d_gens, k, in, F, out);
    return cudaGetLastError();
}

cudaError_t launch_hash_insert(uint64_t* table, uint64_t mask, const uint64_t* keys,
                               unsigned long long N, uint64_t* out, unsigned long long* count,
                               int* fail, int grid, cudaStream_t st) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    hash_insert_kernel<<<grid, 256, 0, st>>>(table, mask, keys, N, out, count, fail);
    finish_insert_count_kernel<<<1, 1, 0, st>>>(count, fail);
    return cudaGetLastError();
}

}  // namespace cg
