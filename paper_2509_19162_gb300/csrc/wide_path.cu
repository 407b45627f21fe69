// Growth with two-word (128-bit) keys: vectors whose n elements of w bits need more than 64 bits
// (Schreier coset graphs of long vectors, Sections 3.1.2 and 3.2, and permutations of more than
// 16 elements from the identity).  The same BFS layer step as the one-word hash strategy -- every
// generator applied to every frontier state, insert-if-absent into the visited set, append of
// the new states -- in one persistent cooperative launch with one grid barrier per layer.
//
// The visited set is an open-addressing table of 16-byte slots (empty = all ones) probed
// linearly; every probe is one 128-bit compare-and-swap (atom.cas.b128), which both reads the
// slot and claims it when empty, so no torn 16-byte read can ever be mistaken for a key.
#include <cstdint>

#include "cg_device.cuh"
#include "cg_kernels.h"

namespace cg {

namespace {

constexpr int kWideBlock = 256;
constexpr int kWideStage = 256;            // staged new states per warp
constexpr uint64_t kWideMaxProbe = 64;
constexpr uint64_t kWideMaxProbeRebuild = 1ull << 16;
constexpr int kWideSmemGens = 16;
constexpr uint64_t kTag124 = (1ull << 60) - 1;   // mask of hi below the tag bits 124-127

__device__ __forceinline__ bool key_eq(const Key128& a, const Key128& b) { return a.lo == b.lo && a.hi == b.hi; }

__device__ __forceinline__ Key128 rotl128(Key128 x, unsigned r) {
    if (r & 64u) {
        const uint64_t t = x.lo;
        x.lo = x.hi;
        x.hi = t;
    }
    r &= 63u;
    if (r == 0) return x;
    Key128 y;
    y.lo = (x.lo << r) | (x.hi >> (64u - r));
    y.hi = (x.hi << r) | (x.lo >> (64u - r));
    return y;
}

__device__ __forceinline__ Key128 shr128(Key128 x, int r) {   // r in [0, 128)
    Key128 y;
    if (r >= 64) { y.lo = x.hi >> (r - 64); y.hi = 0; }
    else if (r == 0) { y = x; }
    else { y.lo = (x.lo >> r) | (x.hi << (64 - r)); y.hi = x.hi >> r; }
    return y;
}

__device__ __forceinline__ Key128 shl128(Key128 x, int r) {   // r in [0, 128)
    Key128 y;
    if (r >= 64) { y.hi = x.lo << (r - 64); y.lo = 0; }
    else if (r == 0) { y = x; }
    else { y.hi = (x.hi << r) | (x.lo >> (64 - r)); y.lo = x.lo << r; }
    return y;
}

// t[i] = s[g[i]] on two-word keys (WideGen).
__device__ __forceinline__ Key128 apply_wide(const WideGen& g, Key128 s) {
    if (g.kind == 1) {
        Key128 r;
        r.lo = __brevll(s.hi);
        r.hi = __brevll(s.lo);
        if (g.width >= 2) {
            r.lo = ((r.lo >> 1) & 0x5555555555555555ull) | ((r.lo & 0x5555555555555555ull) << 1);
            r.hi = ((r.hi >> 1) & 0x5555555555555555ull) | ((r.hi & 0x5555555555555555ull) << 1);
        }
        if (g.width == 4) {
            r.lo = ((r.lo >> 2) & 0x3333333333333333ull) | ((r.lo & 0x3333333333333333ull) << 2);
            r.hi = ((r.hi >> 2) & 0x3333333333333333ull) | ((r.hi & 0x3333333333333333ull) << 2);
        }
        const int sh = g.rev_shift;
        r = sh >= 0 ? shr128(r, sh) : shl128(r, -sh);
        Key128 t;
        t.lo = (s.lo & ~g.mlo[0]) | (r.lo & g.mlo[0]);
        t.hi = (s.hi & ~g.mhi[0]) | (r.hi & g.mhi[0]);
        return t;
    }
    Key128 t{0, 0};
    const uint32_t nt = g.nterms;
    for (uint32_t i = 0; i < nt; ++i) {
        const Key128 r = rotl128(s, g.rot[i]);
        t.lo |= r.lo & g.mlo[i];
        t.hi |= r.hi & g.mhi[i];
    }
    return t;
}

__device__ __forceinline__ uint64_t hash128(const Key128& k) { return mix64(k.lo ^ mix64(k.hi)); }

__device__ __forceinline__ Key128 cas128(Key128* addr, const Key128& cmp, const Key128& val) {
    Key128 old;
    asm volatile("{\n\t.reg .b128 d, c, v;\n\t"
                 "mov.b128 c, {%2, %3};\n\t"
                 "mov.b128 v, {%4, %5};\n\t"
                 "atom.global.cas.b128 d, [%6], c, v;\n\t"
                 "mov.b128 {%0, %1}, d;\n\t}"
                 : "=l"(old.lo), "=l"(old.hi)
                 : "l"(cmp.lo), "l"(cmp.hi), "l"(val.lo), "l"(val.hi), "l"(addr)
                 : "memory");
    return old;
}

// Insert-if-absent: 1 inserted, 0 present, -1 no free slot within max_probe slots.
__device__ __forceinline__ int table_insert128(Key128* table, uint64_t mask, const Key128& key,
                                               uint64_t max_probe) {
    const Key128 empty{~0ull, ~0ull};
    uint64_t h = hash128(key) & mask;
    for (uint64_t p = 0; p < max_probe; ++p) {
        const Key128 old = cas128(table + h, empty, key);
        if (key_eq(old, empty)) return 1;
        if (key_eq(old, key)) return 0;
        h = (h + 1) & mask;
    }
    return -1;
}

__device__ __forceinline__ void wide_flush(Key128* buf, int& cnt, WideDev* J, int lane) {
    if (cnt == 0) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&J->tail, (unsigned long long)cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    bool over = false;
    for (int i = lane; i < cnt; i += 32) {
        const unsigned long long pos = base + i;
        if (pos < J->keys_cap) J->keys[pos] = buf[i];
        else over = true;
    }
    if (__any_sync(0xffffffffu, over) && lane == 0) atomicExch(&J->overflow, 1);
    cnt = 0;
    __syncwarp();
}

// One unit: 32 frontier states (one per lane), every generator applied to each.  A tagged state
// skips the generator that leads back to its parent (when every active lane is tagged, each lane
// runs only the other k - 1 generators).
__device__ __forceinline__ void wide_unit(WideDev* J, const WideGen* gens, unsigned long long idx,
                                          unsigned long long hi, Key128* buf, int& cnt, int lane) {
    const bool active = idx < hi;
    Key128 s{0, 0};
    if (active) {
        const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2*>(J->keys + idx));
        s.lo = v.x;
        s.hi = v.y;
    }
    const bool tagged = J->tagged != 0;
    unsigned tag = 0;
    if (tagged) {
        tag = (unsigned)(s.hi >> 60);
        s.hi &= kTag124;
    }
    const int k = J->k;
    const bool skip = tagged && __all_sync(0xffffffffu, !active || tag != 0);
    const int iters = skip ? k - 1 : k;
    for (int j = 0; j < iters; ++j) {
        const int g = (skip && (int)tag - 1 <= j) ? j + 1 : j;
        const Key128 t = apply_wide(gens[g], s);
        int res = 0;
        if (active && tag != (unsigned)(g + 1)) res = table_insert128(J->table, J->table_mask, t, kWideMaxProbe);
        if (__any_sync(0xffffffffu, res < 0)) {
            if (lane == 0) atomicExch(&J->overflow, 1);
            return;
        }
        const unsigned fresh = __ballot_sync(0xffffffffu, res == 1);
        if (res == 1) {
            Key128 o = t;
            if (tagged) o.hi |= (uint64_t)gens[g].inv_tag << 60;
            buf[cnt + __popc(fresh & lanemask_lt())] = o;
        }
        cnt += __popc(fresh);
        __syncwarp();
        if (cnt > kWideStage - 32) wide_flush(buf, cnt, J, lane);
    }
}

// Close a layer (one thread of the block that arrived last): |L_{r+1}| = tail - hi, stop tests.
__device__ void wide_close(WideDev* J, Ctl* ctl) {
    volatile WideDev* V = J;
    const int status0 = V->status;
    if (status0 == kRunning) {
        const unsigned long long hi = V->hi, tail = V->tail;
        int status = kRunning;
        if (V->overflow) {
            status = kNeedMem;
        } else if (tail == hi) {
            status = kDone;
        } else {
            const int radius = V->radius + 1;
            const unsigned long long fresh = tail - hi;
            J->layer_sizes[radius] = fresh;
            V->radius = radius;
            V->lo = hi;
            V->hi = tail;
            if (J->max_radius >= 0 && radius >= J->max_radius) status = kTruncRadius;
            else if (J->stop_above > 0 && fresh > J->stop_above) status = kTruncAbove;
            else if (radius + 1 >= J->layers_cap) status = kTruncRadius;
        }
        if (status != kRunning) V->status = status;
    }
    atomicAdd(&ctl->rounds, 1);
    __threadfence();
}

__global__ void __launch_bounds__(kWideBlock, 2)
wide_grow_kernel(WideDev* J, Ctl* ctl, int max_rounds, uint64_t timeout_ns) {
    __shared__ Key128 s_stage[kWideBlock / 32][kWideStage];
    __shared__ WideGen s_gens[kWideSmemGens];
    __shared__ unsigned long long s_lo, s_hi, s_unit;
    __shared__ int s_run;
    const WideGen* gens = J->gens;
    if (J->k <= kWideSmemGens) {
        for (int j = threadIdx.x; j < J->k; j += blockDim.x) s_gens[j] = J->gens[j];
        __syncthreads();
        gens = s_gens;
    }
    const int lane = threadIdx.x & 31;
    Key128* buf = s_stage[threadIdx.x >> 5];
    unsigned nbar = 0;                      // grid barriers this block has passed
    for (int round = 0; round < max_rounds; ++round) {
        if (threadIdx.x == 0) {
            s_run = ld_relaxed_int(&J->status) == kRunning;
            s_lo = ld_relaxed_ull(&J->lo);
            s_hi = ld_relaxed_ull(&J->hi);
        }
        __syncthreads();
        if (!s_run) break;
        const unsigned long long lo = s_lo, hi = s_hi;
        const unsigned long long total = (hi - lo + 31) >> 5;
        const unsigned long long ub = total * blockIdx.x / gridDim.x, ue = total * (blockIdx.x + 1) / gridDim.x;
        if (threadIdx.x == 0) s_unit = ub;
        __syncthreads();
        int cnt = 0;
        for (;;) {
            unsigned long long u = 0;
            if (lane == 0) u = atomicAdd(&s_unit, 1ull);
            u = __shfl_sync(0xffffffffu, u, 0);
            if (u >= ue) break;
            wide_unit(J, gens, lo + (u << 5) + lane, hi, buf, cnt, lane);
            if (__any_sync(0xffffffffu, ld_relaxed_int(&J->overflow))) break;
        }
        wide_flush(buf, cnt, J, lane);
        unsigned long long word = 0;
        const int arrive = grid_arrive(ctl, timeout_ns, word, nbar++);
        if (arrive < 0) return;
        if (arrive == 1) {
            if (threadIdx.x == 0) wide_close(J, ctl);
            grid_release(ctl, word, 0);
        }
    }
}

__global__ void wide_init_kernel(WideDev* J) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    J->keys[0] = J->start;
    table_insert128(J->table, J->table_mask, J->start, kWideMaxProbe);
    J->layer_sizes[0] = 1;
    J->lo = 0;
    J->hi = 1;
    J->tail = 1;
    J->radius = 0;
    J->overflow = 0;
    J->status = J->max_radius == 0 ? kTruncRadius : kRunning;
}

// Re-insert keys[0, count) (tags stripped) into a cleared table after the key array grew.
__global__ void wide_rebuild_kernel(const Key128* keys, unsigned long long count, Key128* table,
                                    uint64_t mask, int tagged, int* err) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < count;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        Key128 kk = keys[i];
        if (tagged) kk.hi &= kTag124;
        if (table_insert128(table, mask, kk, kWideMaxProbeRebuild) < 0) atomicExch(err, CG_EDEVICE);
    }
}

}  // namespace

int wide_max_grid(int device) {
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wide_grow_kernel, kWideBlock, 0) != cudaSuccess)
        return 0;
    return sms * per_sm;
}

cudaError_t launch_wide_init(WideDev* d, cudaStream_t st) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    wide_init_kernel<<<1, 32, 0, st>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_wide_grow(WideDev* d, Ctl* ctl, int grid, int max_rounds, uint64_t timeout_ns,
                             cudaStream_t st) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kWideBlock);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, wide_grow_kernel, d, ctl, max_rounds, timeout_ns);
}

cudaError_t launch_wide_rebuild(const Key128* keys, unsigned long long count, Key128* table, uint64_t mask,
                                int tagged, int* d_err, int grid, cudaStream_t st) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    if (count == 0) return cudaSuccess;
    wide_rebuild_kernel<<<grid, 256, 0, st>>>(keys, count, table, mask, tagged, d_err);
    return cudaGetLastError();
}

}  // namespace cg
