// Owner partition of a layer step's candidates for a growth sharded over P ranks (one graph, one
// exchange per layer): every rank expands its share of the frontier, and each candidate goes to
// the rank that owns it, owner(t) = mix64(t) mod P, which deduplicates it against its own share
// of the visited states (Sections 3.1.2-3.1.3: the BFS layer step, split by an owner hash).
//
// Two passes over the frontier shard, both expanding it on the fly: the first counts the
// candidates per owner (block histograms in shared memory, one atomic per owner and block), the
// second scatters each candidate into its owner's range at a cursor advanced with one atomic
// per owner and warp (lanes with the same owner found by match_any).  Order within an owner's
// range is not specified: the owner's insert-if-absent does not depend on it.
#include <cstdint>

#include "cg_device.cuh"
#include "cg_kernels.h"

namespace cg {

namespace {

constexpr int kBlock = 256;

__global__ void __launch_bounds__(kBlock)
owner_count_kernel(const GenSM* __restrict__ gens, int k, const uint64_t* __restrict__ in,
                   unsigned long long F, int P, unsigned long long* __restrict__ counts) {
    extern __shared__ unsigned s_cnt[];
    for (int p = threadIdx.x; p < P; p += blockDim.x) s_cnt[p] = 0;
    __syncthreads();
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < F; i += stride) {
        const uint64_t s = in[i];
        for (int j = 0; j < k; ++j) atomicAdd(&s_cnt[mix64(apply_gen(gens[j], s)) % (unsigned)P], 1u);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < P; p += blockDim.x)
        if (s_cnt[p]) atomicAdd(counts + p, (unsigned long long)s_cnt[p]);
}

__global__ void __launch_bounds__(kBlock)
owner_scatter_kernel(const GenSM* __restrict__ gens, int k, const uint64_t* __restrict__ in,
                     unsigned long long F, int P, unsigned long long* __restrict__ cursor,
                     uint64_t* __restrict__ out, unsigned long long cap, int* err) {
    const int lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    // the warp walks its range together, so that match_any sees all lanes
    const unsigned long long first = blockIdx.x * (unsigned long long)blockDim.x + (threadIdx.x & ~31u);
    for (unsigned long long w = first; w < F; w += stride) {
        const unsigned long long i = w + lane;
        const bool valid = i < F;
        const uint64_t s = valid ? in[i] : 0;
        for (int j = 0; j < k; ++j) {
            const uint64_t t = apply_gen(gens[j], s);
            const unsigned owner = valid ? (unsigned)(mix64(t) % (unsigned)P) : 0xFFFFFFFFu;
            const unsigned peers = __match_any_sync(0xffffffffu, owner);
            const int leader = __ffs(peers) - 1;
            unsigned long long base = 0;
            if (valid && lane == leader) base = atomicAdd(cursor + owner, (unsigned long long)__popc(peers));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (valid) {
                const unsigned long long pos = base + __popc(peers & lanemask_lt());
                if (pos < cap) out[pos] = t;
                else atomicExch(err, CG_EDEVICE);
            }
        }
    }
}

__global__ void exclusive_scan_small_kernel(const unsigned long long* counts, int P,
                                            unsigned long long* cursor) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned long long acc = 0;
        for (int p = 0; p < P; ++p) {
            cursor[p] = acc;
            acc += counts[p];
        }
    }
}

}  // namespace

cudaError_t launch_owner_partition(const GenSM* d_gens, int k, const uint64_t* in, unsigned long long F,
                                   int P, unsigned long long* d_counts, unsigned long long* d_cursor,
                                   uint64_t* out, unsigned long long cap, int* d_err, int grid,
                                   cudaStream_t st) {
    (void)cudaGetLastError();   // clear a stale error: the check after the launch is about this one
    cudaError_t e = cudaMemsetAsync(d_counts, 0, sizeof(unsigned long long) * P, st);
    if (e != cudaSuccess || F == 0) return e;
    owner_count_kernel<<<grid, kBlock, sizeof(unsigned) * P, st>>>(d_gens, k, in, F, P, d_counts);
    exclusive_scan_small_kernel<<<1, 32, 0, st>>>(d_counts, P, d_cursor);
    owner_scatter_kernel<<<grid, kBlock, 0, st>>>(d_gens, k, in, F, P, d_cursor, out, cap, d_err);
    return cudaGetLastError();
}

}  // namespace cg
