// Launchers of the sort strategy's kernels (sort_path.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "cg_internal.h"

namespace cg {

// Device scratch of the sort primitives for up to n keys, carved from one caller buffer.
struct SortScratch {
    uint64_t* keys_tmp;                 // n keys (ping-pong buffer, also compaction output)
    unsigned* hist;                     // per-tile digit histograms / scanned offsets
    unsigned long long* scan_desc;      // look-back descriptors of the histogram scan
    unsigned long long* compact_desc;   // look-back descriptors of the compaction
    unsigned char* flags;               // n keep-flags
    unsigned* tickets;                  // [0] scan, [1] compaction
    int* err;                           // 0 or a CG_E* code
    unsigned long long n;
};

size_t sort_scratch_bytes(unsigned long long n);
SortScratch carve_sort_scratch(void* scratch, unsigned long long n);

cudaError_t launch_expand_all(const GenSM* d_gens, int k, const uint64_t* in, unsigned long long F,
                              uint64_t* out, cudaStream_t st);
cudaError_t launch_radix_sort(uint64_t* keys, unsigned long long n, int bits, const SortScratch& s,
                              cudaStream_t st);
cudaError_t launch_unique_difference(const uint64_t* a, unsigned long long na, const uint64_t* const* bs,
                                     const unsigned long long* nbs, int nb_sets, uint64_t* out,
                                     unsigned long long* d_count, const SortScratch& s, cudaStream_t st);

}  // namespace cg
