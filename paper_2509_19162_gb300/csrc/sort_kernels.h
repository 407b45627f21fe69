// Launchers of the sort strategy's kernels (sort_path.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "cg_internal.h"

namespace cg {

// Device scratch of the sort primitives for up to n keys, carved from one caller buffer:
// a ping-pong key buffer, the digit histograms of every pass, and the control words and
// look-back descriptors that the single-pass (per digit) scatter and the compaction chain
// their tiles with.
struct SortScratch {
    uint64_t* keys_tmp;                 // n keys
    int* err;                           // 0 or a CG_E* code (cleared by the caller)
    unsigned long long* ghist;          // kSortMaxPasses x 256 digit counts
    unsigned* ctl;                      // tile tickets: [p] pass p, [15] the compaction
    unsigned long long* desc;           // look-back descriptors: tiles x 256
    unsigned long long n;
    size_t reset_bytes;                 // bytes from ghist that a sort clears (to the end)
};

constexpr int kSortMaxPasses = 8;

size_t sort_scratch_bytes(unsigned long long n);
SortScratch carve_sort_scratch(void* scratch, unsigned long long n);

// Candidates generated on the fly: candidate i of [0, k F) is generator i / F applied to
// frontier[i % F] (expand fused into the sort's first reads).
struct ExpandSrc {
    const GenSM* gens;
    int k;
    const uint64_t* frontier;
    unsigned long long F;
};

cudaError_t launch_expand_all(const GenSM* d_gens, int k, const uint64_t* in, unsigned long long F,
                              uint64_t* out, cudaStream_t st);
// Sort keys[0, n) ascending on their bits [lo, bits) (higher bits zero; lo > 0 only when the
// bits below lo are decided by the others, as the element at position 0 of a permutation is),
// in place.
cudaError_t launch_radix_sort(uint64_t* keys, unsigned long long n, int bits, const SortScratch& s,
                              cudaStream_t st, int lo = 0);
// Generate the k F candidates of src and write them sorted to out (k F keys, not s.keys_tmp).
cudaError_t launch_expand_sort(const ExpandSrc& src, uint64_t* out, int bits, const SortScratch& s,
                               cudaStream_t st, int lo = 0);
// out = the keys of sorted a that are first of their run and absent from every sorted b_j (at
// most 2 sets), in order; *d_count = their number.
cudaError_t launch_unique_difference(const uint64_t* a, unsigned long long na, const uint64_t* const* bs,
                                     const unsigned long long* nbs, int nb_sets, uint64_t* out,
                                     unsigned long long* d_count, const SortScratch& s, cudaStream_t st);

// 8-bit LSD passes over key bits [lo, bits).
int sort_passes(int bits, int lo = 0);
// Digit histograms (s.ghist[p * 256 + d], every pass p, digit p at bit lo + 8 p) of the
// candidates of src.
cudaError_t launch_candidate_hist(const ExpandSrc& src, int bits, const SortScratch& s, cudaStream_t st,
                                  int lo = 0);
// The candidates of src whose digit at `shift` lies in [d0, d1), appended to out (cap keys) in no
// particular order; *d_count receives their number (d_err set if out is too small).
cudaError_t launch_expand_filter(const ExpandSrc& src, int shift, unsigned d0, unsigned d1, uint64_t* out,
                                 unsigned long long cap, unsigned long long* d_count, int* d_err,
                                 cudaStream_t st);
// keys[i] &= mask, i < n.
cudaError_t launch_mask_keys(uint64_t* keys, unsigned long long n, uint64_t mask, cudaStream_t st);

// ---- small layer steps in one block ----------------------------------------------------------
// Layer steps whose k F_r candidates, F_r and F_{r-1} are at most kSmallStep run back to back by
// one block in shared memory (candidates generated, bitonic-sorted, first of run and absent from
// L_r and L_{r-1} kept, compacted in order into the third layer buffer), with the stop tests of
// the host's loop, until a step is too large or the growth stops: one launch and no host round
// trip for the first and last layers of a growth.
constexpr int kSmallStep = 4096;
constexpr int kSmallMaxSteps = 256;

struct SmallSteps {                 // device memory, read and written by the kernel
    int cur, prev;                  // layer buffers of L_r and L_{r-1} (the third receives L_{r+1})
    int radius;
    int status;                     // kRunning: stopped at a step too large for one block
    unsigned long long Fcur, Fprev;
    int nsteps;                     // steps run by this launch
    int pad;
    unsigned long long sizes[kSmallMaxSteps];   // |L_{r+1}| of each of them
};

// L[3]: the three layer buffers (each of at least kSmallStep keys); layers_done: layer sizes
// recorded before this launch (the layer array holds at most kMaxLayers).
cudaError_t launch_small_steps(const GenSM* d_gens, int k, uint64_t* L0, uint64_t* L1, uint64_t* L2,
                               int max_radius, unsigned long long stop_above, int layers_done,
                               SmallSteps* d_state, cudaStream_t st);

}  // namespace cg
