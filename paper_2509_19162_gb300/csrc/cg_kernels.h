// Launchers of the growth kernels (defined in the .cu files of this directory).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "cg_internal.h"

namespace cg {

// hash strategy (hash_path.cu)
int hash_grow_block();
// Co-resident blocks of the persistent kernel variant (multi: launches of several jobs).
int hash_grow_max_grid(int device, int ilp, bool multi = false);
// Initialise every job (only_fresh = 0) or only the jobs whose status is kFresh, then lay out
// the first round's work over all running jobs.
cudaError_t launch_init_jobs(JobDev* d_jobs, int njobs, unsigned long long* d_ubeg, Ctl* d_ctl,
                             cudaStream_t st, int only_fresh = 0);
cudaError_t launch_resume_units(JobDev* d_jobs, int njobs, unsigned long long* d_ubeg, Ctl* d_ctl,
                                cudaStream_t st);
// n > 0: the jobs' n, for the kernel variants compiled per n (a single rank-bitmap job).
// d_adm (device): a batch launch that admits the jobs as the window allows (AdmitDev); ubeg then
// holds max_active + 1 entries and launch_admit_first must run first (on a zeroed control block).
// host_job: for a launch of one job, the host's copy of its descriptor (the static fields the
// device copy holds at this launch); the single-job kernels take them as a parameter.  Without
// it one job runs through the kernel for several jobs.
cudaError_t launch_hash_grow(JobDev* d_jobs, int njobs, unsigned long long* d_ubeg, Ctl* d_ctl,
                             int grid, int max_rounds, uint64_t timeout_ns, int ilp,
                             cudaStream_t st, int n = 0, const AdmitDev* d_adm = nullptr,
                             const JobDev* host_job = nullptr);
cudaError_t launch_admit_first(JobDev* d_jobs, unsigned long long* d_ubeg, Ctl* d_ctl,
                               const AdmitDev* d_adm, cudaStream_t st);
cudaError_t launch_rebuild_table(const uint64_t* keys, unsigned long long count, uint64_t* table,
                                 uint64_t mask, uint64_t key_mask, int* d_err, int grid,
                                 cudaStream_t st);
cudaError_t launch_rebuild_bitmap(const uint64_t* keys, unsigned long long count, unsigned* bm,
                                  uint64_t words, int n, int* d_err, int grid, cudaStream_t st);
cudaError_t launch_expand(const GenSM* d_gens, int k, const uint64_t* in, unsigned long long F,
                          uint64_t* out, int grid, cudaStream_t st);
cudaError_t launch_hash_insert(uint64_t* table, uint64_t mask, const uint64_t* keys,
                               unsigned long long N, uint64_t* out, unsigned long long* count,
                               int* fail, int grid, cudaStream_t st);

// owner partition of a sharded layer step (shard_path.cu): the k F candidates of in[0, F) grouped
// by owner mix64(t) mod P into out (cap keys); d_counts[p] receives owner p's count, d_cursor
// (P entries, scratch) ends at each owner's range end.  d_err set if out is too small.
cudaError_t launch_owner_partition(const GenSM* d_gens, int k, const uint64_t* in, unsigned long long F,
                                   int P, unsigned long long* d_counts, unsigned long long* d_cursor,
                                   uint64_t* out, unsigned long long cap, int* d_err, int grid,
                                   cudaStream_t st);

// two-word keys (wide_path.cu): one growth of vectors of more than 64 bits
int wide_max_grid(int device);
cudaError_t launch_wide_init(WideDev* d, cudaStream_t st);
cudaError_t launch_wide_grow(WideDev* d, Ctl* ctl, int grid, int max_rounds, uint64_t timeout_ns,
                             cudaStream_t st);
cudaError_t launch_wide_rebuild(const Key128* keys, unsigned long long count, Key128* table, uint64_t mask,
                                int tagged, int* d_err, int grid, cudaStream_t st);

// sweep strategy (sweep_path.cu)
int sweep_max_grid(int device, int ilp, int n);
cudaError_t launch_sweep_init(SweepDev* d, cudaStream_t st);
// Block order of a sweep round (CG_OPT_SWEEP_ORDER): auto (rank order for layers whose nonempty
// blocks fill at least a quarter of S_n when the visited bitmap is larger than L2, else order of
// discovery), discovery, rank.
constexpr int kSweepOrderAuto = 0, kSweepOrderList = 1, kSweepOrderRank = 2;
cudaError_t launch_sweep_grow(SweepDev* d, Ctl* ctl, int grid, int max_rounds, uint64_t timeout_ns,
                              int ilp, int n, int order, cudaStream_t st);
// Unrank the states of one layer (bitmap F, block list L[0, nlist)) into out[0, cap); *count
// (zeroed by the caller) receives the number of states.
cudaError_t launch_sweep_export(const unsigned* F, const unsigned* L, unsigned long long nlist, int n,
                                uint64_t* out, unsigned long long cap, unsigned long long* count,
                                int grid, cudaStream_t st);
// Position-major Lehmer rank of packed permutations, and its inverse.
cudaError_t launch_pos_rank(const uint64_t* keys, unsigned long long count, int n, uint64_t* out,
                            int grid, cudaStream_t st);
cudaError_t launch_pos_unrank(const uint64_t* ranks, unsigned long long count, int n, uint64_t* out,
                              int grid, cudaStream_t st);

}  // namespace cg
