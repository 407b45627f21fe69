/*
 * cg_growth.h -- C ABI of the GB300 (sm_103a) Cayley-graph growth library.
 *
 * The library computes the growth function of a permutation Cayley graph: the sizes of the
 * spheres S_r = { v : d(v, e) = r } around the identity e, r = 0..diameter or up to a radius
 * limit (Section 2.1, Definition "Growth"; diameter = number of layers - 1).  d is the word
 * metric of the generating set.  Each layer step applies every generator to every frontier
 * state, deduplicates the results and removes states already seen (Sections 3.1.2-3.1.3: all
 * of the paper's growth algorithms are breadth-first searches that differ in data layout).
 *
 * Conventions shared by every entry point:
 *  - A permutation of {0..n-1}, n <= 16, is given in one-line form as n bytes p[0..n-1].
 *    A generator g acts on a state s by gather: t[i] = s[g[i]].  (The growth is the same
 *    under scatter or left multiplication; see the readings in the design notes.)
 *  - A state is stored as a packed key: uint64 with element i in bits [4i, 4i+4).
 *  - Return codes: 0 = success, > 0 = informational (the run stopped early, every reported
 *    layer is exact), < 0 = error (nothing reported may be trusted).  cg_strerror() names
 *    every code.
 *  - "device pointer" arguments are CUDA global-memory addresses on the current device;
 *    "host pointer" arguments are ordinary (pageable or pinned) host memory.
 *  - A stream argument is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *  - No entry point takes ownership of caller memory.
 */
#ifndef CG_GROWTH_H
#define CG_GROWTH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------------------- */
#define CG_OK               0
#define CG_TRUNC_RADIUS     1  /* stopped at max_radius; layers 0..max_radius are exact    */
#define CG_TRUNC_MEMCAP     2  /* stopped because the next layer did not fit in mem_cap      */
#define CG_TRUNC_ABOVE      3  /* stopped after the first layer larger than stop_above       */
#define CG_EINVAL          -1  /* bad argument: n not in [1,16], k < 1, a row that is not a
                                  permutation, a null pointer, or an output array too small  */
#define CG_ENOTCLOSED      -2  /* inverse_closed = 1 but the set is not closed under inverse */
#define CG_ENOMEM          -3  /* a device allocation failed                                 */
#define CG_ECUDA           -4  /* a CUDA runtime call failed                                 */
#define CG_EDEVICE         -5  /* a kernel reported an internal error (error word set)       */
#define CG_ETIMEOUT        -6  /* a bounded device-side wait ran out; the kernel returned    */
#define CG_ETOOBIG         -7  /* the problem exceeds the fixed scratch of
                                  cg_growth_run_noalloc (CG_NOALLOC_MAX_*)                    */

/* ---- strategies (cg_growth_set_option(h, CG_OPT_STRATEGY, ...)) --------------------- */
#define CG_STRATEGY_AUTO    0  /* library chooses: BITMAP when eligible, SWEEP when the states
                                  of BITMAP do not fit but the sweep's bitmaps do, else HASH  */
#define CG_STRATEGY_HASH    1  /* visited open-addressing hash set; any generating set        */
#define CG_STRATEGY_SORT    2  /* sorted layers, radix sort + unique + merge-path difference
                                  against layers r and r-1; inverse-closed sets only          */
#define CG_STRATEGY_BITMAP  3  /* visited set = one bit per element of S_n, indexed by Lehmer
                                  rank; any generating set; needs n <= 14 and a bitmap of at
                                  most half of mem_cap and 16 GiB (else CG_EINVAL at run).
                                  AUTO picks it when it fits and the group fills at least 1/512
                                  of S_n, else HASH                                           */
#define CG_STRATEGY_SWEEP   4  /* bitmask BFS (Section 3.1.3): the visited set and two
                                  layers are bitmaps over the n! Lehmer ranks (3 bits per
                                  element of S_n, nothing per state), so the whole of S_14 fits
                                  in 33.4 GB; any generating set; start with distinct values;
                                  needs n <= 14 and the bitmaps within mem_cap (else CG_EINVAL
                                  at run)                                                      */

/* ---- options ------------------------------------------------------------------------ */
#define CG_OPT_STRATEGY     1  /* one of CG_STRATEGY_*                                        */
#define CG_OPT_STOP_ABOVE   2  /* > 0: stop after the first layer with more states than this */
#define CG_OPT_KEEP_LAST    3  /* 1: keep the last layer's states for cg_growth_last_layer    */
#define CG_OPT_GRID         4  /* > 0: blocks of the persistent launch (capped at co-residency);
                                  0: library chooses                                          */
#define CG_OPT_ILP          5  /* 1..4: generators whose probe sequences one thread advances
                                  together, probing one slot per step; 9..12: the same with
                                  ILP = value - 8, probing a whole 32-byte sector per step;
                                  0: library chooses                                          */
#define CG_OPT_SWEEP_ORDER  9  /* CG_STRATEGY_SWEEP: order in which a round takes the layer's
                                  nonempty 1024-rank blocks.  0 = auto (rank order when they
                                  fill at least a quarter of S_n and the visited bitmap, n!/8
                                  bytes, is larger than L2; else the order of discovery);
                                  1 = order of discovery; 2 = rank order.  The layers are the
                                  same in every order                                          */
/* batch options (cg_batch_set_option; CG_OPT_ILP and CG_OPT_GRID apply there too, 1..4)      */
#define CG_OPT_BATCH_WAVE_L2 6 /* cap on the summed visited-set bytes of one launch:
                                  0 = half of L2 (default), -1 = none                          */
#define CG_OPT_BATCH_VISITED 7 /* CG_STRATEGY_AUTO (rank bitmap for dense groups of n <= 12),
                                  CG_STRATEGY_HASH (hash tables only) or CG_STRATEGY_BITMAP
                                  (rank bitmap whenever n <= 12 and it fits)                   */
#define CG_OPT_GRAPH         8 /* 1 (default): when the batch's buffers stay allocated
                                  between runs, capture a whole run as a CUDA graph at its
                                  first run and replay it afterwards; 0: plain launches       */
#define CG_OPT_BATCH_ACTIVE 10 /* most jobs a batch launch grows at once (0 = min(jobs, 2048)) */
#define CG_OPT_UNIT         11 /* batch: frontier states per warp work unit, 32 x {1, 2, 4, 8}
                                  (4 = default)                                                */

/* ---- device memory ------------------------------------------------------------------ */
/*
 * Optional allocator used for every device buffer the library owns (for example PyTorch's
 * caching allocator).  alloc(bytes, stream, ctx) returns a device pointer aligned to 256 bytes
 * or NULL; free(p, stream, ctx) releases it.  Passing NULL for both restores the default
 * (cudaMallocAsync from a private memory pool that keeps freed memory cached).
 * Not thread-safe with concurrent create/run calls; set it once at start-up.
 */
typedef void* (*cg_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*cg_free_fn)(void* p, void* stream, void* ctx);
int cg_set_allocator(cg_alloc_fn alloc, cg_free_fn free_fn, void* ctx);

/* ---- single growth job -------------------------------------------------------------- */
typedef struct cg_growth* cg_growth_t;

/*
 * Create a growth job for the subgroup generated by gens (Section 2.1, Def. "Growth": the job's
 * result is the sphere sizes of the Cayley graph of <gens> around the identity, or around a
 * start vector, cg_growth_set_start).
 *   n, k            permutation length (1..128) and number of generators (>= 1).  From the
 *                   identity n <= 16 packs 4 bits per element in one 64-bit key and
 *                   17 <= n <= 25 packs 5 bits per element in two words (CG_EINVAL at run
 *                   beyond, or when a generator has more than 32 distinct offsets i - g[i]);
 *                   longer vectors grow only from a start vector.
 *   gens            host pointer, k*n bytes, row-major: gens[j*n + i] = image of i under
 *                   generator j.  Copied; the caller keeps ownership.  Identity rows are
 *                   ignored, duplicate rows are allowed.
 *   inverse_closed  1: the caller states the set is closed under inverse (checked on the
 *                   host: CG_ENOTCLOSED if false); this allows the two-layer strategies.
 *                   0: directed growth (full visited set).
 *   max_radius      < 0: unlimited; otherwise stop after layer max_radius.
 *   mem_cap         upper bound in bytes on the device memory the job may own (0 = 160 GiB).
 *   out             receives the handle.
 * The handle owns all device buffers; nothing is allocated until the first run.
 * Errors: CG_EINVAL, CG_ENOTCLOSED.
 */
int cg_growth_create(int n, int k, const uint8_t* gens, int inverse_closed, int max_radius,
                     uint64_t mem_cap, cg_growth_t* out);

/*
 * Grow from a central state instead of the identity (Section 3.1.2: a Schreier coset graph is
 * given by a vector whose stabiliser is the subgroup; its growth is that of the vector's orbit,
 * Section 5.2).  start: host pointer, n values in 0..15, repeats allowed; copied.  NULL restores
 * the identity.  States are packed with the narrowest element width w of 1, 2, 4 bits that
 * holds the values (4 for a permutation of n <= 16), in one 64-bit key when n * w <= 64 and
 * every generator has a one-word form, else in two words (n * w <= 128: 4-bit vectors up to
 * n = 32, 2-bit up to 64, binary up to 128; CG_EINVAL beyond).  Two-word keys run the hash
 * strategy only (AUTO or HASH; others fail at run with CG_EINVAL).  A start with repeated values
 * needs the HASH or SORT strategy (AUTO picks HASH; BITMAP then fails at run with CG_EINVAL).
 * A start whose values are all equal is fixed by every generator: its growth is {1}.  Releases
 * buffers sized for an earlier start.  Errors: CG_EINVAL (also a generator that fits neither
 * the shift-and-mask form, at most 16 distinct offsets in one word or 32 in two, nor the
 * reversal of one contiguous range).
 */
int cg_growth_set_start(cg_growth_t h, const uint8_t* start);

/* Set an option (CG_OPT_*) before cg_growth_run.  Errors: CG_EINVAL. */
int cg_growth_set_option(cg_growth_t h, int option, int64_t value);

/*
 * Run the growth on the caller's stream and wait for it (the stream is synchronised before
 * returning).  layer_sizes_out is a host pointer with room for cap entries; on return
 * layer_sizes_out[r] = |S_r| for r = 0..(*num_layers_out - 1), layer_sizes_out[0] = 1.  The
 * sum is the order of the generated subgroup when the growth ran to the end.
 * Returns CG_OK (growth ended: the last layer is the farthest), CG_TRUNC_* (stopped early;
 * every reported layer is exact), or an error.  If cap is too small the call returns
 * CG_EINVAL and writes the number of layers it needs to *num_layers_out.
 * A handle may be run again; each run starts from the identity (or the start vector).
 * The layer step (Sections 3.1.2-3.1.3): every generator applied to every state of layer r,
 * candidates deduplicated and stripped of visited states; the strategy picks the data layout.
 */
int cg_growth_run(cg_growth_t h, void* cuda_stream, uint64_t* layer_sizes_out, int cap,
                  int* num_layers_out);

/*
 * Bits per element of the packed keys of a growth: 4 for permutations, and for a start vector
 * with repeated values the narrowest of 1, 2, 4 that holds its largest value (element i in bits
 * [w i, w i + w)).  Returns 0 for a NULL handle.
 */
int cg_growth_key_width(cg_growth_t h);

/* 64-bit words per packed key: 1, or 2 for keys of more than 64 bits (see cg_growth_set_start
 * and the identity of n > 16); 0 for a NULL handle. */
int cg_growth_key_words(cg_growth_t h);

/*
 * Copy the packed keys of the last reported layer (the antipodes when the growth ended) to
 * host memory keys_out (room for cap keys), in no particular order, element i of a state in
 * bits [w i, w i + w) with w = cg_growth_key_width(h); *count_out receives the layer size.
 * Two-word keys (cg_growth_key_words = 2) take two entries a state, low word first, and cap
 * then counts states (keys_out holds 2 cap words).  Needs CG_OPT_KEEP_LAST = 1 before the run
 * (two-word keys are always kept).  Errors: CG_EINVAL (cap too small: *count_out still
 * written), CG_ECUDA.
 */
int cg_growth_last_layer(cg_growth_t h, uint64_t* keys_out, uint64_t cap, uint64_t* count_out);

/*
 * Measurements of the last cg_growth_run on this handle.  kernel_ms is the summed duration of
 * the layer-step kernel launches, timed with CUDA events recorded on the run's stream around
 * each launch; launches counts every kernel of this library the run launched; h2d_bytes and
 * d2h_bytes count the bytes the run copied between host and device.  Errors: CG_EINVAL.
 */
typedef struct cg_growth_stats {
    double kernel_ms;
    int launches;
    int rounds;                 /* layer steps executed by the device */
    uint64_t h2d_bytes;
    uint64_t d2h_bytes;
    uint64_t state_capacity;    /* states the job's buffers hold */
    uint64_t table_slots;       /* visited-table slots (hash strategy) */
    int strategy_used;          /* CG_STRATEGY_HASH, _SORT, _BITMAP or _SWEEP: what the run used */
    int probe_variant;          /* kernel variant of the run (generators probed together) */
    int switched_to_sort;       /* 1: AUTO, inverse-closed set: the states stored by the hash or
                                   bitmap path outgrew mem_cap at layer sort_from + 1, and the
                                   sorted layer step (which keeps only the last two layers) took
                                   the growth on from layer sort_from; strategy_used is then
                                   CG_STRATEGY_SORT.  0: no switch                              */
    int sort_from;
} cg_growth_stats;
int cg_growth_get_stats(cg_growth_t h, cg_growth_stats* out);

/* Order of the group generated by the handle's generators (host Schreier-Sims). */
uint64_t cg_growth_group_order(cg_growth_t h);

/* Release the handle and every device buffer it owns (the layers, visited set and scratch of
 * the growth of Sections 2.1 and 3.1.2-3.1.3; buffers from a user allocator go back through its
 * free callback).  NULL is accepted.  Returns CG_OK. */
int cg_growth_destroy(cg_growth_t h);

/* Human-readable name of a return code (static string). */
const char* cg_strerror(int code);

/* Name of the last CUDA error that a call on this thread reported as CG_ECUDA or CG_ENOMEM,
 * with the library source line that saw it ("" if none); valid until the next call on this
 * thread. */
const char* cg_last_error_detail(void);

/* ---- batched growth of many independent jobs ------------------------------------------ */
typedef struct cg_batch* cg_batch_t;

/*
 * Create a batch of njobs independent growth jobs that run together in one persistent
 * launch per call.  Job j has permutation length n[j], k[j] generators at
 * gens + gens_offset[j] (host, k[j]*n[j] bytes row-major), inverse_closed[j] and
 * max_radius[j] (< 0: unlimited).  mem_cap bounds the device memory of the whole batch
 * (0 = 160 GiB).  Errors: CG_EINVAL, CG_ENOTCLOSED (names no job; check each set first).
 */
int cg_batch_create(int njobs, const int* n, const int* k, const uint8_t* gens,
                    const uint64_t* gens_offset, const int* inverse_closed,
                    const int* max_radius, uint64_t mem_cap, cg_batch_t* out);

/*
 * Run every job of the batch to its end on the caller's stream and wait for it.
 *   layer_sizes_out  host, njobs*cap entries: job j's growth at [j*cap, j*cap + layers[j]).
 *   num_layers_out   host, njobs entries.
 *   status_out       host, njobs entries: each job's own return code (CG_OK, CG_TRUNC_*, or
 *                    an error); may be NULL.
 * Returns CG_OK when every job ended or stopped on its limits, otherwise the first error.
 * If cap is too small for some job the call returns CG_EINVAL.
 */
int cg_batch_run(cg_batch_t b, void* cuda_stream, uint64_t* layer_sizes_out, int cap,
                 int* num_layers_out, int* status_out);

/*
 * Cap on the summed visited-set bytes (rank bitmaps and hash tables) of the jobs that one launch
 * of cg_batch_run grows together.  Every candidate state costs one random access to its job's
 * visited set; while the sets of the running jobs fit in L2 those accesses stay on chip, so the
 * batch is split into launches ("waves") whose sets fit.  A job whose set alone exceeds the cap
 * does not count against it.  bytes = 0: half of the device's L2 (the default);
 * UINT64_MAX: no cap (waves bounded by the memory budget only).  No paper counterpart: the
 * paper grows one graph at a time.  Errors: CG_EINVAL.
 */
int cg_batch_set_wave_l2(cg_batch_t b, uint64_t bytes);

/*
 * Set a batch option (CG_OPT_ILP, CG_OPT_GRID, CG_OPT_BATCH_WAVE_L2, CG_OPT_BATCH_VISITED,
 * CG_OPT_GRAPH) before cg_batch_run.  The batch is planned at its first run: visited-set kind per
 * job, waves, and, when every wave fits mem_cap together, device buffers kept between runs.
 * Changing an option (other than CG_OPT_GRAPH) drops the plan.  Errors: CG_EINVAL.
 */
int cg_batch_set_option(cg_batch_t b, int option, int64_t value);

/* Measurements of the last cg_batch_run (as cg_growth_get_stats).  Errors: CG_EINVAL. */
int cg_batch_get_stats(cg_batch_t b, cg_growth_stats* out);

/* Release the batch and its device buffers.  NULL is accepted. */
int cg_batch_destroy(cg_batch_t b);

/* ---- serving: continuous batching of growth jobs ---------------------------------------- */
/*
 * A request loop for many growth jobs of different n, generator sets and radius caps.  Jobs are
 * queued by cg_server_submit (host only, no GPU work) and admitted into one of max_slots
 * device slots, first come first served, while the sum of their predicted device memory stays
 * within mem_budget.  The prediction bounds the states a job can reach by its radius cap
 * (sphere r of an out-degree-k graph holds at most k (k-1)^(r-1) states when the set is
 * inverse-closed, k^r otherwise, and never more than the group order), stored with the cheaper
 * visited set (hash table, or the rank bitmap for n <= 14), capped at job_mem_cap bytes per job,
 * the job's share of the budget (a job that needs more stops with CG_TRUNC_MEMCAP; its reported
 * layers are exact).  A job predicted to reach at least CG_SERVER_SOLO_STATES states fills the
 * GPU by itself: when it reaches the head of the queue, cg_server_step grows it alone with the
 * single-job kernels
 * (same visited set and share, so the same layers) before the batched launch.  Each
 * cg_server_step admits what fits, then runs up to rounds_per_step layer steps of
 * every admitted job in one persistent launch on the caller's stream (jobs' states stay on the
 * device between steps), waits for it, and retires the jobs that ended, releasing their slot
 * and memory.  Results are the same as cg_growth_run's for the same job with the same memory.
 *   cg_server_create   mem_budget 0 = 160 GiB; job_mem_cap 0 = mem_budget / 64 (at least 1 MiB),
 *                      so that at least 64 jobs of any size can run together.  Errors: CG_EINVAL.
 *   cg_server_submit   arguments as cg_growth_create; *job_id_out receives the job's id.
 *                      Errors: CG_EINVAL (also more than 128 distinct generators), CG_ENOTCLOSED.
 *   cg_server_step     *active_out: jobs admitted after the step; *finished_out: jobs that
 *                      ended in this call.  Errors: CG_ENOMEM, CG_ECUDA, CG_ETIMEOUT.
 *   cg_server_finished pops up to cap ids of ended jobs (in ending order) into ids_out.
 *   cg_server_result   copies an ended job's growth (its own return code in *status_out) and
 *                      forgets it; CG_EINVAL with *num_layers_out = -1 if it has not ended, or
 *                      with the needed size if cap is too small.
 *   cg_server_load     jobs queued, jobs admitted, device bytes admitted jobs hold.
 *   cg_server_predict  host only (no GPU work, no server needed): the admission plan of a job
 *                      under the per-job share job_mem_cap (> 0): *states_out the predicted
 *                      states up to its radius cap, *granted_out the states it may store (less
 *                      than the prediction: the job may stop with CG_TRUNC_MEMCAP), *bytes_out
 *                      the device bytes it is admitted with, *visited_out its visited set
 *                      (CG_STRATEGY_HASH or CG_STRATEGY_BITMAP).  Any output may be NULL.
 *                      Errors: CG_EINVAL, CG_ENOTCLOSED.
 */
#define CG_SERVER_SOLO_STATES (1u << 24)
typedef struct cg_server* cg_server_t;
int cg_server_create(uint64_t mem_budget, int max_slots, uint64_t job_mem_cap, int rounds_per_step,
                     cg_server_t* out);
int cg_server_submit(cg_server_t s, int n, int k, const uint8_t* gens, int inverse_closed,
                     int max_radius, uint64_t* job_id_out);
int cg_server_predict(int n, int k, const uint8_t* gens, int inverse_closed, int max_radius,
                      uint64_t job_mem_cap, uint64_t* states_out, uint64_t* granted_out,
                      uint64_t* bytes_out, int* visited_out);
int cg_server_step(cg_server_t s, void* cuda_stream, int* active_out, int* finished_out);
int cg_server_finished(cg_server_t s, uint64_t* ids_out, int cap, int* count_out);
int cg_server_result(cg_server_t s, uint64_t job_id, uint64_t* layers_out, int cap,
                     int* num_layers_out, int* status_out);
int cg_server_load(cg_server_t s, int* queued, int* active, uint64_t* used_bytes);
int cg_server_destroy(cg_server_t s);

/* ---- growth without allocation ------------------------------------------------------- */
/*
 * The paper has no counterpart to this entry point; it exists for callers that cannot allocate
 * device memory when they need a growth -- code inside a memory-capped sandbox or a
 * pre-reserved pool, a latency-critical process that forbids cudaMalloc (which can synchronise
 * the device) after start-up, or a plugin whose host application owns every allocation.
 *
 * cg_growth_run_noalloc computes the same growth as cg_growth_create + cg_growth_run +
 * cg_growth_destroy (hash strategy, same kernels) but calls no cudaMalloc, cudaFree or other
 * allocating routine.  Its buffers live in one fixed device array inside the library
 * (about 24.2 MiB: CG_NOALLOC_MAX_STATES states plus a visited table of twice that many
 * slots), which every GPU that loads the library holds until the process exits.
 *   n, k, gens, inverse_closed, max_radius   as for cg_growth_create (gens: host pointer).
 *   cuda_stream                              stream to run on; synchronised before returning.
 *   layer_sizes_out, cap, num_layers_out     as for cg_growth_run (host pointers).
 * Limits: at most CG_NOALLOC_MAX_GENS distinct non-identity generators (identity rows and
 * repeated rows are dropped first, as cg_growth_create does), and the growth may visit at most
 * CG_NOALLOC_MAX_STATES states (for a complete growth: the group order); beyond either the
 * call returns CG_ETOOBIG and reports nothing.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress)
 * and caches it; make that first call before any stream capture on that device.  The cached
 * address does not survive cudaDeviceReset: do not call this entry point on a device after
 * resetting it in the same process.
 * All calls share the array, which keeps the last call's contents; each call clears what
 * must start empty.  Calls are serialised on the host and wait for their stream, so they do
 * not overlap; anything else that touched the array while a call runs would race with it.
 * Returns the same codes as cg_growth_run, plus CG_ETOOBIG.
 */
#define CG_NOALLOC_MAX_STATES (1u << 20)
#define CG_NOALLOC_MAX_GENS   256
int cg_growth_run_noalloc(int n, int k, const uint8_t* gens, int inverse_closed, int max_radius,
                          void* cuda_stream, uint64_t* layer_sizes_out, int cap,
                          int* num_layers_out);

/* ---- sharded layer step (one graph over P ranks, one exchange per layer) ------------------ */
/*
 * The BFS layer step (Sections 3.1.2-3.1.3) split over P ranks by an owner hash: state t
 * belongs to rank owner(t) = mix64(t) mod P (mix64: the 64-bit MurmurHash3 finaliser of the
 * packed key).  Each rank expands its share of layer r, sends every candidate to its owner (one
 * all-to-all of packed keys), and each owner keeps the candidates absent from its share of the
 * visited states (cg_hash_insert); the new shares form layer r+1, whose size is the sum over
 * ranks (one all-reduce).  The exchange itself is the caller's (the Python driver uses
 * torch.distributed: NCCL on GPUs).
 *
 * cg_shard_owner    host only: owner(key) for P ranks (P >= 1), or CG_EINVAL.
 * cg_shard_expand   expand frontier[0, F) (device, packed untagged keys, n <= 16) by the k
 *                   generators (host, k*n bytes as for cg_growth_create, copied) and write the
 *                   k*F candidates to out (device, cap >= k*F keys) grouped by owner: owner p's
 *                   candidates are out[o_p, o_p + counts_out[p]), o_p = sum of the counts before
 *                   p, in no particular order.  counts_out: host, P entries.  Waits for the
 *                   stream.  Errors: CG_EINVAL (bad rows, P not in [1, 4096], cap too small),
 *                   CG_ENOMEM, CG_ECUDA.
 */
int cg_shard_owner(uint64_t key, int P);
int cg_shard_expand(int n, int k, const uint8_t* gens, const uint64_t* frontier, uint64_t F, int P,
                    uint64_t* out, uint64_t cap, uint64_t* counts_out, void* cuda_stream);

/* ---- step-level kernels (device pointers, asynchronous on the given stream) ----------- */

/*
 * Expand (one layer step's neighbour generation): out[j*F + i] = gens[j] applied to
 * frontier[i] by gather, for i < F, j < k.  frontier and out are device pointers (out has
 * k*F keys); gens is a host pointer (k*n bytes).  Errors: CG_EINVAL, CG_ECUDA.
 */
int cg_expand(int n, int k, const uint8_t* gens, const uint64_t* frontier, uint64_t F,
              uint64_t* out, void* cuda_stream);

/*
 * Insert-if-absent of N keys into an open-addressing table (linear probing, empty slot =
 * 0xFFFFFFFFFFFFFFFF, so that key must not be inserted).  table: device, `slots` entries,
 * slots a power of two, initialised with cg_hash_clear.  Keys not yet present are appended,
 * once each, to new_out (device, room for N keys, in no particular order) and their number is
 * written to *new_count (device uint64, overwritten).  Concurrent duplicate keys in the input
 * are inserted once.  The table must keep at least one empty slot; a probe sequence longer
 * than the table sets *new_count to UINT64_MAX.  Errors: CG_EINVAL, CG_ECUDA.
 */
int cg_hash_insert(uint64_t* table, uint64_t slots, const uint64_t* keys, uint64_t N,
                   uint64_t* new_out, uint64_t* new_count, void* cuda_stream);

/*
 * Radix sort + unique (the sort strategy's dedup step).  keys: device, n uint64 values whose bits
 * at and above key_bits are zero (packed keys of n-element permutations have key_bits = 4n);
 * sorted ascending in place (LSD radix sort, 8-bit digits, one stable single-sweep pass per
 * digit with a decoupled look-back per digit value).  The distinct values,
 * ascending, are written to out (device, room for n) and their number to *d_count (device
 * uint64).  scratch: device buffer of at least cg_sort_unique_scratch_bytes(n) bytes, owned by
 * the caller, contents undefined afterwards.  Asynchronous on the stream.
 * Errors: CG_EINVAL, CG_ECUDA.
 */
size_t cg_sort_unique_scratch_bytes(uint64_t n);
int cg_sort_unique(uint64_t* keys, uint64_t n, int key_bits, uint64_t* out, uint64_t* d_count,
                   void* scratch, size_t scratch_bytes, void* cuda_stream);

/*
 * Set difference (the sort strategy's removal of seen states, K4): out = the distinct
 * values of a that occur in neither b nor c, ascending; *d_count = their number (device uint64).
 * a, b, c: device, each sorted ascending (a may hold duplicates; b or c may be NULL with length
 * 0).  scratch as for cg_sort_unique with n = na.  Asynchronous on the stream.
 * Errors: CG_EINVAL, CG_ECUDA.
 */
int cg_set_difference(const uint64_t* a, uint64_t na, const uint64_t* b, uint64_t nb,
                      const uint64_t* c, uint64_t nc, uint64_t* out, uint64_t* d_count,
                      void* scratch, size_t scratch_bytes, void* cuda_stream);

/* Fill a table of `slots` entries (device) with the empty marker of cg_hash_insert.
 * Errors: CG_EINVAL (NULL table with slots > 0), CG_ECUDA. */
int cg_hash_clear(uint64_t* table, uint64_t slots, void* cuda_stream);

/*
 * Index of a permutation in the sweep strategy's bitmaps (the bitmask BFS of Section 3.1.3):
 * the position-major Lehmer rank  rank(s) = sum_{i=1}^{n-1} d_i * i!,  d_i = #{j < i : s_j < s_i},
 * a bijection from S_n onto 0..n!-1 (identity -> n!-1, full reversal -> 0).
 * cg_perm_rank: keys (device, count packed permutations of 0..n-1, element i in bits 4i..4i+3)
 *   -> ranks (device, count).  A key that is not a permutation of 0..n-1 gives an unspecified
 *   value.
 * cg_perm_unrank: ranks (device, count values < n!) -> keys (device).  A rank >= n! gives an
 *   unspecified key.
 * 1 <= n <= 16.  Asynchronous on the stream.  Errors: CG_EINVAL (n out of range, null pointer
 * with count > 0), CG_ECUDA.
 */
int cg_perm_rank(int n, const uint64_t* keys, uint64_t count, uint64_t* ranks, void* cuda_stream);
int cg_perm_unrank(int n, const uint64_t* ranks, uint64_t count, uint64_t* keys, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* CG_GROWTH_H */
