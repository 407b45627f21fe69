// Internal types shared by the host driver and the kernels of the growth library.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace cg {

constexpr uint64_t kEmpty = ~0ull;   // empty hash slot: never a valid permutation key, n >= 2
constexpr int kMaxN = 16;            // permutations from the identity: 4 bits per element
constexpr int kMaxElems = 64;        // coset vectors: n elements of `width` bits, n * width <= 64
constexpr int kMaxTerms = 16;
constexpr int kMaxLayers = 16384;    // device layer-size array per job

// A generator acting on packed keys (element i in bits [w i, w i + w), w = 1, 2 or 4).
// kind 0, shift-and-mask form: the gather t[i] = s[g[i]] moves element g[i] to element i, a
// rotation of the key by w*(i - g[i]) bits; positions sharing one offset form one term:
// t = OR_t rotl(s, rot[t]) & mask[t].  Cyclic shifts need 2 terms, adjacent transpositions 3,
// any generator <= n, so every generator of n <= 16 elements.
// kind 1, the reversal of the element range [a, b], for long vectors where it would need more
// than kMaxTerms terms: the whole key is bit-reversed (elements land in reverse order, each
// with its bits reversed), the bits of every element put back in order, and the result shifted
// so that element e lands on a + b - e: t = (s & ~mask[0]) | (shift(rev(s), rev_shift) & mask[0]).
// Other generators of more than kMaxTerms offsets are not supported (CG_EINVAL at create).
struct GenSM {
    uint32_t nterms;
    uint32_t inv_tag;   // 1 + index of this generator's inverse in the set (< 15), or 0
    uint8_t kind;
    uint8_t width;      // bits per element
    int16_t rev_shift;  // kind 1: right shift (bits) of the reversed key; negative: left shift
    uint8_t rot[kMaxTerms];
    uint64_t mask[kMaxTerms];
};

// Keys of more than 64 bits (two words): vectors of n elements of w bits with 64 < n w <= 128 --
// coset vectors of 4-bit values up to n = 32, 2-bit up to 64, 1-bit up to 128, and permutations
// of 17..25 elements from the identity with 5-bit elements.  Element i occupies bits
// [w i, w i + w) of the 128-bit number hi:lo.
struct alignas(16) Key128 {
    uint64_t lo, hi;
};

constexpr int kMaxWideElems = 128;
constexpr int kMaxWideTerms = 32;

// A generator acting on two-word keys: kind 0 is the shift-and-mask form over 128 bits (one term
// per distinct element offset, at most kMaxWideTerms); kind 1 the reversal of the element range
// covered by mask (bit-reverse the 128-bit key, put each element's bits back in order, shift by
// rev_shift bits: right if positive).
struct WideGen {
    uint32_t nterms;
    uint32_t inv_tag;   // 1 + index of the inverse (< 15), or 0
    uint8_t kind;
    uint8_t width;
    int16_t rev_shift;
    uint8_t rot[kMaxWideTerms];
    uint64_t mlo[kMaxWideTerms];
    uint64_t mhi[kMaxWideTerms];
};

// One growth with two-word keys (hash strategy): every layer back to back in `keys`, the visited
// set an open-addressing table of 16-byte slots (empty = all ones).  A state found by generator g
// carries the tag (1 + index of g's inverse) in bits 124-127 when n w <= 124.
struct alignas(128) WideDev {
    Key128* keys;
    uint64_t keys_cap;
    Key128* table;
    uint64_t table_mask;
    const WideGen* gens;
    uint64_t* layer_sizes;
    uint64_t stop_above;
    Key128 start;
    int k;
    int n;
    int layers_cap;
    int max_radius;
    int tagged;
    int pad0;
    alignas(128) unsigned long long lo;     // frontier = keys[lo, hi)
    unsigned long long hi;
    unsigned long long tail;
    int radius;
    int status;
    int overflow;
    int pad1;
};

// States found by generator j are stored with tag (1 + index of j's inverse) in key bits 60-63
// when the key leaves them free (n * width <= 60): that inverse leads back to the state's
// parent, in the previous layer, so the expansion skips it.  The visited set always holds
// untagged keys.
constexpr uint64_t kKeyBits60 = (1ull << 60) - 1;

constexpr int kVisitHash = 0;
constexpr int kVisitBitmap = 2;

enum JobStatus : int {
    kRunning = 0,
    kDone = 1,          // empty next layer: growth complete
    kTruncRadius = 2,   // reached max_radius (or the layer array's capacity)
    kTruncAbove = 3,    // recorded the first layer larger than stop_above
    kNeedMem = 4,       // the layer being built did not fit; layers up to `radius` are exact
    kDeviceError = 5,
    kFresh = 6,         // admitted, not yet initialised (the next init launch sets it up)
    kEmptySlot = 7,     // no job in this slot
};

// One growth job of the hash strategy as the persistent kernel sees it.
// 256 bytes: the read-only fields fill the first 128-byte line, the fields updated during a
// run (read by every SM, bumped with atomics) live alone in the second.
struct alignas(128) JobDev {
    // static, written by the host
    uint64_t* keys;            // all layers back to back; layer r = keys[off_r, off_{r+1})
    uint64_t keys_cap;
    uint64_t* table;           // visited set, table_mask + 1 slots
    uint64_t table_mask;
    const GenSM* gens;         // k entries
    uint64_t* layer_sizes;     // device, layers_cap entries; [0] = 1
    uint64_t stop_above;       // 0: none
    int k;
    int n;
    int layers_cap;
    int max_radius;            // < 0: unlimited
    int mode;                  // visited set: 0 hash table, 2 rank bitmap (kVisitBitmap)
    int use_start;             // 1: grow from start_key (a central state), 0: from the identity
    uint64_t bitmap_words;     // bitmap mode: 32-bit words in `table` (ceil(n!/32))
    uint64_t start_key;        // packed start vector when use_start
    int tagged;                // 1: keys leave bits 60-63 free for the parent-edge tag
    int closed;                // 1: every generator's inverse is in the set (every state but
                               //    the start carries a parent-edge tag)
    // dynamic, updated between rounds by block 0
    alignas(128) unsigned long long lo;     // frontier = keys[lo, hi)
    unsigned long long hi;
    unsigned long long tail;   // append cursor (atomic during a round)
    int radius;                // radius of the frontier layer
    int status;                // JobStatus
    int overflow;              // set during a round: keys or table ran out
    int pad;
};
// The round close loads (lo, hi) and (tail, radius | status << 32) as two 16-byte vectors.
static_assert(offsetof(JobDev, lo) % 16 == 0 && offsetof(JobDev, hi) == offsetof(JobDev, lo) + 8,
              "JobDev: lo, hi must form one aligned 16-byte vector");
static_assert(offsetof(JobDev, tail) % 16 == 0 && offsetof(JobDev, radius) == offsetof(JobDev, tail) + 8 &&
                  offsetof(JobDev, status) == offsetof(JobDev, radius) + 4,
              "JobDev: tail, radius, status must form one aligned 16-byte vector");

// One growth of the sweep strategy: the visited set and two layers are bitmaps over the
// position-major Lehmer ranks 0..n!-1 (one bit per element of S_n each: 3 bits per element, as in
// the bitmask BFS of Section 3.1.3).  Layer r lives in F[r & 1]; its nonempty 1024-rank blocks
// (32 words of F) are listed, once each, in L[r & 1][0, lcount[r & 1]); S[r & 1] has one bit per
// block and is what makes a block's entry in the list unique.  Round r first clears layer r - 1
// (the other bitmap, its listed blocks) and then writes layer r + 1 there.
struct alignas(128) SweepDev {
    // static, written by the host
    unsigned* V;               // visited
    unsigned* F[2];            // layer r in F[r & 1]; the other holds layer r-1, then r+1
    unsigned* S[2];            // per-block bits of F (one bit per 32 words)
    unsigned* L[2];            // nonempty blocks of F (block index = rank >> 10)
    const GenSM* gens;         // k entries
    uint64_t* layer_sizes;     // layers_cap entries; [0] = 1
    uint64_t nblocks;          // 1024-rank blocks: every F has 32 * nblocks words
    uint64_t stop_above;       // 0: none
    uint64_t start_rank;       // rank of the start state
    int k;
    int n;
    int layers_cap;
    int max_radius;            // < 0: unlimited
    // dynamic, updated during a run
    alignas(128) unsigned long long grab;   // next work item of the round
    unsigned long long fresh;               // states found in the round
    unsigned long long lcount[2];           // entries of L[i]
    int radius;                // radius of the frontier layer
    int status;                // JobStatus
};

// Admission of many jobs into one persistent launch (a batch): the jobs are grown in index
// order, at most max_active at a time and with the visited sets of the active jobs summing to at
// most `window` bytes, so that their random accesses stay in L2.  Whenever jobs end, the block
// that closes the round admits the next ones and sets them up; a job whose visited set alone
// exceeds the window is counted as 0 (it misses L2 wherever it runs).
struct AdmitDev {
    int* act[2];               // active job indices, double-buffered (Ctl::adm.act_sel selects)
    const uint64_t* vis;       // per job: visited-set bytes counted against `window`
    uint64_t window;
    int max_active;            // capacity of each act[]; the unit table holds max_active + 1
    int njobs;
    int unit_mult;             // frontier states per warp work unit: 32 * unit_mult
    int pad;
};

// Control block of the persistent kernel (device memory, zero-initialised by the host).
// Blocks arrive at the grid barrier on kBarGroups group counters, the last of each group on
// the top counter; every counter and the generation word that waiting blocks poll sit in
// their own 128-byte line, so neither arrivals nor polling queue at one L2 slice.
constexpr int kBarGroups = 32;
constexpr int kGenBits = 20;
constexpr unsigned long long kGenMask = (1ull << kGenBits) - 1;

struct alignas(128) Ctl {
    unsigned int bar_count;
    unsigned int pad0[31];
    // Barrier word: the low kGenBits bits count the barriers completed in this launch; the rest
    // is a payload the releasing block hands to every block (for a single job: the size of the
    // next frontier, 0 when the growth stops).
    unsigned long long bar_word;
    unsigned int pad1[30];
    int err;                        // 0, or a CG_E* code set by a kernel
    int rounds;                     // rounds completed
    unsigned long long total_units; // warp work units of the current round
    unsigned int pad2[28];
    // A round's units split into a static part, in equal contiguous ranges per block, and the
    // second half, which blocks that finish their range draw from this counter.
    unsigned long long dyn_next;
    unsigned int pad3[30];
    struct alignas(128) Group {
        unsigned int count;
        unsigned int pad[31];
    } group[kBarGroups];
    // Admission of a batch into one launch (AdmitDev), updated by the block that closes a round.
    struct alignas(128) Admit {
        int act_sel;                    // AdmitDev::act[act_sel] lists the active jobs
        int nactive;
        unsigned long long next_admit;  // next job index to admit
        unsigned long long vis_used;    // counted visited-set bytes of the active jobs
    } adm;
};

}  // namespace cg
